// Safety shield (Alg. 1, Eq. 22) on the curvilinear state (state_kind 1;
// smppi.h): the merit P = C sum_{t<N_r} max{(1 - alpha) h_t - h_{t+1}, 0} with
// h = w^2 - e_y^2 (Eq. 17, 23), its gradient by a reverse-mode adjoint of the
// curvilinear model step over a full tape of the N_r states (no recomputation:
// 9 floats per state fit in shared memory for any T), projected gradient with
// Armijo backtracking (mode 1), the fixed step of Alg. 1 (mode 0) or BFGS
// (mode 2, the solver of bfgs.cuh).
//
// Kernels:
//   curv_repair_kernel       modes 0 and 1, one block per sequence: thread 0
//                            runs the forward pass, the block forms the adjoint's
//                            coefficients and thread 0 its recursion
//                            (curv_block_grad), the lanes of
//                            warp 0 evaluate the trial steps s, s/2, ... in
//                            parallel and the largest accepted step is taken
//                            (the same iterate as sequential backtracking);
//   curv_repair_bfgs_kernel  mode 2, one warp per sequence from a work counter;
//   curv_cost_grad_kernel    J and dJ/dV with running-cost and CBF weights
//                            (smppi_cost_grad), one warp per sequence.
// The merit accumulates in float32 over blocks of 16 steps and float64 across
// them.  The closed-loop step (Eq. 26) may follow in the tail of the block or
// warp that repaired sequence 0.
#include <algorithm>

#include "bfgs.cuh"
#include "bfgs_launch.cuh"

namespace smppi {
namespace {

constexpr int CR_BLK = 128;
constexpr int CR_NF = 9;   // tape fields per state: v_x v_y r s e_y e_psi cos sin h

__device__ __forceinline__ void tape_put(float* tp, int t, const State& x, float h) {
    float* r = tp + (size_t)t * CR_NF;
    r[0] = x.vx; r[1] = x.vy; r[2] = x.r; r[3] = x.X; r[4] = x.Y; r[5] = x.psi;
    r[6] = x.cp; r[7] = x.sp; r[8] = h;
}
__device__ __forceinline__ State tape_state(const float* tp, int t) {
    const float* r = tp + (size_t)t * CR_NF;
    State x;
    x.vx = r[0]; x.vy = r[1]; x.r = r[2]; x.X = r[3]; x.Y = r[4]; x.psi = r[5];
    x.cp = r[6]; x.sp = r[7];
    return x;
}

// Slope of kappa(s) on the interval of the samples that kappa_at uses.
__device__ __forceinline__ float kappa_slope(const DevParams& P, const float* kt, float s) {
    const float sw = fmaf(floorf(s * P.inv_len), -P.track_len, s);
    const int i = min(max((int)(sw * P.kap_scale), 0), P.n_track - 1);
    return (kt[i + 1] - kt[i]) * P.kap_scale;
}

// J = w_run sum_{t=0}^{N} q(x_t) + w_cbf sum_{t<N} C max{(1-alpha) h_t - h_{t+1}, 0}
// of Vw (TRIAL: of u' = clip(Vw - step Dn), with dec = G . (Vw - u'); Dn = G when
// no search direction is given) from x0 over N steps; (0, 1) is the merit P.
// STORE: the states and h into the tape (N + 1 rows).
template <bool STORE, bool TRIAL>
__device__ double curv_forward(const DevParams& P, const float* kt, const State& x0, int N,
                               const float2* Vw, const float2* G, float step, float* tape,
                               double* dec_out, float w_run = 0.0f, float w_cbf = 1.0f,
                               const float2* Dn = nullptr) {
    State x = x0;
    float h_prev = P.w2 - x.Y * x.Y;
    double J = (w_run != 0.0f) ? (double)(w_run * run_cost(P, x.vx, x.Y * x.Y)) : 0.0;
    double dec = 0.0;
    float Jf = 0.0f, decf = 0.0f;
    const float wc = w_cbf * P.C_cbf;
    if (STORE && tape) tape_put(tape, 0, x, h_prev);
    for (int t = 0; t < N; ++t) {
        const float2 v = Vw[t];
        float2 u;
        if (TRIAL) {
            const float2 g = G[t];
            const float2 dn = Dn ? Dn[t] : g;
            u = clamp2(P, make_float2(fmaf(-step, dn.x, v.x), fmaf(-step, dn.y, v.y)));
            decf = fmaf(g.x, v.x - u.x, fmaf(g.y, v.y - u.y, decf));
        } else {
            u = clamp2(P, v);
        }
        model_step_curv(P, kt, x, u.x, u.y);
        const float d2 = x.Y * x.Y;
        const float h = P.w2 - d2;
        if (w_run != 0.0f) Jf = fmaf(w_run, run_cost(P, x.vx, d2), Jf);
        const float a = cbf_arg(P, h_prev, h);
        Jf = (a > 0.0f) ? fmaf(wc, a, Jf) : Jf;
        h_prev = h;
        if (STORE && tape) tape_put(tape, t + 1, x, h);
        if (((t + 1) & 15) == 0) {
            J += (double)Jf;
            dec += (double)decf;
            Jf = 0.0f;
            decf = 0.0f;
        }
    }
    J += (double)Jf;
    dec += (double)decf;
    if (dec_out) *dec_out = dec;
    return J;
}

// Adjoint of one curvilinear model step (model_step_curv): lb = dP/dx_{t+1} on
// entry, dP/dx_t (through the step only) on exit; *gd, *ga = dP/du_t.  The
// velocity part is the Cartesian model's (model_step_adjoint); the kinematics
//   s' = s + dt num / den,  num = v_x cos e_psi - v_y sin e_psi,
//   den = max(1 - kappa(s) e_y, 0.1),  e_y' = e_y + dt (v_x sin e_psi + v_y cos e_psi),
//   e_psi' = e_psi + dt (r - kappa(s) num / den)
// are differentiated with cos, sin e_psi as functions of e_psi.
__device__ void model_step_adjoint_curv(const DevParams& P, const float* kt, const State& x,
                                        float d, State& lb, float* gd, float* ga) {
    const float yf = fmaf(P.lf, x.r, x.vy), yr = fmaf(-P.lr, x.r, x.vy);
    const float bf = atan2_poly(yf, x.vx), br = atan2_poly(yr, x.vx);
    const float af = d - bf, ar = -br;
    float dphf, dphr;
    const float Fyf = P.Fzf * tyre_shape(P, P.B * af, &dphf);
    tyre_shape(P, P.B * ar, &dphr);
    float sd, cd;
    sincos_half(d, &sd, &cd);
    const float cp = x.cp, sp = x.sp;
    const float k = kappa_at(P, kt, x.X);
    const float den_raw = fmaf(-k, x.Y, 1.0f);
    const float den = fmaxf(den_raw, 0.1f);
    const float num = x.vx * cp - x.vy * sp;
    const float sdot = num / den;

    const float gvx = P.dt * lb.vx, gvy = P.dt * lb.vy, gr = P.dt * lb.r;
    const float gs = P.dt * lb.X, gey = P.dt * lb.Y, gep = P.dt * lb.psi;
    State o = lb;   // identity part of x + dt F
    // e_psi' : e_psi_dot = r - kappa sdot
    o.r += gep;
    float kb = -gep * sdot;
    const float sdotb = gs - gep * k;
    // e_y' : e_y_dot = v_x sin e_psi + v_y cos e_psi
    o.vx += gey * sp;
    o.vy += gey * cp;
    float spb = gey * x.vx, cpb = gey * x.vy;
    // s' : sdot = num / den
    const float numb = sdotb / den, denb = -sdotb * sdot / den;
    o.vx += numb * cp;
    o.vy -= numb * sp;
    cpb += numb * x.vx;
    spb -= numb * x.vy;
    if (den_raw > 0.1f) {   // den = 1 - kappa e_y (the guard has no derivative)
        kb -= denb * x.Y;
        o.Y -= denb * k;
    }
    o.X += kb * kappa_slope(P, kt, x.X);
    o.psi += spb * cp - cpb * sp;
    // velocity part: dvx = (Fx - Fyf sd)/m + vy r
    const float Fxb = gvx * P.m_inv;
    float Fyfb = -gvx * sd * P.m_inv;
    float db = -gvx * Fyf * cd * P.m_inv;
    o.vy += gvx * x.r;
    o.r += gvx * x.vy;
    // dvy = (Fyr + Fyf cd)/m - vx r
    float Fyrb = gvy * P.m_inv;
    Fyfb += gvy * cd * P.m_inv;
    db -= gvy * Fyf * sd * P.m_inv;
    o.vx -= gvy * x.r;
    o.r -= gvy * x.vx;
    // dr = (lf Fyf cd - lr Fyr)/Iz
    Fyfb += gr * P.lf * cd * P.Iz_inv;
    db -= gr * P.lf * Fyf * sd * P.Iz_inv;
    Fyrb -= gr * P.lr * P.Iz_inv;
    // tyres and slip angles
    const float afb = Fyfb * P.Fzf * dphf * P.B;
    const float arb = Fyrb * P.Fzr * dphr * P.B;
    db += afb;
    const float bfb = -afb, brb = -arb;
    const float nf = fmaf(x.vx, x.vx, yf * yf), nr = fmaf(x.vx, x.vx, yr * yr);
    const float yfb = nf > 0.0f ? bfb * x.vx / nf : 0.0f;
    const float yrb = nr > 0.0f ? brb * x.vx / nr : 0.0f;
    if (nf > 0.0f) o.vx -= bfb * yf / nf;
    if (nr > 0.0f) o.vx -= brb * yr / nr;
    o.vy += yfb + yrb;
    o.r += P.lf * yfb - P.lr * yrb;
    lb = o;
    *gd = db;
    *ga = P.fx_gain * Fxb;
}

// Gradient G of J (w_run, w_cbf; (0, 1) = the merit) of Vw (one thread): forward
// pass with the tape, then the adjoint from x_N back to x_0.  G_t = 0 for
// N <= t < T and outside the box.
__device__ double curv_merit_grad(const DevParams& P, const float* kt, const State& x0, int N,
                                  int T, const float2* Vw, float2* G, float* tape,
                                  float w_run = 0.0f, float w_cbf = 1.0f) {
    const double J = curv_forward<true, false>(P, kt, x0, N, Vw, nullptr, 0.0f, tape, nullptr,
                                               w_run, w_cbf);
    for (int t = N; t < T; ++t) G[t] = make_float2(0.0f, 0.0f);
    if (N == 0) return J;
    State lam = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    auto h_at = [&](int t) { return tape[(size_t)t * CR_NF + 8]; };
    // direct terms of x_t (t >= 1): w_run dq/dx_t (q = q_v (v_x - v*)^2 + q_d e_y^2 / w^2
    // + C_obs 1(outside), Eq. 24-25) and w_cbf C [-act(t-1, t) + (1 - alpha) act(t, t+1)] dh_t,
    // dh_t / de_y = -2 e_y
    const float wc = w_cbf * P.C_cbf;
    auto direct = [&](int t) {
        const float vx = tape[(size_t)t * CR_NF + 0], ey = tape[(size_t)t * CR_NF + 4];
        if (w_run != 0.0f) {
            lam.vx += w_run * 2.0f * P.q_v * (vx - P.v_target);
            lam.Y += w_run * 2.0f * P.qd_w2 * ey;
        }
        const bool a0 = cbf_arg(P, h_at(t - 1), h_at(t)) > 0.0f;
        const bool a1 = (t < N) && cbf_arg(P, h_at(t), h_at(t + 1)) > 0.0f;
        const float w = (a0 ? -wc : 0.0f) + (a1 ? wc * P.one_m_alpha : 0.0f);
        lam.Y += w * (-2.0f * ey);
    };
    direct(N);
    for (int t = N - 1; t >= 0; --t) {
        const State x = tape_state(tape, t);
        const float2 v = Vw[t];
        const float2 u = clamp2(P, v);
        float gd, ga;
        model_step_adjoint_curv(P, kt, x, u.x, lam, &gd, &ga);
        const bool in0 = v.x >= P.umin0 && v.x <= P.umax0;
        const bool in1 = v.y >= P.umin1 && v.y <= P.umax1;
        G[t] = make_float2(in0 ? gd : 0.0f, in1 ? ga : 0.0f);
        if (t >= 1) direct(t);
    }
    return J;
}

// Gradient G of the merit (running-cost weight 0, CBF weight 1) of Vw by a
// block of BLK threads: thread 0 runs the forward pass into the tape, every
// thread forms the coefficients of its steps' adjoint map, and thread 0 runs
// the recursion over (v_x, v_y, r, s, e_y, e_psi).  The adjoint of the Euler
// step is linear in the adjoint, lambda_t = lambda_{t+1} + E_t' lambda_{t+1}
// + d_t and g_t = B_t' lambda_{t+1}; E_t and B_t are the derivatives of
// model_step_adjoint_curv at (x_t, u_t) scaled by dt, collected per step (the
// velocity block as the Cartesian block gradient, the Frenet kinematics through
// (s, e_y, e_psi)), d_t the CBF penalties' derivative at x_t.  coef: 7 float4
// per step.  G_t = 0 for N <= t < T and outside the box.  The group is NT
// threads of ranks 0..NT-1 synchronised by sync() (the block of the repair
// kernel, the warp of the BFGS solver).
template <class Sync>
__device__ __forceinline__ void curv_group_grad(const DevParams& P, const float* kt,
                                                const State& x0, int N, int T, const float2* Vw,
                                                float2* G, float* tape, float4* coef, int tid,
                                                int NT, const Sync& sync, bool have_tape = false) {
    if (tid == 0 && !have_tape)   // have_tape: the tape already holds Vw's trajectory
        curv_forward<true, false>(P, kt, x0, N, Vw, nullptr, 0.0f, tape, nullptr, 0.0f, 1.0f);
    sync();
    const float dt = P.dt, wc = P.C_cbf;
    auto h_at = [&](int t) { return tape[(size_t)t * CR_NF + 8]; };
    for (int t = tid; t < N; t += NT) {
        const State x = tape_state(tape, t);
        const float2 v = Vw[t];
        const float d = clampf(v.x, P.umin0, P.umax0);
        // velocity part: v_x, v_y, r through the tyre forces (as the Cartesian model)
        const float yf = fmaf(P.lf, x.r, x.vy), yr = fmaf(-P.lr, x.r, x.vy);
        const float bf = atan2_poly(yf, x.vx), br = atan2_poly(yr, x.vx);
        float dphf, dphr;
        const float Fyf = P.Fzf * tyre_shape(P, P.B * (d - bf), &dphf);
        tyre_shape(P, P.B * (-br), &dphr);
        float sd, cd;
        sincos_half(d, &sd, &cd);
        const float kf = P.Fzf * dphf * P.B, kr = P.Fzr * dphr * P.B;
        const float nf = fmaf(x.vx, x.vx, yf * yf), nr = fmaf(x.vx, x.vx, yr * yr);
        const float pf = nf > 0.0f ? -kf * x.vx / nf : 0.0f, qf = nf > 0.0f ? kf * yf / nf : 0.0f;
        const float pr = nr > 0.0f ? -kr * x.vx / nr : 0.0f, qr = nr > 0.0f ? kr * yr / nr : 0.0f;
        const float a1 = -sd * P.m_inv, a2 = cd * P.m_inv, a3 = P.lf * cd * P.Iz_inv;
        const float b2 = P.m_inv, b3 = -P.lr * P.Iz_inv;
        const bool in0 = v.x >= P.umin0 && v.x <= P.umax0, in1 = v.y >= P.umin1 && v.y <= P.umax1;
        // kinematics: s' = num / den, e_y' = eyd, e_psi' = r - kappa s'
        const float cp = x.cp, sp = x.sp;
        const float k = kappa_at(P, kt, x.X);
        const float den_raw = fmaf(-k, x.Y, 1.0f);
        const float den = fmaxf(den_raw, 0.1f), id = 1.0f / den;
        const float num = x.vx * cp - x.vy * sp, eyd = x.vx * sp + x.vy * cp;
        const float sdot = num * id;
        const float g1 = den_raw > 0.1f ? 1.0f : 0.0f;   // the guard has no derivative
        const float ks = kappa_slope(P, kt, x.X);
        float4* c = coef + 7 * t;
        c[0] = make_float4(dt * (qf * a1), dt * (-x.r + qf * a2 + qr * b2),
                           dt * (qf * a3 + qr * b3), dt * (x.r + pf * a1));
        c[1] = make_float4(dt * (pf * a2 + pr * b2), dt * (pf * a3 + pr * b3),
                           dt * (x.vy + P.lf * pf * a1),
                           dt * (-x.vx + P.lf * pf * a2 - P.lr * pr * b2));
        c[2] = make_float4(dt * (P.lf * pf * a3 - P.lr * pr * b3), dt * cp * id, dt * sp,
                           -dt * cp * k * id);
        c[3] = make_float4(-dt * sp * id, dt * cp, dt * sp * k * id,
                           dt * ks * g1 * x.Y * sdot * id);
        c[4] = make_float4(dt * ks * (-sdot - g1 * x.Y * k * sdot * id), dt * g1 * k * sdot * id,
                           -dt * g1 * k * k * sdot * id, -dt * eyd * id);
        c[5] = make_float4(dt * num, dt * eyd * k * id,
                           in0 ? dt * (-Fyf * cd * P.m_inv + kf * a1) : 0.0f,
                           in0 ? dt * (-Fyf * sd * P.m_inv + kf * a2) : 0.0f);
        float dey = 0.0f;   // d_t (t >= 1): the penalties of the pairs (t - 1, t) and (t, t + 1)
        if (t > 0) {
            const float w = (cbf_arg(P, h_at(t - 1), h_at(t)) > 0.0f ? -wc : 0.0f) +
                            (cbf_arg(P, h_at(t), h_at(t + 1)) > 0.0f ? wc * P.one_m_alpha : 0.0f);
            dey = w * (-2.0f * x.Y);
        }
        c[6] = make_float4(in0 ? dt * (-P.lf * Fyf * sd * P.Iz_inv + kf * a3) : 0.0f,
                           in1 ? dt * P.fx_gain * P.m_inv : 0.0f, dey, 0.0f);
    }
    sync();
    if (tid == 0) {
        float lvx = 0.0f, lvy = 0.0f, lr = 0.0f, ls = 0.0f, ley = 0.0f, lep = 0.0f;
        if (N > 0 && cbf_arg(P, h_at(N - 1), h_at(N)) > 0.0f)   // lambda_N = d_N
            ley = -wc * (-2.0f * tape[(size_t)N * CR_NF + 4]);
#pragma unroll 4
        for (int t = N - 1; t >= 0; --t) {
            const float4* c = coef + 7 * t;
            const float4 c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3], c4 = c[4], c5 = c[5],
                         c6 = c[6];
            G[t] = make_float2(fmaf(c5.z, lvx, fmaf(c5.w, lvy, c6.x * lr)), c6.y * lvx);
            const float nvx = lvx + (fmaf(c0.x, lvx, c0.y * lvy) + c0.z * lr +
                                     fmaf(c2.y, ls, fmaf(c2.z, ley, c2.w * lep)));
            const float nvy = lvy + (fmaf(c0.w, lvx, c1.x * lvy) + c1.y * lr +
                                     fmaf(c3.x, ls, fmaf(c3.y, ley, c3.z * lep)));
            const float nr = lr + (fmaf(c1.z, lvx, c1.w * lvy) + fmaf(c2.x, lr, dt * lep));
            const float ns = ls + fmaf(c3.w, ls, c4.x * lep);
            const float ney = ley + fmaf(c4.y, ls, c4.z * lep) + c6.z;
            const float nep = lep + (fmaf(c4.w, ls, c5.x * ley) + c5.y * lep);
            lvx = nvx;
            lvy = nvy;
            lr = nr;
            ls = ns;
            ley = ney;
            lep = nep;
        }
        for (int t = N; t < T; ++t) G[t] = make_float2(0.0f, 0.0f);
    }
    sync();
}

template <int BLK>
__device__ void curv_block_grad(const DevParams& P, const float* kt, const State& x0, int N,
                                int T, const float2* Vw, float2* G, float* tape, float4* coef,
                                bool have_tape = false) {
    curv_group_grad(P, kt, x0, N, T, Vw, G, tape, coef, (int)threadIdx.x, BLK,
                    []() { __syncthreads(); }, have_tape);
}

// The merit of the curvilinear state from x0 for the BFGS solver (bfgs.cuh):
// curv_forward (the merit and a kept trial leave their trajectory on the warp's
// full tape), and its gradient by the warp from that tape (curv_group_grad;
// coef: 7 float4 per step).
struct CurvMerit {
    const float* kt;
    State x0;
    float* tape;
    float4* coef;
    __device__ __forceinline__ double merit(const DevParams& P, const float2* Vw) const {
        return curv_forward<true, false>(P, kt, x0, P.N_r, Vw, nullptr, 0.0f, tape, nullptr);
    }
    __device__ __forceinline__ void grad(const DevParams& P, const float2* Vw, float2* G,
                                         bool have_tape) const {
        curv_group_grad(P, kt, x0, P.N_r, P.T, Vw, G, tape, coef, (int)(threadIdx.x & 31), 32,
                        []() { __syncwarp(); }, have_tape);
    }
    __device__ __forceinline__ double trial(const DevParams& P, const float2* Vw, const float2* G,
                                            const float2* Dn, float a, double* dec,
                                            bool keep) const {
        return curv_forward<true, true>(P, kt, x0, P.N_r, Vw, G, a, keep ? tape : nullptr, dec,
                                        0.0f, 1.0f, Dn);
    }
};

// Bytes of the staged curvature samples (n_track + 1 floats, padded to 16).
__host__ __device__ inline size_t kappa_bytes(int n) { return (size_t)((n + 1 + 3) & ~3) * 4; }

// Bytes of one warp's region of the BFGS kernel: the solver's arrays, a full
// tape of T + 1 states padded to 16, and the gradient's coefficients (7 float4 per
// step, at the next 16-byte boundary); a multiple of 8, so float2 arrays stay aligned.
__host__ __device__ inline size_t curv_bfgs_tape_bytes(int T) {
    return ((size_t)(T + 1) * CR_NF * 4 + 15) & ~size_t(15);
}
__host__ __device__ inline size_t curv_bfgs_warp_bytes(int T) {
    return bfgs_array_bytes(T) + curv_bfgs_tape_bytes(T) + (size_t)T * 112 + 16;
}

struct CurvSmem {
    double P;
    float red[CR_BLK / 32];
    float step;
    int ok;
    int keep;
};

}  // namespace

__global__ void __launch_bounds__(CR_BLK) curv_repair_kernel(
    DevParams P, const float* __restrict__ kappa, const float* __restrict__ x0g, const float* Vin,
    float* Vout, int n_iters, int mode, float delta, double* __restrict__ merit_out,
    int* __restrict__ iters_out, ApplyArgs ap, unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = P.T, N = P.N_r, n = P.n_track;
    float2* Vw = reinterpret_cast<float2*>(smem_raw);
    float2* G = Vw + T;
    float* kt = reinterpret_cast<float*>(G + T);
    float* tape = kt + ((n + 1 + 3) & ~3);
    float4* coef = reinterpret_cast<float4*>(
        (reinterpret_cast<uintptr_t>(tape + (size_t)(T + 1) * CR_NF) + 15) & ~uintptr_t(15));
    __shared__ CurvSmem sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = CR_BLK / 32;
    const int q = blockIdx.x;
    const float2* vin = reinterpret_cast<const float2*>(Vin) + (size_t)q * T;
    for (int t = tid; t < T; t += CR_BLK) Vw[t] = vin[t];
    for (int i = tid; i <= n; i += CR_BLK) kt[i] = kappa[i];
    const State x0 = make_state(x0g + 6 * q);
    __syncthreads();
    double* mrow = merit_out ? merit_out + (size_t)q * (n_iters + 1) : nullptr;
    // the merit passes and the line search's first trial leave their trajectory on
    // the tape: the next gradient skips its forward pass when the tape holds Vw's
    if (tid == 0) sm.P = curv_forward<true, false>(P, kt, x0, N, Vw, nullptr, 0.0f, tape, nullptr);
    __syncthreads();
    double P0 = sm.P;
    bool traj_ok = true;
    int it = 0;
    bool stalled = false;
    for (; it < n_iters; ++it) {
        if (tid == 0 && mrow) mrow[it] = P0;
        if (P0 == 0.0) break;
        curv_block_grad<CR_BLK>(P, kt, x0, N, T, Vw, G, tape, coef, traj_ok);
        if (mode == 0) {
            for (int t = tid; t < N; t += CR_BLK)
                Vw[t] = clamp2(P, make_float2(fmaf(-delta, G[t].x, Vw[t].x),
                                              fmaf(-delta, G[t].y, Vw[t].y)));
            __syncthreads();
            if (tid == 0)
                sm.P = curv_forward<true, false>(P, kt, x0, N, Vw, nullptr, 0.0f, tape, nullptr);
            __syncthreads();
            P0 = sm.P;
            traj_ok = true;
            continue;
        }
        float gm = 0.0f;
        for (int t = tid; t < N; t += CR_BLK) gm = fmaxf(gm, fmaxf(fabsf(G[t].x), fabsf(G[t].y)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
        if (lane == 0) sm.red[warp] = gm;
        __syncthreads();
        gm = sm.red[0];
#pragma unroll
        for (int w = 1; w < NW; ++w) gm = fmaxf(gm, sm.red[w]);
        if (!(gm > 0.0f)) { stalled = true; break; }
        const float s_first = P.ls_s0 / gm;
        if (warp == 0) {
            int best = 0x7fffffff;
            double best_P = 0.0;
            for (int j = lane; j < P.ls_max; j += 32) {
                const float sj = ldexpf(s_first, -j);
                double dec;
                const double Pt =
                    curv_forward<true, true>(P, kt, x0, N, Vw, G, sj, j == 0 ? tape : nullptr, &dec);
                if (Pt <= P0 - (double)P.ls_c * dec && j < best) { best = j; best_P = Pt; }
            }
            int bj = best;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bj = min(bj, __shfl_xor_sync(0xffffffffu, bj, o));
            if (best == bj && bj != 0x7fffffff) {
                sm.P = best_P;
                sm.step = ldexpf(s_first, -bj);
            }
            if (lane == 0) {
                sm.ok = (bj != 0x7fffffff);
                sm.keep = (bj == 0);   // the first trial's trajectory is the new iterate's
            }
        }
        __syncthreads();
        if (!sm.ok) { stalled = true; break; }
        traj_ok = sm.keep != 0;
        const float sa = sm.step;
        for (int t = tid; t < N; t += CR_BLK)
            Vw[t] = clamp2(P, make_float2(fmaf(-sa, G[t].x, Vw[t].x), fmaf(-sa, G[t].y, Vw[t].y)));
        __syncthreads();
        P0 = sm.P;
    }
    if (tid == 0) {
        if (mrow)
            for (int i = it; i <= n_iters; ++i) mrow[i] = P0;
        if (iters_out) iters_out[q] = it;
        if (stalled) atomicOr(status, SMPPI_DEV_STALLED);
        if (!isfinite(P0)) atomicOr(status, SMPPI_DEV_NUMERIC);
    }
    __syncthreads();
    float2* vout = reinterpret_cast<float2*>(Vout) + (size_t)q * T;
    for (int t = tid; t < T; t += CR_BLK) vout[t] = Vw[t];
    if (q == 0 && tid == 0 && ap.x0) closed_loop_step(P, ap, Vw[0]);
}

// J and dJ/dV of n_seq sequences (smppi_cost_grad on the curvilinear state):
// one warp per sequence, lane 0 runs the forward pass into the warp's tape and
// the adjoint; the tape keeps every state (the checkpoint argument does not
// apply).  Gradients of the controls t >= N are 0.
__global__ void __launch_bounds__(32) curv_cost_grad_kernel(
    DevParams P, const float* __restrict__ kappa, int n_seq, const float* __restrict__ x0g,
    const float* __restrict__ Vg, int N, float w_run, float w_cbf, double* __restrict__ J_out,
    float* __restrict__ grad_out, unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = P.T, n = P.n_track, q = blockIdx.x, lane = threadIdx.x;
    float2* Vw = reinterpret_cast<float2*>(smem_raw);
    float2* G = Vw + T;
    float* kt = reinterpret_cast<float*>(G + T);
    float* tape = kt + ((n + 1 + 3) & ~3);
    if (q >= n_seq) return;
    const float2* vin = reinterpret_cast<const float2*>(Vg) + (size_t)q * T;
    for (int t = lane; t < T; t += 32) Vw[t] = vin[t];
    for (int i = lane; i <= n; i += 32) kt[i] = kappa[i];
    __syncwarp();
    if (lane == 0) {
        const State x0 = make_state(x0g + 6 * q);
        const double J = curv_merit_grad(P, kt, x0, N, T, Vw, G, tape, w_run, w_cbf);
        if (J_out) J_out[q] = J;
        if (!isfinite(J)) atomicOr(status, SMPPI_DEV_NUMERIC);
    }
    __syncwarp();
    float2* gout = reinterpret_cast<float2*>(grad_out) + (size_t)q * T;
    for (int t = lane; t < T; t += 32) gout[t] = G[t];
}

cudaError_t launch_cost_grad_curv(const DevParams& P, const float* kappa, int n_seq,
                                  const float* x0, const float* V, int N, float w_run, float w_cbf,
                                  double* J_out, float* grad_out, unsigned* status,
                                  cudaStream_t st) {
    const size_t smem = (size_t)P.T * 16 + (size_t)((P.n_track + 1 + 3) & ~3) * 4 +
                        (size_t)(P.T + 1) * CR_NF * 4;
    cudaError_t e = ensure_smem((const void*)curv_cost_grad_kernel, smem);
    if (e != cudaSuccess) return e;
    curv_cost_grad_kernel<<<n_seq, 32, smem, st>>>(P, kappa, n_seq, x0, V, N, w_run, w_cbf, J_out,
                                                   grad_out, status);
    return cudaGetLastError();
}

cudaError_t launch_repair_curv(const DevParams& P, const float* kappa, int n_seq,
                               const float* x0, const float* V_in, float* V_out, int n_iters,
                               int mode, float delta, double* merit_out, int* iters_out,
                               const ApplyArgs& ap, unsigned* status, cudaStream_t st) {
    const size_t smem = (size_t)P.T * 16 + (size_t)((P.n_track + 1 + 3) & ~3) * 4 +
                        (size_t)(P.T + 1) * CR_NF * 4 + 16 + (size_t)P.T * 7 * 16;
    cudaError_t e = ensure_smem((const void*)curv_repair_kernel, smem);
    if (e != cudaSuccess) return e;
    curv_repair_kernel<<<n_seq, CR_BLK, smem, st>>>(P, kappa, x0, V_in, V_out, n_iters, mode,
                                                    delta, merit_out, iters_out, ap, status);
    return cudaGetLastError();
}


// BFGS repair (mode 2) on the curvilinear state: the solver of bfgs.cuh with
// the curvilinear merit.  A block holds a few warps that share the staged
// curvature samples; warps take sequences from an atomic counter.
__global__ void __launch_bounds__(32 * BFGS_WPB_MAX, 2) curv_repair_bfgs_kernel(
    DevParams P, const float* __restrict__ kappa, const float* __restrict__ x0g, const float* Vin,
    float* Vout, int n_seq, int n_iters, float* __restrict__ Hws, unsigned* __restrict__ next,
    double* __restrict__ merit_out, int* __restrict__ iters_out, ApplyArgs ap,
    unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = P.T, nt = P.n_track, n = 2 * P.N_r;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    float* kt = reinterpret_cast<float*>(smem_raw);
    unsigned char* wbase = smem_raw + kappa_bytes(nt) + (size_t)warp * curv_bfgs_warp_bytes(T);
    const BfgsArrays a = bfgs_arrays(wbase, T);
    float* tape = reinterpret_cast<float*>(wbase + bfgs_array_bytes(T));
    float4* coef = reinterpret_cast<float4*>(
        (reinterpret_cast<uintptr_t>(wbase + bfgs_array_bytes(T) + curv_bfgs_tape_bytes(T)) + 15) &
        ~uintptr_t(15));
    float* H = Hws + ((size_t)blockIdx.x * wpb + warp) * n * n;

    for (int i = threadIdx.x; i <= nt; i += blockDim.x) kt[i] = kappa[i];
    __syncthreads();

    for (;;) {
        int q = 0;
        if (lane == 0) q = (int)atomicAdd(next, 1u);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= n_seq) break;
        const float2* vin = reinterpret_cast<const float2*>(Vin) + (size_t)q * T;
        for (int t = lane; t < T; t += 32) a.Vw[t] = vin[t];
        __syncwarp();
        const CurvMerit f{kt, make_state(x0g + 6 * q), tape, coef};
        double P0;
        bool stalled;
        const int it = bfgs_solve(P, f, a, H, n_iters,
                                  merit_out ? merit_out + (size_t)q * (n_iters + 1) : nullptr, &P0,
                                  &stalled);
        if (lane == 0) {
            if (iters_out) iters_out[q] = it;
            if (stalled) atomicOr(status, SMPPI_DEV_STALLED);
            if (!isfinite(P0)) atomicOr(status, SMPPI_DEV_NUMERIC);
        }
        float2* vout = reinterpret_cast<float2*>(Vout) + (size_t)q * T;
        for (int t = lane; t < T; t += 32) vout[t] = a.Vw[t];
        if (q == 0 && lane == 0 && ap.x0) closed_loop_step(P, ap, a.Vw[0]);
        __syncwarp();   // the warp's shared memory is reused by its next sequence
    }
}

int curv_bfgs_grid(const DevParams& P, int n_seq, int sms, int* wpb_out) {
    return bfgs_shape((const void*)curv_repair_bfgs_kernel, kappa_bytes(P.n_track),
                      curv_bfgs_warp_bytes(P.T), P.N_r, n_seq, sms, wpb_out);
}

cudaError_t launch_repair_bfgs_curv(const DevParams& P, const float* kappa, int n_seq,
                                    const float* x0, const float* V_in, float* V_out, int n_iters,
                                    void* ws, int grid, int wpb, double* merit_out, int* iters_out,
                                    const ApplyArgs& ap, unsigned* status, cudaStream_t st) {
    const size_t smem = kappa_bytes(P.n_track) + (size_t)wpb * curv_bfgs_warp_bytes(P.T);
    cudaError_t e = ensure_smem((const void*)curv_repair_bfgs_kernel, smem);
    if (e != cudaSuccess) return e;
    unsigned* next = static_cast<unsigned*>(ws);
    float* H = reinterpret_cast<float*>(static_cast<unsigned char*>(ws) + 16);
    e = cudaMemsetAsync(next, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    curv_repair_bfgs_kernel<<<grid, 32 * wpb, smem, st>>>(P, kappa, x0, V_in, V_out, n_seq, n_iters,
                                                          H, next, merit_out, iters_out, ap, status);
    return cudaGetLastError();
}

}  // namespace smppi
