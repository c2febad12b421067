// Safety shield (Alg. 1, Eq. 22): reverse-mode adjoint of the deterministic
// rollout cost with checkpointing, Armijo / fixed-step repair, and the
// closed-loop step (Alg. 2 ExecuteCommand + warm start, Eq. 26).
//
// One thread owns one control sequence.  The forward sweep stores the state
// every `ck` steps (checkpoints, ~sqrt(T) of them); the backward sweep walks
// the checkpoint segments from last to first, recomputes each segment's states
// from its checkpoint and runs the hand-derived adjoint of the Euler step
// through them.  With ck <= 0 the forward sweep stores every state instead
// (full tape, no recomputation).  Per-sequence arrays live in a workspace laid
// out [slot][field][sequence] so that a warp's accesses are coalesced.
#include "kernels.cuh"

namespace smppi {

namespace {

struct Tape {
    float* base;
    int ms, seq;
    __device__ __forceinline__ float& at(int slot, int f) const {
        return base[((size_t)slot * NFIELD + f) * ms + seq];
    }
    __device__ __forceinline__ void put(int slot, const State& x, int s, float h, float hp) const {
        at(slot, 0) = x.vx; at(slot, 1) = x.vy; at(slot, 2) = x.r;
        at(slot, 3) = x.X; at(slot, 4) = x.Y; at(slot, 5) = x.psi;
        at(slot, 6) = x.cp; at(slot, 7) = x.sp;
        at(slot, 8) = __int_as_float(s); at(slot, 9) = h; at(slot, 10) = hp;
    }
    __device__ __forceinline__ void get(int slot, State& x, int& s, float& h, float& hp) const {
        x.vx = at(slot, 0); x.vy = at(slot, 1); x.r = at(slot, 2);
        x.X = at(slot, 3); x.Y = at(slot, 4); x.psi = at(slot, 5);
        x.cp = at(slot, 6); x.sp = at(slot, 7);
        s = __float_as_int(at(slot, 8)); h = at(slot, 9); hp = at(slot, 10);
    }
};

__device__ __forceinline__ float2 clamp2(const DevParams& P, float2 v) {
    return make_float2(clampf(v.x, P.umin0, P.umax0), clampf(v.y, P.umin1, P.umax1));
}

// Direct derivative of the cost terms at x_t (segment s, h_{t-1}, h_t, h_{t+1}):
//   w_run dq/dx_t + w_cbf C [act(t-1,t) (-dh_t/dx_t) + act(t,t+1) (1-alpha) dh_t/dx_t],
// dh/d(X,Y) = -2 r, dq/d(X,Y) = (q_d / w^2) 2 r, dq/dv_x = 2 q_v (v_x - v_target).
__device__ __forceinline__ void add_direct(const DevParams& P, const float4* seg, const float* inv,
                                           const State& x, int s, bool act_prev, bool act_next,
                                           float w_run, float w_cbf, State& lam) {
    const float2 r = seg_offset(seg, inv, s, x.X, x.Y);
    float ch = 0.0f;
    if (act_prev) ch -= w_cbf * P.C_cbf;
    if (act_next) ch += w_cbf * P.C_cbf * P.one_m_alpha;
    // dJ/d(e_y^2) = w_run q_d / w^2 - ch  (since h = w^2 - e_y^2)
    const float cd2 = 2.0f * (w_run * P.qd_w2 - ch);
    lam.X += cd2 * r.x;
    lam.Y += cd2 * r.y;
    lam.vx += w_run * 2.0f * P.q_v * (x.vx - P.v_target);
}

// Forward rollout of u_t = clamp(Vw_t - step G_t) for N steps from x0 (segment s0).
// Returns J in float64 and, when STORE, fills the tape (every state when
// ck <= 0, else every ck-th).  dec_out (optional) = sum_t G_t . (Vw_t - u'_t)
// where u'_t = clip(Vw_t - step G_t) (the Armijo decrease term).  The terms are
// summed in float32 over blocks of 16 steps and the block sums in float64
// (FP64 arithmetic is slow on this part; one FP64 add per 16 steps).
template <bool STORE, bool TRIAL>
__device__ double forward_cost(const DevParams& P, const float4* seg, const float* inv,
                               const State& x0, int s0, int N, const float2* Vw, const float2* G,
                               float step, int ms, int seq, float w_run, float w_cbf, int ck,
                               const Tape& tape, double* dec_out) {
    State x = x0;
    int s = s0;
    float d2 = seg_d2(seg, inv, s, x.X, x.Y);
    float h_prev = P.w2 - d2, h_pp = h_prev;
    double J = (double)(w_run * run_cost(P, x.vx, d2));
    double dec = 0.0;
    float Jf = 0.0f, decf = 0.0f;
    const float wc = w_cbf * P.C_cbf;
    const bool full = ck <= 0;
    for (int t = 0; t < N; ++t) {
        if (STORE) {
            if (full) tape.put(t, x, s, h_prev, h_pp);
            else if (t % ck == 0) tape.put(t / ck, x, s, h_prev, h_pp);
        }
        float2 v = Vw[(size_t)t * ms + seq];
        float2 u;
        if (TRIAL) {
            const float2 g = G[(size_t)t * ms + seq];
            u = clamp2(P, make_float2(fmaf(-step, g.x, v.x), fmaf(-step, g.y, v.y)));
            decf = fmaf(g.x, v.x - u.x, fmaf(g.y, v.y - u.y, decf));
        } else {
            u = clamp2(P, v);
        }
        model_step(P, x, u.x, u.y);
        s = track_follow(seg, inv, P.n_track, s, x.X, x.Y, d2);
        const float h = P.w2 - d2;
        if (w_run != 0.0f) Jf = fmaf(w_run, run_cost(P, x.vx, d2), Jf);
        const float a = cbf_arg(P, h_prev, h);
        if (a > 0.0f) Jf = fmaf(wc, a, Jf);
        h_pp = h_prev;
        h_prev = h;
        if ((t & 15) == 15) {
            J += (double)Jf;
            dec += (double)decf;
            Jf = 0.0f;
            decf = 0.0f;
        }
    }
    J += (double)Jf;
    dec += (double)decf;
    if (STORE && full) tape.put(N, x, s, h_prev, h_pp);
    if (dec_out) *dec_out = dec;
    return J;
}

// Cost and gradient of one sequence (forward with tape + backward adjoint).
// Writes G_t = dJ/dv_t for t < N (0 for N <= t < T).
__device__ double seq_cost_grad(const DevParams& P, const float4* seg, const float* inv,
                                const State& x0, int s0, int N, int T, const float2* Vw, float2* G,
                                int ms, int seq, float w_run, float w_cbf, int ck,
                                const Tape& tape) {
    const double J = forward_cost<true, false>(P, seg, inv, x0, s0, N, Vw, nullptr, 0.0f, ms, seq,
                                               w_run, w_cbf, ck, tape, nullptr);
    for (int t = N; t < T; ++t) G[(size_t)t * ms + seq] = make_float2(0.0f, 0.0f);
    if (N == 0) return J;
    const bool full = ck <= 0;
    const int nck = full ? 1 : (N + ck - 1) / ck;
    const int rb = full ? 0 : nck;  // first slot of the recomputed segment
    State lam = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int c = nck - 1; c >= 0; --c) {
        const int t0 = full ? 0 : c * ck;
        const int t1 = full ? N : min(t0 + ck, N);
        if (!full) {
            // recompute states t0..t1 from checkpoint c
            State x;
            int s;
            float h, hp;
            tape.get(c, x, s, h, hp);
            tape.put(rb, x, s, h, hp);
            for (int i = 1; i <= t1 - t0; ++i) {
                const float2 u = clamp2(P, Vw[(size_t)(t0 + i - 1) * ms + seq]);
                model_step(P, x, u.x, u.y);
                float d2;
                s = track_follow(seg, inv, P.n_track, s, x.X, x.Y, d2);
                hp = h;
                h = P.w2 - d2;
                tape.put(rb + i, x, s, h, hp);
            }
        }
        if (c == nck - 1) {
            // lambda_N = direct term at x_N (only the pair (N-1, N))
            State x;
            int s;
            float h, hp;
            tape.get(rb + (t1 - t0), x, s, h, hp);
            add_direct(P, seg, inv, x, s, cbf_arg(P, hp, h) > 0.0f, false, w_run, w_cbf, lam);
        }
        for (int t = t1 - 1; t >= t0; --t) {
            const int i = rb + (t - t0);
            State x;
            int s;
            float h, hp;
            tape.get(i, x, s, h, hp);
            const float h_next = tape.at(i + 1, 9);
            const float2 v = Vw[(size_t)t * ms + seq];
            const float2 u = clamp2(P, v);
            float gd, ga;
            model_step_adjoint(P, x, u.x, u.y, lam, &gd, &ga);
            const bool in0 = v.x >= P.umin0 && v.x <= P.umax0;
            const bool in1 = v.y >= P.umin1 && v.y <= P.umax1;
            G[(size_t)t * ms + seq] = make_float2(in0 ? gd : 0.0f, in1 ? ga : 0.0f);
            if (t >= 1)
                add_direct(P, seg, inv, x, s, cbf_arg(P, hp, h) > 0.0f,
                           cbf_arg(P, h, h_next) > 0.0f, w_run, w_cbf, lam);
        }
    }
    return J;
}

// Closed-loop step (Alg. 2 ExecuteCommand + warm start, Eq. 26), one thread:
// x0 <- f(x0, clamp(v_exec)) + w_n, V <- shift(V).
__device__ void closed_loop_step(const DevParams& P, const ApplyArgs& ap, float2 v_exec) {
    const uint32_t nn = ap.n + (ap.iter_dev ? *ap.iter_dev : 0u);
    State x = make_state(ap.x0);
    model_step(P, x, clampf(v_exec.x, P.umin0, P.umax0), clampf(v_exec.y, P.umin1, P.umax1));
    const uint4 r = philox10(make_uint4(0u, 0u, nn, ap.ctr3), P);
    const float2 z = box_muller(r.x, r.y);
    ap.x0[0] = x.vx;
    ap.x0[1] = fmaf(P.dsig0, z.x, x.vy);
    ap.x0[2] = fmaf(P.dsig1, z.y, x.r);
    ap.x0[3] = x.X;
    ap.x0[4] = x.Y;
    ap.x0[5] = x.psi;
    float2* V = reinterpret_cast<float2*>(ap.V);
    for (int t = 0; t + 1 < P.T; ++t) V[t] = V[t + 1];
    if (ap.iter_dev) *ap.iter_dev += 1u;
}

}  // namespace

__global__ void seg_table_kernel(const float* __restrict__ xy, int n, float4* __restrict__ seg,
                                 float* __restrict__ inv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = (i + 1 == n) ? 0 : i + 1;
    const float ax = xy[2 * i], ay = xy[2 * i + 1];
    const float dx = xy[2 * j] - ax, dy = xy[2 * j + 1] - ay;
    seg[i] = make_float4(ax, ay, dx, dy);
    inv[i] = 1.0f / fmaf(dx, dx, dy * dy);
}

// Global nearest segment of each x0 (one warp per sequence).
__global__ void seg0_kernel(DevParams P, const float4* __restrict__ seg,
                            const float* __restrict__ inv, int n_seq, const float* __restrict__ x0,
                            int* __restrict__ seg0) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= n_seq) return;
    const float X = x0[6 * w + 3], Y = x0[6 * w + 4];
    float bd = 3.0e38f;
    int bi = 0x7fffffff;
    for (int i = lane; i < P.n_track; i += 32) {
        const float d = seg_d2(seg, inv, i, X, Y);
        if (d < bd) { bd = d; bi = i; }
    }
    warp_argmin(bd, bi);
    if (lane == 0) seg0[w] = bi;
}

constexpr int REP_BLK = 64;

__device__ __forceinline__ void stage_track(const DevParams& P, const float4* __restrict__ segg,
                                            const float* __restrict__ invg, float4* seg,
                                            float* inv) {
    for (int i = threadIdx.x; i < P.n_track; i += blockDim.x) {
        seg[i] = segg[i];
        inv[i] = invg[i];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(REP_BLK) cost_grad_kernel(
    DevParams P, const float4* __restrict__ segg, const float* __restrict__ invg, RepairWs ws,
    int n_seq, const float* __restrict__ x0g, const float* __restrict__ Vg, int N, float w_run,
    float w_cbf, int ck, double* __restrict__ J_out, float* __restrict__ grad_out,
    unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* seg = reinterpret_cast<float4*>(smem_raw);
    float* inv = reinterpret_cast<float*>(seg + P.n_track);
    stage_track(P, segg, invg, seg, inv);
    const int q = blockIdx.x * REP_BLK + threadIdx.x;
    if (q >= n_seq) return;
    const int T = P.T, ms = ws.max_seq;
    const float2* Vrow = reinterpret_cast<const float2*>(Vg) + (size_t)q * T;
    for (int t = 0; t < T; ++t) ws.Vw[(size_t)t * ms + q] = Vrow[t];
    const State x0 = make_state(x0g + 6 * q);
    const Tape tape{ws.tape, ms, q};
    const double J = seq_cost_grad(P, seg, inv, x0, ws.seg0[q], N, T, ws.Vw, ws.G, ms, q, w_run,
                                   w_cbf, ck, tape);
    if (J_out) J_out[q] = J;
    if (!isfinite(J)) atomicOr(status, SMPPI_DEV_NUMERIC);
    float2* grow = reinterpret_cast<float2*>(grad_out) + (size_t)q * T;
    for (int t = 0; t < T; ++t) grow[t] = ws.G[(size_t)t * ms + q];
}

__global__ void __launch_bounds__(REP_BLK) repair_kernel(
    DevParams P, const float4* __restrict__ segg, const float* __restrict__ invg, RepairWs ws,
    int n_seq, const float* __restrict__ x0g, const float* Vin, float* Vout, int n_iters,
    int mode, float delta, double* __restrict__ merit_out, int* __restrict__ iters_out,
    ApplyArgs ap, unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* seg = reinterpret_cast<float4*>(smem_raw);
    float* inv = reinterpret_cast<float*>(seg + P.n_track);
    stage_track(P, segg, invg, seg, inv);
    const int q = blockIdx.x * REP_BLK + threadIdx.x;
    if (q >= n_seq) return;
    const int T = P.T, N = P.N_r, ms = ws.max_seq;
    const float2* vin = reinterpret_cast<const float2*>(Vin) + (size_t)q * T;
    float2* vout = reinterpret_cast<float2*>(Vout) + (size_t)q * T;
    for (int t = 0; t < T; ++t) ws.Vw[(size_t)t * ms + q] = vin[t];
    const State x0 = make_state(x0g + 6 * q);
    const int s0 = ws.seg0[q];
    const Tape tape{ws.tape, ms, q};
    double P0 = forward_cost<false, false>(P, seg, inv, x0, s0, N, ws.Vw, nullptr, 0.0f, ms, q,
                                           0.0f, 1.0f, 0, tape, nullptr);
    int it = 0;
    bool stalled = false;
    for (; it < n_iters; ++it) {
        if (merit_out) merit_out[(size_t)q * (n_iters + 1) + it] = P0;
        if (P0 == 0.0) break;
        seq_cost_grad(P, seg, inv, x0, s0, N, T, ws.Vw, ws.G, ms, q, 0.0f, 1.0f, ws.ck, tape);
        if (mode == 0) {
            for (int t = 0; t < N; ++t) {
                const size_t o = (size_t)t * ms + q;
                const float2 v = ws.Vw[o], g = ws.G[o];
                ws.Vw[o] = clamp2(P, make_float2(fmaf(-delta, g.x, v.x), fmaf(-delta, g.y, v.y)));
            }
            P0 = forward_cost<false, false>(P, seg, inv, x0, s0, N, ws.Vw, nullptr, 0.0f, ms, q,
                                            0.0f, 1.0f, 0, tape, nullptr);
            continue;
        }
        float gmax = 0.0f;
        for (int t = 0; t < N; ++t) {
            const float2 g = ws.G[(size_t)t * ms + q];
            gmax = fmaxf(gmax, fmaxf(fabsf(g.x), fabsf(g.y)));
        }
        if (!(gmax > 0.0f)) { stalled = true; break; }
        float s = P.ls_s0 / gmax;
        bool accepted = false;
        for (int j = 0; j < P.ls_max; ++j) {
            double dec;
            const double Pt = forward_cost<false, true>(P, seg, inv, x0, s0, N, ws.Vw, ws.G, s, ms,
                                                        q, 0.0f, 1.0f, 0, tape, &dec);
            if (Pt <= P0 - (double)P.ls_c * dec) {
                for (int t = 0; t < N; ++t) {
                    const size_t o = (size_t)t * ms + q;
                    const float2 v = ws.Vw[o], g = ws.G[o];
                    ws.Vw[o] = clamp2(P, make_float2(fmaf(-s, g.x, v.x), fmaf(-s, g.y, v.y)));
                }
                P0 = Pt;
                accepted = true;
                break;
            }
            s *= 0.5f;
        }
        if (!accepted) { stalled = true; break; }
    }
    if (merit_out)
        for (int i = it; i <= n_iters; ++i) merit_out[(size_t)q * (n_iters + 1) + i] = P0;
    if (iters_out) iters_out[q] = it;
    if (stalled) atomicOr(status, SMPPI_DEV_STALLED);
    if (!isfinite(P0)) atomicOr(status, SMPPI_DEV_NUMERIC);
    for (int t = 0; t < T; ++t) vout[t] = ws.Vw[(size_t)t * ms + q];
    if (q == 0 && ap.x0) closed_loop_step(P, ap, ws.Vw[0]);
}

// Safety shield for few sequences: one block per sequence, everything in
// shared memory (track table staged by a bulk copy, controls, gradient,
// checkpoint tape), the Armijo trial steps s, s/2, s/4, ... evaluated in
// parallel by the lanes of warp 0 (lane j: s 2^-j), the largest accepted step
// taken: the same iterate as sequential backtracking.
constexpr int REPB_BLK = 64;

__global__ void __launch_bounds__(REPB_BLK) repair_block_kernel(
    DevParams P, const float4* __restrict__ segg, const float* __restrict__ invg, int inv_pad,
    const float* __restrict__ x0g, const float* Vin, float* Vout, int n_iters, int mode,
    float delta, int ck, double* __restrict__ merit_out, int* __restrict__ iters_out, ApplyArgs ap,
    unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = P.T, N = P.N_r, n = P.n_track;
    float4* seg = reinterpret_cast<float4*>(smem_raw);
    float* inv = reinterpret_cast<float*>(seg + n);
    float2* Vw = reinterpret_cast<float2*>(inv + inv_pad);
    float2* G = Vw + T;
    float* tape_s = reinterpret_cast<float*>(G + T);
    __shared__ __align__(8) uint64_t bar;
    __shared__ double s_P;
    __shared__ float s_red[REPB_BLK / 32];
    __shared__ int s_redi[REPB_BLK / 32];
    __shared__ int s_seg0;
    __shared__ float s_step;
    __shared__ bool s_ok;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = blockIdx.x;

    // stage the track (bulk copy) and this sequence's controls
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (tid == 0) {
        const uint32_t b_seg = (uint32_t)n * 16u, b_inv = (uint32_t)inv_pad * 4u;
        mbar_expect_tx(&bar, b_seg + b_inv);
        bulk_g2s(seg, segg, b_seg, &bar);
        bulk_g2s(inv, invg, b_inv, &bar);
    }
    const float2* vin = reinterpret_cast<const float2*>(Vin) + (size_t)q * T;
    for (int t = tid; t < T; t += REPB_BLK) Vw[t] = vin[t];
    const State x0 = make_state(x0g + 6 * q);
    if (!mbar_wait_bounded(&bar, 0)) {
        atomicOr(status, SMPPI_DEV_TIMEOUT);
        mbar_wait_bounded(&bar, 0);   // give the copy in flight a second chance to land
        return;
    }
    // nearest segment of x0 (lowest index on ties)
    float bd = 3.0e38f;
    int bi = 0x7fffffff;
    for (int i = tid; i < n; i += REPB_BLK) {
        const float d = seg_d2(seg, inv, i, x0.X, x0.Y);
        if (d < bd) { bd = d; bi = i; }
    }
    warp_argmin(bd, bi);
    if (lane == 0) { s_red[warp] = bd; s_redi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < REPB_BLK / 32; ++w)
            if (s_red[w] < bd || (s_red[w] == bd && s_redi[w] < bi)) { bd = s_red[w]; bi = s_redi[w]; }
        s_seg0 = bi;
    }
    __syncthreads();
    const int s0 = s_seg0;
    const Tape tape{tape_s, 1, 0};
    if (tid == 0)
        s_P = forward_cost<false, false>(P, seg, inv, x0, s0, N, Vw, nullptr, 0.0f, 1, 0, 0.0f,
                                         1.0f, 0, tape, nullptr);
    __syncthreads();
    double P0 = s_P;
    int it = 0;
    bool stalled = false;
    for (; it < n_iters; ++it) {
        if (tid == 0 && merit_out) merit_out[(size_t)q * (n_iters + 1) + it] = P0;
        if (P0 == 0.0) break;
        if (tid == 0) seq_cost_grad(P, seg, inv, x0, s0, N, T, Vw, G, 1, 0, 0.0f, 1.0f, ck, tape);
        __syncthreads();
        if (mode == 0) {
            for (int t = tid; t < N; t += REPB_BLK)
                Vw[t] = clamp2(P, make_float2(fmaf(-delta, G[t].x, Vw[t].x),
                                              fmaf(-delta, G[t].y, Vw[t].y)));
            __syncthreads();
            if (tid == 0)
                s_P = forward_cost<false, false>(P, seg, inv, x0, s0, N, Vw, nullptr, 0.0f, 1, 0,
                                                 0.0f, 1.0f, 0, tape, nullptr);
            __syncthreads();
            P0 = s_P;
            continue;
        }
        // |g|_inf
        float gm = 0.0f;
        for (int t = tid; t < N; t += REPB_BLK)
            gm = fmaxf(gm, fmaxf(fabsf(G[t].x), fabsf(G[t].y)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
        if (lane == 0) s_red[warp] = gm;
        __syncthreads();
        gm = s_red[0];
        for (int w = 1; w < REPB_BLK / 32; ++w) gm = fmaxf(gm, s_red[w]);
        if (!(gm > 0.0f)) { stalled = true; break; }
        const float s_first = P.ls_s0 / gm;
        if (warp == 0) {
            // lane j tries s_first 2^-j (j = lane, lane + 32, ...); keep the smallest accepted j
            int best = 0x7fffffff;
            double best_P = 0.0;
            for (int j = lane; j < P.ls_max; j += 32) {
                const float sj = ldexpf(s_first, -j);
                double dec;
                const double Pt = forward_cost<false, true>(P, seg, inv, x0, s0, N, Vw, G, sj, 1,
                                                            0, 0.0f, 1.0f, 0, tape, &dec);
                if (Pt <= P0 - (double)P.ls_c * dec && j < best) { best = j; best_P = Pt; }
            }
            int bj = best;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bj = min(bj, __shfl_xor_sync(0xffffffffu, bj, o));
            if (best == bj && bj != 0x7fffffff) {   // the owning lane publishes
                s_P = best_P;
                s_step = ldexpf(s_first, -bj);
            }
            if (lane == 0) s_ok = (bj != 0x7fffffff);
        }
        __syncthreads();
        if (!s_ok) { stalled = true; break; }
        const float sa = s_step;
        for (int t = tid; t < N; t += REPB_BLK)
            Vw[t] = clamp2(P, make_float2(fmaf(-sa, G[t].x, Vw[t].x), fmaf(-sa, G[t].y, Vw[t].y)));
        __syncthreads();
        P0 = s_P;
    }
    if (tid == 0) {
        if (merit_out)
            for (int i = it; i <= n_iters; ++i) merit_out[(size_t)q * (n_iters + 1) + i] = P0;
        if (iters_out) iters_out[q] = it;
        if (stalled) atomicOr(status, SMPPI_DEV_STALLED);
        if (!isfinite(P0)) atomicOr(status, SMPPI_DEV_NUMERIC);
    }
    float2* vout = reinterpret_cast<float2*>(Vout) + (size_t)q * T;
    for (int t = tid; t < T; t += REPB_BLK) vout[t] = Vw[t];
    if (q == 0 && tid == 0 && ap.x0) closed_loop_step(P, ap, Vw[0]);
}

// Closed-loop step as its own launch (V_exec may alias ap.V: it is read first).
__global__ void apply_kernel(DevParams P, ApplyArgs ap, const float* V_exec) {
    const float2 v = reinterpret_cast<const float2*>(V_exec)[0];
    closed_loop_step(P, ap, v);
}

// ----------------------------------------------------------------------------
cudaError_t launch_seg_table(const float* xy, int n, float4* seg, float* inv, cudaStream_t st) {
    seg_table_kernel<<<(n + 127) / 128, 128, 0, st>>>(xy, n, seg, inv);
    return cudaGetLastError();
}

cudaError_t launch_seg0(const DevParams& P, const float4* seg, const float* inv, int n_seq,
                        const float* x0, int* seg0, cudaStream_t st) {
    const int warps_per_block = 4;
    seg0_kernel<<<(n_seq + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(
        P, seg, inv, n_seq, x0, seg0);
    return cudaGetLastError();
}

static size_t track_smem(int n) { return (size_t)n * (sizeof(float4) + sizeof(float)); }

cudaError_t launch_cost_grad(const DevParams& P, const float4* seg, const float* inv,
                             const RepairWs& ws, int n_seq, const float* x0, const float* V, int N,
                             float w_run, float w_cbf, int ck, double* J_out, float* grad_out,
                             unsigned* status, cudaStream_t st) {
    const size_t smem = track_smem(P.n_track);
    cudaError_t e = ensure_smem((const void*)cost_grad_kernel, smem);
    if (e != cudaSuccess) return e;
    cost_grad_kernel<<<(n_seq + REP_BLK - 1) / REP_BLK, REP_BLK, smem, st>>>(
        P, seg, inv, ws, n_seq, x0, V, N, w_run, w_cbf, ck, J_out, grad_out, status);
    return cudaGetLastError();
}

cudaError_t launch_repair(const DevParams& P, const float4* seg, const float* inv,
                          const RepairWs& ws, int n_seq, const float* x0, const float* V_in,
                          float* V_out, int n_iters, int mode, float delta, double* merit_out,
                          int* iters_out, const ApplyArgs& ap, unsigned* status,
                          cudaStream_t st) {
    if (n_seq <= REPAIR_BLOCK_MAX_SEQ) {
        const int inv_pad = (P.n_track + 3) & ~3;
        const size_t smem = (size_t)P.n_track * 16 + (size_t)inv_pad * 4 + (size_t)P.T * 16 +
                            (size_t)(P.T + 2) * NFIELD * 4;
        cudaError_t e = ensure_smem((const void*)repair_block_kernel, smem);
        if (e != cudaSuccess) return e;
        repair_block_kernel<<<n_seq, REPB_BLK, smem, st>>>(P, seg, inv, inv_pad, x0, V_in, V_out,
                                                           n_iters, mode, delta, ws.ck, merit_out,
                                                           iters_out, ap, status);
        return cudaGetLastError();
    }
    const size_t smem = track_smem(P.n_track);
    cudaError_t e = ensure_smem((const void*)repair_kernel, smem);
    if (e != cudaSuccess) return e;
    repair_kernel<<<(n_seq + REP_BLK - 1) / REP_BLK, REP_BLK, smem, st>>>(
        P, seg, inv, ws, n_seq, x0, V_in, V_out, n_iters, mode, delta, merit_out, iters_out, ap,
        status);
    return cudaGetLastError();
}

cudaError_t launch_apply(const DevParams& P, const ApplyArgs& ap, const float* V_exec,
                         cudaStream_t st) {
    apply_kernel<<<1, 1, 0, st>>>(P, ap, V_exec);
    return cudaGetLastError();
}

}  // namespace smppi
