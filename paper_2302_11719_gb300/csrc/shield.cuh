// Safety-shield building blocks shared by the repair kernels and the batched
// persistent kernel: the deterministic rollout cost of Eq. 22 (and of the
// running + CBF cost), its reverse-mode adjoint with checkpointing, the
// block-level repair of one sequence (Alg. 1 with Armijo backtracking) and the
// closed-loop step (Alg. 2 ExecuteCommand + warm start, Eq. 26).
#pragma once

#include "kernels.cuh"
#include <type_traits>

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
__device__ __forceinline__ void add_direct(const DevParams& P, const float4* rec,
                                           const State& x, int s, bool act_prev, bool act_next,
                                           float w_run, float w_cbf, State& lam) {
    const float2 r = rec_offset(rec, s, x.X, x.Y);
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
// Returns J in float64 and, when STORE (and the tape has a base), fills the tape
// (every state when ck <= 0, else every ck-th).  dec_out (optional) = sum_t G_t . (Vw_t - u'_t)
// where u'_t = clip(Vw_t - step Dn_t) (the Armijo decrease term), Dn = G when
// no search direction is given (the gradient step).  The terms are
// summed in float32 over blocks of 16 steps and the block sums in float64
// (FP64 arithmetic is slow on this part; one FP64 add per 16 steps).
//
// The loop is software-pipelined like rollout_sample: in iteration t the
// dynamics x_t -> x_{t+1} are issued together with the track projection, cost
// and tape entry of x_t, which they do not depend on.
template <bool STORE, bool TRIAL, bool FAST = false>
__device__ double forward_cost(const DevParams& P, const float4* rec,
                               const State& x0, int s0, int N, const float2* Vw, const float2* G,
                               float step, int ms, int seq, float w_run, float w_cbf, int ck,
                               const Tape& tape, double* dec_out, const float2* Dn = nullptr) {
    State x = x0;
    int s = s0;
    float d2 = rec_d2_seg(rec, s, x.X, x.Y);
    float h_prev = P.w2 - d2, h_pp = h_prev;
    double J = (double)(w_run * run_cost(P, x.vx, d2));
    double dec = 0.0;
    float Jf = 0.0f, decf = 0.0f;
    const float wc = w_cbf * P.C_cbf;
    const bool full = ck <= 0;
    if (STORE && N > 0 && tape.base) tape.put(0, x, s, h_prev, h_pp);
    auto control = [&](int t) {
        const float2 v = Vw[(size_t)t * ms + seq];
        if (TRIAL) {
            const float2 g = G[(size_t)t * ms + seq];
            const float2 dn = Dn ? Dn[(size_t)t * ms + seq] : g;
            const float2 u = clamp2(P, make_float2(fmaf(-step, dn.x, v.x), fmaf(-step, dn.y, v.y)));
            decf = fmaf(g.x, v.x - u.x, fmaf(g.y, v.y - u.y, decf));
            return u;
        }
        return clamp2(P, v);
    };
    // cost of state x_t (its predecessor's h is h_prev) and its tape entry
    auto settle = [&](const State& xs, int t) {
        bool nofb = false;
        s = walk_rec<false>(rec, P.n_track, s, xs.X, xs.Y, d2, nofb);
        const float h = P.w2 - d2;
        const float q = run_cost(P, xs.vx, d2);
        Jf = (w_run != 0.0f) ? fmaf(w_run, q, Jf) : Jf;
        const float a = cbf_arg(P, h_prev, h);
        Jf = (a > 0.0f) ? fmaf(wc, a, Jf) : Jf;
        h_pp = h_prev;
        h_prev = h;
        if (STORE && tape.base && (full ? true : (t % ck == 0)) && (t < N || full))
            tape.put(full ? t : t / ck, xs, s, h_prev, h_pp);
        if ((t & 15) == 0) {
            J += (double)Jf;
            dec += (double)decf;
            Jf = 0.0f;
            decf = 0.0f;
        }
    };
    if (N > 0) {
        const float2 u0 = control(0);
        model_step<FAST>(P, x, u0.x, u0.y);
    }
    for (int t = 1; t < N; ++t) {
        const float2 u = control(t);
        State xn = x;
        model_step<FAST>(P, xn, u.x, u.y);
        settle(x, t);
        x = xn;
    }
    if (N > 0) settle(x, N);
    J += (double)Jf;
    dec += (double)decf;
    if (dec_out) *dec_out = dec;
    return J;
}

// ---------------------------------------------------------------------------
// Merit of Vw (forward_cost with w_run = 0, w_cbf = 1, no tape: the DCBF
// violation sum of Eq. 22) split across warps of the block so that the
// serial chains run side by side: the model recurrence on one thread and the
// track walk with the DCBF terms on a whole warp that follows the published
// positions.  Arithmetic and summation order are those of forward_cost.
// Progress is published every MERIT_PUB steps; every wait is bounded (past
// the limit: SMPPI_DEV_TIMEOUT and the merit is reported as 0).
// ---------------------------------------------------------------------------
constexpr int MERIT_PUB = 8;
constexpr int MERIT_WAIT_LIMIT = 1 << 24;

// Bounded spin of one thread on a shared-memory counter that another warp of
// the block advances: true once *flag >= target, false after MERIT_WAIT_LIMIT
// tries (about a quarter of a second), when the caller records
// SMPPI_DEV_TIMEOUT and goes on without the value.
__device__ __forceinline__ bool spin_until_geq(const volatile int* flag, int target) {
    int tries = 0;
    while (*flag < target && tries <= MERIT_WAIT_LIMIT) ++tries;
    return tries <= MERIT_WAIT_LIMIT;
}

// The trajectory a merit pass leaves for the block gradient (shared memory; a
// null member stores nothing): ang[t] = (psi, cos psi, sin psi) of x_{t+1},
// t = 0..N-1; sg[t] and hh[t] = the tracked segment and h = w^2 - e_y^2 of x_t,
// t = 0..N.
struct MeritTraj {
    float4* ang = nullptr;
    int* sg = nullptr;
    float* hh = nullptr;
};

// The follower warp: positions pos[t - 1] = (X, Y) of x_t, t = 1..N, ready when
// *prog >= t (published in chunks of MERIT_PUB).  For a chunk, lane l holds the
// segment s - 1 + l of the window around the segment s where the chunk starts
// and evaluates its squared distance to every position of the chunk.  For each
// position every lane then forms its walk map: where the descent walk that
// starts at lane l ends (forward to the first lane above l whose successor is
// not strictly closer; at l when l + 1 is not closer and l - 1 is not closer
// either; -1 for a backward step or a walk that reaches the window's last
// lane).  The walk of the chunk is the composition of its positions' maps,
// formed by a doubling scan (three rounds of shuffles for eight positions), so
// the end lane of every position is known after three shuffle latencies
// rather than after a chain of eight decodes.  From the first position whose
// walk leaves the window, lane 0 finishes one segment at a time (walk_seq_rec)
// for that position and the rest of the chunk.
// The DCBF terms are summed as forward_cost sums them: float32 over blocks of
// 16 steps, then each block's sum added to a float64 total in order.  With
// chunks of 8 starting at t = 1 a block ends only at a chunk's last position,
// so the float64 add runs once per block, after that chunk.
// With sg / hh (MeritTraj) lane 0 also stores each position's segment and h.
// Returns J on every lane.
__device__ __forceinline__ double merit_follow_warp(const DevParams& P, const float4* rec,
                                                    const State& x0, int s0, int N,
                                                    const float2* pos, volatile int* prog,
                                                    unsigned* status, int* sg = nullptr,
                                                    float* hh = nullptr) {
    static_assert(MERIT_PUB == 8, "the float64 adds assume chunks of 8 steps starting at t = 1");
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, n = P.n_track;
    int s = s0;
    float d2 = rec_d2_seg(rec, s, x0.X, x0.Y);
    float h_prev = P.w2 - d2;
    double J = (double)(0.0f * run_cost(P, x0.vx, d2));
    float Jf = 0.0f;
    bool timed_out = false;
    if (sg && lane == 0) {
        sg[0] = s0;
        hh[0] = h_prev;
    }
    for (int t0 = 1; t0 <= N; t0 += MERIT_PUB) {
        const int t1 = min(N, t0 + MERIT_PUB - 1), nq = t1 - t0 + 1;
        const bool ok = spin_until_geq(prog, t1);
        if (__any_sync(FULL, !ok)) {   // warp-uniform
            if (lane == 0) atomicOr(status, SMPPI_DEV_TIMEOUT);
            timed_out = true;
            break;
        }
        __threadfence_block();
        int j = s - 1 + lane;
        if (j < 0) j += n;
        while (j >= n) j -= n;
        // this lane's segment j (first half of record j + 1), loaded once per chunk
        const float4 nA = rec[3 * (j + 1)], nD = rec[3 * (j + 1) + 1], Dn = rec[3 * (j + 1) + 2];
        float dq[MERIT_PUB];
        int M[MERIT_PUB];
        int jq[MERIT_PUB];     // end lane and h of each position (stored when sg is given)
        float hq[MERIT_PUB];
#pragma unroll
        for (int q = 0; q < MERIT_PUB; ++q) {
            const float2 xy = pos[t0 - 1 + min(q, nq - 1)];
            const float ex = xy.x + nA.x, ey = xy.y + nA.z;   // rec_d2_seg's arithmetic
            const float tt = __saturatef(fmaf(ex, Dn.x, ey * Dn.z));
            const float rx = fmaf(tt, nD.x, ex), ry = fmaf(tt, nD.z, ey);
            dq[q] = fmaf(rx, rx, ry * ry);
            const float dn = __shfl_down_sync(FULL, dq[q], 1);
            const float dp = __shfl_up_sync(FULL, dq[q], 1);
            const bool fwd = lane < 31 && dn < dq[q];            // d(l + 1) < d(l)
            const unsigned fw = __ballot_sync(FULL, fwd);
            const int Lf = __ffs(~fw & ~((2u << lane) - 1u)) - 1;
            const bool back = lane == 0 || dp < dq[q];           // d(l - 1) < d(l) or unknown
            M[q] = fwd ? ((Lf < 0 || Lf >= 31) ? -1 : Lf) : (back ? -1 : lane);
        }
        // M[q] <- the walk over positions 0..q from this lane (-1 once it leaves);
        // q descending so that M[q - k] is still the previous round's
#pragma unroll
        for (int k = 1; k < MERIT_PUB; k <<= 1) {
#pragma unroll
            for (int q = MERIT_PUB - 1; q >= k; --q) {
                const int src = M[q - k];
                const int v = __shfl_sync(FULL, M[q], src & 31);
                M[q] = src < 0 ? -1 : v;
            }
        }
        // the walks start at lane 1 (segment s); qs = the first position that leaves
        // the window; each kept position's DCBF term of Eq. 17 in order (C max(a, 0)
        // equals forward_cost's conditional term exactly)
        int L = 1, qs = nq;
#pragma unroll
        for (int q = 0; q < MERIT_PUB; ++q) {
            const int Lq = __shfl_sync(FULL, M[q], 1);
            const float dd = __shfl_sync(FULL, dq[q], Lq & 31);
            const bool go = q < qs && Lq >= 0;
            qs = (q < qs && Lq < 0) ? q : qs;
            L = go ? Lq : L;
            const float h = P.w2 - dd;
            const float a = cbf_arg(P, h_prev, h);
            Jf = go ? fmaf(P.C_cbf, fmaxf(a, 0.0f), Jf) : Jf;
            h_prev = go ? h : h_prev;
            jq[q] = Lq;
            hq[q] = h;
        }
        if (sg && lane == 0) {   // unrolled: jq and hq stay in registers
#pragma unroll
            for (int q = 0; q < MERIT_PUB; ++q) {
                if (q < qs) {
                    int sq = s - 1 + jq[q];
                    if (sq < 0) sq += n;
                    while (sq >= n) sq -= n;
                    sg[t0 + q] = sq;
                    hh[t0 + q] = hq[q];
                }
            }
        }
        int scur = s - 1 + L;
        if (scur < 0) scur += n;
        while (scur >= n) scur -= n;
        // from qs on: lane 0 walks one segment at a time (rare)
#pragma unroll 1
        for (int q = qs; q < nq; ++q) {
            const float2 p = pos[t0 - 1 + q];
            int sr = 0;
            float dr = 0.0f;
            if (lane == 0) sr = walk_seq_rec(rec, n, scur, p.x, p.y, dr);
            scur = __shfl_sync(FULL, sr, 0);
            const float h = P.w2 - __shfl_sync(FULL, dr, 0);
            const float a = cbf_arg(P, h_prev, h);
            Jf = fmaf(P.C_cbf, fmaxf(a, 0.0f), Jf);
            h_prev = h;
            if (sg && lane == 0) {
                sg[t0 + q] = scur;
                hh[t0 + q] = h;
            }
        }
        s = scur;
        if (nq == MERIT_PUB && ((t1 & 15) == 0)) {   // a block of 16 steps ends here
            J += (double)Jf;
            Jf = 0.0f;
        }
    }
    J += (double)Jf;
    return timed_out ? 0.0 : J;
}

// Two warps: thread 0 integrates the model (any parameters); warp 1 follows.
// BLK >= 64; buf holds 8 N bytes.  side(lane) runs on warp 2 meanwhile (BLK >= 96).
template <bool FAST, class Side>
__device__ __forceinline__ void merit_split(const DevParams& P, const float4* rec,
                                            const State& x0, int s0, int N, const float2* Vw,
                                            float* buf, volatile int* prog, double* out,
                                            volatile int* done, unsigned* status,
                                            const Side& side) {
    const int tid = threadIdx.x;
    float2* pos = reinterpret_cast<float2*>(buf);            // (X, Y) of x_{t+1}
    if (tid == 0) {
        *prog = 0;
        *done = 0;
    }
    __syncthreads();
    if (tid == 0) {
        State x = x0;
        for (int t = 0; t < N; ++t) {
            const float2 u = clamp2(P, Vw[t]);
            model_step<FAST>(P, x, u.x, u.y);
            pos[t] = make_float2(x.X, x.Y);
            if ((t + 1) % MERIT_PUB == 0 || t + 1 == N) {
                __threadfence_block();
                *prog = t + 1;
            }
        }
    } else if ((tid >> 5) == 1) {
        const double J = merit_follow_warp(P, rec, x0, s0, N, pos, prog, status);
        if (tid == 32) {
            *out = J;
            __threadfence_block();
            *done = 1;
        }
    } else if ((tid >> 5) == 2) {
        side(tid & 31);
    }
    __syncwarp();
}

// The merit pass's rows in its buffer (only 8-byte aligned in some callers:
// rounded up to 16 bytes for the float4 rows; the tape scratch has
// 44 (T + 2) >= 44 N + 15 bytes): ctl[t] = (Bd, kx, ky, kr) and bx[t] of step t,
// vel[t] = (v_x, v_y, r) of x_t, pos[t] = (X, Y) of x_{t+1}.
struct MeritRows {
    float4* ctl;
    float4* vel;
    float2* pos;
    float* bx;
};

__device__ __forceinline__ MeritRows merit_rows(float* buf, int N) {
    MeritRows m;
    m.ctl = reinterpret_cast<float4*>((reinterpret_cast<uintptr_t>(buf) + 15) & ~uintptr_t(15));
    m.vel = m.ctl + N;
    m.pos = reinterpret_cast<float2*>(m.vel + N);
    m.bx = reinterpret_cast<float*>(m.pos + N);
    return m;
}

// Three warps for the C = 1.5 model: thread 0 runs the velocity recurrence
// (tyre forces; the control factors of every step, vel_coef, are precomputed
// by the whole block), thread 32 the pose recurrence from the published
// velocities, warp 2 the track walk from the published positions.
// BLK >= 96; buf holds 44 N + 15 bytes (merit_rows); prog two counters.  tr:
// the trajectory kept for the block gradient (members may be null).
// side(lane) runs on warp 3 meanwhile (BLK >= 128).
template <class Side>
__device__ __forceinline__ void merit_split3(const DevParams& P, const float4* rec,
                                             const State& x0, int s0, int N, const float2* Vw,
                                             float* buf, volatile int* prog, double* out,
                                             volatile int* done, unsigned* status,
                                             const MeritTraj& tr, const Side& side) {
    const int tid = threadIdx.x;
    const MeritRows mr = merit_rows(buf, N);
    float4* ctl = mr.ctl;
    float4* vel = mr.vel;
    float2* pos = mr.pos;
    float* bx = mr.bx;
    if (tid == 0) {
        prog[0] = 0;
        prog[1] = 0;
        *done = 0;
    }
    for (int t = tid; t < N; t += blockDim.x) {
        const float2 u = clamp2(P, Vw[t]);
        float sd, cd;
        sincos_half(u.x, &sd, &cd);
        const VelCoef k = vel_coef(P, u.x, sd, cd, u.y);
        ctl[t] = make_float4(k.Bd, k.kx, k.ky, k.kr);
        bx[t] = k.bx;
    }
    __syncthreads();
    if (tid == 0) {
        float vx = x0.vx, vy = x0.vy, r = x0.r;
        for (int t = 0; t < N; ++t) {
            vel[t] = make_float4(vx, vy, r, 0.0f);
            if ((t + 1) % MERIT_PUB == 0 || t + 1 == N) {
                __threadfence_block();
                prog[0] = t + 1;
            }
            const float4 c = ctl[t];
            vel_step_fast(P, vx, vy, r, VelCoef{c.x, c.y, c.z, c.w, bx[t]});
        }
    } else if (tid == 32) {
        float X = x0.X, Y = x0.Y, psi = x0.psi, cp = x0.cp, sp = x0.sp;
        for (int t = 0; t < N; ++t) {
            // the velocities arrive MERIT_PUB at a time: wait at the start of each chunk
            if (t % MERIT_PUB == 0) {
                if (!spin_until_geq(prog, min(N, t + MERIT_PUB))) {
                    atomicOr(status, SMPPI_DEV_TIMEOUT);
                    break;
                }
                __threadfence_block();
            }
            const float4 v = vel[t];
            pose_step_fast(P, v.x, v.y, v.z, X, Y, psi, cp, sp);
            pos[t] = make_float2(X, Y);
            if (tr.ang) tr.ang[t] = make_float4(psi, cp, sp, 0.0f);
            if ((t + 1) % MERIT_PUB == 0 || t + 1 == N) {
                __threadfence_block();
                prog[1] = t + 1;
            }
        }
    } else if ((tid >> 5) == 2) {
        const double J = merit_follow_warp(P, rec, x0, s0, N, pos, prog + 1, status, tr.sg,
                                           tr.hh);
        if (tid == 64) {
            *out = J;
            __threadfence_block();
            *done = 1;
        }
    } else if ((tid >> 5) == 3) {
        side(tid & 31);
    }
    __syncwarp();
}

// Cost and gradient of one sequence (forward with tape + backward adjoint).
// Writes G_t = dJ/dv_t for t < N (0 for N <= t < T).
template <bool FAST = false>
__device__ double seq_cost_grad(const DevParams& P, const float4* rec,
                                const State& x0, int s0, int N, int T, const float2* Vw, float2* G,
                                int ms, int seq, float w_run, float w_cbf, int ck,
                                const Tape& tape) {
    const double J = forward_cost<true, false, FAST>(P, rec, x0, s0, N, Vw, nullptr, 0.0f, ms, seq,
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
                model_step<FAST>(P, x, u.x, u.y);
                float d2;
                bool nofb = false;
                s = walk_rec<false>(rec, P.n_track, s, x.X, x.Y, d2, nofb);
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
            add_direct(P, rec, x, s, cbf_arg(P, hp, h) > 0.0f, false, w_run, w_cbf, lam);
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
                add_direct(P, rec, x, s, cbf_arg(P, hp, h) > 0.0f,
                           cbf_arg(P, h, h_next) > 0.0f, w_run, w_cbf, lam);
        }
    }
    return J;
}

// Shared-memory workspace of the block gradient: the trajectory a merit pass
// keeps (MeritTraj) and five float4 of adjoint coefficients per step.
struct GradWs {
    MeritTraj tr;
    float4* coef;
    float2* vt;     // [T] the controls of the line search's first trial
};

// Bytes of a GradWs for horizon T (with 16 bytes for alignment), and its
// carving from the memory at p.
__host__ __device__ constexpr size_t grad_ws_bytes(int T) {
    return (size_t)T * 16 + (size_t)T * 80 + (size_t)(T + 1) * 8 + (size_t)T * 8 + 16;
}

__device__ __forceinline__ GradWs grad_ws_at(unsigned char* p, int T) {
    GradWs g;
    g.tr.ang = reinterpret_cast<float4*>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
    g.coef = g.tr.ang + T;
    g.tr.sg = reinterpret_cast<int*>(g.coef + 5 * T);
    g.tr.hh = reinterpret_cast<float*>(g.tr.sg + T + 1);
    g.vt = reinterpret_cast<float2*>(g.tr.hh + T + 1);
    return g;
}

// Where the penalty part of step t >= 1 reads its inputs: h_{t-1}, h_t, h_{t+1}
// and the tracked segment of x_t.
struct PenIn {
    float hm, h, hn;
    int sg;
};

// Coefficients of the adjoint map of step t (5 float4; block_cost_grad states
// the map) at the state x_t: velocity (vx, vy, r), position (X, Y), heading
// (cp, sp) = (cos psi, sin psi); v the control of step t; for t >= 1 the
// penalty part from pen() (a PenIn; the segment is clamped to the track: a
// merit pass whose wait gave up leaves it unset, and the TIMEOUT bit reports
// that case).
template <class Pen>
__device__ __forceinline__ void cart_grad_coef(const DevParams& P, const float4* rec, int t,
                                               float vx, float vy, float r, float X, float Y,
                                               float cp, float sp, float2 v, const Pen& pen,
                                               float4* c) {
    const float dt = P.dt, wc = P.C_cbf;
    const float d = clampf(v.x, P.umin0, P.umax0);
    const float yf = fmaf(P.lf, r, vy), yr = fmaf(-P.lr, r, vy);
    const float bf = atan2_poly(yf, vx), br = atan2_poly(yr, vx);
    float dphf, dphr;
    const float Fyf = P.Fzf * tyre_shape(P, P.B * (d - bf), &dphf);
    tyre_shape(P, P.B * (-br), &dphr);
    float sd, cd;
    if (P.steer_small) sincos_half(d, &sd, &cd);
    else sincosf(d, &sd, &cd);
    const float dX = vx * cp - vy * sp, dY = vx * sp + vy * cp;
    // lateral-force adjoints Fyf_b = a1 g_vx + a2 g_vy + a3 g_r, Fyr_b = b2 g_vy + b3 g_r;
    // through the tyres and the slip angles they reach v_x (q), v_y and r (p)
    const float kf = P.Fzf * dphf * P.B, kr = P.Fzr * dphr * P.B;
    const float nf = fmaf(vx, vx, yf * yf), nr = fmaf(vx, vx, yr * yr);
    const float pf = nf > 0.0f ? -kf * vx / nf : 0.0f, qf = nf > 0.0f ? kf * yf / nf : 0.0f;
    const float pr = nr > 0.0f ? -kr * vx / nr : 0.0f, qr = nr > 0.0f ? kr * yr / nr : 0.0f;
    const float a1 = -sd * P.m_inv, a2 = cd * P.m_inv, a3 = P.lf * cd * P.Iz_inv;
    const float b2 = P.m_inv, b3 = -P.lr * P.Iz_inv;
    const bool in0 = v.x >= P.umin0 && v.x <= P.umax0, in1 = v.y >= P.umin1 && v.y <= P.umax1;
    c[0] = make_float4(dt * (qf * a1), dt * (-r + qf * a2 + qr * b2), dt * (qf * a3 + qr * b3),
                       dt * (r + pf * a1));
    c[1] = make_float4(dt * (pf * a2 + pr * b2), dt * (pf * a3 + pr * b3),
                       dt * (vy + P.lf * pf * a1), dt * (-vx + P.lf * pf * a2 - P.lr * pr * b2));
    c[2] = make_float4(dt * (P.lf * pf * a3 - P.lr * pr * b3), dt * cp, dt * sp, dt * dX);
    c[3] = make_float4(dt * dY, in0 ? dt * (-Fyf * cd * P.m_inv + kf * a1) : 0.0f,
                       in0 ? dt * (-Fyf * sd * P.m_inv + kf * a2) : 0.0f,
                       in0 ? dt * (-P.lf * Fyf * sd * P.Iz_inv + kf * a3) : 0.0f);
    // d_t (t >= 1): the penalties of the pairs (t - 1, t) and (t, t + 1) through e_y^2
    float ddX = 0.0f, ddY = 0.0f;
    if (t > 0) {
        const PenIn q = pen();
        float ch = 0.0f;
        if (cbf_arg(P, q.hm, q.h) > 0.0f) ch -= wc;
        if (cbf_arg(P, q.h, q.hn) > 0.0f) ch += wc * P.one_m_alpha;
        const float2 ro = rec_offset(rec, min(max(q.sg, 0), P.n_track - 1), X, Y);
        ddX = -2.0f * ch * ro.x;
        ddY = -2.0f * ch * ro.y;
    }
    c[4] = make_float4(in1 ? dt * P.fx_gain * P.m_inv : 0.0f, ddX, ddY, 0.0f);
}

// The recursion of the gradient on one thread: lambda_N = d_N (the penalty of
// the last pair: hN() = (h_{N-1}, h_N), and where it is active xN() = (X, Y) of
// x_N and its segment), then G_t and lambda_t for t = N - 1 .. 0 from the
// coefficients; G_t = 0 for N <= t < T.
template <class HN, class XN>
__device__ __forceinline__ void cart_grad_recur(const DevParams& P, const float4* rec, int N,
                                                int T, const float4* coef, float2* G,
                                                const HN& hN, const XN& xN) {
    const float dt = P.dt, wc = P.C_cbf;
    float lvx = 0.0f, lvy = 0.0f, lr = 0.0f, lX = 0.0f, lY = 0.0f, lp = 0.0f;
    if (N > 0) {
        const float2 hh = hN();
        if (cbf_arg(P, hh.x, hh.y) > 0.0f) {
            const float3 p = xN();
            const float2 ro = rec_offset(rec, min(max(__float_as_int(p.z), 0), P.n_track - 1),
                                         p.x, p.y);
            lX = 2.0f * wc * ro.x;
            lY = 2.0f * wc * ro.y;
        }
    }
#pragma unroll 4
    for (int t = N - 1; t >= 0; --t) {
        const float4* c = coef + 5 * t;
        const float4 c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3], c4 = c[4];
        G[t] = make_float2(fmaf(c3.y, lvx, fmaf(c3.z, lvy, c3.w * lr)), c4.x * lvx);
        const float nvx = lvx + (fmaf(c0.x, lvx, c0.y * lvy) + fmaf(c0.z, lr, fmaf(c2.y, lX, c2.z * lY)));
        const float nvy = lvy + (fmaf(c0.w, lvx, c1.x * lvy) + fmaf(c1.y, lr, fmaf(c2.y, lY, -c2.z * lX)));
        const float nr = lr + (fmaf(c1.z, lvx, c1.w * lvy) + fmaf(c2.x, lr, dt * lp));
        const float np = lp + fmaf(c2.w, lY, -c3.x * lX);
        lX += c4.y;
        lY += c4.z;
        lvx = nvx;
        lvy = nvy;
        lr = nr;
        lp = np;
    }
    for (int t = N; t < T; ++t) G[t] = make_float2(0.0f, 0.0f);
}

// Gradient G_t = dP/dv_t of the merit P (the CBF objective of Eq. 22: running-cost
// weight 0, CBF weight 1) by the whole block, from the trajectory of Vw that the
// last merit pass left (merit_rows of buf, gw.tr).  The adjoint of the Euler
// step is linear in the adjoint: lambda_t = lambda_{t+1} + E_t' lambda_{t+1}
// + d_t and g_t = B_t' lambda_{t+1}, with E_t, B_t the derivatives of
// model_step at (x_t, u_t) scaled by dt (those of model_step_adjoint, collected
// per step) and d_t the CBF penalties' derivative at x_t (add_direct).  Every
// thread forms the coefficients of its steps; thread 0 then runs the recursion
// over (v_x, v_y, r, X, Y, psi).  Writes G_t for t < N (0 for N <= t < T).
// The stored segments are clamped to the track (a merit pass whose wait gave up
// leaves them unset; the TIMEOUT bit reports that case).
template <int BLK>
__device__ void block_cost_grad(const DevParams& P, const float4* rec, const State& x0, int N,
                                int T, const float2* Vw, float2* G, float* buf,
                                const GradWs& gw) {
    const int tid = threadIdx.x;
    const MeritRows mr = merit_rows(buf, N);
    for (int t = tid; t < N; t += BLK) {
        const float4 v4 = mr.vel[t];
        float X = x0.X, Y = x0.Y, cp = x0.cp, sp = x0.sp;
        if (t > 0) {
            const float2 p = mr.pos[t - 1];
            const float4 a = gw.tr.ang[t - 1];
            X = p.x;
            Y = p.y;
            cp = a.y;
            sp = a.z;
        }
        cart_grad_coef(P, rec, t, v4.x, v4.y, v4.z, X, Y, cp, sp, Vw[t],
                       [&]() {
                           return PenIn{gw.tr.hh[t - 1], gw.tr.hh[t], gw.tr.hh[t + 1],
                                        gw.tr.sg[t]};
                       },
                       gw.coef + 5 * t);
    }
    __syncthreads();
    if (tid == 0)
        cart_grad_recur(
            P, rec, N, T, gw.coef, G,
            [&]() { return make_float2(gw.tr.hh[N - 1], gw.tr.hh[N]); },
            [&]() {
                const float2 p = mr.pos[N - 1];
                return make_float3(p.x, p.y, __int_as_float(gw.tr.sg[N]));
            });
    __syncthreads();
}

// The same gradient by a group of NT threads (rank 0..NT-1, synchronised by
// sync()) from a full tape of the trajectory that rank 0 writes first
// (forward_cost, every state) unless have_tape says the tape already holds that
// of Vw: the warp of the BFGS solver.  coef: 5 float4 per step.
template <bool FAST, class Sync>
__device__ __forceinline__ void tape_cost_grad(const DevParams& P, const float4* rec,
                                               const State& x0, int s0, int N, int T,
                                               const float2* Vw, float2* G, const Tape& tape,
                                               float4* coef, int rank, int NT, const Sync& sync,
                                               bool have_tape = false) {
    if (rank == 0 && !have_tape)
        forward_cost<true, false, FAST>(P, rec, x0, s0, N, Vw, nullptr, 0.0f, 1, 0, 0.0f, 1.0f,
                                        0, tape, nullptr);
    sync();
    for (int t = rank; t < N; t += NT) {
        const State x = {tape.at(t, 0), tape.at(t, 1), tape.at(t, 2), tape.at(t, 3),
                         tape.at(t, 4), tape.at(t, 5), tape.at(t, 6), tape.at(t, 7)};
        cart_grad_coef(P, rec, t, x.vx, x.vy, x.r, x.X, x.Y, x.cp, x.sp, Vw[t],
                       [&]() {
                           return PenIn{tape.at(t, 10), tape.at(t, 9), tape.at(t + 1, 9),
                                        __float_as_int(tape.at(t, 8))};
                       },
                       coef + 5 * t);
    }
    sync();
    if (rank == 0)
        cart_grad_recur(
            P, rec, N, T, coef, G, [&]() { return make_float2(tape.at(N, 10), tape.at(N, 9)); },
            [&]() { return make_float3(tape.at(N, 3), tape.at(N, 4), tape.at(N, 8)); });
    sync();
}

// Closed-loop step (Alg. 2 ExecuteCommand + warm start, Eq. 26), one thread:
// x0 <- f(x0, clamp(v_exec)) + w_n, V <- shift(V).
__device__ void closed_loop_step(const DevParams& P, const ApplyArgs& ap, float2 v_exec) {
    const uint32_t nn = ap.n + (ap.iter_dev ? *ap.iter_dev : 0u);
    State x = make_state(ap.x0);
    if (P.state_kind == 1)
        model_step_curv(P, ap.kappa, x, clampf(v_exec.x, P.umin0, P.umax0),
                        clampf(v_exec.y, P.umin1, P.umax1));
    else
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


// Work that a caller of repair_in_block hands to an otherwise idle warp during
// the first merit pass (side(lane) on all lanes of that warp); NoSide: none.
struct NoSide {
    __device__ void operator()(int) const {}
};

// Shared-memory scratch of repair_in_block.
struct RepairSmem {
    double P;
    double dec;        // the Armijo decrease term of the first trial (block_grad)
    int prog[2];       // progress counters of merit_split / merit_split3
    int done;          // set by the merit follower once P is written
    float red[32];
    float step;
    int ok;
};

// Safety shield of one sequence by one block of BLK threads (Alg. 1 with
// Armijo backtracking, mode 1; fixed step, mode 0).  rec: the staged
// track; Vw [T]: the controls, repaired in place; G [T], tape_s [(T+2) NFIELD]:
// shared-memory scratch.  The Armijo trial steps s, s/2, s/4, ... are
// evaluated in parallel by the lanes of warp 0 (lane j: s 2^-j) and the
// largest accepted step is taken: the same iterate as sequential backtracking.
// The gradient comes from thread 0 (seq_cost_grad).  merit_row (optional):
// n_iters + 1 merits; *iters_done: iterations run (0: Vw is unchanged).  side:
// run by an idle warp during the first merit pass (BLK >= 128).  gw (C = 1.5
// model, BLK >= 128): the gradient is formed by the block (block_cost_grad) from
// the trajectory the merit pass keeps there, instead of by thread 0.  Returns the
// final merit.
template <int BLK, bool FAST = false, class Side = NoSide>
__device__ double repair_in_block(const DevParams& P, const float4* rec,
                                  const State& x0, int s0, float2* Vw, float2* G, float* tape_s,
                                  int n_iters, int mode, float delta, int ck, double* merit_row,
                                  int* iters_done, unsigned* status, RepairSmem& sm,
                                  const Side& side = Side(), const GradWs* gw = nullptr) {
    static_assert(BLK >= 128 || std::is_same<Side, NoSide>::value, "side work needs a fourth warp");
    const int T = P.T, N = P.N_r;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = BLK / 32;
    const Tape tape{tape_s, 1, 0};
    // every thread waits (bounded) for the follower's completion flag before it
    // reads the merit, so that the branch on P below is taken by the whole block
    // the first merit pass keeps no trajectory (most updates need no repair and
    // keeping it costs that pass about 2 us); a repair's gradient first runs a
    // pass that keeps it
    const bool block_grad = FAST && BLK >= 128 && gw != nullptr;
    bool traj_ok = false;   // the kept trajectory is that of the current Vw
    auto merit = [&](const auto& sd, bool keep, const float2* ctrl) {
        if (FAST && BLK >= 96)
            merit_split3(P, rec, x0, s0, N, ctrl, tape_s, sm.prog, &sm.P, &sm.done, status,
                         (block_grad && keep) ? gw->tr : MeritTraj{}, sd);
        else
            merit_split<FAST>(P, rec, x0, s0, N, ctrl, tape_s, sm.prog, &sm.P, &sm.done, status,
                              sd);
        __syncthreads();
        if (!spin_until_geq(&sm.done, 1) && tid == 0) atomicOr(status, SMPPI_DEV_TIMEOUT);
        __threadfence_block();
        __syncthreads();
    };
    merit(side, false, Vw);
    double P0 = sm.P;
    int it = 0;
    bool stalled = false;
    for (; it < n_iters; ++it) {
        if (tid == 0 && merit_row) merit_row[it] = P0;
        if (P0 == 0.0) break;
        if (block_grad) {
            if (!traj_ok) merit(NoSide(), true, Vw);   // keeps the trajectory of the current iterate
            traj_ok = true;
            block_cost_grad<BLK>(P, rec, x0, N, T, Vw, G, tape_s, *gw);
        } else {
            if (tid == 0)
                seq_cost_grad<FAST>(P, rec, x0, s0, N, T, Vw, G, 1, 0, 0.0f, 1.0f, ck, tape);
            __syncthreads();
        }
        if (mode == 0) {
            for (int t = tid; t < N; t += BLK)
                Vw[t] = clamp2(P, make_float2(fmaf(-delta, G[t].x, Vw[t].x),
                                              fmaf(-delta, G[t].y, Vw[t].y)));
            __syncthreads();
            merit(NoSide(), true, Vw);
            P0 = sm.P;
            continue;
        }
        // |g|_inf
        float gm = 0.0f;
        for (int t = tid; t < N; t += BLK) gm = fmaxf(gm, fmaxf(fabsf(G[t].x), fabsf(G[t].y)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
        if (lane == 0) sm.red[warp] = gm;
        __syncthreads();
        gm = sm.red[0];
#pragma unroll
        for (int w = 1; w < NW; ++w) gm = fmaxf(gm, sm.red[w]);
        if (!(gm > 0.0f)) { stalled = true; break; }
        const float s_first = P.ls_s0 / gm;
        int j0 = 0;   // the first trial the lanes evaluate
        if (block_grad && P.ls_max > 0) {
            // the full step s_first (accepted in about two of three iterations) by the
            // three-warp merit pass on the trial controls, whose kept trajectory then
            // serves the next gradient; only when it is rejected do the lanes try the
            // shorter steps (the same iterate as sequential backtracking)
            float2* Vt = gw->vt;
            float dpart = 0.0f;
            for (int t = tid; t < N; t += BLK) {
                const float2 v = Vw[t], g = G[t];
                const float2 u = clamp2(P, make_float2(fmaf(-s_first, g.x, v.x),
                                                       fmaf(-s_first, g.y, v.y)));
                Vt[t] = u;
                dpart = fmaf(g.x, v.x - u.x, fmaf(g.y, v.y - u.y, dpart));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dpart += __shfl_xor_sync(0xffffffffu, dpart, o);
            __syncthreads();   // every thread has read sm.red for |g|_inf
            if (lane == 0) sm.red[warp] = dpart;
            __syncthreads();
            if (tid == 0) {
                double dec = 0.0;
                for (int w = 0; w < NW; ++w) dec += (double)sm.red[w];
                sm.dec = dec;
            }
            merit(NoSide(), true, Vt);
            const double Pt = sm.P;
            if (Pt <= P0 - (double)P.ls_c * sm.dec) {
                for (int t = tid; t < N; t += BLK) Vw[t] = Vt[t];
                __syncthreads();
                P0 = Pt;
                traj_ok = true;
                continue;
            }
            traj_ok = false;
            j0 = 1;
        }
        if (warp == 0) {
            // lane j tries s_first 2^-j (j = j0 + lane, j0 + lane + 32, ...); keep the
            // smallest accepted j
            int best = 0x7fffffff;
            double best_P = 0.0;
            for (int j = j0 + lane; j < P.ls_max; j += 32) {
                const float sj = ldexpf(s_first, -j);
                double dec;
                const double Pt = forward_cost<false, true, FAST>(P, rec, x0, s0, N, Vw, G, sj, 1,
                                                            0, 0.0f, 1.0f, 0, tape, &dec);
                if (Pt <= P0 - (double)P.ls_c * dec && j < best) { best = j; best_P = Pt; }
            }
            int bj = best;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bj = min(bj, __shfl_xor_sync(0xffffffffu, bj, o));
            if (best == bj && bj != 0x7fffffff) {   // the owning lane publishes
                sm.P = best_P;
                sm.step = ldexpf(s_first, -bj);
            }
            if (lane == 0) sm.ok = (bj != 0x7fffffff);
        }
        __syncthreads();
        if (!sm.ok) { stalled = true; break; }
        const float sa = sm.step;
        for (int t = tid; t < N; t += BLK)
            Vw[t] = clamp2(P, make_float2(fmaf(-sa, G[t].x, Vw[t].x), fmaf(-sa, G[t].y, Vw[t].y)));
        __syncthreads();
        P0 = sm.P;
        traj_ok = false;
    }
    if (tid == 0) {
        if (merit_row)
            for (int i = it; i <= n_iters; ++i) merit_row[i] = P0;
        if (iters_done) *iters_done = it;
        if (stalled) atomicOr(status, SMPPI_DEV_STALLED);
        if (!isfinite(P0)) atomicOr(status, SMPPI_DEV_NUMERIC);
    }
    __syncthreads();
    return P0;
}

// Nearest segment of (X, Y) over the whole track by one block (lowest index on
// ties); every thread gets the result (segment 0 and the NUMERIC bit when no
// distance is finite, seg_or_zero).
template <int BLK>
__device__ int block_nearest_segment(const float4* rec, int n, float X, float Y,
                                     float* red_f, int* red_i, float* d2_out, unsigned* status) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float bd = 3.0e38f;
    int bi = 0x7fffffff;
    for (int i = tid; i < n; i += BLK) {
        const float d = rec_d2_seg(rec, i, X, Y);
        if (d < bd) { bd = d; bi = i; }
    }
    warp_argmin(bd, bi);
    if (lane == 0) { red_f[warp] = bd; red_i[warp] = bi; }
    __syncthreads();
    bd = red_f[0];
    bi = red_i[0];
    for (int w = 1; w < BLK / 32; ++w)
        if (red_f[w] < bd || (red_f[w] == bd && red_i[w] < bi)) { bd = red_f[w]; bi = red_i[w]; }
    __syncthreads();
    const int s0 = seg_or_zero(bi, n, tid == 0 ? status : nullptr);
    if (d2_out) *d2_out = (s0 == bi) ? bd : rec_d2_seg(rec, s0, X, Y);
    return s0;
}

}  // namespace
}  // namespace smppi
