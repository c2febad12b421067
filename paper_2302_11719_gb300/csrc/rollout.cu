// MPPI iteration kernels (Alg. 2 sampling loop + OptimalControl; Eq. 10-12,
// 17-20): K sampled rollouts with the DCBF-augmented cost, then the min-
// shifted softmin weights and the weighted noise sum.
//
// Launch 1 (rollouts): grid = ceil(K / BLK), one thread per rollout.  Shared
//   memory holds the centreline segment table and the nominal sequence V.  Each
//   thread steps its rollout in registers; the noise of the next pair of steps
//   is drawn from Philox while the current pair is integrated (never stored).
//   Writes S_k and the block minimum of S.  For C = 1.5 and |steer| <= 1/2 the
//   packed kernel runs instead: one thread steps two rollouts (k, k + BLK of
//   its block) with FFMA2 / FADD2 / FMUL2 and reads the segment-pair table.
// Launch 2 (update): G <= #SMs blocks of UPD_BLK threads.  Every block takes
//   m = min_k S_k from the block minima, computes omega_k = exp(-(S_k - m)/lambda)
//   for its contiguous slice of k (all of them enter eta), and regenerates the
//   noise only of rollouts with omega_k > w_skip = 1e-8 / (K max|eps|): the
//   dropped terms change V+ by at most K w_skip max|eps| / eta <= 1e-8 (eta >= 1
//   because the arg-min has weight 1).  With lambda = 1 and the cost spread of
//   these problems that leaves a small fraction of K.  The last block to
//   finish (device-scope ticket) sums the non-empty block partials in float64
//   and writes V+ = clamp(V + A / eta).
#include <atomic>

#include "rollout2.cuh"
#include "shield.cuh"

namespace smppi {

namespace {

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

}  // namespace

// Stage the segment-pair table (one bulk copy, bounded wait), V and the
// nearest segment of x0 (block argmin, lowest index on ties).  Returns false
// (status set, copy drained) if the copy did not complete.
template <int BLK>
__device__ __forceinline__ bool stage_problem(const DevParams& P, const float4* __restrict__ recg,
                                              const float* __restrict__ Vg,
                                              const float* __restrict__ x0g,
                                              float4* rec, float4* Vs, uint64_t* bar, int* s_flag,
                                              int* s_seg0, float* s_d20, float* red_f,
                                              int* red_i, unsigned* status) {
    const int tid = threadIdx.x, n = P.n_track;
    griddep_launch_dependents();
    griddep_wait();
    if (tid == 0) {
        *s_flag = 0;
        mbar_init(bar, 1);
        const uint32_t bytes = (uint32_t)rec_table_bytes(n);
        mbar_expect_tx(bar, bytes);
        bulk_g2s(rec, recg, bytes, bar);
    }
    for (int t = tid; t < P.T; t += BLK) {
        const float2 v = reinterpret_cast<const float2*>(Vg)[t];
        Vs[t] = make_float4(v.x, v.y, P.gis0 * v.x, P.gis1 * v.y);   // (v, gamma Sigma^-1 v)
    }
    __syncthreads();
    if (!mbar_wait_bounded(bar, 0u)) *s_flag = 1;
    __syncthreads();
    if (*s_flag) {
        if (tid == 0) {
            atomicOr(status, SMPPI_DEV_TIMEOUT);
            mbar_wait_bounded(bar, 0u);   // let the copy in flight land before the block exits
        }
        return false;
    }
    const float X0 = x0g[3], Y0 = x0g[4];
    float bd = 3.0e38f;
    int bi = 0x7fffffff;
    for (int i = tid; i < n; i += BLK) {
        const float d = rec_d2_seg(rec, i, X0, Y0);
        if (d < bd) { bd = d; bi = i; }
    }
    warp_argmin(bd, bi);
    const int warp = tid >> 5, lane = tid & 31;
    if (lane == 0) { red_f[warp] = bd; red_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < BLK / 32; ++w)
            if (red_f[w] < bd || (red_f[w] == bd && red_i[w] < bi)) { bd = red_f[w]; bi = red_i[w]; }
        const int s0 = seg_or_zero(bi, n, status);
        *s_seg0 = s0;
        *s_d20 = (s0 == bi) ? bd : rec_d2_seg(rec, s0, X0, Y0);
    }
    __syncthreads();
    return true;
}

// Launch 1: one thread per rollout.  FAST: model parameters of the
// branch-free model step (see model_step).
template <int BLK, bool DUMP, bool FAST>
__global__ void __launch_bounds__(BLK) mppi_rollout_kernel(
    DevParams P, const float* __restrict__ x0g, const float* __restrict__ Vg,
    const float4* __restrict__ recg, uint32_t iter, uint32_t ctr3,
    const uint32_t* __restrict__ iter_dev, float* __restrict__ S_out, float* __restrict__ traj,
    float* __restrict__ blk_min, int* __restrict__ seg0_out, unsigned* __restrict__ status,
    uint32_t k_off) {
    constexpr int NW = BLK / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = P.T;
    float4* rec = reinterpret_cast<float4*>(smem_raw);
    float4* Vs = rec + 3 * (P.n_track + 5);
    __shared__ __align__(8) uint64_t bar;
    __shared__ float red_f[NW];
    __shared__ int red_i[NW];
    __shared__ int s_seg0, s_flag;
    __shared__ float s_d20;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = blockIdx.x * BLK + tid;
    const bool active = k < P.K;

    if (!stage_problem<BLK>(P, recg, Vg, x0g, rec, Vs, &bar, &s_flag, &s_seg0, &s_d20,
                            red_f, red_i, status))
        return;
    if (iter_dev) iter += *iter_dev;
    if (blockIdx.x == 0 && tid == 0 && seg0_out) *seg0_out = s_seg0;
    float S = 3.0e38f;
    if (active) {
        S = rollout_sample<FAST, DUMP>(P, rec, Vs, make_state(x0g), s_seg0, s_d20,
                                       (uint32_t)k + k_off, iter, ctr3,
                                       DUMP ? traj + (size_t)k * (T + 1) * 6 : nullptr);
        S_out[k] = S;
        if (!isfinite(S)) atomicOr(status, SMPPI_DEV_NUMERIC);
    }
    const float m = warp_min(active ? S : 3.0e38f);
    if (lane == 0) red_f[warp] = m;
    __syncthreads();
    if (tid == 0) {
        float mb = red_f[0];
#pragma unroll
        for (int w = 1; w < NW; ++w) mb = fminf(mb, red_f[w]);
        blk_min[blockIdx.x] = mb;
    }
}

// Partial of one rollout block (Eq. 10-11 over its rollouts, min-shifted by its
// own minimum m_b; the merge rescales it by exp(-(m_b - m)/lambda)):
// part_eta = sum_k exp(-(S_k - m_b)/lambda) and part_acc[2t + j] = the same
// weights times eps_{k,t,j}, summed over the rollouts whose weight exceeds
// w_skip, with the noise regenerated.  The taken rollouts are listed in thread
// order (rollout a, then b, of each thread); thread (slot c, pair p)
// accumulates list items c, c + C, ... for pair p and the slots are added in
// slot order: a fixed summation order.  smem: l_k, l_w [2 BLK], acc_s [2T].
template <int BLK>
__device__ __forceinline__ void block_partial(const DevParams& P, float m_b, float2 S, bool act_a,
                                              bool act_b, uint32_t ka, uint32_t kb, uint32_t iter,
                                              uint32_t ctr3, int* l_k, float* l_w, float* acc_s,
                                              float* red, int* w_cnt, float* part_acc,
                                              double* part_eta, int* part_has) {
    constexpr int NW = BLK / 32;
    constexpr int PP = (SMPPI_MAX_T / 2 + BLK - 1) / BLK;   // pairs per thread at most
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = P.T, T2 = 2 * T, npair = (T + 1) >> 1;
    const float wa = act_a ? expf((m_b - S.x) * P.lam_inv) : 0.0f;
    const float wb = act_b ? expf((m_b - S.y) * P.lam_inv) : 0.0f;
    const bool ta = wa > P.w_skip, tb = wb > P.w_skip;
    const int ntake = (int)ta + (int)tb;
    int incl = ntake;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    float e = wa + wb;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 31) w_cnt[warp] = incl;
    if (lane == 0) red[warp] = e;
    for (int j = tid; j < T2; j += BLK) acc_s[j] = 0.0f;
    __syncthreads();
    int off = incl - ntake, tot = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        if (w < warp) off += w_cnt[w];
        tot += w_cnt[w];
    }
    if (ta) { l_k[off] = (int)ka; l_w[off] = wa; ++off; }
    if (tb) { l_k[off] = (int)kb; l_w[off] = wb; }
    __syncthreads();
    const int C = npair <= BLK ? BLK / npair : 1;
    const int c = npair <= BLK ? tid / npair : 0;
    const int pb = npair <= BLK ? tid % npair : tid;
    float ac[PP][4];
#pragma unroll
    for (int u = 0; u < PP; ++u) ac[u][0] = ac[u][1] = ac[u][2] = ac[u][3] = 0.0f;
    if (c < C) {
        for (int i = c; i < tot; i += C) {
#pragma unroll
            for (int u = 0; u < PP; ++u) {
                const int p = pb + u * BLK;
                if ((u > 0 && npair <= BLK) || p >= npair) break;
                const uint4 r = philox10(make_uint4((uint32_t)l_k[i], (uint32_t)p, iter, ctr3), P);
                const float2 ze = box_muller(r.x, r.y), zo = box_muller(r.z, r.w);
                const float w0 = l_w[i] * P.sig0, w1 = l_w[i] * P.sig1;
                ac[u][0] = fmaf(w0, ze.x, ac[u][0]);
                ac[u][1] = fmaf(w1, ze.y, ac[u][1]);
                ac[u][2] = fmaf(w0, zo.x, ac[u][2]);
                ac[u][3] = fmaf(w1, zo.y, ac[u][3]);
            }
        }
    }
    for (int cc = 0; cc < C; ++cc) {
        if (c == cc) {
#pragma unroll
            for (int u = 0; u < PP; ++u) {
                const int p = pb + u * BLK;
                if ((u > 0 && npair <= BLK) || p >= npair) break;
                acc_s[4 * p] += ac[u][0];
                acc_s[4 * p + 1] += ac[u][1];
                if (2 * p + 1 < T) {
                    acc_s[4 * p + 2] += ac[u][2];
                    acc_s[4 * p + 3] += ac[u][3];
                }
            }
        }
        __syncthreads();
    }
    for (int j = tid; j < T2; j += BLK) part_acc[j] = acc_s[j];
    if (tid == 0) {
        float eta = red[0];
#pragma unroll
        for (int w = 1; w < NW; ++w) eta += red[w];
        *part_eta = (double)eta;
        *part_has = tot > 0;
    }
}

// Launch 1, packed form: thread t of block b steps rollouts 2 b BLK + t and
// 2 b BLK + BLK + t together (rollout2.cuh).  The segment-pair table arrives
// by one bulk copy; V is laid out as broadcast pairs.  Built for MINB = 2 and
// 3 resident blocks per SM: a grid that fits in one wave at two blocks per SM
// runs the MINB = 2 build (the compiler keeps more values in registers: 4 %
// faster at K = 65536), a larger one the MINB = 3 build (<= 168 registers, a
// third block per SM: 1 % faster at K = 262144 than MINB = 2).
template <bool DUMP, bool PART, int MINB>
__global__ void __launch_bounds__(ROLL2_BLK, MINB) mppi_rollout2_kernel(
    DevParams P, const float* __restrict__ x0g, const float* __restrict__ Vg,
    const float4* __restrict__ recg, uint32_t iter, uint32_t ctr3,
    const uint32_t* __restrict__ iter_dev, float* __restrict__ S_out, float* __restrict__ traj,
    float* __restrict__ blk_min, int* __restrict__ seg0_out, unsigned* __restrict__ status,
    uint32_t k_off, BlockPartials part) {
    constexpr int BLK = ROLL2_BLK, NW = BLK / 32;
    griddep_launch_dependents();
    griddep_wait();
    if (iter_dev) iter += *iter_dev;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = P.T, n = P.n_track;
    float4* rec = reinterpret_cast<float4*>(smem_raw);
    float4* Vp = rec + 3 * (n + 5);
    __shared__ __align__(8) uint64_t bar;
    __shared__ float red_f[NW];
    __shared__ int red_i[NW];
    __shared__ int s_seg0, s_fail;
    __shared__ float s_d20;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid == 0) {
        s_fail = 0;
        mbar_init(&bar, 1);
        const uint32_t bytes = (uint32_t)rec_table_bytes(n);
        mbar_expect_tx(&bar, bytes);
        bulk_g2s(rec, recg, bytes, &bar);
    }
    for (int t = tid; t < T; t += BLK) {
        const float2 v = reinterpret_cast<const float2*>(Vg)[t];
        const float g0 = P.gis0 * v.x, g1 = P.gis1 * v.y;
        Vp[2 * t] = make_float4(v.x, v.x, v.y, v.y);
        Vp[2 * t + 1] = make_float4(g0, g0, g1, g1);
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0u)) s_fail = 1;
    __syncthreads();
    if (s_fail) {
        if (tid == 0) {
            atomicOr(status, SMPPI_DEV_TIMEOUT);
            mbar_wait_bounded(&bar, 0u);   // let the copy in flight land before the block exits
        }
        return;
    }
    // global nearest segment of x0 (lowest index on ties)
    const float X0 = x0g[3], Y0 = x0g[4];
    float bd = 3.0e38f;
    int bi = 0x7fffffff;
    for (int i = tid; i < n; i += BLK) {
        const float d = rec_d2_seg(rec, i, X0, Y0);
        if (d < bd) { bd = d; bi = i; }
    }
    warp_argmin(bd, bi);
    if (lane == 0) { red_f[warp] = bd; red_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < NW; ++w)
            if (red_f[w] < bd || (red_f[w] == bd && red_i[w] < bi)) { bd = red_f[w]; bi = red_i[w]; }
        const int s0 = seg_or_zero(bi, n, status);
        s_seg0 = s0;
        s_d20 = (s0 == bi) ? bd : rec_d2_seg(rec, s0, X0, Y0);
        if (blockIdx.x == 0 && seg0_out) *seg0_out = s0;
    }
    __syncthreads();

    const int ka = blockIdx.x * 2 * BLK + tid, kb = ka + BLK;
    const bool act_a = ka < P.K, act_b = kb < P.K;
    float* ta = (DUMP && act_a) ? traj + (size_t)ka * (T + 1) * 6 : nullptr;
    float* tb = (DUMP && act_b) ? traj + (size_t)kb * (T + 1) * 6 : nullptr;
    const float2 S = x2::rollout2<DUMP>(P, rec, Vp, make_state(x0g), s_seg0, s_d20,
                                        (uint32_t)ka + k_off, (uint32_t)kb + k_off, iter, ctr3,
                                        ta, tb);
    if (act_a) {
        S_out[ka] = S.x;
        if (!isfinite(S.x)) atomicOr(status, SMPPI_DEV_NUMERIC);
    }
    if (act_b) {
        S_out[kb] = S.y;
        if (!isfinite(S.y)) atomicOr(status, SMPPI_DEV_NUMERIC);
    }
    const float m = warp_min(fminf(act_a ? S.x : 3.0e38f, act_b ? S.y : 3.0e38f));
    if (lane == 0) red_f[warp] = m;
    __syncthreads();
    __shared__ float s_mb;
    if (tid == 0) {
        float mb = red_f[0];
#pragma unroll
        for (int w = 1; w < NW; ++w) mb = fminf(mb, red_f[w]);
        blk_min[blockIdx.x] = mb;
        s_mb = mb;
    }
    if (PART) {   // this block's min-shifted partial of the update (merged by the next launch)
        __shared__ int w_cnt[NW];
        __syncthreads();
        float* acc_s = reinterpret_cast<float*>(Vp + 2 * T);
        int* l_k = reinterpret_cast<int*>(acc_s + 2 * T);
        float* l_w = reinterpret_cast<float*>(l_k + 2 * BLK);
        block_partial<BLK>(P, s_mb, S, act_a, act_b, (uint32_t)ka + k_off, (uint32_t)kb + k_off,
                           iter, ctr3, l_k, l_w, acc_s, red_f, w_cnt,
                           part.acc + (size_t)blockIdx.x * 2 * T, part.eta + blockIdx.x,
                           part.has + blockIdx.x);
    }
}

// Segment-pair records j = 0 .. n + 4 (segments j - 1 and j, mod n).
__global__ void rec_table_kernel(const float* __restrict__ xy, int n, float4* __restrict__ rec) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n + 5) return;
    float ax[2], ay[2], dx[2], dy[2], gx[2], gy[2];
    for (int h = 0; h < 2; ++h) {
        const int i = (j - 1 + h + n) % n, i1 = (i + 1 == n) ? 0 : i + 1;
        ax[h] = xy[2 * i];
        ay[h] = xy[2 * i + 1];
        dx[h] = xy[2 * i1] - ax[h];
        dy[h] = xy[2 * i1 + 1] - ay[h];
        const float l2 = fmaf(dx[h], dx[h], dy[h] * dy[h]);
        const float inv = l2 > 0.0f ? 1.0f / l2 : 0.0f;
        gx[h] = dx[h] * inv;
        gy[h] = dy[h] * inv;
    }
    rec[3 * j] = make_float4(-ax[0], -ax[1], -ay[0], -ay[1]);
    rec[3 * j + 1] = make_float4(-dx[0], -dx[1], -dy[0], -dy[1]);
    rec[3 * j + 2] = make_float4(gx[0], gx[1], gy[0], gy[1]);
}

// Launch 2: weights, weighted noise sum of the rollouts whose weight exceeds
// w_skip, last-block float64 merge.  blk_min may be NULL (then m = min of S).
// part_has[b] != 0 when block b's noise sums are not all zero.
constexpr int UPD_PER_T = 8;                  // slice values per thread in one pass
constexpr int UPD_LIST = UPD_PER_T * UPD_BLK;  // list of taken rollouts of one pass

//
// SHIELD: the last block then also runs the safety shield on V+ (Alg. 1,
// repair_in_block; V_safe out) and the closed-loop step (x0 <- f(x0, v_0^safe)
// + w, V <- shift(V+), Eq. 26), so that one control update is two launches.
// Every block bulk-copies the segment-pair table into its shared memory at
// entry (overlapping the weight pass); the non-last blocks wait for their copy
// before they exit.
struct ShieldTail {
    const float4* rec;      // segment-pair table (global)
    const int* seg0;        // nearest segment of x0 (written by the rollout launch)
    float* x0;              // in/out state
    float* V_safe;          // out: repaired controls
    int n_repair, ck;
    double* merit_out;      // optional: n_repair + 1 merits
    uint32_t ctr3_dist;     // counter word of the disturbance
};

// x_{n+1} = f(x_n, clamp(v_0)) + w_n (Eq. 26), w_n on (v_y, r) from the Philox
// counter (0, 0, iter, ctr3); xn gets (v_x, v_y, r, X, Y, psi).
__device__ __forceinline__ void closed_loop_next(const DevParams& P, const State& x0, float2 v0,
                                                 uint32_t iter, uint32_t ctr3, float* xn) {
    State x = x0;
    model_step(P, x, clampf(v0.x, P.umin0, P.umax0), clampf(v0.y, P.umin1, P.umax1));
    const uint4 r = philox10(make_uint4(0u, 0u, iter, ctr3), P);
    const float2 z = box_muller(r.x, r.y);
    xn[0] = x.vx;
    xn[1] = fmaf(P.dsig0, z.x, x.vy);
    xn[2] = fmaf(P.dsig1, z.y, x.r);
    xn[3] = x.X;
    xn[4] = x.Y;
    xn[5] = x.psi;
}

// The closed-loop work that does not wait for the merit of V+: V <- shift(V+),
// V_safe <- V+ and the next state from v_0 = V+_0, all right unless the shield
// then repairs V+ (shield_tail redoes V_safe and the state in that case).  Run
// by an idle warp during the first merit pass.
struct TailSide {
    const DevParams* P;
    const float2* Vplus;   // shared
    float2* Vs_out;        // global
    float2* V2;            // global
    State x0;
    uint32_t iter, ctr3;
    float* xn;             // shared, 6 floats
    __device__ void operator()(int lane) const {
        const int T = P->T;
        for (int t = lane; t < T; t += 32) {
            Vs_out[t] = Vplus[t];
            V2[t] = Vplus[t + 1 < T ? t + 1 : T - 1];   // warm start: shift(V+)
        }
        if (lane == 0) closed_loop_next(*P, x0, Vplus[0], iter, ctr3, xn);
    }
};

// The safety shield on V+ (Alg. 1 with Armijo backtracking, repair_in_block;
// V_safe out) and the closed-loop step (x0 <- f(x0, v_0^safe) + w, V <- shift(V+),
// Eq. 26) by one block of BLK threads.  smem_raw: the segment-pair table, whose
// bulk copy completes on bar, then room for the repair's controls, gradient and
// tape; Vplus: V+ in shared memory.  With the shield on, the closed-loop writes
// for an unrepaired V+ run during the merit pass (TailSide); after a repair
// V_safe and the state are written again from the repaired controls.
template <int BLK, bool FAST>
__device__ __forceinline__ void shield_tail(const DevParams& P, unsigned char* smem_raw,
                                            uint64_t* bar, const float2* Vplus, float* V,
                                            uint32_t iter, uint32_t n_upd, uint32_t* iter_dev,
                                            const ShieldTail& sh, unsigned* status,
                                            bool block_grad = false,
                                            const float* x0_in = nullptr,
                                            const int* seg0_in = nullptr) {
    __shared__ int s_fail, s_iters;
    __shared__ float s_xn[6];
    __shared__ RepairSmem rsm;
    const int tid = threadIdx.x, T = P.T;
    float4* rec = reinterpret_cast<float4*>(smem_raw);
    float2* Vw = reinterpret_cast<float2*>(rec + 3 * (P.n_track + 5));
    float2* G2 = Vw + T;
    float* tape_s = reinterpret_cast<float*>(G2 + T);
    // the block gradient's workspace follows the tape scratch (block_grad only)
    const GradWs gws =
        grad_ws_at(reinterpret_cast<unsigned char*>(tape_s + (size_t)(T + 2) * NFIELD), T);
    if (tid == 0) {
        s_fail = 0;
        s_iters = 0;
    }
    __syncthreads();
    if (!mbar_wait_bounded(bar, 0u)) s_fail = 1;
    __syncthreads();
    if (s_fail) {
        if (tid == 0) {
            atomicOr(status, SMPPI_DEV_TIMEOUT);
            mbar_wait_bounded(bar, 0u);
        }
        return;
    }
    for (int t = tid; t < T; t += BLK) Vw[t] = Vplus[t];
    __syncthreads();
    const State x0 = make_state(x0_in ? x0_in : sh.x0);   // x0_in: already loaded
    float2* Vs_out = reinterpret_cast<float2*>(sh.V_safe);
    float2* V2 = reinterpret_cast<float2*>(V);
    if (sh.n_repair > 0) {
        const TailSide side{&P, Vplus, Vs_out, V2, x0, iter, sh.ctr3_dist, s_xn};
        repair_in_block<BLK, FAST>(P, rec, x0, seg0_in ? *seg0_in : sh.seg0[0], Vw, G2, tape_s,
                                   sh.n_repair, 1, 0.0f,
                                   sh.ck, sh.merit_out, &s_iters, status, rsm, side,
                                   block_grad ? &gws : nullptr);
        if (s_iters != 0) {   // V+ was repaired: V_safe and the step from the new controls
            for (int t = tid; t < T; t += BLK) Vs_out[t] = Vw[t];
            if (tid == 0) closed_loop_next(P, x0, Vw[0], iter, sh.ctr3_dist, s_xn);
        }
    } else {
        for (int t = tid; t < T; t += BLK) {
            Vs_out[t] = Vw[t];
            V2[t] = Vplus[t + 1 < T ? t + 1 : T - 1];   // warm start: shift(V+)
        }
        if (tid == 0) closed_loop_next(P, x0, Vw[0], iter, sh.ctr3_dist, s_xn);
    }
    if (tid == 0) {   // x0 <- f(x0, clamp(v_0^safe)) + w_n
        for (int i = 0; i < 6; ++i) sh.x0[i] = s_xn[i];
        if (iter_dev) *iter_dev = n_upd + 1u;
    }
}

template <bool SHIELD, bool FAST>
__global__ void __launch_bounds__(UPD_BLK) mppi_update_kernel(
    DevParams P, const float* __restrict__ S, const float* __restrict__ blk_min, int n_min,
    float* V, uint32_t iter, uint32_t ctr3, uint32_t* __restrict__ iter_dev,
    float* __restrict__ part_acc, double* __restrict__ part_eta, int* __restrict__ part_has,
    unsigned* __restrict__ ticket, unsigned* __restrict__ status, ShieldTail sh,
    uint32_t k_off, double* __restrict__ partial_out) {
    constexpr int NW = UPD_BLK / 32;
    constexpr int PER_T = UPD_PER_T;
    griddep_launch_dependents();
    griddep_wait();
    const uint32_t n_upd = iter_dev ? *iter_dev : 0u;
    iter += n_upd;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    if (SHIELD && threadIdx.x == 0) {
        mbar_init(&bar, 1);
        const uint32_t bytes = (uint32_t)rec_table_bytes(P.n_track);
        mbar_expect_tx(&bar, bytes);
        bulk_g2s(reinterpret_cast<float4*>(smem_raw), sh.rec, bytes, &bar);
    }
    __shared__ float red_f[NW];
    __shared__ int l_k[UPD_LIST];
    __shared__ float l_w[UPD_LIST];
    __shared__ int w_cnt[NW];
    __shared__ __align__(16) float acc_s[2 * SMPPI_MAX_T];   // read as float2 by the shield
    __shared__ bool s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = P.K, T = P.T, T2 = 2 * T, npair = (T + 1) >> 1;

    // global minimum of the costs
    float m = 3.0e38f;
    if (blk_min) {
        for (int b = tid; b < n_min; b += UPD_BLK) m = fminf(m, blk_min[b]);
    } else {
        for (int k = tid; k < K; k += UPD_BLK) m = fminf(m, S[k]);
    }
    m = warp_min(m);
    if (lane == 0) red_f[warp] = m;
    __syncthreads();
    m = red_f[0];
#pragma unroll
    for (int w = 1; w < NW; ++w) m = fminf(m, red_f[w]);

    const int per = (K + gridDim.x - 1) / gridDim.x;
    const int k_lo = blockIdx.x * per, k_hi = min(K, k_lo + per);
    // thread (slot c, pair p) accumulates omega eps for pair p over list items c, c + C, ...
    const int C = UPD_BLK / npair;          // >= 1 because npair <= SMPPI_MAX_T / 2
    const int c = tid / npair, p = tid % npair;
    const bool worker = c < C;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    float eta_t = 0.0f;
    int has = 0;
    for (int kb = k_lo; kb < k_hi; kb += PER_T * UPD_BLK) {
        // weights of up to PER_T values per thread (loads issued together), k in order
        float om[PER_T];
        int ntake = 0;
#pragma unroll
        for (int u = 0; u < PER_T; ++u) {
            const int k = kb + tid * PER_T + u;
            om[u] = (k < k_hi) ? expf((m - __ldg(&S[k])) * P.lam_inv) : 0.0f;
            eta_t += om[u];
            ntake += om[u] > P.w_skip;
        }
        // block prefix sum of the per-thread counts (thread order = k order)
        int incl = ntake;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) w_cnt[warp] = incl;
        __syncthreads();
        int off = incl - ntake, tot = 0;
        for (int w = 0; w < NW; ++w) {
            if (w < warp) off += w_cnt[w];
            tot += w_cnt[w];
        }
#pragma unroll
        for (int u = 0; u < PER_T; ++u) {
            if (om[u] > P.w_skip) {     // tot <= PER_T * UPD_BLK = UPD_LIST: no overflow
                l_k[off] = kb + tid * PER_T + u;
                l_w[off] = om[u];
                ++off;
            }
        }
        __syncthreads();
        const int nl = tot;
        has |= (nl > 0);
        if (worker) {
            for (int i = c; i < nl; i += C) {
                const uint4 r =
                    philox10(make_uint4((uint32_t)l_k[i] + k_off, (uint32_t)p, iter, ctr3), P);
                const float2 ze = box_muller(r.x, r.y), zo = box_muller(r.z, r.w);
                const float w0 = l_w[i] * P.sig0, w1 = l_w[i] * P.sig1;
                a0 = fmaf(w0, ze.x, a0);
                a1 = fmaf(w1, ze.y, a1);
                a2 = fmaf(w0, zo.x, a2);
                a3 = fmaf(w1, zo.y, a3);
            }
        }
        __syncthreads();
    }
    // block normaliser (float within the block; FP64 math is slow on this part and
    // is kept to the cross-block merge) and per-pair sums over the slots, in slot order
    float eta_f = eta_t;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) eta_f += __shfl_xor_sync(0xffffffffu, eta_f, o);
    if (lane == 0) red_f[warp] = eta_f;
    for (int j = tid; j < T2; j += UPD_BLK) acc_s[j] = 0.0f;
    __syncthreads();
    float eta = 0.0f;
#pragma unroll
    for (int w = 0; w < NW; ++w) eta += red_f[w];
    if (has) {
        for (int cc = 0; cc < C; ++cc) {
            if (worker && c == cc) {
                acc_s[4 * p] += a0;
                acc_s[4 * p + 1] += a1;
                if (2 * p + 1 < T) {
                    acc_s[4 * p + 2] += a2;
                    acc_s[4 * p + 3] += a3;
                }
            }
            __syncthreads();
        }
        float* pa = part_acc + (size_t)blockIdx.x * T2;
        for (int j = tid; j < T2; j += UPD_BLK) pa[j] = acc_s[j];
    }
    if (tid == 0) {
        part_eta[blockIdx.x] = (double)eta;
        part_has[blockIdx.x] = has;
    }

    // the last block merges the partials in block order (float64)
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) {
        if (SHIELD && tid == 0) mbar_wait_bounded(&bar, 0u);   // the copy lands before exit
        return;
    }
    __threadfence();
    const int G = gridDim.x;            // <= UPD_BLK
    const int hb = (tid < G) ? __ldcg(&part_has[tid]) : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, hb != 0);
    if (lane == 0) w_cnt[warp] = __popc(bal);
    __syncthreads();
    int off = 0, nz = 0;
    for (int w = 0; w < NW; ++w) {
        if (w < warp) off += w_cnt[w];
        nz += w_cnt[w];
    }
    if (hb) l_k[off + __popc(bal & ((1u << lane) - 1u))] = tid;
    // eta = sum_b eta_b in float64 by warp 0 (fixed order: lane-strided, then a tree)
    __shared__ double s_inv_eta;
    if (warp == 0) {
        double e_sum = 0.0;
        for (int b = lane; b < G; b += 32) e_sum += __ldcg(&part_eta[b]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e_sum += __shfl_xor_sync(0xffffffffu, e_sum, o);
        if (lane == 0) {
            s_inv_eta = 1.0 / e_sum;
            if (partial_out) {
                partial_out[0] = (double)m;
                partial_out[1] = e_sum;
            }
        }
    }
    __syncthreads();
    const double inv_eta = s_inv_eta;
    for (int j = tid; j < T2; j += UPD_BLK) {
        double A = 0.0;
        int i = 0;
        for (; i + 8 <= nz; i += 8) {      // 8 independent loads in flight, summed in order
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcg(&part_acc[(size_t)l_k[i + u] * T2 + j]);
#pragma unroll
            for (int u = 0; u < 8; ++u) A += (double)v[u];
        }
        for (; i < nz; ++i) A += (double)__ldcg(&part_acc[(size_t)l_k[i] * T2 + j]);
        if (partial_out) {          // slice partial: V is left as it is
            partial_out[2 + j] = A;
            continue;
        }
        const float lo = (j & 1) ? P.umin1 : P.umin0, hi = (j & 1) ? P.umax1 : P.umax0;
        const float v = (float)fma(A, inv_eta, (double)V[j]);
        if (!isfinite(v)) atomicOr(status, SMPPI_DEV_NUMERIC);
        V[j] = clampf(v, lo, hi);
        if (SHIELD) acc_s[j] = V[j];    // V+ (the merge no longer needs acc_s)
    }
    if (tid == 0) *ticket = 0u;
    if (!SHIELD || partial_out) return;

    // ---- safety shield on V+ (Alg. 1) and closed-loop step (Eq. 26) ----
    shield_tail<UPD_BLK, FAST>(P, smem_raw, &bar, reinterpret_cast<const float2*>(acc_s), V, iter,
                               n_upd, iter_dev, sh, status);
}

// One control update after a rollout launch that wrote block partials: the
// merge of the partials into V+ (Eq. 10-11; the log-sum-exp rescaling
// c_b = exp(-(m_b - m)/lambda) with m the smallest block minimum; the
// normaliser in float64, the noise sum in float32 compensated, both in a fixed
// order; blocks whose whole contribution c_b eta_b is below w_skip are left out
// of the noise sum, which moves V+ by at most w_skip max|eps| each),
// then the shield and the closed-loop step (shield_tail).  One block; the
// track table is staged before the wait on the rollout launch.
template <bool FAST>
__global__ void __launch_bounds__(UPD_BLK) mppi_merge_shield_kernel(
    DevParams P, int nb, const float* __restrict__ blk_min, BlockPartials part, float* V,
    uint32_t iter, uint32_t* __restrict__ iter_dev, unsigned* __restrict__ status,
    ShieldTail sh) {
    constexpr int NW = UPD_BLK / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ float s_c[MERGE_MAX_BLOCKS];
    __shared__ int l_b[MERGE_MAX_BLOCKS];
    __shared__ __align__(16) float vplus[2 * SMPPI_MAX_T];   // read as float2 by the shield
    __shared__ float red_f[NW];
    __shared__ double red_d[NW];
    __shared__ int w_cnt[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T2 = 2 * P.T;
    griddep_launch_dependents();
    if (tid == 0) {   // the track table is constant: staged before the wait
        mbar_init(&bar, 1);
        const uint32_t bytes = (uint32_t)rec_table_bytes(P.n_track);
        mbar_expect_tx(&bar, bytes);
        bulk_g2s(reinterpret_cast<float4*>(smem_raw), sh.rec, bytes, &bar);
    }
    griddep_wait();
    const uint32_t n_upd = iter_dev ? *iter_dev : 0u;
    iter += n_upd;
    // every block's (m_b, eta_b, has_b) loaded at once into registers (one round trip)
    constexpr int PB = MERGE_MAX_BLOCKS / UPD_BLK;
    float mb[PB];
    double eb[PB];
    int hb[PB];
#pragma unroll
    for (int u = 0; u < PB; ++u) {
        const int b = tid + u * UPD_BLK;
        mb[u] = b < nb ? __ldcg(&blk_min[b]) : 3.0e38f;
        eb[u] = b < nb ? __ldcg(&part.eta[b]) : 0.0;
        hb[u] = b < nb ? __ldcg(&part.has[b]) : 0;
    }
    // loaded in the same round trip and used only later: V (the first control of
    // this thread), x0 and the start segment of the shield
    const float v_pre = tid < T2 ? __ldcg(&V[tid]) : 0.0f;
    float x0r[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) x0r[i] = __ldcg(&sh.x0[i]);
    const int seg0r = __ldcg(sh.seg0);
    // m = min_b m_b
    float m = mb[0];
#pragma unroll
    for (int u = 1; u < PB; ++u) m = fminf(m, mb[u]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red_f[warp] = m;
    __syncthreads();
    m = red_f[0];
#pragma unroll
    for (int w = 1; w < NW; ++w) m = fminf(m, red_f[w]);
    // c_b (float32: its rounding rescales eta_b and A_b alike) and the normaliser
    // eta = sum c_b eta_b and 1/eta in float64 (fixed order: thread-strided, the
    // warp's butterfly, then the warps in order)
    double eta = 0.0;
#pragma unroll
    for (int u = 0; u < PB; ++u) {
        const int b = tid + u * UPD_BLK;
        if (b < nb) {
            const float c = expf((m - mb[u]) * P.lam_inv);
            const double ce = (double)c * eb[u];
            eta += ce;
            s_c[b] = (hb[u] && ce > (double)P.w_skip) ? c : 0.0f;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) eta += __shfl_xor_sync(0xffffffffu, eta, o);
    if (lane == 0) red_d[warp] = eta;
    __syncthreads();
    // 1/eta, one float64 division for the block (the warps' sums in order): with
    // fewer controls than threads a thread without a control forms it while the
    // others sum the noise, else thread 0 first
    __shared__ double s_inv;
    const bool late = T2 < UPD_BLK;
    auto form_inv = [&]() {
        double e = red_d[0];
#pragma unroll
        for (int w = 1; w < NW; ++w) e += red_d[w];
        s_inv = 1.0 / e;
    };
    if (!late) {
        if (tid == 0) form_inv();
        __syncthreads();
    }
    // the blocks that enter the noise sum, in block order
    int nz = 0;
    for (int b0 = 0; b0 < nb; b0 += UPD_BLK) {
        const int b = b0 + tid;
        const bool sel = b < nb && s_c[b] != 0.0f;
        const unsigned bal = __ballot_sync(0xffffffffu, sel);
        if (lane == 0) w_cnt[warp] = __popc(bal);
        __syncthreads();
        int off = nz;
        for (int w = 0; w < warp; ++w) off += w_cnt[w];
        if (sel) l_b[off + __popc(bal & ((1u << lane) - 1u))] = b;
        for (int w = 0; w < NW; ++w) nz += w_cnt[w];
        __syncthreads();
    }
    if (late && tid == UPD_BLK - 1) form_inv();
    auto form = [&](int j, float A, float cmp) {
        const float lo = (j & 1) ? P.umin1 : P.umin0, hi = (j & 1) ? P.umax1 : P.umax0;
        const float vj = j == tid ? v_pre : V[j];
        const float v = (float)fma((double)__fadd_rn(A, cmp), s_inv, (double)vj);
        if (!isfinite(v)) atomicOr(status, SMPPI_DEV_NUMERIC);
        vplus[j] = clampf(v, lo, hi);
    };
    float A_own = 0.0f, cmp_own = 0.0f;   // the sum of this thread's control (late)
    // A_j = sum_b c_b A_b[j] in block order by the compensated dot product of
    // Ogita, Rump and Oishi (Dot2: each product's rounding error from an FMA, each
    // sum's from the two-sum, both carried in a second accumulator), as accurate
    // as the sum in twice the float32 precision rounded once
    for (int j = tid; j < T2; j += UPD_BLK) {
        float A = 0.0f, cmp = 0.0f;
        auto add = [&](float c, float v) {
            const float t = __fmul_rn(c, v);
            const float et = fmaf(c, v, -t);
            const float sum = __fadd_rn(A, t);
            const float bv = __fsub_rn(sum, A);
            const float es = __fadd_rn(__fsub_rn(A, __fsub_rn(sum, bv)), __fsub_rn(t, bv));
            cmp = __fadd_rn(cmp, __fadd_rn(es, et));
            A = sum;
        };
        int i = 0;
        for (; i + 8 <= nz; i += 8) {      // 8 independent loads in flight, summed in order
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcg(&part.acc[(size_t)l_b[i + u] * T2 + j]);
#pragma unroll
            for (int u = 0; u < 8; ++u) add(s_c[l_b[i + u]], v[u]);
        }
        for (; i < nz; ++i) add(s_c[l_b[i]], __ldcg(&part.acc[(size_t)l_b[i] * T2 + j]));
        if (late) {
            A_own = A;
            cmp_own = cmp;
        } else {
            form(j, A, cmp);
        }
    }
    if (late) {
        __syncthreads();
        if (tid < T2) form(tid, A_own, cmp_own);
    }
    shield_tail<UPD_BLK, FAST>(P, smem_raw, &bar, reinterpret_cast<const float2*>(vplus), V, iter,
                               n_upd, iter_dev, sh, status, true, x0r, &seg0r);
}

// Control noise exactly as the rollout kernels draw it (test access).
__global__ void debug_noise_kernel(DevParams P, uint32_t iter, uint32_t ctr3, int K, int T,
                                   float* __restrict__ eps, uint32_t* __restrict__ raw) {
    const int npair = (T + 1) >> 1;
    const long long total = (long long)K * npair;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / npair), p = (int)(i % npair);
        // the rollout kernels' form (first two rounds split), checked against the
        // oracle's Philox word for word
        uint4 r, r2;
        x2::philox_pair_words(P, x2::philox_pair_setup(P, (uint32_t)k, (uint32_t)k, iter, ctr3),
                              (uint32_t)p, r, r2);
        if (raw) {
            uint32_t* o = raw + i * 4;
            o[0] = r.x; o[1] = r.y; o[2] = r.z; o[3] = r.w;
        }
        if (eps) {
            const float2 ze = box_muller(r.x, r.y);
            float* e = eps + ((size_t)k * T + 2 * p) * 2;
            e[0] = P.sig0 * ze.x;
            e[1] = P.sig1 * ze.y;
            if (2 * p + 1 < T) {
                const float2 zo = box_muller(r.z, r.w);
                e[2] = P.sig0 * zo.x;
                e[3] = P.sig1 * zo.y;
            }
        }
    }
}

// The library's hand-written elementary functions on given arguments (test
// access).  Packed forms (fn 1, 3, 6, 7, 8) take elements 2i and 2i + 1 as the
// two halves of one register pair.  ref receives CUDA's own function of the
// same arguments.
__global__ void debug_elementary_kernel(int fn, int n, const float* __restrict__ a,
                                        const float* __restrict__ b, float* __restrict__ out,
                                        float* __restrict__ ref) {
    using namespace x2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool packed = fn == 1 || fn == 3 || (fn >= 6 && fn <= 8);
    const int i0 = packed ? 2 * i : i;
    if (i0 >= n) return;
    const int i1 = (packed && i0 + 1 < n) ? i0 + 1 : i0;
    const f2 A = make_float2(a[i0], a[i1]), B = make_float2(b[i0], b[i1]);
    f2 o = A, r = A;
    switch (fn) {
        case 0: o.x = atan2_poly(A.x, B.x); r.x = atan2f(A.x, B.x); break;
        case 1: o = atan2_2(A, B); r = make_float2(atan2f(A.x, B.x), atan2f(A.y, B.y)); break;
        case 2: o.x = tyre15(A.x); r.x = sinf(1.5f * atanf(A.x)); break;
        case 3: o = tyre15_2(A); r = make_float2(sinf(1.5f * atanf(A.x)), sinf(1.5f * atanf(A.y))); break;
        case 4: { float sn, cs; sincos_half(A.x, &sn, &cs); o.x = sn; r.x = sinf(A.x); } break;
        case 5: { float sn, cs; sincos_half(A.x, &sn, &cs); o.x = cs; r.x = cosf(A.x); } break;
        case 6: { f2 sn, cs; sincos_half2(A, sn, cs); o = sn; r = make_float2(sinf(A.x), sinf(A.y)); } break;
        case 7: { f2 sn, cs; sincos_half2(A, sn, cs); o = cs; r = make_float2(cosf(A.x), cosf(A.y)); } break;
        case 8: o = atan2_2_lat(A, B); r = make_float2(atan2f(A.x, B.x), atan2f(A.y, B.y)); break;
        default: o.x = rsqrt_n(A.x); r.x = rsqrtf(A.x); break;
    }
    out[i0] = o.x;
    ref[i0] = r.x;
    if (packed && i1 != i0) {
        out[i1] = o.y;
        ref[i1] = r.y;
    }
}

// Merge of slice partials (m_g, eta_g, A_g) into V+ (Eq. 10-11 over the union
// of the slices): omega_k = exp(-(S_k - m)/lambda) = c_g exp(-(S_k - m_g)/lambda)
// for k in slice g, c_g = exp(-(m_g - m)/lambda), m = min_g m_g, so eta and the
// weighted noise sum are the c_g-weighted sums of the slices' (float64, in
// slice order).  With one slice c_0 = 1 and V+ is the single update's, bit for
// bit.
__global__ void __launch_bounds__(UPD_BLK) mppi_merge_kernel(DevParams P, int n_parts,
                                                             const double* __restrict__ parts,
                                                             float* V, unsigned* status) {
    __shared__ double s_c[MERGE_MAX_PARTS];
    __shared__ double s_inv_eta;
    const int T2 = 2 * P.T, W = T2 + 2, tid = threadIdx.x;
    if (tid == 0) {
        double m = parts[0];
        for (int g = 1; g < n_parts; ++g) m = fmin(m, parts[(size_t)g * W]);
        const double lam_inv = (double)P.lam_inv;
        double eta = 0.0;
        for (int g = 0; g < n_parts; ++g) {
            const double c = exp(-(parts[(size_t)g * W] - m) * lam_inv);
            s_c[g] = c;
            eta += c * parts[(size_t)g * W + 1];
        }
        s_inv_eta = 1.0 / eta;
    }
    __syncthreads();
    const double inv_eta = s_inv_eta;
    for (int j = tid; j < T2; j += UPD_BLK) {
        double A = 0.0;
        for (int g = 0; g < n_parts; ++g) A += s_c[g] * parts[(size_t)g * W + 2 + j];
        const float lo = (j & 1) ? P.umin1 : P.umin0, hi = (j & 1) ? P.umax1 : P.umax0;
        const float v = (float)fma(A, inv_eta, (double)V[j]);
        if (!isfinite(v)) atomicOr(status, SMPPI_DEV_NUMERIC);
        V[j] = clampf(v, lo, hi);
    }
}

// ----------------------------------------------------------------------------
// Host-side launchers
// ----------------------------------------------------------------------------
// Launch with programmatic stream serialization (see griddep_wait).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), int grid, int block, size_t smem,
                              cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}
size_t rollout_smem_bytes(int n_track, int T) {
    // the packed kernel's V pairs take two float4 per step, the scalar kernel's one;
    // the block partials add 2T floats and the list of taken rollouts
    return rec_table_bytes(n_track) + (size_t)T * 2 * sizeof(float4) +
           (size_t)T * 2 * sizeof(float) + (size_t)ROLL2_BLK * 4 * sizeof(float);
}

static bool packed_rollout(const DevParams& P) { return P.tyre15 && P.steer_small; }

int rollout_blocks(const DevParams& P) {
    return packed_rollout(P) ? (P.K + 2 * ROLL2_BLK - 1) / (2 * ROLL2_BLK)
                             : (P.K + ROLL_BLK - 1) / ROLL_BLK;
}

cudaError_t launch_rec_table(const float* track_xy, int n, float4* rec, cudaStream_t st) {
    rec_table_kernel<<<(n + 5 + 127) / 128, 128, 0, st>>>(track_xy, n, rec);
    return cudaGetLastError();
}

// SM count of the current device, cached per device ordinal (every thread
// that fills an entry writes the same value).
static int device_sms() {
    constexpr int MAX_DEV = 64;
    static std::atomic<int> sms_of[MAX_DEV];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    int sms = dev < MAX_DEV ? sms_of[dev].load(std::memory_order_relaxed) : 0;
    if (sms < 1) {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            sms < 1)
            sms = 1;
        if (dev < MAX_DEV) sms_of[dev].store(sms, std::memory_order_relaxed);
    }
    return sms;
}

int update_grid(int K) {
    const int sms = device_sms();
    const int by_k = (K + UPD_BLK - 1) / UPD_BLK;
    int g = by_k < sms ? by_k : sms;
    return g < UPD_BLK ? g : UPD_BLK;   // the merge lists at most UPD_BLK partials
}

bool merge_shield_applies(const DevParams& P) {
    return packed_rollout(P) && rollout_blocks(P) <= MERGE_MAX_BLOCKS;
}

cudaError_t launch_rollout(const DevParams& P, bool dump, const float* x0, const float* V,
                           const float4* rec, uint32_t iter, uint32_t ctr3,
                           const uint32_t* iter_dev, float* S_out, float* traj, float* blk_min,
                           int* seg0_out, unsigned* status, cudaStream_t st, uint32_t k_off,
                           BlockPartials part) {
    if (packed_rollout(P)) {
        const bool with_part = part.acc != nullptr;
        size_t smem = rec_table_bytes(P.n_track) + (size_t)P.T * 2 * sizeof(float4);
        if (with_part) smem += (size_t)P.T * 2 * sizeof(float) + (size_t)ROLL2_BLK * 4 * sizeof(float);
        const bool one_wave = rollout_blocks(P) <= 2 * device_sms();
        auto kern = dump ? mppi_rollout2_kernel<true, false, 3>
                    : with_part ? (one_wave ? mppi_rollout2_kernel<false, true, 2>
                                            : mppi_rollout2_kernel<false, true, 3>)
                                : (one_wave ? mppi_rollout2_kernel<false, false, 2>
                                            : mppi_rollout2_kernel<false, false, 3>);
        cudaError_t e = ensure_smem((const void*)kern, smem);
        if (e != cudaSuccess) return e;
        return launch_pdl(kern, rollout_blocks(P), ROLL2_BLK, smem, st, P, x0, V, rec, iter, ctr3,
                          iter_dev, S_out, traj, blk_min, seg0_out, status, k_off, part);
    }
    const int nblk = (P.K + ROLL_BLK - 1) / ROLL_BLK;
    const size_t smem = rec_table_bytes(P.n_track) + (size_t)P.T * sizeof(float4);
    auto kern = dump ? mppi_rollout_kernel<ROLL_BLK, true, false>
                     : mppi_rollout_kernel<ROLL_BLK, false, false>;
    cudaError_t e = ensure_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, nblk, ROLL_BLK, smem, st, P, x0, V, rec, iter, ctr3, iter_dev, S_out,
                      traj, blk_min, seg0_out, status, k_off);
}

cudaError_t launch_update(const DevParams& P, const float* S, const float* blk_min, int n_min,
                          float* V, uint32_t iter, uint32_t ctr3, uint32_t* iter_dev,
                          float* part_acc, double* part_eta, int* part_has, unsigned* ticket,
                          unsigned* status, cudaStream_t st) {
    return launch_pdl(mppi_update_kernel<false, false>, update_grid(P.K), UPD_BLK, 0, st, P, S,
                      blk_min, n_min, V, iter, ctr3, iter_dev, part_acc, part_eta, part_has, ticket,
                      status, ShieldTail{}, 0u, (double*)nullptr);
}

cudaError_t launch_update_partial(const DevParams& P, const float* S, const float* blk_min,
                                  int n_min, const float* V, uint32_t iter, uint32_t ctr3,
                                  float* part_acc, double* part_eta, int* part_has,
                                  unsigned* ticket, unsigned* status, uint32_t k_off,
                                  double* partial_out, cudaStream_t st) {
    // V is only read when partial_out is given
    return launch_pdl(mppi_update_kernel<false, false>, update_grid(P.K), UPD_BLK, 0, st, P, S,
                      blk_min, n_min, const_cast<float*>(V), iter, ctr3, (uint32_t*)nullptr,
                      part_acc, part_eta, part_has, ticket, status, ShieldTail{}, k_off,
                      partial_out);
}

cudaError_t launch_merge(const DevParams& P, int n_parts, const double* parts, float* V,
                         unsigned* status, cudaStream_t st) {
    // an ordinary launch: the partials may come from another library's kernels (a collective)
    mppi_merge_kernel<<<1, UPD_BLK, 0, st>>>(P, n_parts, parts, V, status);
    return cudaGetLastError();
}

cudaError_t launch_update_shield(const DevParams& P, const float* S, const float* blk_min,
                                 int n_min, float* V, uint32_t iter, uint32_t ctr3,
                                 uint32_t* iter_dev, float* part_acc, double* part_eta,
                                 int* part_has, unsigned* ticket, unsigned* status,
                                 const float4* rec, const int* seg0, float* x0, float* V_safe,
                                 int n_repair, int ck, double* merit_out, uint32_t ctr3_dist,
                                 cudaStream_t st) {
    const size_t smem = rec_table_bytes(P.n_track) + (size_t)P.T * 16 +
                        (size_t)(P.T + 2) * NFIELD * 4;
    const ShieldTail sh{rec, seg0, x0, V_safe, n_repair, ck, merit_out, ctr3_dist};
    auto kern = (P.tyre15 && P.steer_small) ? mppi_update_kernel<true, true>
                                             : mppi_update_kernel<true, false>;
    cudaError_t e = ensure_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, update_grid(P.K), UPD_BLK, smem, st, P, S, blk_min, n_min, V, iter,
                      ctr3, iter_dev, part_acc, part_eta, part_has, ticket, status, sh, 0u,
                      (double*)nullptr);
}

cudaError_t launch_merge_shield(const DevParams& P, int nb, const float* blk_min,
                                BlockPartials part, float* V, uint32_t iter, uint32_t* iter_dev,
                                unsigned* status, const float4* rec, const int* seg0, float* x0,
                                float* V_safe, int n_repair, int ck, double* merit_out,
                                uint32_t ctr3_dist, cudaStream_t st) {
    const size_t smem = rec_table_bytes(P.n_track) + (size_t)P.T * 16 +
                        (size_t)(P.T + 2) * NFIELD * 4 + grad_ws_bytes(P.T);
    const ShieldTail sh{rec, seg0, x0, V_safe, n_repair, ck, merit_out, ctr3_dist};
    auto kern = (P.tyre15 && P.steer_small) ? mppi_merge_shield_kernel<true>
                                             : mppi_merge_shield_kernel<false>;
    cudaError_t e = ensure_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, 1, UPD_BLK, smem, st, P, nb, blk_min, part, V, iter, iter_dev, status,
                      sh);
}

cudaError_t launch_debug_elementary(int fn, int n, const float* a, const float* b, float* out,
                                   float* ref, cudaStream_t st) {
    const int items = (fn == 1 || fn == 3 || (fn >= 6 && fn <= 8)) ? (n + 1) / 2 : n;
    debug_elementary_kernel<<<(items + 255) / 256, 256, 0, st>>>(fn, n, a, b, out, ref);
    return cudaGetLastError();
}

cudaError_t launch_debug_noise(const DevParams& P, uint32_t iter, uint32_t ctr3, int K, int T,
                               float* eps, uint32_t* raw, cudaStream_t st) {
    const long long total = (long long)K * ((T + 1) / 2);
    int grid = (int)((total + 255) / 256);
    if (grid > 4096) grid = 4096;
    if (grid < 1) grid = 1;
    debug_noise_kernel<<<grid, 256, 0, st>>>(P, iter, ctr3, K, T, eps, raw);
    return cudaGetLastError();
}

}  // namespace smppi
