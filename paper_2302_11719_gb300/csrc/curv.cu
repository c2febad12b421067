// Rollouts of the curvilinear state variant (state_kind 1; smppi.h): the
// (s, e_y, e_psi) state of the paper's AutoRally model (Sec. VI-A) on the
// centreline curvature kappa(s).  e_y is a state, so the rollout loop has no
// track-distance search: h = w^2 - e_y^2 (Eq. 23) and the running cost
// (Eq. 24-25) read it directly, and the only track data a step touches are two
// curvature samples.
//
// Same layout and launch shape as the Cartesian packed kernel: two rollouts
// per thread on the packed FP32 datapath (FFMA2 / FADD2 / FMUL2), ROLL2_BLK
// threads per block, noise regenerated from Philox, V staged as broadcast
// pairs; the curvature samples are staged in shared memory.
#include "kernels.cuh"
#include "rollout2.cuh"

namespace smppi {
namespace x2 {

// kappa(s) of both halves (s modulo L, linear between the staged samples).
__device__ __forceinline__ f2 kappa2(const DevParams& P, const float* kt, f2 s) {
    const f2 q = make_float2(floorf(s.x * P.inv_len), floorf(s.y * P.inv_len));
    const f2 x = mul(fma(q, bc(-P.track_len), s), bc(P.kap_scale));
    const int ia = min(max((int)x.x, 0), P.n_track - 1);
    const int ib = min(max((int)x.y, 0), P.n_track - 1);
    const f2 f = make_float2(x.x - (float)ia, x.y - (float)ib);
    const f2 k0 = make_float2(kt[ia], kt[ib]);
    const f2 k1 = make_float2(kt[ia + 1], kt[ib + 1]);
    return fma(f, add(k1, neg(k0)), k0);
}

// One explicit Euler step of both rollouts (C = 1.5, |steer| <= 1/2): the
// velocity part as in model_step2, then the curvilinear kinematics
//   s' = (v_x cos e_psi - v_y sin e_psi) / max(1 - kappa e_y, 0.1),
//   e_y' = v_x sin e_psi + v_y cos e_psi,  e_psi' = r - kappa s',
// with (cos, sin) e_psi (cp, sp) rotated by dt e_psi'.  X, Y, psi of State2
// hold s, e_y, e_psi; e_psi itself is carried only when PSI (trajectory dumps).
template <bool PSI>
__device__ __forceinline__ void model_step2_curv(const DevParams& P, const float* kt, State2& x,
                                                 f2 d, f2 a) {
    const f2 bf = atan2_2(fma(bc(P.lf), x.r, x.vy), x.vx);
    const f2 br = atan2_2(fma(bc(-P.lr), x.r, x.vy), x.vx);
    const f2 Fyf = mul(bc(P.Fzf), tyre15_2(mul(bc(P.B), fma(bf, bc(-1.0f), d))));
    const f2 Fyr = mul(bc(P.Fzr), tyre15_2(mul(bc(-P.B), br)));
    f2 sd, cd;
    sincos_half2(d, sd, cd);
    const f2 Fx = mul(bc(P.fx_gain), a);
    const f2 dvx = fma(fma(neg(Fyf), sd, Fx), bc(P.m_inv), mul(x.vy, x.r));
    const f2 dvy = fma(fma(Fyf, cd, Fyr), bc(P.m_inv), mul(neg(x.vx), x.r));
    const f2 dr = mul(fma(mul(bc(P.lf), Fyf), cd, mul(bc(-P.lr), Fyr)), bc(P.Iz_inv));
    const f2 k = kappa2(P, kt, x.X);
    const f2 den = fma(neg(k), x.Y, bc(1.0f));
    const f2 inv = make_float2(rcp_approx(fmaxf(den.x, 0.1f)), rcp_approx(fmaxf(den.y, 0.1f)));
    const f2 sdot = mul(fma(x.vx, x.cp, mul(neg(x.vy), x.sp)), inv);
    const f2 eydot = fma(x.vx, x.sp, mul(x.vy, x.cp));
    const f2 dpsi = mul(bc(P.dt), fma(neg(k), sdot, x.r));
    f2 sa, ca;
    sincos_half2(dpsi, sa, ca);
    if (fabsf(dpsi.x) > 0.5f) sincosf(dpsi.x, &sa.x, &ca.x);
    if (fabsf(dpsi.y) > 0.5f) sincosf(dpsi.y, &sa.y, &ca.y);
    const f2 dt = bc(P.dt);
    x.vx = fma(dt, dvx, x.vx);
    x.vy = fma(dt, dvy, x.vy);
    x.r = fma(dt, dr, x.r);
    x.X = fma(dt, sdot, x.X);
    x.Y = fma(dt, eydot, x.Y);
    if (PSI) x.psi = add(x.psi, dpsi);
    const f2 cp0 = x.cp;
    x.cp = fma(x.cp, ca, mul(neg(x.sp), sa));
    x.sp = fma(x.sp, ca, mul(cp0, sa));
}

// Cost of the states x_t of both rollouts (e_y^2 = x.Y^2): q (Eq. 24-25) and
// the DCBF penalty of (x_{t-1}, x_t) (Eq. 17).
__device__ __forceinline__ void curv_cost2(const DevParams& P, const State2& x, f2& h_prev,
                                           f2& acc) {
    const f2 d2 = mul(x.Y, x.Y);
    const f2 h = fma(d2, bc(-1.0f), bc(P.w2));
    const f2 ev = add(x.vx, bc(-P.v_target));
    f2 q = fma(mul(bc(P.q_v), ev), ev, mul(bc(P.qd_w2), d2));
    if (d2.x > P.w2) q.x += P.C_obs;
    if (d2.y > P.w2) q.y += P.C_obs;
    const f2 c = fma(bc(P.one_m_alpha), h_prev, add(d2, bc(-P.w2)));   // (1-alpha) h_prev - h
    acc = add(acc, fma(bc(P.C_cbf), make_float2(fmaxf(c.x, 0.0f), fmaxf(c.y, 0.0f)), q));
    h_prev = h;
}

// Costs S~ of rollouts ka and kb (Alg. 2 sampling loop; Eq. 12, 17-20, 24-25).
template <bool DUMP>
__device__ __forceinline__ f2 rollout2_curv(const DevParams& P, const float* kt, const float4* Vp,
                                            const State& x0, uint32_t ka, uint32_t kb,
                                            uint32_t iter, uint32_t ctr3, float* ta, float* tb) {
    const int T = P.T, npair = (T + 1) >> 1;
    const float d20 = x0.Y * x0.Y, h0 = P.w2 - d20;
    f2 h_prev = bc(h0);
    f2 acc = bc(run_cost(P, x0.vx, d20) + P.C_cbf * fmaxf(cbf_arg(P, h0, h0), 0.0f));
    State2 x = broadcast(x0);
    if (DUMP) dump2(ta, tb, 0, x);
    f2 za0, za1, zb0, zb1;
    const PhiloxPair ph = philox_pair_setup(P, ka, kb, iter, ctr3);
    noise_pair2(P, ph, 0u, za0, za1, zb0, zb1);
    for (int p = 0; p < npair; ++p) {   // steps 2p and 2p + 1 (< T)
        f2 na0, na1, nb0, nb1;
        if (p + 1 < npair) noise_pair2(P, ph, (uint32_t)(p + 1), na0, na1, nb0, nb1);
        f2 d, a;
        perturb2(P, Vp[4 * p], Vp[4 * p + 1], za0, za1, acc, d, a);
        model_step2_curv<DUMP>(P, kt, x, d, a);
        curv_cost2(P, x, h_prev, acc);
        if (DUMP) dump2(ta, tb, 2 * p + 1, x);
        if (2 * p + 1 < T) {
            perturb2(P, Vp[4 * p + 2], Vp[4 * p + 3], zb0, zb1, acc, d, a);
            model_step2_curv<DUMP>(P, kt, x, d, a);
            curv_cost2(P, x, h_prev, acc);
            if (DUMP) dump2(ta, tb, 2 * p + 2, x);
        }
        za0 = na0; za1 = na1; zb0 = nb0; zb1 = nb1;
    }
    return acc;
}

}  // namespace x2

// Curvilinear rollouts: rollouts k and k + ROLL2_BLK of each block on one
// thread; S_out [K], blk_min [blocks]; traj (DUMP) [K][T + 1][6].
template <bool DUMP>
__global__ void __launch_bounds__(ROLL2_BLK, 2) mppi_rollout_curv_kernel(
    DevParams P, const float* __restrict__ kappa, const float* __restrict__ x0g,
    const float* __restrict__ Vg, uint32_t iter, uint32_t ctr3,
    const uint32_t* __restrict__ iter_dev, float* __restrict__ S_out,
    float* __restrict__ traj, float* __restrict__ blk_min, unsigned* __restrict__ status,
    uint32_t k_off) {
    constexpr int BLK = ROLL2_BLK, NW = BLK / 32;
    griddep_launch_dependents();
    griddep_wait();
    if (iter_dev) iter += *iter_dev;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = P.T, n = P.n_track;
    float4* Vp = reinterpret_cast<float4*>(smem_raw);
    float* kt = reinterpret_cast<float*>(Vp + 2 * T);
    __shared__ float red_f[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int t = tid; t < T; t += BLK) {
        const float2 v = reinterpret_cast<const float2*>(Vg)[t];
        const float g0 = P.gis0 * v.x, g1 = P.gis1 * v.y;
        Vp[2 * t] = make_float4(v.x, v.x, v.y, v.y);
        Vp[2 * t + 1] = make_float4(g0, g0, g1, g1);
    }
    for (int i = tid; i <= n; i += BLK) kt[i] = kappa[i];
    __syncthreads();

    const int ka = blockIdx.x * 2 * BLK + tid, kb = ka + BLK;
    const bool act_a = ka < P.K, act_b = kb < P.K;
    float* ta = (DUMP && act_a) ? traj + (size_t)ka * (T + 1) * 6 : nullptr;
    float* tb = (DUMP && act_b) ? traj + (size_t)kb * (T + 1) * 6 : nullptr;
    const float2 S = x2::rollout2_curv<DUMP>(P, kt, Vp, make_state(x0g), (uint32_t)ka + k_off,
                                             (uint32_t)kb + k_off, iter, ctr3, ta, tb);
    if (act_a) {
        S_out[ka] = S.x;
        if (!isfinite(S.x)) atomicOr(status, SMPPI_DEV_NUMERIC);
    }
    if (act_b) {
        S_out[kb] = S.y;
        if (!isfinite(S.y)) atomicOr(status, SMPPI_DEV_NUMERIC);
    }
    float m = fminf(act_a ? S.x : 3.0e38f, act_b ? S.y : 3.0e38f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red_f[warp] = m;
    __syncthreads();
    if (tid == 0) {
        float mb = red_f[0];
#pragma unroll
        for (int w = 1; w < NW; ++w) mb = fminf(mb, red_f[w]);
        blk_min[blockIdx.x] = mb;
    }
}

size_t curv_rollout_smem_bytes(int n_track, int T) {
    return (size_t)T * 2 * sizeof(float4) + (size_t)(n_track + 1) * sizeof(float);
}

cudaError_t launch_rollout_curv(const DevParams& P, const float* kappa, bool dump, const float* x0,
                                const float* V, uint32_t iter, uint32_t ctr3,
                                const uint32_t* iter_dev, float* S_out, float* traj,
                                float* blk_min, unsigned* status, cudaStream_t st,
                                uint32_t k_off) {
    const size_t smem = curv_rollout_smem_bytes(P.n_track, P.T);
    auto kern = dump ? mppi_rollout_curv_kernel<true> : mppi_rollout_curv_kernel<false>;
    cudaError_t e = ensure_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(rollout_blocks(P));
    cfg.blockDim = dim3(ROLL2_BLK);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, P, kappa, x0, V, iter, ctr3, iter_dev, S_out, traj,
                              blk_min, status, k_off);
}

}  // namespace smppi
