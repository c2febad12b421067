// MPPI iteration kernels: K sampled rollouts with the DCBF-augmented cost,
// the min-shifted softmin weights and the weighted noise sum (Alg. 2 sampling
// loop + OptimalControl; Eq. 10-12, 17-20).
//
// Layout of one launch (K rollouts, horizon T):
//   grid = ceil(K / BLK) blocks, one thread per rollout.  Shared memory holds
//   the centreline segment table, the nominal sequence V and the per-warp
//   partial sums.  Each thread steps its rollout in registers, drawing the
//   noise from Philox as it goes (never stored).  The block then reduces its
//   costs to a local minimum m_b and normaliser eta_b = sum exp(-(S - m_b)/lambda)
//   and, in a second pass over the same rollouts, regenerates the noise and
//   accumulates sum_k omega_k eps_{k,t} for every t.  A small merge kernel
//   rescales the per-block partials by exp(-(m_b - m)/lambda) and sums them in
//   float64 to V+ = clamp(V + A / eta).
#include "kernels.cuh"

namespace smppi {

namespace {

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace

// Stage the centreline segment table, V and the nearest segment of x0.
template <int BLK>
__device__ __forceinline__ void stage_problem(const DevParams& P, const float4* __restrict__ segg,
                                              const float* __restrict__ invg,
                                              const float* __restrict__ Vg, const State& x0,
                                              float4* seg, float* inv, float2* Vs, int* s_seg0,
                                              float* s_d20, float* red_f, int* red_i) {
    const int tid = threadIdx.x;
    for (int i = tid; i < P.n_track; i += BLK) {
        seg[i] = segg[i];
        inv[i] = invg[i];
    }
    for (int t = tid; t < P.T; t += BLK) Vs[t] = reinterpret_cast<const float2*>(Vg)[t];
    __syncthreads();
    // global nearest segment of x0 (lowest index on ties)
    float bd = 3.0e38f;
    int bi = 0x7fffffff;
    for (int i = tid; i < P.n_track; i += BLK) {
        const float d = seg_d2(seg, inv, i, x0.X, x0.Y);
        if (d < bd) { bd = d; bi = i; }
    }
    warp_argmin(bd, bi);
    const int warp = tid >> 5, lane = tid & 31;
    if (lane == 0) { red_f[warp] = bd; red_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < BLK / 32; ++w)
            if (red_f[w] < bd || (red_f[w] == bd && red_i[w] < bi)) { bd = red_f[w]; bi = red_i[w]; }
        *s_seg0 = bi;
        *s_d20 = bd;
    }
    __syncthreads();
}

// One block of rollouts (MODE_ROLL / MODE_DUMP) or of given costs (MODE_FROM_S).
template <int BLK, int MODE>
__global__ void __launch_bounds__(BLK) mppi_rollout_kernel(
    DevParams P, const float* __restrict__ x0g, const float* __restrict__ Vg,
    const float4* __restrict__ segg, const float* __restrict__ invg, uint32_t iter,
    uint32_t ctr3, const uint32_t* __restrict__ iter_dev, const float* __restrict__ S_in,
    float* __restrict__ S_out, float* __restrict__ traj, float* __restrict__ part_acc,
    float2* __restrict__ part_mh, unsigned* __restrict__ status) {
    constexpr int NW = BLK / 32;
    if (iter_dev) iter += *iter_dev;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = P.T, n = P.n_track;
    float4* seg = reinterpret_cast<float4*>(smem_raw);
    float* inv = reinterpret_cast<float*>(seg + n);
    float2* Vs = reinterpret_cast<float2*>(inv + n + (n & 1));
    float* wacc = reinterpret_cast<float*>(Vs + T);  // [NW][2T]
    __shared__ float red_f[NW];
    __shared__ int red_i[NW];
    __shared__ int s_seg0;
    __shared__ float s_d20;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = blockIdx.x * BLK + tid;
    const bool active = k < P.K;

    State x = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (MODE != MODE_FROM_S) {
        x.vx = x0g[0]; x.vy = x0g[1]; x.r = x0g[2]; x.X = x0g[3]; x.Y = x0g[4]; x.psi = x0g[5];
    }

    float S = 3.0e38f;
    if (MODE == MODE_FROM_S) {
        for (int t = tid; t < T; t += BLK) Vs[t] = reinterpret_cast<const float2*>(Vg)[t];
        __syncthreads();
        if (active) S = S_in[k];
    } else {
        stage_problem<BLK>(P, segg, invg, Vg, x, seg, inv, Vs, &s_seg0, &s_d20, red_f, red_i);
        if (active) {
            int s = s_seg0;
            float d2 = s_d20;
            float h_prev = P.w2 - d2;
            float acc = run_cost(P, x.vx, d2) + P.C_cbf * fmaxf(cbf_arg(P, h_prev, h_prev), 0.0f);
            if (MODE == MODE_DUMP) {
                float* tr = traj + (size_t)k * (T + 1) * 6;
                tr[0] = x.vx; tr[1] = x.vy; tr[2] = x.r; tr[3] = x.X; tr[4] = x.Y; tr[5] = x.psi;
            }
            uint4 rnd = make_uint4(0, 0, 0, 0);
            for (int t = 0; t < T; ++t) {
                if ((t & 1) == 0)
                    rnd = philox10(make_uint4((uint32_t)k, (uint32_t)(t >> 1), iter, ctr3), P.key0,
                                   P.key1);
                const float2 z = (t & 1) ? box_muller(rnd.z, rnd.w) : box_muller(rnd.x, rnd.y);
                const float2 v = Vs[t];
                const float u0 = fmaf(P.sig0, z.x, v.x), u1 = fmaf(P.sig1, z.y, v.y);
                acc = fmaf(P.gis0 * v.x, u0, acc);
                acc = fmaf(P.gis1 * v.y, u1, acc);
                model_step(P, x, clampf(u0, P.umin0, P.umax0), clampf(u1, P.umin1, P.umax1));
                s = track_follow(seg, inv, n, s, x.X, x.Y, d2);
                const float h = P.w2 - d2;
                acc += run_cost(P, x.vx, d2) + P.C_cbf * fmaxf(cbf_arg(P, h_prev, h), 0.0f);
                h_prev = h;
                if (MODE == MODE_DUMP) {
                    float* tr = traj + ((size_t)k * (T + 1) + t + 1) * 6;
                    tr[0] = x.vx; tr[1] = x.vy; tr[2] = x.r; tr[3] = x.X; tr[4] = x.Y; tr[5] = x.psi;
                }
            }
            S = acc;
            if (S_out) S_out[k] = S;
            if (!isfinite(S)) atomicOr(status, SMPPI_DEV_NUMERIC);
        }
    }

    // block minimum and normaliser (Eq. 11 with the block-local shift m_b)
    float m = warp_min(active ? S : 3.0e38f);
    if (lane == 0) red_f[warp] = m;
    __syncthreads();
    float mb = red_f[0];
#pragma unroll
    for (int w = 1; w < NW; ++w) mb = fminf(mb, red_f[w]);
    __syncthreads();
    const float om = active ? expf((mb - S) * P.lam_inv) : 0.0f;
    const float es = warp_sum(om);
    if (lane == 0) red_f[warp] = es;
    __syncthreads();
    if (tid == 0) {
        float eta = 0.0f;
        for (int w = 0; w < NW; ++w) eta += red_f[w];
        part_mh[blockIdx.x] = make_float2(mb, eta);
    }

    // second pass: regenerate eps_{k,t} and accumulate omega_k eps_{k,t} (Eq. 10)
    const bool warp_active = __any_sync(0xffffffffu, om > 0.0f);
    float* wa = wacc + warp * 2 * T;
    const int npair = (T + 1) >> 1;
    for (int p = 0; p < npair; ++p) {
        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
        if (warp_active) {
            const uint4 rnd = philox10(make_uint4((uint32_t)k, (uint32_t)p, iter, ctr3), P.key0, P.key1);
            const float2 ze = box_muller(rnd.x, rnd.y);
            const float2 zo = box_muller(rnd.z, rnd.w);
            a0 = warp_sum(om * P.sig0 * ze.x);
            a1 = warp_sum(om * P.sig1 * ze.y);
            a2 = warp_sum(om * P.sig0 * zo.x);
            a3 = warp_sum(om * P.sig1 * zo.y);
        }
        if (lane == 0) {
            wa[4 * p] = a0;
            wa[4 * p + 1] = a1;
            if (2 * p + 1 < T) {
                wa[4 * p + 2] = a2;
                wa[4 * p + 3] = a3;
            }
        }
    }
    __syncthreads();
    for (int j = tid; j < 2 * T; j += BLK) {
        float s = 0.0f;
#pragma unroll
        for (int w = 0; w < NW; ++w) s += wacc[w * 2 * T + j];
        part_acc[(size_t)blockIdx.x * 2 * T + j] = s;
    }
}

// Merge the per-block partials (float64): m = min_b m_b, scale_b =
// exp(-(m_b - m)/lambda), eta = sum_b eta_b scale_b, A_j = sum_b acc_bj scale_b,
// V+_j = clamp(V_j + A_j / eta).  grid = ceil(2T / 32), block = (32, 8).
__global__ void __launch_bounds__(256) mppi_merge_kernel(DevParams P,
                                                         const float* __restrict__ part_acc,
                                                         const float2* __restrict__ part_mh,
                                                         int nblk, float* __restrict__ V,
                                                         unsigned* __restrict__ status) {
    __shared__ float s_m[8];
    __shared__ double s_d[8][33];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int T2 = 2 * P.T;
    float m = 3.0e38f;
    for (int b = tid; b < nblk; b += 256) m = fminf(m, part_mh[b].x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (tx == 0) s_m[ty] = m;
    __syncthreads();
    m = s_m[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) m = fminf(m, s_m[w]);
    // eta (every block computes it; nblk is small)
    double eta = 0.0;
    for (int b = tid; b < nblk; b += 256) {
        const float2 mh = part_mh[b];
        eta += (double)mh.y * (double)expf((m - mh.x) * P.lam_inv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) eta += __shfl_xor_sync(0xffffffffu, eta, o);
    if (tx == 0) s_d[ty][32] = eta;
    __syncthreads();
    eta = 0.0;
    for (int w = 0; w < 8; ++w) eta += s_d[w][32];
    const int j = blockIdx.x * 32 + tx;
    double a = 0.0;
    if (j < T2) {
        for (int b = ty; b < nblk; b += 8) {
            const float sc = expf((m - part_mh[b].x) * P.lam_inv);
            a += (double)part_acc[(size_t)b * T2 + j] * (double)sc;
        }
    }
    s_d[ty][tx] = a;
    __syncthreads();
    if (ty == 0 && j < T2) {
        double A = 0.0;
        for (int w = 0; w < 8; ++w) A += s_d[w][tx];
        const float lo = (j & 1) ? P.umin1 : P.umin0, hi = (j & 1) ? P.umax1 : P.umax0;
        const float v = (float)((double)V[j] + A / eta);
        if (!isfinite(v)) atomicOr(status, SMPPI_DEV_NUMERIC);
        V[j] = clampf(v, lo, hi);
    }
}

// Control noise exactly as the rollout kernels draw it (test access).
__global__ void debug_noise_kernel(DevParams P, uint32_t iter, uint32_t ctr3, int K, int T,
                                   float* __restrict__ eps, uint32_t* __restrict__ raw) {
    const int npair = (T + 1) >> 1;
    const long long total = (long long)K * npair;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / npair), p = (int)(i % npair);
        const uint4 r = philox10(make_uint4((uint32_t)k, (uint32_t)p, iter, ctr3), P.key0, P.key1);
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

// ----------------------------------------------------------------------------
// Host-side launchers
// ----------------------------------------------------------------------------
size_t rollout_smem_bytes(int n_track, int T) {
    return (size_t)n_track * sizeof(float4) + (size_t)(n_track + (n_track & 1)) * sizeof(float) +
           (size_t)T * sizeof(float2) + (size_t)(ROLL_BLK / 32) * 2 * T * sizeof(float);
}

cudaError_t launch_rollout(const DevParams& P, int mode, const float* x0, const float* V,
                           const float4* seg, const float* inv, uint32_t iter, uint32_t ctr3,
                           const uint32_t* iter_dev, const float* S_in, float* S_out, float* traj, float* part_acc,
                           float2* part_mh, unsigned* status, cudaStream_t st) {
    const int nblk = (P.K + ROLL_BLK - 1) / ROLL_BLK;
    const size_t smem = rollout_smem_bytes(P.n_track, P.T);
    auto kern = mppi_rollout_kernel<ROLL_BLK, MODE_ROLL>;
    if (mode == MODE_DUMP) kern = mppi_rollout_kernel<ROLL_BLK, MODE_DUMP>;
    if (mode == MODE_FROM_S) kern = mppi_rollout_kernel<ROLL_BLK, MODE_FROM_S>;
    cudaError_t e = ensure_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<nblk, ROLL_BLK, smem, st>>>(P, x0, V, seg, inv, iter, ctr3, iter_dev, S_in, S_out, traj,
                                       part_acc, part_mh, status);
    return cudaGetLastError();
}

cudaError_t launch_merge(const DevParams& P, const float* part_acc, const float2* part_mh,
                         int nblk, float* V, unsigned* status, cudaStream_t st) {
    dim3 grid((2 * P.T + 31) / 32), block(32, 8);
    mppi_merge_kernel<<<grid, block, 0, st>>>(P, part_acc, part_mh, nblk, V, status);
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
