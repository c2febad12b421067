// BFGS repair: the solver Sec. IV-B names for the local problem of Eq. 22, run
// for a fixed number of iterations.  The variant (box projection, Armijo on the
// projected path, binding coordinates held, gradient-step restarts) is stated
// with smppi_repair's mode 2 in smppi.h.
//
// One block per sequence on a persistent grid.  The n x n inverse-Hessian
// approximation H (n = 2 N_r controls) of the sequence a block works on lives
// in that block's slice of a global workspace, small enough to stay in L2;
// the O(n^2) parts (H y, H_FF g_F, the rank-two update) are spread over the
// block, one warp per row for the products so that the row reads coalesce.
// Thread 0 computes the adjoint gradient (seq_cost_grad); the lanes of warp 0
// evaluate the line-search trials a = 1, 1/2, ... in parallel and the largest
// accepted a is taken, the same iterate as sequential backtracking.
#include <algorithm>

#include "shield.cuh"

namespace smppi {

constexpr int BFGS_BLK = 256;
constexpr size_t BFGS_WS_MAX = size_t(256) << 20;   // bytes of H slices at most

namespace {

constexpr int BNW = BFGS_BLK / 32;

struct BfgsSmem {
    double P;               // merit of the iterate the block agrees on
    double red[BNW][3];     // block sums
    float redf[BNW];        // block maxima
    float step;             // accepted trial step a
    int ok;                 // a trial was accepted
};

// Sums of a, b, c over the block (the same value, in the same order, on every thread).
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, BfgsSmem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
        sm.red[warp][0] = a;
        sm.red[warp][1] = b;
        sm.red[warp][2] = c;
    }
    __syncthreads();
    a = b = c = 0.0;
#pragma unroll
    for (int w = 0; w < BNW; ++w) {
        a += sm.red[w][0];
        b += sm.red[w][1];
        c += sm.red[w][2];
    }
    __syncthreads();
}

__device__ __forceinline__ float block_max(float v, BfgsSmem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sm.redf[warp] = v;
    __syncthreads();
    v = sm.redf[0];
#pragma unroll
    for (int w = 1; w < BNW; ++w) v = fmaxf(v, sm.redf[w]);
    __syncthreads();
    return v;
}

// out_i = sum_{j} M_ij x_j over the rows i < n (row-major n x n), one warp per
// row; with mask, only rows and columns whose flag is set (others give 0).
__device__ __forceinline__ void block_matvec(const float* __restrict__ M, const float* x, int n,
                                             const unsigned char* mask, float* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < n; i += BNW) {
        float a = 0.0f;
        if (!mask || mask[i]) {
            const float* row = M + (size_t)i * n;
            for (int j = lane; j < n; j += 32)
                if (!mask || mask[j]) a = fmaf(row[j], x[j], a);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) out[i] = a;
    }
    __syncthreads();
}

}  // namespace

template <bool FAST>
__global__ void __launch_bounds__(BFGS_BLK) repair_bfgs_kernel(
    DevParams P, const float4* __restrict__ recg, const float* __restrict__ x0g, const float* Vin,
    float* Vout, int n_seq, int n_iters, int ck, float* __restrict__ Hws,
    double* __restrict__ merit_out, int* __restrict__ iters_out, ApplyArgs ap,
    unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = P.T, N = P.N_r, nt = P.n_track, n = 2 * N;
    float4* rec = reinterpret_cast<float4*>(smem_raw);
    float2* Vw = reinterpret_cast<float2*>(rec + 3 * (nt + 5));   // iterate z (first N)
    float2* G = Vw + T;                                              // gradient at z
    float2* Gp = G + T;                                              // gradient at the previous z
    float2* Sv = Gp + T;                                             // last step s = z' - z
    float2* Dn = Sv + T;                                             // negated direction
    float* Yv = reinterpret_cast<float*>(Dn + T);                    // y = g - g_prev (n)
    float* Hy = Yv + 2 * T;                                          // H y (n)
    unsigned char* fr = reinterpret_cast<unsigned char*>(Hy + 2 * T);   // free coordinate flags
    float* tape_s = reinterpret_cast<float*>(fr + ((2 * T + 15) & ~15));
    __shared__ BfgsSmem sm;
    __shared__ float s_red[BNW];
    __shared__ int s_redi[BNW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Tape tape{tape_s, 1, 0};
    float* H = Hws + (size_t)blockIdx.x * n * n;
    const float* zf = reinterpret_cast<const float*>(Vw);
    const float* gf = reinterpret_cast<const float*>(G);
    const float* gpf = reinterpret_cast<const float*>(Gp);
    const float* sf = reinterpret_cast<const float*>(Sv);
    float* dnf = reinterpret_cast<float*>(Dn);

    for (int i = tid; i < 3 * (nt + 5); i += BFGS_BLK) rec[i] = recg[i];
    __syncthreads();

    for (int q = blockIdx.x; q < n_seq; q += gridDim.x) {
        const float2* vin = reinterpret_cast<const float2*>(Vin) + (size_t)q * T;
        for (int t = tid; t < T; t += BFGS_BLK) Vw[t] = vin[t];
        const State x0 = make_state(x0g + 6 * q);
        __syncthreads();
        const int s0 = block_nearest_segment<BFGS_BLK>(rec, nt, x0.X, x0.Y, s_red, s_redi, nullptr);
        double* mrow = merit_out ? merit_out + (size_t)q * (n_iters + 1) : nullptr;
        if (tid == 0)
            sm.P = forward_cost<false, false, FAST>(P, rec, x0, s0, N, Vw, nullptr, 0.0f, 1, 0, 0.0f,
                                                    1.0f, 0, tape, nullptr);
        __syncthreads();
        double P0 = sm.P;
        bool H_set = false, have_step = false, stalled = false;
        int it = 0;
        for (; it < n_iters; ++it) {
            if (tid == 0 && mrow) mrow[it] = P0;
            if (P0 == 0.0) break;
            if (tid == 0) seq_cost_grad<FAST>(P, rec, x0, s0, N, T, Vw, G, 1, 0, 0.0f, 1.0f, ck, tape);
            __syncthreads();
            // curvature pair of the last accepted step and the inverse update
            //   H <- (I - rho s y') H (I - rho y s') + rho s s'
            //      = H - rho (s (Hy)' + (Hy) s') + (rho^2 y'Hy + rho) s s'   (H symmetric)
            if (have_step) {
                double sy = 0.0, yy = 0.0, ss = 0.0;
                for (int i = tid; i < n; i += BFGS_BLK) {
                    const float y = gf[i] - gpf[i];
                    Yv[i] = y;
                    sy += (double)sf[i] * y;
                    yy += (double)y * y;
                    ss += (double)sf[i] * sf[i];
                }
                block_sum3(sy, yy, ss, sm);
                if (sy > 1e-5 * sqrt(ss * yy)) {
                    if (!H_set) {
                        const float h0 = (float)(sy / yy);
                        for (int k = tid; k < n * n; k += BFGS_BLK) H[k] = (k % (n + 1) == 0) ? h0 : 0.0f;
                        __syncthreads();
                        H_set = true;
                    }
                    block_matvec(H, Yv, n, nullptr, Hy);
                    double yHy = 0.0, d1 = 0.0, d2 = 0.0;
                    for (int i = tid; i < n; i += BFGS_BLK) yHy += (double)Yv[i] * Hy[i];
                    block_sum3(yHy, d1, d2, sm);
                    const float rho = (float)(1.0 / sy);
                    const float cs = (float)(yHy / (sy * sy) + 1.0 / sy);
                    for (int k = tid; k < n * n; k += BFGS_BLK) {
                        const int i = k / n, j = k - i * n;
                        const float si = sf[i], sj = sf[j];
                        H[k] = fmaf(cs * si, sj, fmaf(-rho, fmaf(si, Hy[j], Hy[i] * sj), H[k]));
                    }
                    __syncthreads();
                }
            }
            // |g|_inf and the binding coordinates (at a bound, gradient pushing outward)
            float gm = 0.0f;
            for (int i = tid; i < n; i += BFGS_BLK) {
                const float g = gf[i], z = zf[i];
                const float lo = (i & 1) ? P.umin1 : P.umin0, hi = (i & 1) ? P.umax1 : P.umax0;
                fr[i] = !((z <= lo && g > 0.0f) || (z >= hi && g < 0.0f));
                gm = fmaxf(gm, fabsf(g));
            }
            gm = block_max(gm, sm);
            if (!(gm > 0.0f)) { stalled = true; break; }
            const float s_first = P.ls_s0 / gm;
            // direction (negated): Dn = H_FF g_F, or the scaled gradient step
            if (H_set) {
                block_matvec(H, gf, n, fr, dnf);
                double gHg = 0.0, d1 = 0.0, d2 = 0.0;
                for (int i = tid; i < n; i += BFGS_BLK) gHg += (double)gf[i] * dnf[i];
                block_sum3(gHg, d1, d2, sm);
                if (!(gHg > 0.0)) H_set = false;      // g'd = -g'Dn >= 0: not a descent direction
            }
            if (!H_set) {
                for (int i = tid; i < n; i += BFGS_BLK) dnf[i] = fr[i] ? s_first * gf[i] : 0.0f;
                __syncthreads();
            }
            // Armijo on the projected path (trials in parallel on warp 0); if the
            // direction came from H and nothing is accepted, once more along the
            // gradient step
            for (int pass = 0; pass < 2; ++pass) {
                if (warp == 0) {
                    int best = 0x7fffffff;
                    double best_P = 0.0;
                    for (int j = lane; j < P.ls_max; j += 32) {
                        const float a = ldexpf(1.0f, -j);
                        double dec;
                        const double Pt = forward_cost<false, true, FAST>(
                            P, rec, x0, s0, N, Vw, G, a, 1, 0, 0.0f, 1.0f, 0, tape, &dec, Dn);
                        if (dec > 0.0 && Pt <= P0 - (double)P.ls_c * dec && j < best) {
                            best = j;
                            best_P = Pt;
                        }
                    }
                    int bj = best;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) bj = min(bj, __shfl_xor_sync(0xffffffffu, bj, o));
                    if (best == bj && bj != 0x7fffffff) {
                        sm.P = best_P;
                        sm.step = ldexpf(1.0f, -bj);
                    }
                    if (lane == 0) sm.ok = (bj != 0x7fffffff);
                }
                __syncthreads();
                if (sm.ok || !H_set) break;
                H_set = false;
                for (int i = tid; i < n; i += BFGS_BLK) dnf[i] = fr[i] ? s_first * gf[i] : 0.0f;
                __syncthreads();
            }
            if (!sm.ok) { stalled = true; break; }
            const float a = sm.step;
            for (int t = tid; t < N; t += BFGS_BLK) {
                const float2 v = Vw[t], dn = Dn[t];
                const float2 u = clamp2(P, make_float2(fmaf(-a, dn.x, v.x), fmaf(-a, dn.y, v.y)));
                Sv[t] = make_float2(u.x - v.x, u.y - v.y);
                Gp[t] = G[t];
                Vw[t] = u;
            }
            __syncthreads();
            P0 = sm.P;
            have_step = true;
        }
        if (tid == 0) {
            if (mrow)
                for (int i = it; i <= n_iters; ++i) mrow[i] = P0;
            if (iters_out) iters_out[q] = it;
            if (stalled) atomicOr(status, SMPPI_DEV_STALLED);
            if (!isfinite(P0)) atomicOr(status, SMPPI_DEV_NUMERIC);
        }
        float2* vout = reinterpret_cast<float2*>(Vout) + (size_t)q * T;
        for (int t = tid; t < T; t += BFGS_BLK) vout[t] = Vw[t];
        if (q == 0 && tid == 0 && ap.x0) closed_loop_step(P, ap, Vw[0]);
        __syncthreads();   // shared memory is reused by the next sequence
    }
}

size_t bfgs_smem_bytes(const DevParams& P) {
    const size_t T = (size_t)P.T;
    return rec_table_bytes(P.n_track) + 5 * T * 8 + 2 * T * 8 + ((2 * T + 15) & ~size_t(15)) +
           (T + 2) * NFIELD * 4;
}

// Blocks of the persistent grid: resident blocks, at most n_seq, and few
// enough that their H slices fit in BFGS_WS_MAX.
int bfgs_grid(const DevParams& P, int n_seq, int sms) {
    const bool fast = P.tyre15 && P.steer_small;
    const void* kern = fast ? (const void*)repair_bfgs_kernel<true> : (const void*)repair_bfgs_kernel<false>;
    const size_t smem = bfgs_smem_bytes(P);
    if (ensure_smem(kern, smem) != cudaSuccess) return 0;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, BFGS_BLK, smem) != cudaSuccess)
        return 0;
    const size_t n = 2 * (size_t)P.N_r;
    const size_t per = std::max<size_t>(1, n * n * sizeof(float));
    const int by_ws = (int)std::max<size_t>(1, BFGS_WS_MAX / per);
    return std::max(1, std::min({n_seq, std::max(1, bps) * sms, by_ws}));
}

size_t bfgs_ws_bytes(const DevParams& P, int grid) {
    const size_t n = 2 * (size_t)P.N_r;
    return std::max<size_t>(16, (size_t)grid * n * n * sizeof(float));
}

cudaError_t launch_repair_bfgs(const DevParams& P, const float4* rec, int n_seq, const float* x0,
                               const float* V_in, float* V_out, int n_iters, int ck, float* H_ws,
                               int grid, double* merit_out, int* iters_out, const ApplyArgs& ap,
                               unsigned* status, cudaStream_t st) {
    const bool fast = P.tyre15 && P.steer_small;
    auto kern = fast ? repair_bfgs_kernel<true> : repair_bfgs_kernel<false>;
    const size_t smem = bfgs_smem_bytes(P);
    cudaError_t e = ensure_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, BFGS_BLK, smem, st>>>(P, rec, x0, V_in, V_out, n_seq, n_iters, ck, H_ws, merit_out,
                                        iters_out, ap, status);
    return cudaGetLastError();
}

}  // namespace smppi
