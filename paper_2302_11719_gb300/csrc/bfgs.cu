// BFGS repair: the solver Sec. IV-B names for the local problem of Eq. 22, run
// for a fixed number of iterations.  The variant (box projection, Armijo on the
// projected path, binding coordinates held, gradient-step restarts) is stated
// with smppi_repair's mode 2 in smppi.h.
//
// One WARP per sequence: lane 0 computes the adjoint gradient (seq_cost_grad,
// a serial chain), the lanes evaluate the line-search trials a = 1, 1/2, ...
// in parallel (the largest accepted a is taken: the same iterate as
// sequential backtracking), and the O(n^2) parts (H y, H_FF g_F, the rank-two
// update, n = 2 N_r) are spread over the lanes.  A block holds a few warps
// that share the staged track table; warps take sequences from an atomic
// counter, so the sequences that need many iterations do not hold up a fixed
// share of the others.
//
// H of the sequence a warp works on lives in that warp's slice of a global
// workspace, small enough to stay in L2.  The update is evaluated in a form
// that is symmetric in (i, j) operation by operation (no fused multiply-add),
// so H stays exactly symmetric; products with H then read it by columns,
// H[j][i] = H[i][j], so that the lanes' loads of one j coalesce.
#include <algorithm>

#include "shield.cuh"

namespace smppi {

constexpr int BFGS_WPB_MAX = 4;                      // warps (sequences) per block
constexpr size_t BFGS_WS_MAX = size_t(256) << 20;    // bytes of H slices at most
constexpr int BFGS_ROWS = 8;                         // rows per lane per pass of a product

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// out_i = sum_j H_ji x_j (= (H x)_i, H symmetric) for i < n, lanes over i;
// with mask, only the flagged rows and columns (other rows give 0).
__device__ __forceinline__ void warp_symv(const float* __restrict__ H, const float* x, int n,
                                          const unsigned char* mask, float* out) {
    const int lane = threadIdx.x & 31;
    for (int i0 = lane; i0 < n; i0 += 32 * BFGS_ROWS) {
        float acc[BFGS_ROWS];
#pragma unroll
        for (int r = 0; r < BFGS_ROWS; ++r) acc[r] = 0.0f;
        for (int j = 0; j < n; ++j) {
            if (mask && !mask[j]) continue;          // the same j on every lane
            const float xj = x[j];
            const float* col = H + (size_t)j * n;
#pragma unroll
            for (int r = 0; r < BFGS_ROWS; ++r) {
                const int i = i0 + 32 * r;
                if (i < n) acc[r] = fmaf(col[i], xj, acc[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < BFGS_ROWS; ++r) {
            const int i = i0 + 32 * r;
            if (i < n) out[i] = (mask && !mask[i]) ? 0.0f : acc[r];
        }
    }
    __syncwarp();
}

}  // namespace

// Bytes of one warp's shared-memory region for horizon T (a multiple of 8, so
// every warp's float2 arrays stay aligned): five float2 arrays of T, two float
// arrays of 2T, 2T flag bytes and the tape, the last two padded to 16 bytes.
__host__ __device__ inline size_t bfgs_warp_bytes(int T) {
    const size_t t = (size_t)T;
    return 5 * t * 8 + 2 * t * 8 + ((2 * t + 15) & ~size_t(15)) +
           ((((t + 2) * NFIELD * 4) + 15) & ~size_t(15));
}

template <bool FAST>
__global__ void __launch_bounds__(32 * BFGS_WPB_MAX) repair_bfgs_kernel(
    DevParams P, const float4* __restrict__ recg, const float* __restrict__ x0g, const float* Vin,
    float* Vout, int n_seq, int n_iters, int ck, float* __restrict__ Hws,
    unsigned* __restrict__ next, double* __restrict__ merit_out, int* __restrict__ iters_out,
    ApplyArgs ap, unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = P.T, N = P.N_r, nt = P.n_track, n = 2 * N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    float4* rec = reinterpret_cast<float4*>(smem_raw);
    unsigned char* wbase = smem_raw + rec_table_bytes(nt) + (size_t)warp * bfgs_warp_bytes(T);
    float2* Vw = reinterpret_cast<float2*>(wbase);   // iterate z (first N)
    float2* G = Vw + T;                              // gradient at z
    float2* Gp = G + T;                              // gradient at the previous z
    float2* Sv = Gp + T;                             // last step s = z' - z
    float2* Dn = Sv + T;                             // negated direction
    float* Yv = reinterpret_cast<float*>(Dn + T);    // y = g - g_prev (n)
    float* Hy = Yv + 2 * T;                          // H y (n)
    unsigned char* fr = reinterpret_cast<unsigned char*>(Hy + 2 * T);   // free coordinate flags
    float* tape_s = reinterpret_cast<float*>(fr + ((2 * T + 15) & ~15));
    const Tape tape{tape_s, 1, 0};
    float* H = Hws + ((size_t)blockIdx.x * wpb + warp) * n * n;
    const float* zf = reinterpret_cast<const float*>(Vw);
    const float* gf = reinterpret_cast<const float*>(G);
    const float* gpf = reinterpret_cast<const float*>(Gp);
    const float* sf = reinterpret_cast<const float*>(Sv);
    float* dnf = reinterpret_cast<float*>(Dn);

    for (int i = threadIdx.x; i < 3 * (nt + 5); i += blockDim.x) rec[i] = recg[i];
    __syncthreads();

    for (;;) {
        int q = 0;
        if (lane == 0) q = (int)atomicAdd(next, 1u);
        q = __shfl_sync(FULL, q, 0);
        if (q >= n_seq) break;
        const float2* vin = reinterpret_cast<const float2*>(Vin) + (size_t)q * T;
        for (int t = lane; t < T; t += 32) Vw[t] = vin[t];
        const State x0 = make_state(x0g + 6 * q);
        // global nearest segment of x0 (lowest index on ties)
        float bd = 3.0e38f;
        int s0 = 0x7fffffff;
        for (int i = lane; i < nt; i += 32) {
            const float d = rec_d2_seg(rec, i, x0.X, x0.Y);
            if (d < bd) { bd = d; s0 = i; }
        }
        warp_argmin(bd, s0);
        __syncwarp();
        double* mrow = merit_out ? merit_out + (size_t)q * (n_iters + 1) : nullptr;
        double P0 = 0.0;
        if (lane == 0)
            P0 = forward_cost<false, false, FAST>(P, rec, x0, s0, N, Vw, nullptr, 0.0f, 1, 0, 0.0f,
                                                  1.0f, 0, tape, nullptr);
        P0 = __shfl_sync(FULL, P0, 0);
        bool H_set = false, have_step = false, stalled = false;
        int it = 0;
        for (; it < n_iters; ++it) {
            if (lane == 0 && mrow) mrow[it] = P0;
            if (P0 == 0.0) break;
            if (lane == 0) seq_cost_grad<FAST>(P, rec, x0, s0, N, T, Vw, G, 1, 0, 0.0f, 1.0f, ck, tape);
            __syncwarp();
            // curvature pair of the last accepted step and the inverse update
            //   H <- (I - rho s y') H (I - rho y s') + rho s s'
            //      = H - rho (s (Hy)' + (Hy) s') + (rho^2 y'Hy + rho) s s'   (H symmetric)
            if (have_step) {
                double sy = 0.0, yy = 0.0, ss = 0.0;
                for (int i = lane; i < n; i += 32) {
                    const float y = gf[i] - gpf[i];
                    Yv[i] = y;
                    sy += (double)sf[i] * y;
                    yy += (double)y * y;
                    ss += (double)sf[i] * sf[i];
                }
                sy = warp_sum(sy);
                yy = warp_sum(yy);
                ss = warp_sum(ss);
                __syncwarp();
                if (sy > 1e-5 * sqrt(ss * yy)) {
                    if (!H_set) {
                        const float h0 = (float)(sy / yy);
                        for (int k = lane; k < n * n; k += 32) H[k] = (k % (n + 1) == 0) ? h0 : 0.0f;
                        __syncwarp();
                        H_set = true;
                    }
                    warp_symv(H, Yv, n, nullptr, Hy);
                    double yHy = 0.0;
                    for (int i = lane; i < n; i += 32) yHy += (double)Yv[i] * Hy[i];
                    yHy = warp_sum(yHy);
                    const float rho = (float)(1.0 / sy);
                    const float cs = (float)(yHy / (sy * sy) + 1.0 / sy);
                    for (int k = lane; k < n * n; k += 32) {
                        const int i = k / n, j = k - i * n;
                        const float si = sf[i], sj = sf[j];
                        const float cross = __fadd_rn(__fmul_rn(si, Hy[j]), __fmul_rn(sj, Hy[i]));
                        const float delta = __fsub_rn(__fmul_rn(cs, __fmul_rn(si, sj)), __fmul_rn(rho, cross));
                        H[k] = __fadd_rn(H[k], delta);
                    }
                    __syncwarp();
                }
            }
            // |g|_inf and the binding coordinates (at a bound, gradient pushing outward)
            float gm = 0.0f;
            for (int i = lane; i < n; i += 32) {
                const float g = gf[i], z = zf[i];
                const float lo = (i & 1) ? P.umin1 : P.umin0, hi = (i & 1) ? P.umax1 : P.umax0;
                fr[i] = !((z <= lo && g > 0.0f) || (z >= hi && g < 0.0f));
                gm = fmaxf(gm, fabsf(g));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(FULL, gm, o));
            __syncwarp();
            if (!(gm > 0.0f)) { stalled = true; break; }
            const float s_first = P.ls_s0 / gm;
            // direction (negated): Dn = H_FF g_F, or the scaled gradient step
            if (H_set) {
                warp_symv(H, gf, n, fr, dnf);
                double gHg = 0.0;
                for (int i = lane; i < n; i += 32) gHg += (double)gf[i] * dnf[i];
                gHg = warp_sum(gHg);
                if (!(gHg > 0.0)) H_set = false;      // g'd = -g'Dn >= 0: not a descent direction
            }
            if (!H_set) {
                for (int i = lane; i < n; i += 32) dnf[i] = fr[i] ? s_first * gf[i] : 0.0f;
                __syncwarp();
            }
            // Armijo on the projected path (trials in parallel on the lanes); if the
            // direction came from H and nothing is accepted, once more along the
            // gradient step
            int bj = 0x7fffffff;
            double best_P = 0.0;
            for (int pass = 0; pass < 2; ++pass) {
                int best = 0x7fffffff;
                double bp = 0.0;
                for (int j = lane; j < P.ls_max; j += 32) {
                    const float a = ldexpf(1.0f, -j);
                    double dec;
                    const double Pt = forward_cost<false, true, FAST>(P, rec, x0, s0, N, Vw, G, a, 1, 0,
                                                                      0.0f, 1.0f, 0, tape, &dec, Dn);
                    if (dec > 0.0 && Pt <= P0 - (double)P.ls_c * dec && j < best) {
                        best = j;
                        bp = Pt;
                    }
                }
                bj = best;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) bj = min(bj, __shfl_xor_sync(FULL, bj, o));
                // the lane that owns trial bj (j = lane + 32 m) holds its merit
                best_P = __shfl_sync(FULL, bp, (bj == 0x7fffffff) ? 0 : (bj & 31));
                if (bj != 0x7fffffff || !H_set) break;
                H_set = false;
                for (int i = lane; i < n; i += 32) dnf[i] = fr[i] ? s_first * gf[i] : 0.0f;
                __syncwarp();
            }
            if (bj == 0x7fffffff) { stalled = true; break; }
            const float a = ldexpf(1.0f, -bj);
            for (int t = lane; t < N; t += 32) {
                const float2 v = Vw[t], dn = Dn[t];
                const float2 u = clamp2(P, make_float2(fmaf(-a, dn.x, v.x), fmaf(-a, dn.y, v.y)));
                Sv[t] = make_float2(u.x - v.x, u.y - v.y);
                Gp[t] = G[t];
                Vw[t] = u;
            }
            __syncwarp();
            P0 = best_P;
            have_step = true;
        }
        if (lane == 0) {
            if (mrow)
                for (int i = it; i <= n_iters; ++i) mrow[i] = P0;
            if (iters_out) iters_out[q] = it;
            if (stalled) atomicOr(status, SMPPI_DEV_STALLED);
            if (!isfinite(P0)) atomicOr(status, SMPPI_DEV_NUMERIC);
        }
        float2* vout = reinterpret_cast<float2*>(Vout) + (size_t)q * T;
        for (int t = lane; t < T; t += 32) vout[t] = Vw[t];
        if (q == 0 && lane == 0 && ap.x0) closed_loop_step(P, ap, Vw[0]);
        __syncwarp();   // the warp's shared memory is reused by its next sequence
    }
}

namespace {

const void* bfgs_kernel(const DevParams& P) {
    return (P.tyre15 && P.steer_small) ? (const void*)repair_bfgs_kernel<true>
                                       : (const void*)repair_bfgs_kernel<false>;
}

// Warps per block: as many as fit next to the track table (at most BFGS_WPB_MAX).
int bfgs_wpb(const DevParams& P) {
    int dev = 0, max_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t track = rec_table_bytes(P.n_track), per = bfgs_warp_bytes(P.T);
    if ((size_t)max_optin < track + per) return 0;
    return (int)std::min<size_t>(BFGS_WPB_MAX, ((size_t)max_optin - track) / per);
}

}  // namespace

// Launch shape of the BFGS repair: blocks of `wpb` warps, as many blocks as
// are resident, no more warps than sequences, and few enough warp slots that
// their H slices fit in BFGS_WS_MAX.  Returns the block count (0: no fit).
int bfgs_grid(const DevParams& P, int n_seq, int sms, int* wpb_out) {
    const int wpb = bfgs_wpb(P);
    if (wpb < 1) return 0;
    const size_t smem = rec_table_bytes(P.n_track) + (size_t)wpb * bfgs_warp_bytes(P.T);
    const void* kern = bfgs_kernel(P);
    if (ensure_smem(kern, smem) != cudaSuccess) return 0;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, 32 * wpb, smem) != cudaSuccess)
        return 0;
    const size_t n = 2 * (size_t)P.N_r;
    const size_t per = std::max<size_t>(1, n * n * sizeof(float));
    const int by_ws = (int)std::max<size_t>(1, BFGS_WS_MAX / per / wpb);
    const int by_seq = (n_seq + wpb - 1) / wpb;
    if (wpb_out) *wpb_out = wpb;
    return std::max(1, std::min({by_seq, std::max(1, bps) * sms, by_ws}));
}

// Workspace: a 16-byte work counter, then one H slice per warp slot.
size_t bfgs_ws_bytes(const DevParams& P, int grid, int wpb) {
    const size_t n = 2 * (size_t)P.N_r;
    return 16 + (size_t)grid * wpb * n * n * sizeof(float);
}

cudaError_t launch_repair_bfgs(const DevParams& P, const float4* rec, int n_seq, const float* x0,
                               const float* V_in, float* V_out, int n_iters, int ck, void* ws,
                               int grid, int wpb, double* merit_out, int* iters_out,
                               const ApplyArgs& ap, unsigned* status, cudaStream_t st) {
    const size_t smem = rec_table_bytes(P.n_track) + (size_t)wpb * bfgs_warp_bytes(P.T);
    const void* kern = bfgs_kernel(P);
    cudaError_t e = ensure_smem(kern, smem);
    if (e != cudaSuccess) return e;
    unsigned* next = static_cast<unsigned*>(ws);
    float* H = reinterpret_cast<float*>(static_cast<unsigned char*>(ws) + 16);
    e = cudaMemsetAsync(next, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    if (P.tyre15 && P.steer_small)
        repair_bfgs_kernel<true><<<grid, 32 * wpb, smem, st>>>(P, rec, x0, V_in, V_out, n_seq, n_iters,
                                                                ck, H, next, merit_out, iters_out, ap,
                                                                status);
    else
        repair_bfgs_kernel<false><<<grid, 32 * wpb, smem, st>>>(P, rec, x0, V_in, V_out, n_seq, n_iters,
                                                                 ck, H, next, merit_out, iters_out, ap,
                                                                 status);
    return cudaGetLastError();
}

}  // namespace smppi
