// BFGS repair of one sequence on one warp: the solver Sec. IV-B names for the
// local problem of Eq. 22, run for a fixed number of iterations.  The variant
// (box projection, Armijo on the projected path, binding coordinates held,
// gradient-step restarts) is stated with smppi_repair's mode 2 in smppi.h.
// Shared by the kernels of the two state kinds (bfgs.cu: Cartesian state,
// curv_repair.cu: curvilinear state); what differs between them is the merit,
// supplied as an object with
//   double merit(P, Vw)                         lane 0: P(Vw)
//   void   grad(P, Vw, G, have_tape)            all lanes: G = dP/dV at Vw, 0 past
//                                               N_r and for controls outside the box
//                                               (have_tape: the warp's tape already
//                                               holds Vw's trajectory)
//   double trial(P, Vw, G, Dn, a, &dec, keep)   any lane: P(u), u = clip(Vw - a Dn),
//                                               dec = G . (Vw - u); keep: leave u's
//                                               trajectory on the warp's tape
// merit() leaves Vw's trajectory on the tape too.
//
// The warp computes the gradient (lane 0 the forward pass, unless the tape
// already holds the iterate's trajectory, and the adjoint recursion; the lanes
// the coefficients of the steps' adjoint maps), the lanes evaluate the
// line-search trials a = 1, 1/2, ... in parallel (the largest accepted a is
// taken: the same iterate as sequential backtracking), and the products with H
// (n = 2 N_r) are spread over the lanes.
//
// The warp's slice of a global workspace (n^2 floats) holds, when they fit
// (2 n_iters (n + 1) <= n^2, as for any n_iters <= n/2 - 1), the curvature
// pairs since the last restart and H's products are formed from them by the
// two-loop recursion (lm_product; equal to the dense update's in exact
// arithmetic, O(k n) instead of O(n^2) per iteration).  Otherwise it holds H
// itself: the update is evaluated in a form that is symmetric in (i, j)
// operation by operation (no fused multiply-add), so H stays exactly
// symmetric; products with H then read it by columns, H[j][i] = H[i][j], so
// that the lanes' loads of one j coalesce.
#pragma once

#include "shield.cuh"

namespace smppi {

constexpr int BFGS_WPB_MAX = 4;                      // warps (sequences) per block
constexpr size_t BFGS_WS_MAX = size_t(256) << 20;    // bytes of H slices at most
constexpr int BFGS_ROWS = 8;                         // rows per lane per pass of a product
constexpr int BFGS_COLS = 8;                         // columns of H read at once by a product
constexpr int BFGS_UPD = 4;                          // rows of H read at once by the update

namespace {

__device__ __forceinline__ double bfgs_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// out_i = sum_j H_ji x_j (= (H x)_i, H symmetric) for i < n, lanes over i;
// with mask, only the flagged rows and columns (other rows give 0).  The
// columns are read BFGS_COLS at a time, all their loads issued before the
// products, which are then added in column order (H is in global memory: one
// column at a time would wait for each load in turn).
__device__ __forceinline__ void warp_symv(const float* __restrict__ H, const float* x, int n,
                                          const unsigned char* mask, float* out) {
    const int lane = threadIdx.x & 31;
    for (int i0 = lane; i0 < n; i0 += 32 * BFGS_ROWS) {
        float acc[BFGS_ROWS];
#pragma unroll
        for (int r = 0; r < BFGS_ROWS; ++r) acc[r] = 0.0f;
        for (int j0 = 0; j0 < n; j0 += BFGS_COLS) {
            float h[BFGS_COLS][BFGS_ROWS];
#pragma unroll
            for (int u = 0; u < BFGS_COLS; ++u) {
                const int j = j0 + u;
                const bool use = j < n && (!mask || mask[j]);   // the same j on every lane
                const float* col = H + (size_t)j * n;
#pragma unroll
                for (int r = 0; r < BFGS_ROWS; ++r) {
                    const int i = i0 + 32 * r;
                    h[u][r] = (use && i < n) ? __ldcg(col + i) : 0.0f;
                }
            }
#pragma unroll
            for (int u = 0; u < BFGS_COLS; ++u) {
                const int j = j0 + u;
                if (j < n && (!mask || mask[j])) {
                    const float xj = x[j];
#pragma unroll
                    for (int r = 0; r < BFGS_ROWS; ++r)
                        if (i0 + 32 * r < n) acc[r] = fmaf(h[u][r], xj, acc[r]);
                }
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

__device__ __forceinline__ float bfgs_warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Dn = P_F H P_F g for the H that k inverse updates with the stored pairs
// (s_i, y_i, rho_i = 1/(y_i's_i)), oldest first, make of h0 I: the two-loop
// recursion (equal to the dense update's product in exact arithmetic).  S, Y: k
// rows of n floats; rho, alpha: k floats; q: n floats of scratch (shared); fr:
// the free coordinates.  All lanes; the dot products by the warp's butterfly.
__device__ __forceinline__ void lm_product(const float* S, const float* Y, const float* rho,
                                           float* alpha, int k, float h0, int n, const float* g,
                                           const unsigned char* fr, float* q, float* dn) {
    const int lane = threadIdx.x & 31;
    for (int j = lane; j < n; j += 32) q[j] = fr[j] ? g[j] : 0.0f;
    __syncwarp();
    for (int i = k - 1; i >= 0; --i) {
        const float* si = S + (size_t)i * n;
        const float* yi = Y + (size_t)i * n;
        float d = 0.0f;
        for (int j = lane; j < n; j += 32) d = fmaf(__ldcg(si + j), q[j], d);
        const float a = rho[i] * bfgs_warp_sumf(d);
        if (lane == 0) alpha[i] = a;
        for (int j = lane; j < n; j += 32) q[j] = fmaf(-a, __ldcg(yi + j), q[j]);
        __syncwarp();
    }
    for (int j = lane; j < n; j += 32) q[j] *= h0;
    __syncwarp();
    for (int i = 0; i < k; ++i) {
        const float* si = S + (size_t)i * n;
        const float* yi = Y + (size_t)i * n;
        float d = 0.0f;
        for (int j = lane; j < n; j += 32) d = fmaf(__ldcg(yi + j), q[j], d);
        const float c = alpha[i] - rho[i] * bfgs_warp_sumf(d);
        for (int j = lane; j < n; j += 32) q[j] = fmaf(c, __ldcg(si + j), q[j]);
        __syncwarp();
    }
    for (int j = lane; j < n; j += 32) dn[j] = fr[j] ? q[j] : 0.0f;
    __syncwarp();
}

// The warp's working arrays for horizon T: five float2 arrays of T, two float
// arrays of 2T and 2T flag bytes (padded to 16 bytes).
struct BfgsArrays {
    float2* Vw;          // iterate z (first N_r controls; the rest are carried)
    float2* G;           // gradient at z
    float2* Gp;          // gradient at the previous z
    float2* Sv;          // last step s = z' - z
    float2* Dn;          // negated direction
    float* Yv;           // y = g - g_prev (n)
    float* Hy;           // H y (n)
    unsigned char* fr;   // free coordinate flags (n)
};

__host__ __device__ inline size_t bfgs_array_bytes(int T) {
    const size_t t = (size_t)T;
    return 5 * t * 8 + 2 * t * 8 + ((2 * t + 15) & ~size_t(15));
}

__device__ __forceinline__ BfgsArrays bfgs_arrays(unsigned char* base, int T) {
    BfgsArrays a;
    a.Vw = reinterpret_cast<float2*>(base);
    a.G = a.Vw + T;
    a.Gp = a.G + T;
    a.Sv = a.Gp + T;
    a.Dn = a.Sv + T;
    a.Yv = reinterpret_cast<float*>(a.Dn + T);
    a.Hy = a.Yv + 2 * T;
    a.fr = reinterpret_cast<unsigned char*>(a.Hy + 2 * T);
    return a;
}

// Runs up to n_iters BFGS iterations on a.Vw (all lanes of the warp).  mrow:
// P before each iteration and after the last (n_iters + 1 values, repeated
// after an early stop) or null.  Returns the iterations run; *P_out is the
// final merit on every lane, *stalled_out whether the search gave up (no
// accepted step, or a zero gradient with P > 0).
template <class Merit>
__device__ __forceinline__ int bfgs_solve(const DevParams& P, const Merit& f, const BfgsArrays& a,
                                          float* __restrict__ H, int n_iters, double* mrow,
                                          double* P_out, bool* stalled_out) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, N = P.N_r, n = 2 * N;
    const float* zf = reinterpret_cast<const float*>(a.Vw);
    const float* gf = reinterpret_cast<const float*>(a.G);
    const float* gpf = reinterpret_cast<const float*>(a.Gp);
    const float* sf = reinterpret_cast<const float*>(a.Sv);
    float* dnf = reinterpret_cast<float*>(a.Dn);
    double P0 = 0.0;
    if (lane == 0) P0 = f.merit(P, a.Vw);
    P0 = __shfl_sync(FULL, P0, 0);
    bool H_set = false, have_step = false, stalled = false;
    // limited-memory form when the pairs fit in the H slice (at most n_iters of
    // them): S, Y (n_iters rows of n), then rho and alpha (n_iters each)
    const bool lm = (size_t)2 * n_iters * (n + 1) <= (size_t)n * n;
    float* S_st = H;
    float* Y_st = H + (size_t)n_iters * n;
    float* rho_st = H + (size_t)2 * n_iters * n;
    float* alpha_st = rho_st + n_iters;
    int lm_k = 0;
    float lm_h0 = 0.0f;
    // the tape holds the current iterate's trajectory (left by the merit, or by
    // the full-step trial of lane 0 when that step was taken)
    bool traj_ok = true;
    int it = 0;
    for (; it < n_iters; ++it) {
        if (lane == 0 && mrow) mrow[it] = P0;
        if (P0 == 0.0) break;
        f.grad(P, a.Vw, a.G, traj_ok);
        __syncwarp();
        // curvature pair of the last accepted step and the inverse update
        //   H <- (I - rho s y') H (I - rho y s') + rho s s'
        //      = H - rho (s (Hy)' + (Hy) s') + (rho^2 y'Hy + rho) s s'   (H symmetric)
        if (have_step) {
            double sy = 0.0, yy = 0.0, ss = 0.0;
            for (int i = lane; i < n; i += 32) {
                const float y = gf[i] - gpf[i];
                a.Yv[i] = y;
                sy += (double)sf[i] * y;
                yy += (double)y * y;
                ss += (double)sf[i] * sf[i];
            }
            sy = bfgs_warp_sum(sy);
            yy = bfgs_warp_sum(yy);
            ss = bfgs_warp_sum(ss);
            __syncwarp();
            if (lm && sy > 1e-5 * sqrt(ss * yy)) {   // store the pair
                if (!H_set) {
                    lm_h0 = (float)(sy / yy);
                    lm_k = 0;
                    H_set = true;
                }
                for (int i = lane; i < n; i += 32) {
                    S_st[(size_t)lm_k * n + i] = sf[i];
                    Y_st[(size_t)lm_k * n + i] = a.Yv[i];
                }
                if (lane == 0) rho_st[lm_k] = (float)(1.0 / sy);
                ++lm_k;
                __syncwarp();
            } else if (sy > 1e-5 * sqrt(ss * yy)) {
                if (!H_set) {
                    const float h0 = (float)(sy / yy);
                    for (int i = 0; i < n; ++i)
                        for (int j = lane; j < n; j += 32) H[(size_t)i * n + j] = i == j ? h0 : 0.0f;
                    __syncwarp();
                    H_set = true;
                }
                warp_symv(H, a.Yv, n, nullptr, a.Hy);
                double yHy = 0.0;
                for (int i = lane; i < n; i += 32) yHy += (double)a.Yv[i] * a.Hy[i];
                yHy = bfgs_warp_sum(yHy);
                const float rho = (float)(1.0 / sy);
                const float cs = (float)(yHy / (sy * sy) + 1.0 / sy);
                // by column chunks of 32 BFGS_ROWS (s_j and (Hy)_j of a lane's columns held
                // in registers) and BFGS_UPD rows at a time, all loads of H first
                for (int c0 = lane; c0 < n; c0 += 32 * BFGS_ROWS) {
                    float sj[BFGS_ROWS], hyj[BFGS_ROWS];
#pragma unroll
                    for (int u = 0; u < BFGS_ROWS; ++u) {
                        const int j = c0 + 32 * u;
                        sj[u] = j < n ? sf[j] : 0.0f;
                        hyj[u] = j < n ? a.Hy[j] : 0.0f;
                    }
                    for (int i0 = 0; i0 < n; i0 += BFGS_UPD) {
                        float hk[BFGS_UPD][BFGS_ROWS];
#pragma unroll
                        for (int v = 0; v < BFGS_UPD; ++v)
#pragma unroll
                            for (int u = 0; u < BFGS_ROWS; ++u) {
                                const int i = i0 + v, j = c0 + 32 * u;
                                hk[v][u] = (i < n && j < n) ? __ldcg(H + (size_t)i * n + j) : 0.0f;
                            }
#pragma unroll
                        for (int v = 0; v < BFGS_UPD; ++v) {
                            const int i = i0 + v;
                            if (i < n) {
                                const float si = sf[i], hyi = a.Hy[i];
#pragma unroll
                                for (int u = 0; u < BFGS_ROWS; ++u) {
                                    const int j = c0 + 32 * u;
                                    if (j < n) {
                                        const float cross = __fadd_rn(__fmul_rn(si, hyj[u]),
                                                                      __fmul_rn(sj[u], hyi));
                                        const float delta =
                                            __fsub_rn(__fmul_rn(cs, __fmul_rn(si, sj[u])),
                                                      __fmul_rn(rho, cross));
                                        H[(size_t)i * n + j] = __fadd_rn(hk[v][u], delta);
                                    }
                                }
                            }
                        }
                    }
                }
                __syncwarp();
            }
        }
        // |g|_inf and the binding coordinates (at a bound, gradient pushing outward)
        float gm = 0.0f;
        for (int i = lane; i < n; i += 32) {
            const float g = gf[i], z = zf[i];
            const float lo = (i & 1) ? P.umin1 : P.umin0, hi = (i & 1) ? P.umax1 : P.umax0;
            a.fr[i] = !((z <= lo && g > 0.0f) || (z >= hi && g < 0.0f));
            gm = fmaxf(gm, fabsf(g));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(FULL, gm, o));
        __syncwarp();
        if (!(gm > 0.0f)) { stalled = true; break; }
        const float s_first = P.ls_s0 / gm;
        // direction (negated): Dn = H_FF g_F, or the scaled gradient step
        if (H_set) {
            if (lm) lm_product(S_st, Y_st, rho_st, alpha_st, lm_k, lm_h0, n, gf, a.fr, a.Hy, dnf);
            else warp_symv(H, gf, n, a.fr, dnf);
            double gHg = 0.0;
            for (int i = lane; i < n; i += 32) gHg += (double)gf[i] * dnf[i];
            gHg = bfgs_warp_sum(gHg);
            if (!(gHg > 0.0)) H_set = false;      // g'd = -g'Dn >= 0: not a descent direction
        }
        if (!H_set) {
            for (int i = lane; i < n; i += 32) dnf[i] = a.fr[i] ? s_first * gf[i] : 0.0f;
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
                double dec;
                const double Pt = f.trial(P, a.Vw, a.G, a.Dn, ldexpf(1.0f, -j), &dec, j == 0);
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
            for (int i = lane; i < n; i += 32) dnf[i] = a.fr[i] ? s_first * gf[i] : 0.0f;
            __syncwarp();
        }
        if (bj == 0x7fffffff) { stalled = true; break; }
        traj_ok = bj == 0;   // the full step's trial trajectory is the new iterate's
        const float al = ldexpf(1.0f, -bj);
        for (int t = lane; t < N; t += 32) {
            const float2 v = a.Vw[t], dn = a.Dn[t];
            const float2 u = clamp2(P, make_float2(fmaf(-al, dn.x, v.x), fmaf(-al, dn.y, v.y)));
            a.Sv[t] = make_float2(u.x - v.x, u.y - v.y);
            a.Gp[t] = a.G[t];
            a.Vw[t] = u;
        }
        __syncwarp();
        P0 = best_P;
        have_step = true;
    }
    if (lane == 0 && mrow)
        for (int i = it; i <= n_iters; ++i) mrow[i] = P0;
    *P_out = P0;
    *stalled_out = stalled;
    return it;
}

}  // namespace
}  // namespace smppi
