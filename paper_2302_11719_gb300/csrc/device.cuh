// Device building blocks of the Shield-MPPI hot path (sm_103a, FP32 SIMT).
//
// Method: arXiv 2302.11719.  Vehicle model x_{k+1} = f(x_k, u_k) (Eq. 1) is the
// dynamic single-track car with static axle loads and Fy = Fz sin(C atan(B a))
// tyres, integrated by explicit Euler; safe set h = w^2 - e_y^2 (Eq. 23);
// running cost q (Eq. 24-25); DCBF penalty C max{(1-alpha) h_{k-1} - h_k, 0}
// (Eq. 17, alpha = the paper's beta of Eq. 15).  No tensor cores: nothing here
// is a dense contraction; the hot loop is FP32 FMA/ALU/SFU work in registers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/smppi.h"

namespace smppi {

// Parameters as the kernels use them (derived once on the host).
struct DevParams {
    float lf, lr, B, Ct, Fzf, Fzr, fx_gain, m_inv, Iz_inv, dt;
    float sig0, sig1;            // noise std
    float gis0, gis1;            // gamma / sigma^2 (control term of Alg. 2)
    float lam_inv;               // 1 / lambda
    float one_m_alpha, C_cbf;    // (1 - alpha), C
    float q_v, v_target, qd_w2, C_obs, w2;
    float umin0, umin1, umax0, umax1;
    float dsig0, dsig1;          // disturbance std on (v_y, r)
    float ls_s0, ls_c;
    int ls_max;
    int K, T, N_r, n_track;
    uint32_t key0, key1;
};

struct State {
    float vx, vy, r, X, Y, psi;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of
//   (c0..c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// (m + 1/2) 2^-23 with m = x >> 9: exact in float32, in (0, 1).
__device__ __forceinline__ float u01(uint32_t x) {
    return fmaf(__uint2float_rn(x >> 9), 0x1p-23f, 0x1p-24f);
}

// Box-Muller pair (library logf / sqrtf / sincospif).
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b) {
    const float r = sqrtf(-2.0f * logf(u01(a)));
    float s, c;
    sincospif(2.0f * u01(b), &s, &c);
    return make_float2(r * c, r * s);
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) {
    return fminf(fmaxf(v, lo), hi);
}

// ---------------------------------------------------------------------------
// One explicit Euler step of the single-track model (Eq. 1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void model_step(const DevParams& P, State& x, float d, float a) {
    const float bf = atan2f(fmaf(P.lf, x.r, x.vy), x.vx);
    const float br = atan2f(fmaf(-P.lr, x.r, x.vy), x.vx);
    const float Fyf = P.Fzf * sinf(P.Ct * atanf(P.B * (d - bf)));
    const float Fyr = P.Fzr * sinf(P.Ct * atanf(P.B * (-br)));
    float sd, cd, sp, cp;
    sincosf(d, &sd, &cd);
    sincosf(x.psi, &sp, &cp);
    const float Fx = P.fx_gain * a;
    const float dvx = fmaf(Fx - Fyf * sd, P.m_inv, x.vy * x.r);
    const float dvy = fmaf(Fyr + Fyf * cd, P.m_inv, -x.vx * x.r);
    const float dr = (P.lf * Fyf * cd - P.lr * Fyr) * P.Iz_inv;
    const float dX = x.vx * cp - x.vy * sp;
    const float dY = x.vx * sp + x.vy * cp;
    const float dpsi = x.r;
    x.vx = fmaf(P.dt, dvx, x.vx);
    x.vy = fmaf(P.dt, dvy, x.vy);
    x.r = fmaf(P.dt, dr, x.r);
    x.X = fmaf(P.dt, dX, x.X);
    x.Y = fmaf(P.dt, dY, x.Y);
    x.psi = fmaf(P.dt, dpsi, x.psi);
}

// Reverse-mode adjoint of model_step at (x, d, a): given lb = dJ/dx_{t+1},
// overwrite lb with dJ/dx_t through the dynamics and return dJ/du_t in
// (*gd, *ga).  Hand-derived from the forward formulas above.
__device__ __forceinline__ void model_step_adjoint(const DevParams& P, const State& x, float d,
                                                   float a, State& lb, float* gd, float* ga) {
    (void)a;
    const float yf = fmaf(P.lf, x.r, x.vy), yr = fmaf(-P.lr, x.r, x.vy);
    const float bf = atan2f(yf, x.vx), br = atan2f(yr, x.vx);
    const float af = d - bf, ar = -br;
    const float phf = atanf(P.B * af), phr = atanf(P.B * ar);
    float sphf, cphf, sphr, cphr;
    sincosf(P.Ct * phf, &sphf, &cphf);
    sincosf(P.Ct * phr, &sphr, &cphr);
    const float Fyf = P.Fzf * sphf;
    (void)sphr;
    float sd, cd, sp, cp;
    sincosf(d, &sd, &cd);
    sincosf(x.psi, &sp, &cp);
    const float dX = x.vx * cp - x.vy * sp;
    const float dY = x.vx * sp + x.vy * cp;

    const float gvx = P.dt * lb.vx, gvy = P.dt * lb.vy, gr = P.dt * lb.r;
    const float gX = P.dt * lb.X, gY = P.dt * lb.Y, gpsi = P.dt * lb.psi;
    State o = lb;  // identity part of x + dt F
    // kinematics
    o.vx += gX * cp + gY * sp;
    o.vy += gY * cp - gX * sp;
    o.psi += gY * dX - gX * dY;
    o.r += gpsi;
    // dvx = (Fx - Fyf sd)/m + vy r
    float Fxb = gvx * P.m_inv;
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
    // tyres: Fy = Fz sin(Ct atan(B alpha))
    const float afb = Fyfb * P.Fzf * P.Ct * cphf * P.B / fmaf(P.B * af, P.B * af, 1.0f);
    const float arb = Fyrb * P.Fzr * P.Ct * cphr * P.B / fmaf(P.B * ar, P.B * ar, 1.0f);
    db += afb;
    const float bfb = -afb, brb = -arb;
    // slip: b = atan2(y, vx): db/dy = vx / (vx^2 + y^2), db/dvx = -y / (vx^2 + y^2)
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

// ---------------------------------------------------------------------------
// Track: closed polyline, segment i = (A_i, D_i = A_{i+1} - A_i) plus 1/|D_i|^2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float seg_d2(const float4* __restrict__ seg,
                                        const float* __restrict__ inv, int i, float X, float Y) {
    const float4 s = seg[i];
    const float ex = X - s.x, ey = Y - s.y;
    const float tau = __saturatef(fmaf(ex, s.z, ey * s.w) * inv[i]);
    const float rx = fmaf(-tau, s.z, ex), ry = fmaf(-tau, s.w, ey);
    return fmaf(rx, rx, ry * ry);
}

// Offset vector from the nearest point of segment i to (X, Y); d(e_y^2)/d(X,Y) = 2 r.
__device__ __forceinline__ float2 seg_offset(const float4* __restrict__ seg,
                                             const float* __restrict__ inv, int i, float X,
                                             float Y) {
    const float4 s = seg[i];
    const float ex = X - s.x, ey = Y - s.y;
    const float tau = __saturatef(fmaf(ex, s.z, ey * s.w) * inv[i]);
    return make_float2(fmaf(-tau, s.z, ex), fmaf(-tau, s.w, ey));
}

// Continuous tracking of the nearest segment: walk forward while the next
// segment is strictly closer, else backward while the previous one is.
__device__ __forceinline__ int track_follow(const float4* __restrict__ seg,
                                            const float* __restrict__ inv, int n, int s, float X,
                                            float Y, float& d2) {
    float d = seg_d2(seg, inv, s, X, Y);
    int nx = (s + 1 == n) ? 0 : s + 1;
    float dn = seg_d2(seg, inv, nx, X, Y);
    if (dn < d) {
        for (int it = 0; it < n && dn < d; ++it) {
            s = nx;
            d = dn;
            nx = (s + 1 == n) ? 0 : s + 1;
            dn = seg_d2(seg, inv, nx, X, Y);
        }
    } else {
        int pv = (s == 0) ? n - 1 : s - 1;
        float dp = seg_d2(seg, inv, pv, X, Y);
        for (int it = 0; it < n && dp < d; ++it) {
            s = pv;
            d = dp;
            pv = (s == 0) ? n - 1 : s - 1;
            dp = seg_d2(seg, inv, pv, X, Y);
        }
    }
    d2 = d;
    return s;
}

// Running cost q (Eq. 24-25) given e_y^2.
__device__ __forceinline__ float run_cost(const DevParams& P, float vx, float d2) {
    const float ev = vx - P.v_target;
    float q = fmaf(P.q_v * ev, ev, P.qd_w2 * d2);
    if (d2 > P.w2) q += P.C_obs;
    return q;
}

// DCBF violation (1 - alpha) h_prev - h (penalty C max(., 0), Eq. 17).
__device__ __forceinline__ float cbf_arg(const DevParams& P, float h_prev, float h) {
    return fmaf(P.one_m_alpha, h_prev, -h);
}

// Warp-level argmin of (d2, index) with lowest index on ties.
__device__ __forceinline__ void warp_argmin(float& d, int& i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float od = __shfl_xor_sync(0xffffffffu, d, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (od < d || (od == d && oi < i)) {
            d = od;
            i = oi;
        }
    }
}

}  // namespace smppi
