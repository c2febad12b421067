// Device building blocks of the Shield-MPPI hot path (sm_103a, FP32 SIMT).
//
// Method: arXiv 2302.11719.  Vehicle model x_{k+1} = f(x_k, u_k) (Eq. 1) is the
// dynamic single-track car with static axle loads and Fy = Fz sin(C atan(B a))
// tyres, integrated by explicit Euler; safe set h = w^2 - e_y^2 (Eq. 23);
// running cost q (Eq. 24-25); DCBF penalty C max{(1-alpha) h_{k-1} - h_k, 0}
// (Eq. 17, alpha = the paper's beta of Eq. 15).  No tensor cores: nothing here
// is a dense contraction; the hot loop is FP32 FMA/ALU/SFU work in registers.
//
// Elementary functions on the hot path are written here so that each step
// costs few instructions while staying within a few ulp (measured on dense grids
// against float64: atan2 <= 3.8 ulp, the C = 1.5 tyre <= 5.0 ulp, the short
// sin / cos <= 0.8 ulp):
//   atan2   -- octant reduction + a degree-8 polynomial in a^2 for atan(a)/a on
//              [0, 1]: the minimax fit (Remez exchange, absolute error of
//              atan(a) = a p(a^2)) of csrc/atan_minimax.py: 5.8e-9 with exact
//              coefficients, 2.2e-8 with the float32 ones below (ATAN_P0..8);
//              valid for finite arguments with max(|x|, |y|) below 2^126;
//   tyre    -- for C = 1.5, sin(1.5 atan z) by the half-angle identities
//              cos t = 1/sqrt(1+z^2), sin(3t/2) = sin t cos(t/2) + cos t sin(t/2)
//              (no atan, no sin); other C use the library atanf / sinf;
//   heading -- (cos psi, sin psi) is carried with the state and rotated by the
//              Euler increment dt r each step (exactly cos / sin of the Euler
//              psi up to rounding), so no sin / cos of an unbounded angle;
//   small sin / cos -- Taylor series to x^9 / x^10 for |x| <= 1/2 (remainder
//              < 1.2e-11), the library otherwise.
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
    float w_skip;                // weights <= w_skip are left out of the noise sum (<= 1e-8 on V+)
    float one_m_alpha, C_cbf;    // (1 - alpha), C
    float q_v, v_target, qd_w2, C_obs, w2;
    float umin0, umin1, umax0, umax1;
    float dsig0, dsig1;          // disturbance std on (v_y, r)
    float ls_s0, ls_c;
    int ls_max;
    int K, T, N_r, n_track;
    int tyre15;                  // 1 when Ct == 1.5 (half-angle tyre path)
    int steer_small;             // 1 when |steer| <= 1/2 on the whole control box
    uint32_t key0, key1;
    uint32_t rk0[10], rk1[10];   // Philox round keys key + i * Weyl
    // curvilinear state (state_kind 1): x = (v_x, v_y, r, s, e_y, e_psi) held in
    // State's (vx, vy, r, X, Y, psi) with (cp, sp) = (cos, sin) e_psi; the
    // curvature samples are passed to the kernels that need them (a pointer
    // member here would change the register allocation of every kernel)
    int state_kind;
    float kap_scale;             // n_track / L
    float track_len, inv_len;    // L, 1 / L
};

struct State {
    float vx, vy, r, X, Y, psi;
    float cp, sp;                // cos psi, sin psi
};

__device__ __forceinline__ State make_state(const float* x) {
    State s;
    s.vx = x[0]; s.vy = x[1]; s.r = x[2]; s.X = x[3]; s.Y = x[4]; s.psi = x[5];
    sincosf(s.psi, &s.sp, &s.cp);
    return s;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of
//   (c0..c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with the key bumped by the Weyl constants between rounds (round keys are
// precomputed on the host: rk[i] = key + i W).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, const DevParams& P) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        // one 32 x 32 -> 64-bit product gives both halves
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ P.rk0[i], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ P.rk1[i], (uint32_t)p0);
    }
    return c;
}

// (m + 1/2) 2^-23 with m = x >> 9: exact in float32, in (0, 1).
__device__ __forceinline__ float u01(uint32_t x) {
    return fmaf(__uint2float_rn(x >> 9), 0x1p-23f, 0x1p-24f);
}

// 1 / sqrt(x) by the SFU approximation without the denormal path
// (rsqrt.approx.ftz.f32), for arguments that cannot be denormal: for a normal
// x > 0 it is rsqrtf(x) bit for bit (tests/test_gpu_elementary.py checks every
// float in [1/2, 2) and samples of every binade), at about half the latency.
__device__ __forceinline__ float rsqrt_n(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Box-Muller pair (library logf and sincospif; r = sqrt(q) as q rsqrt(q), with
// q = -2 ln u in [1.2e-7, 33.3] for the u of u01).
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b) {
    const float q = -2.0f * logf(u01(a));
    const float r = q * rsqrt_n(q);
    float s, c;
    sincospif(2.0f * u01(b), &s, &c);
    return make_float2(r * c, r * s);
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) {
    return fminf(fmaxf(v, lo), hi);
}

// atan(a) ~ a p(a^2) on [0, 1]: the coefficients of p, highest degree first
// (csrc/atan_minimax.py prints them; a CPU test regenerates and compares them).
constexpr float ATAN_P8 = 2.456725575e-03f;
constexpr float ATAN_P7 = -1.440136135e-02f;
constexpr float ATAN_P6 = 3.978123143e-02f;
constexpr float ATAN_P5 = -7.234857976e-02f;
constexpr float ATAN_P4 = 1.049894616e-01f;
constexpr float ATAN_P3 = -1.416122913e-01f;
constexpr float ATAN_P2 = 1.998590678e-01f;
constexpr float ATAN_P1 = -3.333259821e-01f;
constexpr float ATAN_P0 = 9.999998808e-01f;

// atan2 by octant reduction and the minimax polynomial for atan(a)/a, a in [0, 1].
__device__ __forceinline__ float atan2_poly(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float a = mx > 0.0f ? __fdividef(mn, mx) : 0.0f;
    const float s = a * a;
    float p = ATAN_P8;
    p = fmaf(p, s, ATAN_P7);
    p = fmaf(p, s, ATAN_P6);
    p = fmaf(p, s, ATAN_P5);
    p = fmaf(p, s, ATAN_P4);
    p = fmaf(p, s, ATAN_P3);
    p = fmaf(p, s, ATAN_P2);
    p = fmaf(p, s, ATAN_P1);
    p = fmaf(p, s, ATAN_P0);
    float r = a * p;
    if (ay > ax) r = 1.57079632679f - r;
    if (x < 0.0f) r = 3.14159265359f - r;
    return copysignf(r, y);
}

// sin and cos of |x| <= 1/2 by Taylor series to x^9 / x^10 (remainders below
// 0.5^11 / 11! = 1.2e-11 and 0.5^12 / 12! = 5.1e-13).
__device__ __forceinline__ void sincos_half(float x, float* s, float* c) {
    const float x2 = x * x;
    float ps = 2.7557319223985893e-06f;              //  1/9!
    ps = fmaf(ps, x2, -1.9841269841269841e-04f);     // -1/7!
    ps = fmaf(ps, x2, 8.3333333333333333e-03f);      //  1/5!
    ps = fmaf(ps, x2, -1.6666666666666667e-01f);     // -1/3!
    *s = fmaf(ps * x2, x, x);
    float pc = -2.7557319223985891e-07f;             // -1/10!
    pc = fmaf(pc, x2, 2.4801587301587302e-05f);      //  1/8!
    pc = fmaf(pc, x2, -1.3888888888888889e-03f);     // -1/6!
    pc = fmaf(pc, x2, 4.1666666666666667e-02f);      //  1/4!
    pc = fmaf(pc, x2, -0.5f);                        // -1/2!
    *c = fmaf(pc, x2, 1.0f);
}

__device__ __forceinline__ void sincos_any(float x, float* s, float* c) {
    if (fabsf(x) <= 0.5f) sincos_half(x, s, c);
    else sincosf(x, s, c);
}

// ---------------------------------------------------------------------------
// Packed FP32 pairs (sm_100+: one FFMA2 / FADD2 / FMUL2 does the same IEEE
// operation on both halves of a register pair).
// ---------------------------------------------------------------------------
namespace x2 {

using f2 = float2;

__device__ __forceinline__ f2 bc(float v) { return make_float2(v, v); }
__device__ __forceinline__ f2 add(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 neg(f2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ f2 lo(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ f2 hi(float4 v) { return make_float2(v.z, v.w); }

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// atan2 of both halves: octant reduction and the degree-8 minimax polynomial
// of atan2_poly (ATAN_P0..8).  x = y = 0 gives 0 (mx is kept at or above the smallest
// normal float, so a = 0 there).
__device__ __forceinline__ f2 atan2_2(f2 y, f2 x) {
    const float ax0 = fabsf(x.x), ay0 = fabsf(y.x), ax1 = fabsf(x.y), ay1 = fabsf(y.y);
    const f2 mn = make_float2(fminf(ax0, ay0), fminf(ax1, ay1));
    const float mx0 = fmaxf(fmaxf(ax0, ay0), 1.17549435e-38f);
    const float mx1 = fmaxf(fmaxf(ax1, ay1), 1.17549435e-38f);
    const f2 a = mul(mn, make_float2(rcp_approx(mx0), rcp_approx(mx1)));
    const f2 s = mul(a, a);
    f2 p = fma(bc(ATAN_P8), s, bc(ATAN_P7));
    p = fma(p, s, bc(ATAN_P6));
    p = fma(p, s, bc(ATAN_P5));
    p = fma(p, s, bc(ATAN_P4));
    p = fma(p, s, bc(ATAN_P3));
    p = fma(p, s, bc(ATAN_P2));
    p = fma(p, s, bc(ATAN_P1));
    p = fma(p, s, bc(ATAN_P0));
    f2 r = mul(a, p);
    const f2 r1 = fma(r, bc(-1.0f), bc(1.57079632679f));
    r.x = (ay0 > ax0) ? r1.x : r.x;
    r.y = (ay1 > ax1) ? r1.y : r.y;
    const f2 r2 = fma(r, bc(-1.0f), bc(3.14159265359f));
    r.x = (x.x < 0.0f) ? r2.x : r.x;
    r.y = (x.y < 0.0f) ? r2.y : r.y;
    return make_float2(copysignf(r.x, y.x), copysignf(r.y, y.y));
}

// atan2 of both halves for one-thread recurrences, where the dependent chain
// rather than the instruction count sets the time: the polynomial of atan2_2
// by Estrin's scheme (depth 4 instead of 8, two more products), and the
// octant's fix-up folded into one FMA after it, atan2(y, x) = O + (S a) p(a^2)
// with the offset O in {0, pi/2, pi} and the sign S = +-1 (both carrying the
// sign of y) picked from the comparisons while the reciprocal is in flight.
// One rounding follows the polynomial (atan2_2 has up to three there).
__device__ __forceinline__ f2 atan2_2_lat(f2 y, f2 x) {
    const float ax0 = fabsf(x.x), ay0 = fabsf(y.x), ax1 = fabsf(x.y), ay1 = fabsf(y.y);
    const float mn0 = fminf(ax0, ay0), mn1 = fminf(ax1, ay1);
    const float mx0 = fmaxf(fmaxf(ax0, ay0), 1.17549435e-38f);
    const float mx1 = fmaxf(fmaxf(ax1, ay1), 1.17549435e-38f);
    const f2 rc = make_float2(rcp_approx(mx0), rcp_approx(mx1));
    // ay > ax reflects the result about pi/4 (pi/2 - r), x < 0 about pi/2 (pi - r)
    const bool sw0 = ay0 > ax0, sw1 = ay1 > ax1, ng0 = x.x < 0.0f, ng1 = x.y < 0.0f;
    const unsigned sy0 = __float_as_uint(y.x) & 0x80000000u;
    const unsigned sy1 = __float_as_uint(y.y) & 0x80000000u;
    const float o0 = sw0 ? 1.57079632679f : (ng0 ? 3.14159265359f : 0.0f);
    const float o1 = sw1 ? 1.57079632679f : (ng1 ? 3.14159265359f : 0.0f);
    const f2 O = make_float2(__uint_as_float(__float_as_uint(o0) | sy0),
                             __uint_as_float(__float_as_uint(o1) | sy1));
    const f2 mS = make_float2(
        __uint_as_float(__float_as_uint(mn0) ^ sy0 ^ (sw0 != ng0 ? 0x80000000u : 0u)),
        __uint_as_float(__float_as_uint(mn1) ^ sy1 ^ (sw1 != ng1 ? 0x80000000u : 0u)));
    const f2 a = mul(make_float2(mn0, mn1), rc);
    const f2 aS = mul(mS, rc);
    const f2 s = mul(a, a);
    const f2 s2 = mul(s, s), s4 = mul(s2, s2);
    const f2 q0 = fma(bc(ATAN_P1), s, bc(ATAN_P0));
    const f2 q1 = fma(bc(ATAN_P3), s, bc(ATAN_P2));
    const f2 q2 = fma(bc(ATAN_P5), s, bc(ATAN_P4));
    const f2 q3 = fma(bc(ATAN_P7), s, bc(ATAN_P6));
    const f2 lo4 = fma(q1, s2, q0);                             // P0 + .. + P3 s^3
    const f2 hi4 = fma(fma(bc(ATAN_P8), s2, q3), s2, q2);      // P4 + .. + P8 s^4
    return fma(aS, fma(hi4, s4, lo4), O);
}

// sin(1.5 atan z) of both halves (half-angle identities, as tyre15) as the
// product w ru, with t = atan z, c = cos t = 1 / sqrt(1 + z^2),
// u = cos^2(t/2) = (1 + c) / 2, ru = 1 / cos(t/2) and w = sin t (c/2 + u):
// sin t cos(t/2) + cos t sin(t/2) = (sin t / cos(t/2)) (cos^2(t/2) + cos t / 2).
// A caller can scale w while the second reciprocal square root is in flight.
// (q = 1 + z^2 >= 1 and u in [1/2, 1] are never denormal: rsqrt_n.)
__device__ __forceinline__ void tyre15_2_parts(f2 z, f2& w, f2& ru) {
    const f2 q = fma(z, z, bc(1.0f));
    const f2 c = make_float2(rsqrt_n(q.x), rsqrt_n(q.y));
    const f2 u = fma(bc(0.5f), c, bc(0.5f));
    ru = make_float2(rsqrt_n(u.x), rsqrt_n(u.y));
    w = mul(mul(z, c), fma(bc(0.5f), c, u));
}

__device__ __forceinline__ f2 tyre15_2(f2 z) {
    f2 w, ru;
    tyre15_2_parts(z, w, ru);
    return mul(w, ru);
}

}  // namespace x2

// sin(1.5 atan z) by the half-angle identities (no branch).
__device__ __forceinline__ float tyre15(float z) {
    const float c = rsqrt_n(fmaf(z, z, 1.0f));       // cos t, t = atan z
    const float u = fmaf(0.5f, c, 0.5f);             // cos^2(t/2)
    return z * c * rsqrt_n(u) * fmaf(0.5f, c, u);    // sin t cos(t/2) + cos t sin(t/2)
}

// Lateral tyre force shape sin(Ct atan(z)) and, if dz != nullptr, its
// derivative Ct cos(Ct atan z) / (1 + z^2).
__device__ __forceinline__ float tyre_shape(const DevParams& P, float z, float* dz) {
    if (P.tyre15) {
        const float c = rsqrt_n(fmaf(z, z, 1.0f));   // cos t, t = atan z
        const float s = z * c;                       // sin t
        const float u = fmaf(0.5f, c, 0.5f);         // cos^2(t/2)
        const float ru = rsqrt_n(u);                 // 1 / cos(t/2)
        if (dz) *dz = 1.5f * ru * fmaf(c, u, -0.5f * s * s) * c * c;   // 1.5 cos(1.5 t) cos^2 t
        return s * ru * fmaf(0.5f, c, u);            // sin t cos(t/2) + cos t sin(t/2)
    }
    const float t = atanf(z);
    float sn, cs;
    sincosf(P.Ct * t, &sn, &cs);
    if (dz) *dz = P.Ct * cs / fmaf(z, z, 1.0f);
    return sn;
}

// ---------------------------------------------------------------------------
// One explicit Euler step of the single-track model (Eq. 1).
// ---------------------------------------------------------------------------
// FAST: the parameters satisfy Ct == 1.5 and |steer| <= 1/2 on the control
// box (P.tyre15 && P.steer_small).  The FAST step is split into its velocity
// part (v_x, v_y, r: the tyre forces) and its pose part (X, Y, psi: driven by
// the velocities of the same step) so that the repair's merit pass can run the
// two recurrences on different threads; explicit fmaf fixes the rounding.
//
// Velocity part: (v_x, v_y, r) <- Euler update at steer d with throttle a.
// The per-step factors that depend on the control alone (vel_coef) are formed
// apart from the recurrence; the front and rear axle (slip angle, lateral force)
// run as the two halves of packed instructions (atan2_2_lat, tyre15_2_parts),
// and the lateral forces Fz w ru enter the update as (dt-scaled w) x ru, so
// that two FMAs follow the last reciprocal square root.  This step is the
// dependent chain of every one-thread recurrence (the merit pass, the repair's
// forward and adjoint sweeps).
struct VelCoef {
    float Bd;   // B d
    float kx;   // -dt Fzf sin(d) / m
    float ky;   //  dt Fzf cos(d) / m
    float kr;   //  dt lf Fzf cos(d) / Iz
    float bx;   //  dt fx_gain a / m
};

__device__ __forceinline__ VelCoef vel_coef(const DevParams& P, float d, float sd, float cd,
                                            float a) {
    const float gm = P.dt * P.Fzf * P.m_inv, gi = P.dt * P.lf * P.Fzf * P.Iz_inv;
    return VelCoef{P.B * d, -gm * sd, gm * cd, gi * cd, (P.dt * P.fx_gain * P.m_inv) * a};
}

__device__ __forceinline__ void vel_step_fast(const DevParams& P, float& vx, float& vy, float& r,
                                              const VelCoef& k) {
    const float2 b = x2::atan2_2_lat(make_float2(fmaf(P.lf, r, vy), fmaf(-P.lr, r, vy)),
                                     make_float2(vx, vx));
    float2 w, ru;
    x2::tyre15_2_parts(make_float2(fmaf(-P.B, b.x, k.Bd), -P.B * b.y), w, ru);
    const float gyr = P.dt * P.Fzr * P.m_inv, grr = -(P.dt * P.lr * P.Fzr * P.Iz_inv);
    // dv_x = (Fx - Fyf sin d) / m + v_y r, dv_y = (Fyf cos d + Fyr) / m - v_x r,
    // dr = (lf Fyf cos d - lr Fyr) / Iz, with Fy = Fz w ru
    // __fadd_rn: the product in bx is never contracted into this add, so a step
    // with vel_coef inline rounds as one with the factors read from memory
    const float bxv = fmaf(P.dt * vy, r, __fadd_rn(vx, k.bx));
    const float byv = fmaf(-(P.dt * vx), r, vy);
    vx = fmaf(w.x * k.kx, ru.x, bxv);
    vy = fmaf(w.x * k.ky, ru.x, fmaf(w.y * gyr, ru.y, byv));
    r = fmaf(w.x * k.kr, ru.x, fmaf(w.y * grr, ru.y, r));
}

// Pose part, from the velocities (vx, vy, r) of the same step: (X, Y) by Euler,
// psi += dt r and (cos psi, sin psi) rotated by dt r (library sin / cos when
// |dt r| > 1/2).
__device__ __forceinline__ void pose_step_fast(const DevParams& P, float vx, float vy, float r,
                                               float& X, float& Y, float& psi, float& cp,
                                               float& sp) {
    const float dX = fmaf(vx, cp, -(vy * sp));
    const float dY = fmaf(vx, sp, vy * cp);
    const float dpsi = P.dt * r;
    float sa, ca;
    sincos_half(dpsi, &sa, &ca);
    X = fmaf(P.dt, dX, X);
    Y = fmaf(P.dt, dY, Y);
    psi += dpsi;
    if (fabsf(dpsi) > 0.5f) sincosf(dpsi, &sa, &ca);
    const float cp0 = cp;
    cp = fmaf(cp, ca, -(sp * sa));
    sp = fmaf(sp, ca, cp0 * sa);
}

template <bool FAST = false>
__device__ __forceinline__ void model_step(const DevParams& P, State& x, float d, float a) {
    if (FAST) {
        float sd, cd;
        sincos_half(d, &sd, &cd);
        const float vx = x.vx, vy = x.vy, r = x.r;
        vel_step_fast(P, x.vx, x.vy, x.r, vel_coef(P, d, sd, cd, a));
        pose_step_fast(P, vx, vy, r, x.X, x.Y, x.psi, x.cp, x.sp);
        return;
    }
    const float bf = atan2_poly(fmaf(P.lf, x.r, x.vy), x.vx);
    const float br = atan2_poly(fmaf(-P.lr, x.r, x.vy), x.vx);
    const float Fyf = P.Fzf * tyre_shape(P, P.B * (d - bf), nullptr);
    const float Fyr = P.Fzr * tyre_shape(P, -P.B * br, nullptr);
    float sd, cd;
    if (P.steer_small) sincos_half(d, &sd, &cd);
    else sincosf(d, &sd, &cd);
    const float Fx = P.fx_gain * a;
    const float dvx = fmaf(Fx - Fyf * sd, P.m_inv, x.vy * x.r);
    const float dvy = fmaf(Fyr + Fyf * cd, P.m_inv, -x.vx * x.r);
    const float dr = (P.lf * Fyf * cd - P.lr * Fyr) * P.Iz_inv;
    const float dX = x.vx * x.cp - x.vy * x.sp;
    const float dY = x.vx * x.sp + x.vy * x.cp;
    // heading: psi += dt r, (cos, sin) rotated by the same increment
    const float dpsi = P.dt * x.r;
    float sa, ca;
    sincos_any(dpsi, &sa, &ca);
    const float cp = x.cp * ca - x.sp * sa;
    const float sp = x.sp * ca + x.cp * sa;
    x.vx = fmaf(P.dt, dvx, x.vx);
    x.vy = fmaf(P.dt, dvy, x.vy);
    x.r = fmaf(P.dt, dr, x.r);
    x.X = fmaf(P.dt, dX, x.X);
    x.Y = fmaf(P.dt, dY, x.Y);
    x.psi += dpsi;
    x.cp = cp;
    x.sp = sp;
}

// ---------------------------------------------------------------------------
// Curvilinear state (state_kind 1; smppi.h): x = (v_x, v_y, r, s, e_y, e_psi)
// in State's (vx, vy, r, X, Y, psi), (cp, sp) = (cos e_psi, sin e_psi).
// kappa(s) from the n_track + 1 samples (the last repeats the first), s taken
// modulo the track length L.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float kappa_at(const DevParams& P, const float* kt, float s) {
    const float sw = fmaf(floorf(s * P.inv_len), -P.track_len, s);
    const float x = sw * P.kap_scale;
    const int i = min(max((int)x, 0), P.n_track - 1);
    const float f = x - (float)i;
    const float k0 = kt[i], k1 = kt[i + 1];
    return fmaf(f, k1 - k0, k0);
}

// One explicit Euler step of the curvilinear model (C = 1.5, |steer| <= 1/2):
// the velocity part is the Cartesian model's; then
//   s' = (v_x cos e_psi - v_y sin e_psi) / max(1 - kappa e_y, 0.1),
//   e_y' = v_x sin e_psi + v_y cos e_psi,  e_psi' = r - kappa s',
// with (cos, sin) e_psi rotated by the increment dt e_psi'.
__device__ __forceinline__ void model_step_curv(const DevParams& P, const float* kt, State& x,
                                                float d, float a) {
    float sd, cd;
    sincos_half(d, &sd, &cd);
    const float vx = x.vx, vy = x.vy, r = x.r;
    vel_step_fast(P, x.vx, x.vy, x.r, vel_coef(P, d, sd, cd, a));
    const float k = kappa_at(P, kt, x.X);
    const float den = fmaxf(fmaf(-k, x.Y, 1.0f), 0.1f);
    const float sdot = __fdiv_rn(fmaf(vx, x.cp, -(vy * x.sp)), den);
    const float eydot = fmaf(vx, x.sp, vy * x.cp);
    const float epdot = fmaf(-k, sdot, r);
    const float dpsi = P.dt * epdot;
    float sa, ca;
    sincos_any(dpsi, &sa, &ca);
    x.X = fmaf(P.dt, sdot, x.X);
    x.Y = fmaf(P.dt, eydot, x.Y);
    x.psi += dpsi;
    const float cp0 = x.cp;
    x.cp = fmaf(x.cp, ca, -(x.sp * sa));
    x.sp = fmaf(x.sp, ca, cp0 * sa);
}

// Reverse-mode adjoint of model_step at (x, d, a): given lb = dJ/dx_{t+1},
// overwrite lb with dJ/dx_t through the dynamics and return dJ/du_t in
// (*gd, *ga).  Hand-derived from the forward formulas above (cos / sin psi
// are functions of psi; the adjoint flows through psi only).
__device__ __forceinline__ void model_step_adjoint(const DevParams& P, const State& x, float d,
                                                   float a, State& lb, float* gd, float* ga) {
    (void)a;
    const float yf = fmaf(P.lf, x.r, x.vy), yr = fmaf(-P.lr, x.r, x.vy);
    const float bf = atan2_poly(yf, x.vx), br = atan2_poly(yr, x.vx);
    const float af = d - bf, ar = -br;
    float dphf, dphr;
    const float Fyf = P.Fzf * tyre_shape(P, P.B * af, &dphf);
    tyre_shape(P, P.B * ar, &dphr);
    float sd, cd;
    if (P.steer_small) sincos_half(d, &sd, &cd);
    else sincosf(d, &sd, &cd);
    const float cp = x.cp, sp = x.sp;
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
    // tyres: Fy = Fz shape(B alpha)
    const float afb = Fyfb * P.Fzf * dphf * P.B;
    const float arb = Fyrb * P.Fzr * dphr * P.B;
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
// Track: closed polyline P_0 .. P_{n-1}; segment i runs from A_i = P_i with
// D_i = P_{i+1 mod n} - A_i.  Stored as a table of segment PAIRS built once
// per track (launch_rec_table):
//   record j (j = 0 .. n + 4) = segments (j - 1 mod n, j mod n) as
//     float4 nA = (-A_x, -A_x', -A_y, -A_y'),
//     float4 nD = (-D_x, -D_x', -D_y, -D_y'),
//     float4 Dn = (D_x, D_x', D_y, D_y') / |D|^2   (0 for a zero-length segment)
//   (primes: the second segment).  One record gives the squared distances to
//   two consecutive segments with packed instructions; segment i is the first
//   half of record i + 1.  The squared distance from (X, Y) to segment i is
//   |e - tau D|^2 with e = (X, Y) - A, tau = clamp(e . Dn, 0, 1).
// ---------------------------------------------------------------------------

// Squared distances from (X, Y) to the two segments of record j.
__device__ __forceinline__ float2 rec_d2(const float4* __restrict__ rec, int j, float2 XX,
                                         float2 YY) {
    using namespace x2;
    const float4 nA = rec[3 * j], nD = rec[3 * j + 1], Dn = rec[3 * j + 2];
    const f2 ex = add(XX, lo(nA)), ey = add(YY, hi(nA));
    f2 t = fma(ex, lo(Dn), mul(ey, hi(Dn)));
    t.x = __saturatef(t.x);
    t.y = __saturatef(t.y);
    const f2 rx = fma(t, lo(nD), ex), ry = fma(t, hi(nD), ey);
    return fma(rx, rx, mul(ry, ry));
}

// The same arithmetic for segment i alone (first half of record i + 1).
__device__ __forceinline__ float rec_d2_seg(const float4* __restrict__ rec, int i, float X,
                                            float Y) {
    const float4 nA = rec[3 * (i + 1)], nD = rec[3 * (i + 1) + 1], Dn = rec[3 * (i + 1) + 2];
    const float ex = X + nA.x, ey = Y + nA.z;
    const float t = __saturatef(fmaf(ex, Dn.x, ey * Dn.z));
    const float rx = fmaf(t, nD.x, ex), ry = fmaf(t, nD.z, ey);
    return fmaf(rx, rx, ry * ry);
}

// Offset from the nearest point of segment i to (X, Y): d(e_y^2)/d(X, Y) = 2 r.
__device__ __forceinline__ float2 rec_offset(const float4* __restrict__ rec, int i, float X,
                                             float Y) {
    const float4 nA = rec[3 * (i + 1)], nD = rec[3 * (i + 1) + 1], Dn = rec[3 * (i + 1) + 2];
    const float ex = X + nA.x, ey = Y + nA.z;
    const float t = __saturatef(fmaf(ex, Dn.x, ey * Dn.z));
    return make_float2(fmaf(t, nD.x, ex), fmaf(t, nD.z, ey));
}

// Continuous tracking of the nearest segment (the walk that defines e_y along a
// trajectory): from the previous segment s walk forward while the next segment
// is strictly closer, else backward while the previous one is; one segment at
// a time.
static __device__ __noinline__ int walk_seq_rec(const float4* __restrict__ rec, int n, int s, float X,
                                         float Y, float& d2) {
    float d = rec_d2_seg(rec, s, X, Y);
    int nx = (s + 1 == n) ? 0 : s + 1;
    float dn = rec_d2_seg(rec, nx, X, Y);
    if (dn < d) {
        for (int it = 0; it < n && dn < d; ++it) {
            s = nx;
            d = dn;
            nx = (s + 1 == n) ? 0 : s + 1;
            dn = rec_d2_seg(rec, nx, X, Y);
        }
    } else {
        int pv = (s == 0) ? n - 1 : s - 1;
        float dp = rec_d2_seg(rec, pv, X, Y);
        for (int it = 0; it < n && dp < d; ++it) {
            s = pv;
            d = dp;
            pv = (s == 0) ? n - 1 : s - 1;
            dp = rec_d2_seg(rec, pv, X, Y);
        }
    }
    d2 = d;
    return s;
}

// The descent walk from s evaluated on the window s-1 .. s+4 (three records,
// six packed distances): it ends within s .. s+3; a longer forward walk or
// any backward step reruns walk_seq_rec (or, with SPEC, sets fb and returns a
// segment in [0, n) that the caller discards).  Same result as walk_seq_rec.
template <bool SPEC>
__device__ __forceinline__ int walk_rec(const float4* __restrict__ rec, int n, int s, float X,
                                        float Y, float& d2, bool& fb) {
    const float2 XX = make_float2(X, X), YY = make_float2(Y, Y);
    const float2 p0 = rec_d2(rec, s, XX, YY);       // d(s-1), d(s)
    const float2 p1 = rec_d2(rec, s + 2, XX, YY);   // d(s+1), d(s+2)
    const float2 p2 = rec_d2(rec, s + 4, XX, YY);   // d(s+3), d(s+4)
    const bool f1 = p1.x < p0.y, f2_ = p1.y < p1.x, f3 = p2.x < p1.y, f4 = p2.y < p2.x;
    const bool b1 = p0.x < p0.y;
    const int adv = f1 ? (f2_ ? (f3 ? 3 : 2) : 1) : 0;
    const float dd = f1 ? (f2_ ? (f3 ? p2.x : p1.y) : p1.x) : p0.y;
    const bool out = f1 ? (f2_ && f3 && f4) : b1;
    if (SPEC) fb |= out;
    else if (out) return walk_seq_rec(rec, n, s, X, Y, d2);
    int r = s + adv;
    if (r >= n) r -= n;
    d2 = dd;
    return r;
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

// ---------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may start while its predecessor in the
// stream is still running; griddep_wait() blocks until the predecessor has
// completed and its memory is visible (a no-op without such a predecessor), so
// every read of data another launch produced comes after it.
// griddep_launch_dependents() lets the next such launch start early.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" :::);
}

// ---------------------------------------------------------------------------
// Bulk (TMA, non-tensor) global -> shared copies completed on an mbarrier.
// Addresses 16-byte aligned, sizes multiples of 16 bytes.  The wait is
// bounded: after the limit it reports failure (the caller sets a status bit).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `parity` of the barrier; false if it did not complete in time.
// A try_wait may suspend the thread for a hardware-defined time before it
// returns false, so the wait is bounded in time (MBAR_WAIT_NS of the global
// timer) as well as in tries.
constexpr uint64_t MBAR_WAIT_NS = 250000000ull;   // 0.25 s
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (int i = 0; i < (1 << 22); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > MBAR_WAIT_NS) return false;
    }
    return false;
}

// One sampled rollout step (Alg. 2 inner loop): u = v + eps, control term
// gamma v' Sigma^-1 u, x <- f(x, clamp(u)), project on the track, add q and the
// DCBF penalty (Eq. 12, 17-20).
// vg = (v, gamma Sigma^-1 v) of the step.
__device__ __forceinline__ void rollout_step(const DevParams& P, const float4* rec, float4 vg,
                                             float2 z, State& x, int& s, float& h_prev,
                                             float& acc) {
    const float u0 = fmaf(P.sig0, z.x, vg.x), u1 = fmaf(P.sig1, z.y, vg.y);
    acc = fmaf(vg.z, u0, acc);
    acc = fmaf(vg.w, u1, acc);
    model_step(P, x, clampf(u0, P.umin0, P.umax0), clampf(u1, P.umin1, P.umax1));
    float d2;
    bool fb = false;
    s = walk_rec<false>(rec, P.n_track, s, x.X, x.Y, d2, fb);
    const float h = P.w2 - d2;
    acc += run_cost(P, x.vx, d2) + P.C_cbf * fmaxf(cbf_arg(P, h_prev, h), 0.0f);
    h_prev = h;
}

// Cost of state x_t: walk to its segment, add q(x_t) and the DCBF penalty of
// the pair (x_{t-1}, x_t) (Eq. 17, 24).
__device__ __forceinline__ void track_cost(const DevParams& P, const float4* rec, const State& x,
                                           int& s, float& h_prev, float& acc) {
    float d2;
    bool fb = false;
    s = walk_rec<false>(rec, P.n_track, s, x.X, x.Y, d2, fb);
    const float h = P.w2 - d2;
    acc += run_cost(P, x.vx, d2) + P.C_cbf * fmaxf(cbf_arg(P, h_prev, h), 0.0f);
    h_prev = h;
}

// Perturbed control of one step: u = v + eps (returned clamped to the box) and
// the control term gamma v' Sigma^-1 u added to acc (vg = (v, gamma Sigma^-1 v)).
__device__ __forceinline__ float2 perturb(const DevParams& P, float4 vg, float2 z, float& acc) {
    const float u0 = fmaf(P.sig0, z.x, vg.x), u1 = fmaf(P.sig1, z.y, vg.y);
    acc = fmaf(vg.z, u0, acc);
    acc = fmaf(vg.w, u1, acc);
    return make_float2(clampf(u0, P.umin0, P.umax0), clampf(u1, P.umin1, P.umax1));
}

__device__ __forceinline__ void dump_row(float* tr, int t, const State& x) {
    float* o = tr + (size_t)t * 6;
    o[0] = x.vx; o[1] = x.vy; o[2] = x.r; o[3] = x.X; o[4] = x.Y; o[5] = x.psi;
}

// Trajectory cost S~ of sampled rollout k (Alg. 2 inner loop, Eq. 12, 17-20),
// software-pipelined: the track projection and cost of x_t are issued
// together with the dynamics x_t -> x_{t+1}, which do not depend on them, and
// the noise of the next pair of steps is drawn one pair ahead.  x = x_0 with
// segment s and squared offset d20; Vs[t] = (v_t, gamma Sigma^-1 v_t); traj
// (DUMP only): this rollout's (T + 1) x 6 row.
template <bool FAST, bool DUMP>
__device__ __forceinline__ float rollout_sample(const DevParams& P, const float4* rec,
                                                const float4* Vs, State x, int s,
                                                float d20, uint32_t k, uint32_t iter,
                                                uint32_t ctr3, float* traj) {
    const int T = P.T, npair = (T + 1) >> 1;
    float h_prev = P.w2 - d20;
    float acc = run_cost(P, x.vx, d20) + P.C_cbf * fmaxf(cbf_arg(P, h_prev, h_prev), 0.0f);
    if (DUMP) dump_row(traj, 0, x);
    uint4 r = philox10(make_uint4(k, 0u, iter, ctr3), P);
    float2 za = box_muller(r.x, r.y), zb = box_muller(r.z, r.w);
    // pair 0 (the cost of x_0 is already in acc); afterwards the cost of x is pending
    {
        const uint4 rn = philox10(make_uint4(k, 1u, iter, ctr3), P);
        const float2 na = box_muller(rn.x, rn.y), nb = box_muller(rn.z, rn.w);
        const float2 ua = perturb(P, Vs[0], za, acc);
        model_step<FAST>(P, x, ua.x, ua.y);
        if (DUMP) dump_row(traj, 1, x);
        if (T > 1) {
            const float2 ub = perturb(P, Vs[1], zb, acc);
            State xb = x;
            model_step<FAST>(P, xb, ub.x, ub.y);
            track_cost(P, rec, x, s, h_prev, acc);
            x = xb;
            if (DUMP) dump_row(traj, 2, x);
        }
        za = na;
        zb = nb;
    }
    for (int p = 1; p < npair; ++p) {
        const uint4 rn = philox10(make_uint4(k, (uint32_t)(p + 1), iter, ctr3), P);
        const float2 na = box_muller(rn.x, rn.y), nb = box_muller(rn.z, rn.w);
        const float2 ua = perturb(P, Vs[2 * p], za, acc);
        State xa = x;
        model_step<FAST>(P, xa, ua.x, ua.y);
        track_cost(P, rec, x, s, h_prev, acc);
        if (DUMP) dump_row(traj, 2 * p + 1, xa);
        if (2 * p + 1 < T) {
            const float2 ub = perturb(P, Vs[2 * p + 1], zb, acc);
            State xb = xa;
            model_step<FAST>(P, xb, ub.x, ub.y);
            track_cost(P, rec, xa, s, h_prev, acc);
            x = xb;
            if (DUMP) dump_row(traj, 2 * p + 2, x);
        } else {
            x = xa;
        }
        za = na;
        zb = nb;
    }
    track_cost(P, rec, x, s, h_prev, acc);   // x_T
    return acc;
}

// Result of a nearest-segment search.  The search starts its argmin at an
// out-of-range index, which survives only when no squared distance is below
// 3e38 (a start position that is NaN, infinite or beyond ~1.8e19 m): segment 0
// is taken instead, so that every later table access stays in bounds, and the
// NUMERIC bit of the status word reports the state.
__device__ __forceinline__ int seg_or_zero(int s, int n, unsigned* status) {
    if ((unsigned)s < (unsigned)n) return s;
    if (status) atomicOr(status, SMPPI_DEV_NUMERIC);
    return 0;
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
