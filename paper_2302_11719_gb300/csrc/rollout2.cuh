// Two rollouts per thread on the packed FP32 datapath of sm_100+ (one FFMA2 /
// FADD2 / FMUL2 instruction performs the same IEEE operation on both halves of
// a register pair).  Every float2 below holds (rollout a, rollout b); the
// arithmetic of each half is the scalar model step of Eq. 1 with the costs of
// Eq. 17 and 24-25.  Operations without a packed form (min / max, compares,
// MUFU, integer Philox) run once per half.
//
// Issue slots, not FP32 lanes, bound the single-rollout kernel: at K = 65536 an
// SM scheduler holds at most 4 warps and every model step is ~380 scalar
// instructions.  Packing two rollouts halves the FP32 instruction count.
//
// Track queries read a table of segment PAIRS built once per track:
//   record j (j = 0 .. n + 4) = segments (j - 1 mod n, j mod n) as
//     float4 nA = (-A_x, -A_x', -A_y, -A_y'),
//     float4 nD = (-D_x, -D_x', -D_y, -D_y'),
//     float4 Dn = (D_x, D_x', D_y, D_y') / |D|^2   (0 for a zero-length segment)
//   with A the segment start, D = B - A; primes are the second segment.  One
//   record gives the squared distance to two consecutive segments with packed
//   instructions.  Segment i is the first half of record i + 1.
#pragma once

#include "device.cuh"

namespace smppi {
namespace x2 {

using f2 = float2;

struct State2 {
    f2 vx, vy, r, X, Y, psi, cp, sp;   // psi is carried only when trajectories are dumped
};

__device__ __forceinline__ State2 broadcast(const State& s) {
    State2 x;
    x.vx = bc(s.vx); x.vy = bc(s.vy); x.r = bc(s.r); x.X = bc(s.X); x.Y = bc(s.Y);
    x.psi = bc(s.psi); x.cp = bc(s.cp); x.sp = bc(s.sp);
    return x;
}

// sin and cos of |x| <= 1/2 by Taylor series to x^7 / x^8: the remainders are
// below 0.5^9 / 9! = 5.4e-9 and 0.5^10 / 10! = 2.7e-10, under half an ulp of
// the results (|sin x| >= 0.96 |x|, cos x >= 0.87).
__device__ __forceinline__ void sincos_half2(f2 x, f2& s, f2& c) {
    const f2 x2 = mul(x, x);
    f2 ps = fma(bc(-1.9841269841269841e-04f), x2, bc(8.3333333333333333e-03f));
    ps = fma(ps, x2, bc(-1.6666666666666667e-01f));
    s = fma(mul(ps, x2), x, x);
    f2 pc = fma(bc(2.4801587301587302e-05f), x2, bc(-1.3888888888888889e-03f));
    pc = fma(pc, x2, bc(4.1666666666666667e-02f));
    pc = fma(pc, x2, bc(-0.5f));
    c = fma(pc, x2, bc(1.0f));
}

// One explicit Euler step (Eq. 1) of both rollouts; C = 1.5 and |steer| <= 1/2
// (the kernel is used only for such parameters).  |dt r| > 1/2 falls back to
// the library sincos for that half; with SPEC the step instead sets fb and
// leaves the result to be discarded (the caller replays the step exactly).
template <bool PSI, bool SPEC>
__device__ __forceinline__ void model_step2(const DevParams& P, State2& x, f2 d, f2 a, bool& fb) {
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
    const f2 dX = fma(x.vx, x.cp, mul(neg(x.vy), x.sp));
    const f2 dY = fma(x.vx, x.sp, mul(x.vy, x.cp));
    const f2 dpsi = mul(bc(P.dt), x.r);
    f2 sa, ca;
    sincos_half2(dpsi, sa, ca);
    const f2 dt = bc(P.dt);
    x.vx = fma(dt, dvx, x.vx);
    x.vy = fma(dt, dvy, x.vy);
    x.r = fma(dt, dr, x.r);
    x.X = fma(dt, dX, x.X);
    x.Y = fma(dt, dY, x.Y);
    if (PSI) x.psi = add(x.psi, dpsi);
    if (SPEC) {
        fb |= fmaxf(fabsf(dpsi.x), fabsf(dpsi.y)) > 0.5f;
    } else {
        if (fabsf(dpsi.x) > 0.5f) sincosf(dpsi.x, &sa.x, &ca.x);
        if (fabsf(dpsi.y) > 0.5f) sincosf(dpsi.y, &sa.y, &ca.y);
    }
    const f2 cp0 = x.cp;
    x.cp = fma(x.cp, ca, mul(neg(x.sp), sa));
    x.sp = fma(x.sp, ca, mul(cp0, sa));
}

// Cost of the states x_t of both rollouts: walk to their segments, add q(x_t)
// (Eq. 24-25) and the DCBF penalty of (x_{t-1}, x_t) (Eq. 17).
template <bool SPEC>
__device__ __forceinline__ void track_cost2(const DevParams& P, const float4* rec,
                                            const State2& x, int& sa, int& sb, f2& h_prev,
                                            f2& acc, bool& fb) {
    f2 d2;
    sa = walk_rec<SPEC>(rec, P.n_track, sa, x.X.x, x.Y.x, d2.x, fb);
    sb = walk_rec<SPEC>(rec, P.n_track, sb, x.X.y, x.Y.y, d2.y, fb);
    const f2 h = fma(d2, bc(-1.0f), bc(P.w2));
    const f2 ev = add(x.vx, bc(-P.v_target));
    f2 q = fma(mul(bc(P.q_v), ev), ev, mul(bc(P.qd_w2), d2));
    if (d2.x > P.w2) q.x += P.C_obs;
    if (d2.y > P.w2) q.y += P.C_obs;
    const f2 c = fma(bc(P.one_m_alpha), h_prev, add(d2, bc(-P.w2)));   // (1-alpha) h_prev - h
    acc = add(acc, fma(bc(P.C_cbf), make_float2(fmaxf(c.x, 0.0f), fmaxf(c.y, 0.0f)), q));
    h_prev = h;
}

// Box-Muller of both rollouts: (z_0, z_1) = sqrt(-2 ln u_1) (cos, sin)(2 pi u_2).
__device__ __forceinline__ void box_muller2(uint32_t a1, uint32_t b1, uint32_t a2, uint32_t b2,
                                            f2& z0, f2& z1) {
    const f2 u1 = fma(make_float2(__uint2float_rn(a1 >> 9), __uint2float_rn(b1 >> 9)),
                      bc(0x1p-23f), bc(0x1p-24f));
    const f2 u2 = fma(make_float2(__uint2float_rn(a2 >> 9), __uint2float_rn(b2 >> 9)),
                      bc(0x1p-23f), bc(0x1p-24f));
    const f2 q = mul(bc(-2.0f), make_float2(logf(u1.x), logf(u1.y)));
    const f2 r = mul(q, make_float2(rsqrt_n(q.x), rsqrt_n(q.y)));
    f2 s, c;
    sincospif(2.0f * u2.x, &s.x, &c.x);
    sincospif(2.0f * u2.y, &s.y, &c.y);
    z0 = mul(r, c);
    z1 = mul(r, s);
}

// Philox4x32-10 of the counters (k, p, iter, ctr3) of two rollouts ka, kb for
// successive p, with the parts of the first two rounds that do not depend on p
// formed once (philox10 does the same rounds in full).  Round 0 maps the counter
// to (G0 ^ p, G1, R0, R1): G0 = hi(M1 iter) ^ key0, G1 = lo(M1 iter),
// R0 = hi(M0 k) ^ ctr3 ^ key1, R1 = lo(M0 k).  Round 1 then gives
// (hi(M1 R0) ^ G1 ^ key0', lo(M1 R0), hi(M0 x) ^ R1 ^ key1', lo(M0 x)) with
// x = G0 ^ p, the one product the two rollouts share; rounds 2-9 follow.
struct PhiloxPair {
    uint32_t g0;                 // hi(M1 iter) ^ key0 of round 0
    uint32_t qa0, qa1, sa1;      // rollout a: round-1 words 0 and 1, R1 ^ key1 of round 1
    uint32_t qb0, qb1, sb1;      // rollout b
};

__device__ __forceinline__ PhiloxPair philox_pair_setup(const DevParams& P, uint32_t ka,
                                                        uint32_t kb, uint32_t iter,
                                                        uint32_t ctr3) {
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const unsigned long long gi = (unsigned long long)M1 * iter;
    PhiloxPair s;
    s.g0 = (uint32_t)(gi >> 32) ^ P.rk0[0];
    const uint32_t g1 = (uint32_t)gi;
    auto one = [&](uint32_t k, uint32_t& q0, uint32_t& q1, uint32_t& s1) {
        const unsigned long long pk = (unsigned long long)M0 * k;
        const uint32_t r0 = (uint32_t)(pk >> 32) ^ ctr3 ^ P.rk1[0], r1 = (uint32_t)pk;
        const unsigned long long pr = (unsigned long long)M1 * r0;
        q0 = (uint32_t)(pr >> 32) ^ g1 ^ P.rk0[1];
        q1 = (uint32_t)pr;
        s1 = r1 ^ P.rk1[1];
    };
    one(ka, s.qa0, s.qa1, s.sa1);
    one(kb, s.qb0, s.qb1, s.sb1);
    return s;
}

// Rounds 2-9 of Philox4x32-10 (round keys rk[2..9]).
__device__ __forceinline__ uint4 philox_rounds_2_9(uint4 c, const DevParams& P) {
#pragma unroll
    for (int i = 2; i < 10; ++i) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ P.rk0[i], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ P.rk1[i], (uint32_t)p0);
    }
    return c;
}

// The Philox words of counters (ka, p, iter, ctr3) and (kb, p, iter, ctr3).
__device__ __forceinline__ void philox_pair_words(const DevParams& P, const PhiloxPair& ph,
                                                  uint32_t p, uint4& ra, uint4& rb) {
    const unsigned long long px = (unsigned long long)0xD2511F53u * (ph.g0 ^ p);
    const uint32_t hx = (uint32_t)(px >> 32), lx = (uint32_t)px;
    ra = philox_rounds_2_9(make_uint4(ph.qa0, ph.qa1, hx ^ ph.sa1, lx), P);
    rb = philox_rounds_2_9(make_uint4(ph.qb0, ph.qb1, hx ^ ph.sb1, lx), P);
}

// Noise of steps 2p (zs0, zs1) and 2p + 1 (zt0, zt1) of rollouts ka, kb:
// Philox counter (k, p, iter, ctr3), words 0-1 for step 2p, 2-3 for 2p + 1.
__device__ __forceinline__ void noise_pair2(const DevParams& P, const PhiloxPair& ph, uint32_t p,
                                            f2& zs0, f2& zs1, f2& zt0, f2& zt1) {
    uint4 ra, rb;
    philox_pair_words(P, ph, p, ra, rb);
    box_muller2(ra.x, rb.x, ra.y, rb.y, zs0, zs1);
    box_muller2(ra.z, rb.z, ra.w, rb.w, zt0, zt1);
}

// u = v + sigma z of both rollouts (returned clamped to the control box) and
// the control term gamma v' Sigma^-1 u added to acc.  vv = (v0, v0, v1, v1),
// gg = gamma Sigma^-1 v in the same layout.
__device__ __forceinline__ void perturb2(const DevParams& P, float4 vv, float4 gg, f2 z0, f2 z1,
                                         f2& acc, f2& d, f2& a) {
    const f2 u0 = fma(bc(P.sig0), z0, lo(vv)), u1 = fma(bc(P.sig1), z1, hi(vv));
    acc = fma(lo(gg), u0, acc);
    acc = fma(hi(gg), u1, acc);
    d = make_float2(clampf(u0.x, P.umin0, P.umax0), clampf(u0.y, P.umin0, P.umax0));
    a = make_float2(clampf(u1.x, P.umin1, P.umax1), clampf(u1.y, P.umin1, P.umax1));
}

__device__ __forceinline__ void dump2(float* ta, float* tb, int t, const State2& x) {
    if (ta) {
        float* r = ta + (size_t)t * 6;
        r[0] = x.vx.x; r[1] = x.vy.x; r[2] = x.r.x; r[3] = x.X.x; r[4] = x.Y.x; r[5] = x.psi.x;
    }
    if (tb) {
        float* r = tb + (size_t)t * 6;
        r[0] = x.vx.y; r[1] = x.vy.y; r[2] = x.r.y; r[3] = x.X.y; r[4] = x.Y.y; r[5] = x.psi.y;
    }
}

// Steps 2p and 2p + 1 of both rollouts (x = x_{2p} on entry, x_{2p+2} on
// exit, xa = x_{2p+1}): the cost of x_{2p} is taken while x_{2p+1} is
// integrated, and the cost of x_{2p+1} while x_{2p+2} is.
template <bool PSI, bool SPEC>
__device__ __forceinline__ void pair_steps2(const DevParams& P, const float4* rec,
                                            const float4* Vq, f2 za0, f2 za1, f2 zb0, f2 zb1,
                                            State2& x, State2& xa, int& sa, int& sb, f2& h_prev,
                                            f2& acc, bool& fb) {
    f2 d, a;
    perturb2(P, Vq[0], Vq[1], za0, za1, acc, d, a);
    xa = x;
    model_step2<PSI, SPEC>(P, xa, d, a, fb);
    track_cost2<SPEC>(P, rec, x, sa, sb, h_prev, acc, fb);
    perturb2(P, Vq[2], Vq[3], zb0, zb1, acc, d, a);
    State2 xb = xa;
    model_step2<PSI, SPEC>(P, xb, d, a, fb);
    track_cost2<SPEC>(P, rec, xa, sa, sb, h_prev, acc, fb);
    x = xb;
}

// Costs S~ of rollouts ka and kb (Alg. 2 sampling loop, Eq. 17-20, 24-25).
// Vp[2t] = (v0, v0, v1, v1), Vp[2t + 1] = gamma Sigma^-1 v_t in that layout.
// Software-pipelined: the track cost of x_t is computed while x_{t+1} is
// integrated and the noise of the next two steps is drawn.  The body of the
// main loop is branch-free (one block for the scheduler): its rare fallbacks
// (|dt r| > 1/2, a track walk that leaves its window) only set a flag, and a
// flagged iteration is replayed from its saved start with the exact step.
template <bool DUMP>
__device__ __forceinline__ f2 rollout2(const DevParams& P, const float4* rec,
                                       const float4* Vp, const State& x0, int s0, float d20,
                                       uint32_t ka, uint32_t kb, uint32_t iter, uint32_t ctr3,
                                       float* ta, float* tb) {
    const int T = P.T, nfull = T >> 1;
    const float h0 = P.w2 - d20;
    f2 h_prev = bc(h0);
    f2 acc = bc(run_cost(P, x0.vx, d20) + P.C_cbf * fmaxf(cbf_arg(P, h0, h0), 0.0f));
    State2 x = broadcast(x0);
    int sa = s0, sb = s0;
    bool fb = false;
    if (DUMP) dump2(ta, tb, 0, x);
    f2 za0, za1, zb0, zb1;
    const PhiloxPair ph = philox_pair_setup(P, ka, kb, iter, ctr3);
    noise_pair2(P, ph, 0u, za0, za1, zb0, zb1);
    {   // steps 0 and 1 (the cost of x_0 is already in acc)
        f2 na0, na1, nb0, nb1;
        noise_pair2(P, ph, 1u, na0, na1, nb0, nb1);
        f2 d, a;
        perturb2(P, Vp[0], Vp[1], za0, za1, acc, d, a);
        model_step2<DUMP, false>(P, x, d, a, fb);
        if (DUMP) dump2(ta, tb, 1, x);
        if (T > 1) {
            perturb2(P, Vp[2], Vp[3], zb0, zb1, acc, d, a);
            State2 xb = x;
            model_step2<DUMP, false>(P, xb, d, a, fb);
            track_cost2<false>(P, rec, x, sa, sb, h_prev, acc, fb);
            x = xb;
            if (DUMP) dump2(ta, tb, 2, x);
        }
        za0 = na0; za1 = na1; zb0 = nb0; zb1 = nb1;
    }
    for (int p = 1; p < nfull; ++p) {   // steps 2p, 2p + 1 < T
        f2 na0, na1, nb0, nb1;
        noise_pair2(P, ph, (uint32_t)(p + 1), na0, na1, nb0, nb1);
        const State2 x_in = x;
        const int sa_in = sa, sb_in = sb;
        const f2 hp_in = h_prev, acc_in = acc;
        State2 xa;
        fb = false;
        pair_steps2<DUMP, true>(P, rec, Vp + 4 * p, za0, za1, zb0, zb1, x, xa, sa, sb, h_prev,
                                acc, fb);
        if (fb) {
            x = x_in; sa = sa_in; sb = sb_in; h_prev = hp_in; acc = acc_in;
            pair_steps2<DUMP, false>(P, rec, Vp + 4 * p, za0, za1, zb0, zb1, x, xa, sa, sb,
                                     h_prev, acc, fb);
        }
        if (DUMP) {
            dump2(ta, tb, 2 * p + 1, xa);
            dump2(ta, tb, 2 * p + 2, x);
        }
        za0 = na0; za1 = na1; zb0 = nb0; zb1 = nb1;
    }
    if ((T & 1) && nfull >= 1) {   // odd T: the last step T - 1
        f2 d, a;
        perturb2(P, Vp[2 * (T - 1)], Vp[2 * (T - 1) + 1], za0, za1, acc, d, a);
        State2 xa = x;
        model_step2<DUMP, false>(P, xa, d, a, fb);
        track_cost2<false>(P, rec, x, sa, sb, h_prev, acc, fb);
        x = xa;
        if (DUMP) dump2(ta, tb, T, x);
    }
    track_cost2<false>(P, rec, x, sa, sb, h_prev, acc, fb);   // x_T
    return acc;
}

}  // namespace x2
}  // namespace smppi
