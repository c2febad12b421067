// Shield-MPPI oracle: plain, slow, FP64 CPU implementation of one Shield-MPPI
// control update (Yin, Dawson, Fan, Tsiotras, "Shield Model Predictive Path
// Integral: A Computationally Efficient Robust MPC Approach Using Control
// Barrier Functions", arXiv 2302.11719).
//
// TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA path, never to
// stand in for it: only the tests, the smoke check and the timed CPU baseline
// of bench.py may load it.  It shares no code, header, table or constant
// generator with the CUDA library; the only thing both sides share is the
// seeded input generator module, which holds none of the method's arithmetic.
//
// Everything is double precision.  The noise the method draws comes from this
// file's own Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11), written from that paper's definition.
//
// Structure follows the paper:
//   dynamics x_{k+1} = f(x_k, u_k)                 Eq. 1 (Sec. II), model Sec. VI-A
//   trajectory cost S with control term           Eq. 8 / Eq. 12, Alg. 2
//   DCBF condition / penalty, augmented state      Eq. 14-15, Eq. 17-20 (Sec. III, IV-A)
//   min-shifted weights and control update         Eq. 10-11 (Sec. II)
//   safe set h = w^2 - e_y^2                       Eq. 23 (Sec. VI-B)
//   running cost                                   Eq. 24-25 (Sec. VI-C)
//   local repair of the CBF objective              Eq. 22, Alg. 1 (Sec. IV-B)
//   disturbed closed loop                          Eq. 26 (Sec. VI-F), Alg. 2
//
// Where the paper is silent these readings are taken (their labels are used below):
//   c2  control term gamma * v_t' Sigma^-1 (v_t + eps_t), gamma a parameter;
//   c3  terminal cost phi = q, so S sums q over x_0..x_T;
//   c4  the k = 0 CBF term uses x_{-1} = x_0 (Eq. 20);
//   c7  dynamics see clamp(v + eps); cost and update use the unclamped eps;
//       the update result and every repair iterate are projected on the box;
//   c9  repair = projected gradient with Armijo backtracking (mode 1) or the
//       fixed step of Alg. 1 (mode 0);
//   c27 the BFGS repair (mode 2; the solver Sec. IV-B names for Eq. 22, run
//       for a fixed number of iterations) is box-projected BFGS with Armijo
//       backtracking on the projected path, see bfgs_box below;
//   c12 max(0, .) has derivative 0 at a non-positive argument; clamp(v) has
//       derivative 1 on the closed box and 0 strictly outside it;
//   c13 warm start V <- shift(V^+): drop v_0 and repeat the last control;
//   c15 e_y is the distance to the centreline polyline, tracked continuously
//       from the previous step's segment (the curvilinear coordinate of the
//       paper's model); the first segment is the global nearest one.
//   c28 curvature of the centreline as a function of arc length: turning angle
//       over mean segment length at each vertex, piecewise linear in s between
//       vertices, sampled at n uniform stations and interpolated linearly;
//   c29 curvilinear state (s, e_y, e_psi) of the paper's AutoRally model
//       (Sec. VI-A): Frenet kinematics on that curvature, 1 - kappa e_y held
//       at >= 0.1, h and q from e_y directly.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

// Parameters of one problem.  Values are supplied by the caller; the Python
// wrapper rounds them to the float32 values the GPU path uses so that both
// sides evaluate the same model.
struct OrcParams {
    double m, Iz, lf, lr;      // mass, yaw inertia, CoG to front / rear axle
    double B, Ct, g, fx_gain;  // tyre B and C, gravity, N of rear force per unit throttle
    double dt;                 // Euler step
    double sigma[2];           // noise std of (steer, throttle): Sigma = diag(sigma^2)
    double lambda, gamma;      // temperature (Eq. 11) and control-cost weight (Alg. 2)
    int K, T, N_r;             // rollouts, horizon, repair horizon
    double alpha;              // class-kappa rate p(r) = alpha r (the paper's beta, Eq. 15)
    double C_cbf;              // penalty weight C (Eq. 17)
    double q_v, v_target, q_d, C_obs;  // running cost weights (Eq. 24-25)
    double u_min[2], u_max[2];         // control box
    double half_width;                 // w_T (Eq. 23)
    double dist_sigma[2];              // disturbance std on (v_y, r) (Eq. 26)
    double ls_s0, ls_c;                // Armijo: first step s0/|g|_inf, sufficient decrease c
    int ls_max_halvings;               // trials per line search
    int n_track;                       // centreline points
    const float* track_xy;             // n_track x 2, closed polyline (float32 values)
    uint64_t seed;
    int state_kind;                    // 0: (X, Y, psi), e_y from the polyline; 1: (s, e_y, e_psi)
    const double* kappa;               // state_kind 1: n_track curvature samples (reading c28)
    double track_len;                  // state_kind 1: arc length L of the closed centreline
};

// ---------------------------------------------------------------------------
// Philox4x32-10 and Philox4x64-10 (SC'11).  One round maps the counter block
// (c0, c1, c2, c3) with key (k0, k1) to
//   (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
// and the key is bumped by the Weyl constants between rounds.  The 4x64
// instance exists only so that the round structure can be checked against an
// independent library implementation (numpy.random.Philox).
// ---------------------------------------------------------------------------
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        unsigned __int128 p0 = (unsigned __int128)M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Uniform in (0, 1) from the top 23 bits: (m + 1/2) 2^-23, m = x >> 9.  The
// value is exact in float32 and in float64 and is never 0 or 1.
double orc_uniform(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

// Box-Muller: two uniforms -> two independent standard normals.
void orc_box_muller(uint32_t a, uint32_t b, double z[2]) {
    const double PI = 3.14159265358979323846;
    double u1 = orc_uniform(a), u2 = orc_uniform(b);
    double r = std::sqrt(-2.0 * std::log(u1));
    z[0] = r * std::cos(2.0 * PI * u2);
    z[1] = r * std::sin(2.0 * PI * u2);
}

// Standard normal pair for rollout k, step t of iteration `iter` on random
// stream `stream` (0 = MPPI noise, 1 = disturbance) of problem `instance`.
// Counter = (k, t >> 1, iter, stream | instance << 8), key = seed; even t uses
// output words (0, 1), odd t words (2, 3).
void orc_normal_pair(uint64_t seed, uint32_t iter, uint32_t instance, uint32_t stream,
                     uint32_t k, uint32_t t, double z[2]) {
    uint32_t ctr[4] = {k, t >> 1, iter, stream | (instance << 8)};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    if ((t & 1u) == 0) orc_box_muller(out[0], out[1], z);
    else orc_box_muller(out[2], out[3], z);
}

// MPPI control noise eps_t^k ~ N(0, Sigma) (Sec. II, Alg. 2 "Sample eps^m").
void orc_noise(const OrcParams* p, uint32_t iter, uint32_t instance, uint32_t k, uint32_t t,
               double eps[2]) {
    double z[2];
    orc_normal_pair(p->seed, iter, instance, 0u, k, t, z);
    eps[0] = p->sigma[0] * z[0];
    eps[1] = p->sigma[1] * z[1];
}

// eps for rollouts k0..k0+nk-1 and steps 0..T-1 into out[(i T + t) 2 + j].
void orc_noise_block(const OrcParams* p, uint32_t iter, uint32_t instance, uint32_t k0, int nk,
                     int T, double* out) {
    for (int i = 0; i < nk; ++i)
        for (int t = 0; t < T; ++t)
            orc_noise(p, iter, instance, k0 + (uint32_t)i, (uint32_t)t, out + ((size_t)i * T + t) * 2);
}

// Additive disturbance w_n of the closed loop (Eq. 26): zero except on v_y
// and r, drawn on stream 1 with counter (0, 0, n, 1 | instance << 8).
void orc_disturbance(const OrcParams* p, uint32_t n, uint32_t instance, double w[6]) {
    double z[2];
    orc_normal_pair(p->seed, n, instance, 1u, 0u, 0u, z);
    for (int i = 0; i < 6; ++i) w[i] = 0.0;
    w[1] = p->dist_sigma[0] * z[0];
    w[2] = p->dist_sigma[1] * z[1];
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Forward-mode dual numbers (value + one directional derivative).  Only the
// elementary rules below are used; the gradient of the repair objective comes
// from them, independently of any hand-derived adjoint.
// ---------------------------------------------------------------------------
struct Dual {
    double v, d;
    Dual(double value = 0.0, double deriv = 0.0) : v(value), d(deriv) {}
};
static inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
static inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
static inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
static inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
static inline Dual operator/(Dual a, Dual b) {
    return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
static inline Dual sin(Dual a) { return Dual(std::sin(a.v), std::cos(a.v) * a.d); }
static inline Dual cos(Dual a) { return Dual(std::cos(a.v), -std::sin(a.v) * a.d); }
static inline Dual atan(Dual a) { return Dual(std::atan(a.v), a.d / (1.0 + a.v * a.v)); }
static inline Dual atan2(Dual y, Dual x) {
    double r2 = x.v * x.v + y.v * y.v;
    double dd = (r2 > 0.0) ? (x.v * y.d - y.v * x.d) / r2 : 0.0;
    return Dual(std::atan2(y.v, x.v), dd);
}
static inline double val(double a) { return a; }
static inline double val(Dual a) { return a.v; }

// ---------------------------------------------------------------------------
// Curvature of the closed centreline as a function of arc length (reading
// c28).  Vertex P_i between the segments d_{i-1} = P_i - P_{i-1} and
// d_i = P_{i+1} - P_i (lengths l_{i-1}, l_i):
//   kappa_i = atan2(d_{i-1} x d_i, d_{i-1} . d_i) / ((l_{i-1} + l_i) / 2),
// positive where the centreline turns left.  kappa(s) is piecewise linear
// between the vertex stations s_i = l_0 + ... + l_{i-1} (period L = total
// length); its samples at the n uniform stations s = j L / n form the table
// that the model interpolates linearly.
// ---------------------------------------------------------------------------
extern "C" void orc_curvature_table(const OrcParams* p, double* kappa_out, double* len_out) {
    const int n = p->n_track;
    std::vector<double> len(n), kv(n), st(n + 1, 0.0);
    auto pt = [&](int i, int c) { return (double)p->track_xy[2 * (((i % n) + n) % n) + c]; };
    for (int i = 0; i < n; ++i) {
        len[i] = std::hypot(pt(i + 1, 0) - pt(i, 0), pt(i + 1, 1) - pt(i, 1));
        st[i + 1] = st[i] + len[i];
    }
    for (int i = 0; i < n; ++i) {
        const double ax = pt(i, 0) - pt(i - 1, 0), ay = pt(i, 1) - pt(i - 1, 1);
        const double bx = pt(i + 1, 0) - pt(i, 0), by = pt(i + 1, 1) - pt(i, 1);
        const double turn = std::atan2(ax * by - ay * bx, ax * bx + ay * by);
        kv[i] = turn / (0.5 * (len[(i + n - 1) % n] + len[i]));
    }
    const double L = st[n];
    int seg = 0;
    for (int j = 0; j < n; ++j) {
        const double sj = j * L / n;
        while (seg + 1 < n && st[seg + 1] <= sj) ++seg;
        const double f = (sj - st[seg]) / len[seg];
        kappa_out[j] = (1.0 - f) * kv[seg] + f * kv[(seg + 1) % n];
    }
    *len_out = L;
}

// kappa(s): linear interpolation of the uniform samples, s taken modulo L.
template <class R>
static R kappa_at(const OrcParams* p, R s) {
    const int M = p->n_track;
    const double L = p->track_len;
    const R sw = s - R(std::floor(val(s) / L) * L);
    const R x = sw * R(M / L);
    int i = (int)std::floor(val(x));
    if (i < 0) i = 0;
    if (i > M - 1) i = M - 1;
    const R f = x - R((double)i);
    return R(p->kappa[i]) + f * R(p->kappa[(i + 1) % M] - p->kappa[i]);
}

// ---------------------------------------------------------------------------
// Vehicle model (Sec. VI-A uses a single-track model; its parameters are not
// given, so the dynamic single-track model with Pacejka-type lateral tyre
// forces below is the model this implementation fixes).  State x = (v_x, v_y, r, X, Y,
// psi), control u = (delta, a).  Static axle loads, no drag.
// ---------------------------------------------------------------------------
template <class R>
static void deriv(const OrcParams* p, const R x[6], const R u[2], R xdot[6]) {
    using std::atan; using std::atan2; using std::cos; using std::sin;
    const R vx = x[0], vy = x[1], r = x[2], psi = x[5];
    const R delta = u[0], a = u[1];
    const double Fz_f = p->m * p->g * p->lr / (p->lf + p->lr);
    const double Fz_r = p->m * p->g * p->lf / (p->lf + p->lr);
    // slip angles of the front and rear axle
    R alpha_f = delta - atan2(vy + R(p->lf) * r, vx);
    R alpha_r = -atan2(vy - R(p->lr) * r, vx);
    // lateral forces Fy = D sin(C atan(B alpha)), D = axle normal load
    R Fyf = R(Fz_f) * sin(R(p->Ct) * atan(R(p->B) * alpha_f));
    R Fyr = R(Fz_r) * sin(R(p->Ct) * atan(R(p->B) * alpha_r));
    R Fxr = R(p->fx_gain) * a;
    R sd = sin(delta), cd = cos(delta);
    xdot[0] = (Fxr - Fyf * sd) / R(p->m) + vy * r;
    xdot[1] = (Fyr + Fyf * cd) / R(p->m) - vx * r;
    xdot[2] = (R(p->lf) * Fyf * cd - R(p->lr) * Fyr) / R(p->Iz);
    if (p->state_kind == 1) {
        // curvilinear kinematics (reading c29): x[3] = s, x[4] = e_y, x[5] = e_psi
        const R es = sin(x[5]), ec = cos(x[5]);
        const R k = kappa_at<R>(p, x[3]);
        R den = R(1.0) - k * x[4];
        if (val(den) < 0.1) den = R(0.1);
        xdot[3] = (vx * ec - vy * es) / den;
        xdot[4] = vx * es + vy * ec;
        xdot[5] = r - k * xdot[3];
        return;
    }
    R sp = sin(psi), cp = cos(psi);
    xdot[3] = vx * cp - vy * sp;
    xdot[4] = vx * sp + vy * cp;
    xdot[5] = r;
}

// x_{k+1} = f(x_k, u_k) (Eq. 1): explicit Euler of the model above.
template <class R>
static void step(const OrcParams* p, const R x[6], const R u[2], R xn[6]) {
    R xdot[6];
    deriv<R>(p, x, u, xdot);
    for (int i = 0; i < 6; ++i) xn[i] = x[i] + R(p->dt) * xdot[i];
}

template <class R>
static R clamp_ctrl(const OrcParams* p, int j, R v) {
    // c7 / c12: projection on the control box; derivative 1 on the closed box
    if (val(v) < p->u_min[j]) return R(p->u_min[j]);
    if (val(v) > p->u_max[j]) return R(p->u_max[j]);
    return v;
}

// ---------------------------------------------------------------------------
// Track: closed polyline through the float32 points P_0..P_{n-1}; segment i
// runs from P_i to P_{i+1 mod n}.  e_y^2 is the squared distance to it.
// ---------------------------------------------------------------------------
static inline void seg_geom(const OrcParams* p, int i, double A[2], double D[2]) {
    int j = (i + 1) % p->n_track;
    A[0] = (double)p->track_xy[2 * i];
    A[1] = (double)p->track_xy[2 * i + 1];
    D[0] = (double)p->track_xy[2 * j] - A[0];
    D[1] = (double)p->track_xy[2 * j + 1] - A[1];
}

// Squared distance from (X, Y) to segment i: project, clamp to the segment.
template <class R>
static R seg_dist2(const OrcParams* p, int i, R X, R Y) {
    double A[2], D[2];
    seg_geom(p, i, A, D);
    R ex = X - R(A[0]), ey = Y - R(A[1]);
    double len2 = D[0] * D[0] + D[1] * D[1];
    R tau = (ex * R(D[0]) + ey * R(D[1])) / R(len2);
    if (val(tau) < 0.0) tau = R(0.0);
    if (val(tau) > 1.0) tau = R(1.0);
    R rx = ex - tau * R(D[0]), ry = ey - tau * R(D[1]);
    return rx * rx + ry * ry;
}

extern "C" {

double orc_seg_dist2(const OrcParams* p, int i, double X, double Y) {
    return seg_dist2<double>(p, i, X, Y);
}

// kappa(s) of the curvilinear model (the interpolation above), for the pins.
double orc_kappa_at(const OrcParams* p, double s) { return kappa_at<double>(p, s); }

// Global nearest segment (brute force over all segments, lowest index on ties).
int orc_track_nearest(const OrcParams* p, double X, double Y, double* d2_out) {
    int best = 0;
    double bd = seg_dist2<double>(p, 0, X, Y);
    for (int i = 1; i < p->n_track; ++i) {
        double d = seg_dist2<double>(p, i, X, Y);
        if (d < bd) { bd = d; best = i; }
    }
    if (d2_out) *d2_out = bd;
    return best;
}

// Continuous tracking of the nearest segment (reading c15): starting from the
// previous step's segment, walk forward while the next segment is strictly
// closer, otherwise backward while the previous one is strictly closer.
int orc_track_follow(const OrcParams* p, int seg, double X, double Y, double* d2_out) {
    const int n = p->n_track;
    double d = seg_dist2<double>(p, seg, X, Y);
    int nxt = (seg + 1) % n;
    double dn = seg_dist2<double>(p, nxt, X, Y);
    if (dn < d) {
        for (int it = 0; it < n && dn < d; ++it) {
            seg = nxt; d = dn;
            nxt = (seg + 1) % n;
            dn = seg_dist2<double>(p, nxt, X, Y);
        }
    } else {
        int prv = (seg + n - 1) % n;
        double dp = seg_dist2<double>(p, prv, X, Y);
        for (int it = 0; it < n && dp < d; ++it) {
            seg = prv; d = dp;
            prv = (seg + n - 1) % n;
            dp = seg_dist2<double>(p, prv, X, Y);
        }
    }
    if (d2_out) *d2_out = d;
    return seg;
}

// h(x) = w_T^2 - e_y^2 (Eq. 23).
double orc_h(const OrcParams* p, double d2) { return p->half_width * p->half_width - d2; }

// Running cost q (Eq. 24-25): Q = diag(q_v on v_x, q_d / w^2 on e_y), target
// v_x = v_target, plus C_obs outside the track.
double orc_q(const OrcParams* p, const double x[6], double d2) {
    double w2 = p->half_width * p->half_width;
    double ev = x[0] - p->v_target;
    double q = p->q_v * ev * ev + p->q_d * d2 / w2;
    if (d2 > w2) q += p->C_obs;
    return q;
}

// DCBF violation penalty C max{-h(x_k) + (1 - alpha) h(x_{k-1}), 0} (Eq. 17 /
// Eq. 19 on the augmented state z_k = (x_k, x_{k-1}), Eq. 18).
double orc_cbf_penalty(const OrcParams* p, double h_prev, double h_now) {
    double arg = (1.0 - p->alpha) * h_prev - h_now;
    return arg > 0.0 ? p->C_cbf * arg : 0.0;
}

void orc_deriv(const OrcParams* p, const double x[6], const double u[2], double xdot[6]) {
    deriv<double>(p, x, u, xdot);
}
void orc_step(const OrcParams* p, const double x[6], const double u[2], double xn[6]) {
    step<double>(p, x, u, xn);
}

// One sampled trajectory of Alg. 2 (inner loop over k) for rollout index k:
//   u_t = v_t + eps_t, x_{t+1} = f(x_t, clamp(u_t)),
//   S~ = sum_{t=0}^{T} q(x_t) + gamma sum_t v_t' Sigma^-1 u_t
//        + sum_{t=0}^{T} C_cbf(z_t)   with z_0 = (x_0, x_0)      (Eq. 12, Eq. 20)
// If `noisy` is 0 the noise is zero (the nominal rollout).  traj (T+1)x6 and
// eps Tx2 are optional outputs.
double orc_rollout(const OrcParams* p, const double x0[6], const double* V, uint32_t iter,
                   uint32_t instance, uint32_t k, int noisy, double* traj, double* eps_out) {
    double x[6];
    for (int i = 0; i < 6; ++i) x[i] = x0[i];
    // e_y^2: the tracked polyline distance, or the curvilinear state's own e_y
    const bool curv = p->state_kind == 1;
    double d2 = x[4] * x[4];
    int seg = curv ? 0 : orc_track_nearest(p, x[3], x[4], &d2);
    double h_prev = orc_h(p, d2);
    double S = orc_q(p, x, d2) + orc_cbf_penalty(p, h_prev, h_prev);
    if (traj) for (int i = 0; i < 6; ++i) traj[i] = x[i];
    const double is0 = 1.0 / (p->sigma[0] * p->sigma[0]);
    const double is1 = 1.0 / (p->sigma[1] * p->sigma[1]);
    for (int t = 0; t < p->T; ++t) {
        double eps[2] = {0.0, 0.0};
        if (noisy) orc_noise(p, iter, instance, k, (uint32_t)t, eps);
        if (eps_out) { eps_out[2 * t] = eps[0]; eps_out[2 * t + 1] = eps[1]; }
        double uraw[2] = {V[2 * t] + eps[0], V[2 * t + 1] + eps[1]};
        double u[2] = {clamp_ctrl<double>(p, 0, uraw[0]), clamp_ctrl<double>(p, 1, uraw[1])};
        double xn[6];
        step<double>(p, x, u, xn);
        for (int i = 0; i < 6; ++i) x[i] = xn[i];
        if (curv) d2 = x[4] * x[4];
        else seg = orc_track_follow(p, seg, x[3], x[4], &d2);
        double h = orc_h(p, d2);
        // control term of Alg. 2 (absent when gamma = 0, also for a degenerate Sigma)
        if (p->gamma != 0.0)
            S += p->gamma * (V[2 * t] * uraw[0] * is0 + V[2 * t + 1] * uraw[1] * is1);
        S += orc_q(p, x, d2) + orc_cbf_penalty(p, h_prev, h);
        h_prev = h;
        if (traj) for (int i = 0; i < 6; ++i) traj[6 * (t + 1) + i] = x[i];
    }
    return S;
}

// Min-shifted weights and the Monte-Carlo control update (Eq. 10-11):
//   omega_k = exp(-(S_k - min S) / lambda),
//   v_t^+ = clamp(v_t + sum_k omega_k eps_t^k / sum_k omega_k).
// S is given (K values); the noise is regenerated from the counter.
void orc_update(const OrcParams* p, const double* S, const double* V, uint32_t iter,
                uint32_t instance, double* Vplus, double* omega_out) {
    const int K = p->K, T = p->T;
    double m = S[0];
    for (int k = 1; k < K; ++k) if (S[k] < m) m = S[k];
    std::vector<double> omega(K);
    double eta = 0.0;
    for (int k = 0; k < K; ++k) { omega[k] = std::exp(-(S[k] - m) / p->lambda); eta += omega[k]; }
    std::vector<double> acc(2 * T, 0.0);
    for (int k = 0; k < K; ++k) {
        for (int t = 0; t < T; ++t) {
            double eps[2];
            orc_noise(p, iter, instance, (uint32_t)k, (uint32_t)t, eps);
            acc[2 * t] += omega[k] * eps[0];
            acc[2 * t + 1] += omega[k] * eps[1];
        }
    }
    for (int t = 0; t < T; ++t)
        for (int j = 0; j < 2; ++j)
            Vplus[2 * t + j] = clamp_ctrl<double>(p, j, V[2 * t + j] + acc[2 * t + j] / eta);
    if (omega_out) for (int k = 0; k < K; ++k) omega_out[k] = omega[k] / eta;
}

// The update of Eq. 10-11 over a partition of the rollouts (the sampling loop
// of Alg. 2 is a loop over independent rollouts, so its K rollouts can be
// split into slices): for the slice k_lo .. k_hi - 1 with costs S[0 ..],
//   m_g = min S_k,  eta_g = sum_k exp(-(S_k - m_g) / lambda),
//   A_g[2t + j] = sum_k exp(-(S_k - m_g) / lambda) eps_{k,t,j},
// written to out [2T + 2] = (m_g, eta_g, A_g).
void orc_partial(const OrcParams* p, const double* S, uint32_t iter, uint32_t instance, int k_lo,
                 int k_hi, double* out) {
    const int T = p->T, n = k_hi - k_lo;
    double m = S[0];
    for (int i = 1; i < n; ++i) if (S[i] < m) m = S[i];
    double eta = 0.0;
    std::vector<double> acc(2 * T, 0.0);
    for (int i = 0; i < n; ++i) {
        const double w = std::exp(-(S[i] - m) / p->lambda);
        eta += w;
        for (int t = 0; t < T; ++t) {
            double eps[2];
            orc_noise(p, iter, instance, (uint32_t)(k_lo + i), (uint32_t)t, eps);
            acc[2 * t] += w * eps[0];
            acc[2 * t + 1] += w * eps[1];
        }
    }
    out[0] = m;
    out[1] = eta;
    for (int j = 0; j < 2 * T; ++j) out[2 + j] = acc[j];
}

// V+ from the slices' partials (n_parts x (2T + 2)): with m = min_g m_g the
// weights of slice g are its own times c_g = exp(-(m_g - m) / lambda), so
//   v_t^+ = clamp(v_t + sum_g c_g A_g[t] / sum_g c_g eta_g)
// is the update of Eq. 10-11 over all rollouts of the slices.
void orc_merge(const OrcParams* p, int n_parts, const double* parts, const double* V,
               double* Vplus) {
    const int T = p->T, W = 2 * T + 2;
    double m = parts[0];
    for (int g = 1; g < n_parts; ++g) if (parts[g * W] < m) m = parts[g * W];
    double eta = 0.0;
    std::vector<double> c(n_parts), acc(2 * T, 0.0);
    for (int g = 0; g < n_parts; ++g) {
        c[g] = std::exp(-(parts[g * W] - m) / p->lambda);
        eta += c[g] * parts[g * W + 1];
        for (int j = 0; j < 2 * T; ++j) acc[j] += c[g] * parts[g * W + 2 + j];
    }
    for (int t = 0; t < T; ++t)
        for (int j = 0; j < 2; ++j)
            Vplus[2 * t + j] = clamp_ctrl<double>(p, j, V[2 * t + j] + acc[2 * t + j] / eta);
}

// One MPPI iteration (Alg. 2, the sampling loop and OptimalControl): K noisy
// rollouts, then the update.  The per-rollout costs are computed in parallel
// over k with `nthreads` threads; every reduction runs in index order, so the
// result does not depend on the thread count.
void orc_mppi_step(const OrcParams* p, const double x0[6], const double* V, uint32_t iter,
                   uint32_t instance, double* S_out, double* Vplus, int nthreads) {
    const int K = p->K;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
    for (int k = 0; k < K; ++k)
        S_out[k] = orc_rollout(p, x0, V, iter, instance, (uint32_t)k, 1, nullptr, nullptr);
    (void)nthreads;
    orc_update(p, S_out, V, iter, instance, Vplus, nullptr);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Deterministic (noise-free) cost of a control sequence over the first N
// steps, used by the repair (Eq. 22) and by the gradient checks:
//   J = w_run sum_{t=0}^{N} q(x_t) + w_cbf sum_{t=0}^{N-1} C max{(1-alpha) h_t - h_{t+1}, 0}
// with x_{t+1} = f(x_t, clamp(v_t)).  With (w_run, w_cbf) = (0, 1) this is
// P(V) = -C times the objective of Eq. 22 (maximising the sum of
// min{h_{t+1} - (1-alpha) h_t, 0} is minimising P).  The segment sequence is
// chosen on the values and held fixed for the derivative.
// ---------------------------------------------------------------------------
template <class R>
static R det_cost(const OrcParams* p, const double x0[6], const R* V, int N, double w_run,
                  double w_cbf) {
    R x[6];
    for (int i = 0; i < 6; ++i) x[i] = R(x0[i]);
    double d2v;
    const bool curv = p->state_kind == 1;
    int seg = curv ? 0 : orc_track_nearest(p, x0[3], x0[4], &d2v);
    const double w2 = p->half_width * p->half_width;
    R d2 = curv ? x[4] * x[4] : seg_dist2<R>(p, seg, x[3], x[4]);
    R h_prev = R(w2) - d2;
    R J = R(0.0);
    if (w_run != 0.0) {
        R ev = x[0] - R(p->v_target);
        J = J + R(w_run) * (R(p->q_v) * ev * ev + R(p->q_d / w2) * d2 +
                             R(val(d2) > w2 ? p->C_obs : 0.0));
    }
    for (int t = 0; t < N; ++t) {
        R u[2] = {clamp_ctrl<R>(p, 0, V[2 * t]), clamp_ctrl<R>(p, 1, V[2 * t + 1])};
        R xn[6];
        step<R>(p, x, u, xn);
        for (int i = 0; i < 6; ++i) x[i] = xn[i];
        if (curv) {
            d2 = x[4] * x[4];
        } else {
            seg = orc_track_follow(p, seg, val(x[3]), val(x[4]), &d2v);
            d2 = seg_dist2<R>(p, seg, x[3], x[4]);
        }
        R h = R(w2) - d2;
        if (w_run != 0.0) {
            R ev = x[0] - R(p->v_target);
            J = J + R(w_run) * (R(p->q_v) * ev * ev + R(p->q_d / w2) * d2 +
                                 R(val(d2) > w2 ? p->C_obs : 0.0));
        }
        R arg = R(1.0 - p->alpha) * h_prev - h;
        if (w_cbf != 0.0 && val(arg) > 0.0) J = J + R(w_cbf * p->C_cbf) * arg;
        h_prev = h;
    }
    return J;
}

extern "C" {

double orc_cost(const OrcParams* p, const double x0[6], const double* V, int N, double w_run,
                double w_cbf) {
    return det_cost<double>(p, x0, V, N, w_run, w_cbf);
}

// CBF repair merit P(V) over the repair horizon N_r (Eq. 22, sign-flipped).
double orc_merit(const OrcParams* p, const double x0[6], const double* V) {
    return det_cost<double>(p, x0, V, p->N_r, 0.0, 1.0);
}

// Gradient of J with respect to v_0..v_{N-1} (2N values; the rest of grad,
// up to 2T, is zero) by forward-mode dual numbers, one direction at a time.
double orc_cost_grad(const OrcParams* p, const double x0[6], const double* V, int N, double w_run,
                     double w_cbf, double* grad) {
    std::vector<Dual> Vd(2 * (size_t)p->T);
    for (int i = 0; i < 2 * p->T; ++i) Vd[i] = Dual(V[i], 0.0);
    double J = 0.0;
    for (int i = 0; i < 2 * p->T; ++i) grad[i] = 0.0;
    for (int i = 0; i < 2 * N; ++i) {
        Vd[i].d = 1.0;
        Dual Jd = det_cost<Dual>(p, x0, Vd.data(), N, w_run, w_cbf);
        Vd[i].d = 0.0;
        grad[i] = Jd.d;
        J = Jd.v;
    }
    if (N == 0) J = det_cost<double>(p, x0, V, N, w_run, w_cbf);
    return J;
}

// Safety shield (Alg. 1, reading c9; mode 2 = BFGS, reading c27).  mode 0: n_iters fixed steps
// V <- clip(V - delta grad P).  mode 1: projected gradient with Armijo
// backtracking: s = ls_s0 / |g|_inf, V' = clip(V - s g), accept when
// P(V') <= P(V) - ls_c g'(V - V'), else halve s (ls_max_halvings trials).
// Stops when P = 0 (the CBF condition holds on every pair, so V is already
// safe).  merit_out gets P before each iteration and after the last one
// (n_iters + 1 values, repeated after an early stop).  Returns 0 when the
// loop ended normally, 5 when no trial step was accepted (stalled).
int orc_repair_bfgs(const OrcParams* p, const double x0[6], double* V, int n_iters,
                    double* merit_out, int* iters_done);

int orc_repair(const OrcParams* p, const double x0[6], double* V, int n_iters, int mode,
               double delta, double* merit_out, int* iters_done) {
    if (mode == 2) return orc_repair_bfgs(p, x0, V, n_iters, merit_out, iters_done);
    const int N = p->N_r, T = p->T;
    std::vector<double> g(2 * (size_t)T), Vt(2 * (size_t)T);
    int status = 0, it = 0;
    double P = orc_merit(p, x0, V);
    for (; it < n_iters; ++it) {
        merit_out[it] = P;
        if (P == 0.0) break;
        orc_cost_grad(p, x0, V, N, 0.0, 1.0, g.data());
        if (mode == 0) {
            for (int i = 0; i < 2 * N; ++i) V[i] = clamp_ctrl<double>(p, i & 1, V[i] - delta * g[i]);
            P = orc_merit(p, x0, V);
            continue;
        }
        double gmax = 0.0;
        for (int i = 0; i < 2 * N; ++i) gmax = std::fmax(gmax, std::fabs(g[i]));
        if (gmax == 0.0) { status = 5; break; }
        double s = p->ls_s0 / gmax;
        bool accepted = false;
        for (int j = 0; j < p->ls_max_halvings; ++j) {
            for (int i = 0; i < 2 * T; ++i) Vt[i] = V[i];
            double dec = 0.0;
            for (int i = 0; i < 2 * N; ++i) {
                Vt[i] = clamp_ctrl<double>(p, i & 1, V[i] - s * g[i]);
                dec += g[i] * (V[i] - Vt[i]);
            }
            double Pt = orc_merit(p, x0, Vt.data());
            if (Pt <= P - p->ls_c * dec) {
                for (int i = 0; i < 2 * N; ++i) V[i] = Vt[i];
                P = Pt;
                accepted = true;
                break;
            }
            s *= 0.5;
        }
        if (!accepted) { status = 5; break; }
    }
    for (int i = it; i <= n_iters; ++i) merit_out[i] = P;
    if (iters_done) *iters_done = it;
    return status;
}

// ---------------------------------------------------------------------------
// BFGS (Sec. IV-B names it as the solver of Eq. 22, run for a fixed number of
// iterations; the variant is reading c27).
//
// Inverse update of the n x n matrix H (row-major) from the step s and the
// gradient change y, as defined:
//   H <- (I - rho s y') H (I - rho y s') + rho s s',   rho = 1 / (y' s).
// ---------------------------------------------------------------------------
void orc_bfgs_update(int n, double* H, const double* s, const double* y) {
    double ys = 0.0;
    for (int i = 0; i < n; ++i) ys += y[i] * s[i];
    const double rho = 1.0 / ys;
    std::vector<double> A((size_t)n * n), AH((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)                       // A = I - rho s y'
        for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = (i == j ? 1.0 : 0.0) - rho * s[i] * y[j];
    for (int i = 0; i < n; ++i)                       // A H
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j) AH[(size_t)i * n + j] += A[(size_t)i * n + k] * H[(size_t)k * n + j];
    for (int i = 0; i < n; ++i)                       // (A H) A' + rho s s'
        for (int j = 0; j < n; ++j) {
            double v = 0.0;
            for (int k = 0; k < n; ++k) v += AH[(size_t)i * n + k] * A[(size_t)j * n + k];
            H[(size_t)i * n + j] = v + rho * s[i] * s[j];
        }
}

}  // extern "C"

// Box-constrained BFGS with Armijo backtracking (reading c27), minimising f
// over lo <= z <= hi from z for at most n_iters iterations:
//   - H, the inverse-Hessian approximation, starts unset.  While it is unset
//     the direction is the scaled gradient step of mode 1, d = -(s0/|g|_inf) g.
//   - After an accepted step s = z' - z with y = g(z') - g(z): when
//     s'y > 1e-5 |s| |y|, H is set to (s'y / y'y) I if it was unset and then
//     takes the update of orc_bfgs_update; otherwise H is kept as it is.
//   - Binding coordinates (at a bound with the gradient pushing outward:
//     z_i = lo_i and g_i > 0, or z_i = hi_i and g_i < 0) keep d_i = 0.  With
//     H set, the free coordinates take d_F = -H_FF g_F (H restricted to the
//     free rows and columns); H is unset (and the gradient step taken) when
//     g'd >= 0.
//   - Line search: trials z(a) = clip(z + a d), a = 1, 1/2, 1/4, ...
//     (ls_max trials); the first with dec = g'(z - z(a)) > 0 and
//     f(z(a)) <= f(z) - c dec is accepted.  If none is and d came from H, H
//     is unset and the search is repeated along the gradient step; if none is
//     then, the iteration stops (stalled).
//   - The loop stops early when f = 0 (for the repair: already safe).
// merit_out gets f before each iteration and after the last one (n_iters + 1
// values, repeated after an early stop).  Returns 0, or 5 when stalled.
// F provides double value(const double* z) and void grad(const double* z, double* g).
template <class F>
static int bfgs_box(F& f, int n, const double* lo, const double* hi, double* z, int n_iters,
                    double s0, double c, int ls_max, double* merit_out, int* iters_done) {
    std::vector<double> g(n), gp(n), s(n), y(n), d(n), zt(n), H((size_t)n * n);
    std::vector<char> fr(n);
    bool H_set = false, have_step = false;
    int status = 0, it = 0;
    double fz = f.value(z);
    double gmax = 0.0;
    auto gradient_step = [&]() {
        for (int i = 0; i < n; ++i) d[i] = fr[i] ? -(s0 / gmax) * g[i] : 0.0;
    };
    auto line_search = [&](double* f_new) {
        double a = 1.0;
        for (int j = 0; j < ls_max; ++j) {
            double dec = 0.0;
            for (int i = 0; i < n; ++i) {
                zt[i] = std::fmin(std::fmax(z[i] + a * d[i], lo[i]), hi[i]);
                dec += g[i] * (z[i] - zt[i]);
            }
            if (dec > 0.0) {
                const double ft = f.value(zt.data());
                if (ft <= fz - c * dec) {
                    *f_new = ft;
                    return true;
                }
            }
            a *= 0.5;
        }
        return false;
    };
    for (; it < n_iters; ++it) {
        merit_out[it] = fz;
        if (fz == 0.0) break;
        f.grad(z, g.data());
        if (have_step) {
            double sy = 0.0, yy = 0.0, ss = 0.0;
            for (int i = 0; i < n; ++i) {
                y[i] = g[i] - gp[i];
                sy += s[i] * y[i];
                yy += y[i] * y[i];
                ss += s[i] * s[i];
            }
            if (sy > 1e-5 * std::sqrt(ss * yy)) {
                if (!H_set) {
                    for (size_t k = 0; k < H.size(); ++k) H[k] = 0.0;
                    for (int i = 0; i < n; ++i) H[(size_t)i * n + i] = sy / yy;
                    H_set = true;
                }
                orc_bfgs_update(n, H.data(), s.data(), y.data());
            }
        }
        gmax = 0.0;
        for (int i = 0; i < n; ++i) {
            gmax = std::fmax(gmax, std::fabs(g[i]));
            fr[i] = !((z[i] <= lo[i] && g[i] > 0.0) || (z[i] >= hi[i] && g[i] < 0.0));
        }
        if (gmax == 0.0) { status = 5; break; }
        if (H_set) {
            double gd = 0.0;
            for (int i = 0; i < n; ++i) {
                double v = 0.0;
                if (fr[i])
                    for (int j = 0; j < n; ++j)
                        if (fr[j]) v += H[(size_t)i * n + j] * g[j];
                d[i] = -v;
                gd += g[i] * d[i];
            }
            if (!(gd < 0.0)) {
                H_set = false;
                gradient_step();
            }
        } else {
            gradient_step();
        }
        double f_new = fz;
        bool ok = line_search(&f_new);
        if (!ok && H_set) {
            H_set = false;
            gradient_step();
            ok = line_search(&f_new);
        }
        if (!ok) { status = 5; break; }
        for (int i = 0; i < n; ++i) {
            s[i] = zt[i] - z[i];
            gp[i] = g[i];
            z[i] = zt[i];
        }
        fz = f_new;
        have_step = true;
    }
    for (int i = it; i <= n_iters; ++i) merit_out[i] = fz;
    if (iters_done) *iters_done = it;
    return status;
}

// The repair merit P as a function of the first 2 N_r controls (the rest of V
// held fixed), with its gradient by dual numbers.
struct RepairObjective {
    const OrcParams* p;
    const double* x0;
    std::vector<double> V;
    double value(const double* z) {
        for (int i = 0; i < 2 * p->N_r; ++i) V[i] = z[i];
        return orc_merit(p, x0, V.data());
    }
    void grad(const double* z, double* g) {
        for (int i = 0; i < 2 * p->N_r; ++i) V[i] = z[i];
        std::vector<double> gall(2 * (size_t)p->T);
        orc_cost_grad(p, x0, V.data(), p->N_r, 0.0, 1.0, gall.data());
        for (int i = 0; i < 2 * p->N_r; ++i) g[i] = gall[i];
    }
};

// f(z) = 1/2 z'Az - b'z (A symmetric, row-major), for the checks of bfgs_box.
struct QuadraticObjective {
    int n;
    const double* A;
    const double* b;
    double value(const double* z) {
        double v = 0.0;
        for (int i = 0; i < n; ++i) {
            double Az = 0.0;
            for (int j = 0; j < n; ++j) Az += A[(size_t)i * n + j] * z[j];
            v += 0.5 * z[i] * Az - b[i] * z[i];
        }
        return v;
    }
    void grad(const double* z, double* g) {
        for (int i = 0; i < n; ++i) {
            double Az = 0.0;
            for (int j = 0; j < n; ++j) Az += A[(size_t)i * n + j] * z[j];
            g[i] = Az - b[i];
        }
    }
};

extern "C" {

// BFGS repair of V (mode 2 of orc_repair; reading c27).
int orc_repair_bfgs(const OrcParams* p, const double x0[6], double* V, int n_iters,
                    double* merit_out, int* iters_done) {
    const int n = 2 * p->N_r;
    RepairObjective f{p, x0, std::vector<double>(V, V + 2 * (size_t)p->T)};
    std::vector<double> lo(n), hi(n), z(V, V + n);
    for (int i = 0; i < n; ++i) {
        lo[i] = p->u_min[i & 1];
        hi[i] = p->u_max[i & 1];
    }
    const int st = bfgs_box(f, n, lo.data(), hi.data(), z.data(), n_iters, p->ls_s0, p->ls_c,
                            p->ls_max_halvings, merit_out, iters_done);
    for (int i = 0; i < n; ++i) V[i] = z[i];
    return st;
}

// bfgs_box on the quadratic 1/2 z'Az - b'z (checks of the solver itself).
int orc_bfgs_quadratic(int n, const double* A, const double* b, const double* lo,
                       const double* hi, double* z, int n_iters, double s0, double c, int ls_max,
                       double* merit_out, int* iters_done) {
    QuadraticObjective f{n, A, b};
    return bfgs_box(f, n, lo, hi, z, n_iters, s0, c, ls_max, merit_out, iters_done);
}

// Closed loop (Alg. 2, ExecuteCommand, on the disturbed system Eq. 26):
// x0 <- f(x0, clamp(v0)) + w_n.
void orc_apply(const OrcParams* p, const double x0[6], const double v0[2], uint32_t n,
               uint32_t instance, double x_out[6]) {
    double u[2] = {clamp_ctrl<double>(p, 0, v0[0]), clamp_ctrl<double>(p, 1, v0[1])};
    double w[6];
    step<double>(p, x0, u, x_out);
    orc_disturbance(p, n, instance, w);
    for (int i = 0; i < 6; ++i) x_out[i] += w[i];
}

// Warm start V <- shift(V^+) (Alg. 2, last line; reading c13): drop v_0 and
// repeat the last control.
void orc_shift(const OrcParams* p, const double* Vplus, double* V_out) {
    const int T = p->T;
    for (int t = 0; t + 1 < T; ++t) {
        V_out[2 * t] = Vplus[2 * (t + 1)];
        V_out[2 * t + 1] = Vplus[2 * (t + 1) + 1];
    }
    V_out[2 * (T - 1)] = Vplus[2 * (T - 1)];
    V_out[2 * (T - 1) + 1] = Vplus[2 * (T - 1) + 1];
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"
