/*
 * smppi.h -- C ABI of the GB300 (sm_103a) Shield-MPPI hot path.
 *
 * Method: Yin, Dawson, Fan, Tsiotras, "Shield Model Predictive Path Integral:
 * A Computationally Efficient Robust MPC Approach Using Control Barrier
 * Functions", arXiv 2302.11719.  One Shield-MPPI control update (Alg. 2) is
 *   1. K Gaussian perturbations of the nominal controls V (Sec. II),
 *   2. forward simulation of every perturbed sequence through the vehicle
 *      model x_{k+1} = f(x_k, u_k) (Eq. 1),
 *   3. trajectory cost with the DCBF penalty on the augmented state
 *      (Eq. 12, Eq. 17-20; safe set h = w^2 - e_y^2, Eq. 23; running cost
 *      Eq. 24-25),
 *   4. the min-shifted softmin control update (Eq. 10-11),
 *   5. the safety shield: gradient repair of the CBF objective (Eq. 22,
 *      Alg. 1),
 *   6. execution of v_0^safe on the (disturbed, Eq. 26) system and the warm
 *      start V <- V^+.
 *
 * Conventions of every entry point:
 *   - Arrays are float32 (merits: float64), C-contiguous, in DEVICE memory
 *     unless the argument says host.  The caller owns them; the library never
 *     frees or keeps a caller pointer beyond the call, except params.track_xy,
 *     which must stay valid until smppi_destroy.
 *   - State x = (v_x, v_y, r, X, Y, psi) (6 floats); control u = (delta, a)
 *     (steer in rad, throttle in [-1, 1]); a control sequence is T x 2.
 *     A start state whose position is not finite (or beyond ~1e19 m) has no
 *     nearest centreline segment: the kernels then start from segment 0, set
 *     SMPPI_DEV_NUMERIC and produce NaN costs (V+ then lies on the lower
 *     corner of the control box); the handle stays usable.  Host-buffer calls
 *     refuse an x0 with a non-finite entry or a position beyond 1e18 m with
 *     SMPPI_ERR_ARG before anything is enqueued.
 *     NaN or Inf arising later (in velocities, costs, merits) is flagged as
 *     described below.
 *   - All work is enqueued on the handle's CUDA stream and is asynchronous;
 *     no entry point synchronises unless it says so.  Argument errors are
 *     found on the host before anything is enqueued and return SMPPI_ERR_ARG;
 *     failed CUDA calls return SMPPI_ERR_CUDA.  Conditions found on the device
 *     (NaN/Inf in a state or cost, a stalled line search) are recorded in a
 *     device status word that smppi_sync_status reads.  smppi_last_error gives
 *     a one-line message for the last failure on the handle.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key = seed and
 *     counter = (k, t >> 1, iter, stream | instance << 8); even t uses output
 *     words (0, 1), odd t words (2, 3); Box-Muller on
 *     u = ((x >> 9) + 1/2) 2^-23.  Stream 0 = MPPI noise, stream 1 = closed-
 *     loop disturbance (counter (0, 0, n, 1 | instance << 8)).  Noise is
 *     regenerated where it is used and never stored.
 *   - Not thread-safe per handle; distinct handles are independent.
 */
#ifndef SMPPI_H
#define SMPPI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SMPPI_OK = 0,
    SMPPI_ERR_ARG = 1,      /* invalid argument (null pointer, size or value out of range) */
    SMPPI_ERR_CUDA = 2,     /* a CUDA runtime call or kernel launch failed */
    SMPPI_ERR_NUMERIC = 3,  /* NaN or Inf in a state, cost or merit (device status) */
    SMPPI_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up (device status) */
    SMPPI_ERR_STALLED = 5,  /* the repair line search accepted no trial step */
    SMPPI_ERR_NOMEM = 6     /* workspace allocation failed */
} smppi_status;

/* Device status bits (smppi_sync_status folds them into a status code). */
#define SMPPI_DEV_NUMERIC 1u
#define SMPPI_DEV_TIMEOUT 2u
#define SMPPI_DEV_STALLED 4u

/* Limits of the library. */
#define SMPPI_MAX_T 512        /* horizon */
#define SMPPI_MAX_TRACK 2048   /* centreline points (staged in shared memory) */

/*
 * Problem parameters (host struct, copied at create).  Names follow the paper:
 * lambda = temperature (Eq. 11); gamma = control-cost weight of Alg. 2
 * (Eq. 8 has gamma = lambda); alpha = class-kappa rate p(r) = alpha r, the
 * paper's beta (Eq. 15), so the penalty threshold is (1 - alpha) h(x_{k-1})
 * (Eq. 17); C_cbf = C of Eq. 17; half_width = w_T of Eq. 23; q_v, v_target,
 * q_d, C_obs = the running cost q = q_v (v_x - v_target)^2 + q_d e_y^2 / w^2
 * + C_obs 1(outside) (Eq. 24-25).
 */
typedef struct smppi_params {
    float m, Iz, lf, lr;        /* vehicle: mass, yaw inertia, CoG-axle distances */
    float B, Ct, g, fx_gain;    /* tyre Fy = Fz sin(Ct atan(B slip)), gravity, rear N per throttle */
    float dt;                   /* explicit Euler step (s) */
    float sigma[2];             /* Sigma = diag(sigma^2) of the control noise */
    float lambda, gamma;
    int K, T, N_r;              /* rollouts, horizon (<= SMPPI_MAX_T), repair horizon (<= T) */
    float alpha, C_cbf;
    float q_v, v_target, q_d, C_obs;
    float u_min[2], u_max[2];   /* control box */
    float half_width;
    float dist_sigma[2];        /* disturbance std on (v_y, r) of Eq. 26 */
    float ls_s0, ls_c;          /* Armijo: first step ls_s0 / |g|_inf, sufficient decrease ls_c */
    int ls_max_halvings;        /* trial steps per line search */
    int checkpoint;             /* adjoint checkpoint interval (0 = ceil(sqrt(T))) */
    int max_seq;                /* most sequences one repair / cost_grad call handles */
    int n_track;                /* centreline points, 3..SMPPI_MAX_TRACK */
    const float* track_xy;      /* DEVICE, n_track x 2: closed centreline polyline */
    uint64_t seed;              /* Philox key */
    int state_kind;             /* 0: x = (v_x, v_y, r, X, Y, psi), e_y = distance to the
                                 * polyline (tracked); 1: curvilinear x = (v_x, v_y, r, s,
                                 * e_y, e_psi) of the paper's AutoRally model (Sec. VI-A):
                                 * s = arc length, e_y = lateral offset (left positive),
                                 * e_psi = heading error, on the centreline's curvature
                                 * kappa(s) (see below).  1 needs Ct = 1.5 and
                                 * |steer| <= 1/2; the batch and smppi_step_noalloc
                                 * refuse it; smppi_cost_grad and the repair keep the
                                 * whole trajectory (no checkpoints). */
} smppi_params;

/* Curvilinear state (state_kind = 1):
 *   kappa(s): at each vertex P_i the turning angle between P_i - P_{i-1} and
 *   P_{i+1} - P_i over the mean length of the two segments; piecewise linear in
 *   the arc length between the vertices; sampled at n_track uniform stations
 *   s = j L / n_track (L = the closed polyline's length) and interpolated
 *   linearly between the samples, s taken modulo L.
 *   ds/dt = (v_x cos e_psi - v_y sin e_psi) / max(1 - kappa e_y, 0.1),
 *   de_y/dt = v_x sin e_psi + v_y cos e_psi,  de_psi/dt = r - kappa ds/dt;
 *   explicit Euler like the Cartesian model; h = w^2 - e_y^2 and q use e_y.
 *   smppi_create returns SMPPI_ERR_ARG when two consecutive vertices of the
 *   track coincide (the curvature is undefined there). */

typedef struct smppi_handle smppi_handle;

/* Fill *p with the single-problem defaults (m = 21.7, Iz = 1.12, lf = 0.34,
 * lr = 0.23, B = 4, Ct = 1.5, g = 9.81, fx_gain = 60, dt = 0.02,
 * sigma = (0.15, 0.3), lambda = gamma = 1, K = 256, T = N_r = 50, alpha = 0.3,
 * C_cbf = 1000, q = 2 (v_x - 8)^2 + 100 e_y^2 / w^2, box [-0.5, 0.5] x [-1, 1],
 * w = 2, disturbance 0.3, Armijo 0.1 / 1e-4 / 20, max_seq = 1); track_xy is
 * left NULL. */
void smppi_default_params(smppi_params* p);

/* Create a handle: validates p, copies it, allocates the workspace for p->K
 * rollouts, horizon p->T and p->max_seq repair sequences, and prepares the
 * segment table of the track on `cuda_stream` (a cudaStream_t; NULL = the
 * legacy default stream).  On failure *out is NULL. */
smppi_status smppi_create(const smppi_params* p, void* cuda_stream, smppi_handle** out);

/* Free the workspace after synchronising the handle's stream.  NULL is a no-op. */
smppi_status smppi_destroy(smppi_handle* h);

/* Message of the last failure on h; with h NULL, of the last failed call
 * without a handle (create, smppi_step_noalloc, smppi_debug_wait_timeout) on
 * the calling host thread.  Valid until the next failing call. */
const char* smppi_last_error(const smppi_handle* h);

/* Synchronise the stream, read and clear the device status word; returns
 * SMPPI_OK or the first of NUMERIC / TIMEOUT / STALLED that is set.  If
 * bits_out is not NULL the raw bits are written there (host). */
smppi_status smppi_sync_status(smppi_handle* h, uint32_t* bits_out);

/*
 * One MPPI iteration (Alg. 2, sampling loop + OptimalControl; Eq. 10-12, 20).
 *   x0   [6]        current state
 *   V    [T x 2]    in: nominal controls v_t; out: V^+ (Eq. 10, clamped to the box)
 *   iter            Philox counter word (the control-update index)
 *   instance        Philox counter word (problem index, < 2^24)
 *   S_out [K]       optional (NULL): per-rollout cost S~ (Eq. 20)
 *   traj_out [K x (T+1) x 6]  optional (NULL): every sampled trajectory
 * Rollout costs accumulate in float32; the cross-block min / normaliser merge
 * of Eq. 11 and the weighted noise sum run in float64.
 */
smppi_status smppi_step(smppi_handle* h, const float* x0, float* V, uint32_t iter,
                        uint32_t instance, float* S_out, float* traj_out);

/*
 * Rollouts sharded over several devices or calls (Eq. 10-11 over a partition of
 * the K rollouts; Alg. 2's sampling loop is a parallel loop over them).  The
 * weights are min-shifted per slice and rescaled at the merge, a log-sum-exp
 * merge: omega_k = exp(-(S_k - m)/lambda) = c_g exp(-(S_k - m_g)/lambda) with
 * m = min_g m_g and c_g = exp(-(m_g - m)/lambda).
 *
 * smppi_step_partial runs rollouts k_lo .. k_hi - 1 of iteration (iter,
 * instance) (their Philox counters, so slices of one iteration on different
 * devices draw exactly the noise of the unsharded iteration) and writes
 *   partial_out [2T + 2] (DEVICE, float64) = (m_g, eta_g, A_g[0 .. 2T - 1]):
 *   m_g = min S_k over the slice, eta_g = sum exp(-(S_k - m_g)/lambda) and
 *   A_g[2t + j] = sum exp(-(S_k - m_g)/lambda) eps_{k,t,j} (the noise sum of
 *   rollouts whose slice weight exceeds the skip threshold of all K rollouts).
 * V [T x 2] is read, not written.  0 <= k_lo < k_hi <= K (the handle's K),
 * else SMPPI_ERR_ARG.  Uses the handle's workspace (one slice at a time per
 * handle).
 *
 * smppi_merge_partials forms V <- clamp(V + A / eta) from n_parts partials
 * [n_parts x (2T + 2)] (DEVICE, float64, e.g. gathered from every device by
 * an all-gather), with eta = sum_g c_g eta_g and A = sum_g c_g A_g summed in
 * float64 in slice order, so every device that merges the same partials gets
 * the same V+.  One partial covering all K gives smppi_step's V+ bit for bit.
 * n_parts in [1, 1024], else SMPPI_ERR_ARG.
 */
smppi_status smppi_step_partial(smppi_handle* h, const float* x0, const float* V, uint32_t iter,
                                uint32_t instance, int k_lo, int k_hi, double* partial_out);
smppi_status smppi_merge_partials(smppi_handle* h, int n_parts, const double* partials,
                                  float* V);

/* The control update alone (Eq. 10-11) from given rollout costs S [K]: the
 * noise of iteration (iter, instance) is regenerated.  V [T x 2] in/out as
 * in smppi_step. */
smppi_status smppi_update(smppi_handle* h, const float* S, float* V, uint32_t iter,
                          uint32_t instance);

/*
 * Deterministic cost and its gradient for n_seq independent sequences
 * (n_seq <= max_seq), by a reverse-mode adjoint with checkpoints every
 * `checkpoint` steps (0 = the handle's) and recomputation in the backward
 * sweep; checkpoint < 0 stores the whole trajectory instead (full tape).
 *   J(V) = w_run sum_{t=0}^{N} q(x_t) + w_cbf sum_{t=0}^{N-1} C max{(1-alpha) h_t - h_{t+1}, 0}
 * with x_{t+1} = f(x_t, clamp(v_t)) from x0 (Eq. 1, 17, 23-24); (0, 1) is
 * the repair objective P = -C x (objective of Eq. 22).
 *   x0 [n_seq x 6], V [n_seq x T x 2], N <= T (horizon of the sum),
 *   J_out [n_seq] (float64), grad_out [n_seq x T x 2] (zero for t >= N).
 * max(0, .) has derivative 0 at a non-positive argument; clamp passes the
 * derivative on the closed box and blocks it strictly outside.
 */
smppi_status smppi_cost_grad(smppi_handle* h, int n_seq, const float* x0, const float* V,
                             int N, float w_run, float w_cbf, int checkpoint,
                             double* J_out, float* grad_out);

/*
 * Safety shield (Alg. 1, Eq. 22) on n_seq independent sequences
 * (n_seq <= max_seq): n_iters steps on the first N_r controls of each.
 *   mode 0: V <- clip(V - delta grad P)                      (Alg. 1, fixed step)
 *   mode 1: projected gradient with Armijo backtracking: s = ls_s0 / |g|_inf,
 *           accept clip(V - s g) when P' <= P - ls_c g'(V - V'), else halve s
 *           (ls_max_halvings trials); stop early when P = 0 (already safe).
 *   mode 2: BFGS (the solver Sec. IV-B names), box-projected: an inverse-
 *           Hessian approximation H over the 2 N_r controls, unset at first
 *           (direction = the mode-1 step -(ls_s0/|g|_inf) g); after each
 *           accepted step s with gradient change y and s'y > 1e-5 |s||y|, H
 *           (first (s'y/y'y) I) takes H <- (I - rho s y') H (I - rho y s')
 *           + rho s s', rho = 1/(y's).  Coordinates at a bound whose gradient
 *           pushes outward keep d_i = 0; the others take d = -H_FF g_F (H is
 *           unset again when g'd >= 0).  Trials clip(V + a d), a = 1, 1/2, ...
 *           (ls_max_halvings), accepted when g'(V - V') > 0 and
 *           P' <= P - ls_c g'(V - V'); if none is and d came from H, the search
 *           is repeated along the gradient step.  One warp per sequence (both
 *           state kinds).  When 2 n_iters (2 N_r + 1) <= (2 N_r)^2 the warp keeps
 *           the curvature pairs since the last reset and applies H by the
 *           two-loop recursion (the same H in exact arithmetic), otherwise H
 *           itself.  A mode-2 call that needs more workspace than the handle holds
 *           allocates it (a work counter and (2 N_r)^2 floats per resident
 *           warp, about 256 MB at most).
 *   x0 [n_seq x 6]; V_in, V_out [n_seq x T x 2] (may alias);
 *   merit_out [n_seq x (n_iters + 1)] optional (float64): P before each
 *   iteration and after the last, repeated after an early stop;
 *   iters_out [n_seq] optional (int32): iterations run per sequence.
 * A sequence whose line search accepts nothing keeps its last iterate and
 * sets SMPPI_DEV_STALLED in the status word.  The merit accumulates in float64.
 */
smppi_status smppi_repair(smppi_handle* h, int n_seq, const float* x0, const float* V_in,
                          float* V_out, int n_iters, int mode, float delta,
                          double* merit_out, int* iters_out);

/*
 * Closed-loop step (Alg. 2 ExecuteCommand and warm start; Eq. 26):
 *   x0 [6] in/out:  x0 <- f(x0, clamp(V_exec[0])) + w_n, w_n on stream 1
 *   V  [T x 2] in/out: V <- shift(V) (drop v_0, repeat v_{T-1})
 *   V_exec [T x 2]: the sequence whose first control is executed (V^safe)
 */
smppi_status smppi_apply(smppi_handle* h, float* x0, float* V, const float* V_exec, uint32_t n,
                         uint32_t instance);

/*
 * One whole Shield-MPPI control update (Alg. 2 body) on the handle's stream:
 * smppi_step, then smppi_repair (mode 1, n_repair iterations) of V^+ into
 * V_safe, then the closed-loop step (smppi_apply) with n = iter.
 *   host_buffers = 0: x0 [6], V [T x 2], V_safe [T x 2] are device arrays.
 *   host_buffers = 1: they are host arrays (any host memory); the update
 *   copies x0 and V in and x0, V, V_safe (and the merits) out in one copy each
 *   way through a staging block of the handle and its pinned host mirror
 *   (allocated on first use), replays the copies and the launches from a CUDA
 *   graph the handle keeps per (instance, n_repair, merits), and synchronises
 *   the stream before returning.  Per-kernel timing does not cover these calls.
 *   merit_out [n_repair + 1] optional, device (or host when host_buffers = 1).
 */
smppi_status smppi_shield_update(smppi_handle* h, float* x0, float* V, float* V_safe,
                                 uint32_t iter, uint32_t instance, int n_repair,
                                 double* merit_out, int host_buffers);

/* Capture smppi_shield_update(device buffers) into a CUDA graph owned by the
 * handle and replay it `n_updates` times, iter = iter0 .. iter0 + n_updates-1
 * (the graph is re-instantiated when the arguments change). */
smppi_status smppi_shield_loop(smppi_handle* h, float* x0, float* V, float* V_safe,
                               uint32_t iter0, uint32_t instance, int n_repair, int n_updates);

/*
 * Batched Shield-MPPI: B independent control problems with their own K_i, T_i,
 * centreline and state; one closed-loop update of all of them (Alg. 2 body per
 * problem: sampling loop, OptimalControl, SafetyShield, ExecuteCommand on the
 * disturbed system of Eq. 26, warm start) in ONE persistent launch over a
 * device work queue of (problem, chunk of rollouts) items.  The block that
 * finishes a problem's last chunk forms its V+, repairs it and steps its
 * closed loop while the other blocks keep taking rollout items.
 */
typedef struct smppi_instance_desc {
    int K, T, N_r;              /* rollouts, horizon, repair horizon of this problem */
    int n_track;                /* centreline points (3..SMPPI_MAX_TRACK) */
    float half_width;           /* w_T of Eq. 23 */
    int track_offset;           /* first point of this problem in tracks_xy */
    int V_offset;               /* first control of this problem in the V / V_safe arrays */
} smppi_instance_desc;

typedef struct smppi_batch smppi_batch;

/* Create a batch.  `shared` supplies the parameters common to all problems
 * (model, noise, temperature, cost weights, CBF alpha and C, Armijo settings,
 * checkpoint, seed); its K, T, N_r, n_track, track_xy, half_width and max_seq
 * are ignored.  desc [B] (host) describes each problem; tracks_xy (device)
 * holds all centrelines back to back (2 floats per point), and must stay
 * valid only during this call.  block_rollouts: rollouts per work item (64,
 * 128 or 256), or 0 to let the autotuner pick it together with the grid at
 * the first smppi_batch_step / smppi_batch_loop (it times one update of each
 * candidate on a scratch copy of the state; the caller's arrays are untouched). */
smppi_status smppi_batch_create(const smppi_params* shared, int B,
                                const smppi_instance_desc* desc, const float* tracks_xy,
                                int block_rollouts, void* cuda_stream, smppi_batch** out);
smppi_status smppi_batch_destroy(smppi_batch* b);
/* Message of the last failure on b; with b NULL, of the last failed
 * smppi_batch_create on the calling host thread. */
const char* smppi_batch_last_error(const smppi_batch* b);

/* One closed-loop Shield-MPPI update of all B problems (device arrays):
 *   x0 [B x 6] in/out; V in/out (nominal -> warm start shift(V+)); V_safe out
 *   (the repaired sequences); both indexed by desc[i].V_offset, T_i x 2 each;
 *   iter: update index (Philox counter word and disturbance index);
 *   n_repair: Armijo repair iterations per problem (0 = plain MPPI with the
 *   DCBF cost, V_safe = V+). */
smppi_status smppi_batch_step(smppi_batch* b, float* x0, float* V, float* V_safe,
                              uint32_t iter, int n_repair);

/* n_updates closed-loop updates replayed from a CUDA graph (iter = iter0 ..). */
smppi_status smppi_batch_loop(smppi_batch* b, float* x0, float* V, float* V_safe,
                              uint32_t iter0, int n_repair, int n_updates);

/* Synchronise the batch stream and read / clear its device status word.
 * After SMPPI_DEV_TIMEOUT (a block gave up on a bounded wait and left the
 * launch) the problems' completion counters are cleared as well; the state
 * of the problems that block held (x0, V, V_safe) is then undefined.  While
 * the TIMEOUT bit is set (until this call reads it), batch launches take no
 * further work items, so a launch, and every later replay of a loop, ends
 * within about one wait limit; the problems they do not reach keep their
 * state. */
smppi_status smppi_batch_sync_status(smppi_batch* b, uint32_t* bits_out);

/* The launch shape in use (after autotuning): rollouts per item and grid size. */
smppi_status smppi_batch_config(const smppi_batch* b, int* block_rollouts, int* grid);

/* Safety monitor of the batch (not part of the paper's method; it measures
 * the closed loop the paper evaluates in Sec. VI).  For every problem, the
 * number of executed closed-loop steps x_n -> x_{n+1} since creation (or the
 * last read with reset != 0) that violated the discrete CBF condition of
 * Eq. 15 / 17, h(x_{n+1}) < (1 - alpha) h(x_n), and that ended outside the
 * track, h(x_{n+1}) < 0, with h = w^2 - e_y^2 (Eq. 23) and e_y tracked from
 * x_n's nearest segment (the same projection as the cost).  viol_out and
 * outside_out (host, B each) may be NULL.  Synchronises the batch's stream.
 * The autotuner's timing runs are not counted. */
smppi_status smppi_batch_monitor(smppi_batch* b, uint32_t* viol_out, uint32_t* outside_out,
                                 int reset);

/*
 * smppi_step without any allocation, for callers that cannot allocate device
 * memory: control loops that forbid allocation once running, or runtimes that
 * own every device allocation.  (The paper has no counterpart; this is a
 * deployment variant of smppi_step.)  Same arguments and results as smppi_step
 * (no trajectory dump), but no handle: p is validated and used on every call,
 * and the work is enqueued on `cuda_stream` (a cudaStream_t, NULL = legacy
 * default stream).  Limits: K <= 65536 (SMPPI_ERR_ARG beyond, with a message
 * for smppi_last_error(NULL)), T <= SMPPI_MAX_T, n_track <= SMPPI_MAX_TRACK.
 * Scratch: one fixed 1.4 MB array per GPU inside the library, held until the
 * process exits.  The first call on a device looks up that array's device
 * address; make it before any stream capture.  Later calls outside a capture
 * look the address up again (it does not survive a device reset); calls
 * inside a capture reuse the last one.  Every call on a device shares the
 * array and leaves its contents behind; calls that overlap on the GPU race on
 * it.  Device-side checks are not reported: with a NaN in x0 or in the costs
 * the call still returns SMPPI_OK and V+ lies on the lower corner of the
 * control box.
 */
smppi_status smppi_step_noalloc(const smppi_params* p, const float* x0, float* V, uint32_t iter,
                                uint32_t instance, float* S_out, void* cuda_stream);

/*
 * Per-kernel timing (CUDA events recorded on the handle's stream around each
 * kernel launch).  smppi_timing(h, 1) starts recording, (h, 0) stops it.
 * smppi_timing_read synchronises the stream, writes for each kernel kind k <
 * n_kinds the summed duration in ms (ms_out[k], host) and the number of
 * launches (count_out[k], host), and resets the record.  Kinds:
 */
#define SMPPI_KERNEL_ROLLOUT 0    /* rollouts and trajectory costs */
#define SMPPI_KERNEL_UPDATE 1     /* softmin weights, weighted noise sum, float64 merge -> V+ */
#define SMPPI_KERNEL_SEG0 2       /* nearest segment of x0 */
#define SMPPI_KERNEL_REPAIR 3     /* safety shield iterations */
#define SMPPI_KERNEL_APPLY 4      /* closed-loop step */
#define SMPPI_KERNEL_COST_GRAD 5  /* cost + adjoint gradient */
#define SMPPI_KERNEL_UPDATE_SHIELD 6  /* update -> V+, then (last block) shield and closed-loop step */
#define SMPPI_KERNEL_MERGE 7      /* merge of slice partials -> V+ */
#define SMPPI_KERNEL_KINDS 8
smppi_status smppi_timing(smppi_handle* h, int enable);
smppi_status smppi_timing_read(smppi_handle* h, double* ms_out, int* count_out, int n_kinds);

/*
 * Test access to the device noise generator: for k < K, t < T writes
 * eps_out[(k T + t) 2 + j] = the control noise of rollout k, step t exactly as
 * the rollout kernels draw it (stream 0), and, if raw_out is not NULL,
 * raw_out[(k ceil(T/2) + p) 4 + i] = Philox word i of counter (k, p, iter,
 * instance << 8).  Both device arrays.
 */
smppi_status smppi_debug_noise(smppi_handle* h, uint32_t iter, uint32_t instance, int K, int T,
                               float* eps_out, uint32_t* raw_out);

/*
 * Test access to the hand-written elementary functions of the rollout and
 * repair kernels (no handle; not part of the method): for i < n, out[i] = the
 * library's function and ref[i] = CUDA's own function of the same arguments:
 *   fn 0: atan2(a, b), scalar form      ref atan2f(a, b)
 *   fn 1: atan2(a, b), packed pair form  ref atan2f(a, b)
 *   fn 2: sin(1.5 atan a), scalar        ref sinf(1.5f atanf(a))
 *   fn 3: sin(1.5 atan a), packed        ref sinf(1.5f atanf(a))
 *   fn 4 / 5: sin / cos of a, |a| <= 1/2, scalar   ref sinf / cosf
 *   fn 6 / 7: sin / cos of a, |a| <= 1/2, packed   ref sinf / cosf
 *   fn 8: atan2(a, b), packed pair form of the one-thread recurrences
 *         (Estrin's scheme, octant folded into one FMA)   ref atan2f(a, b)
 *   fn 9: 1 / sqrt(a) without the denormal path, as the tyre and
 *         Box-Muller use it (arguments never denormal)     ref rsqrtf(a)
 * (b is read by fn 0, 1 and 8 only but must not be NULL).  Packed forms evaluate
 * elements 2i and 2i + 1 as the two halves of one instruction.  All arrays
 * DEVICE, float32; asynchronous on cuda_stream; SMPPI_ERR_ARG for another fn,
 * n < 0 or a NULL array.
 */
smppi_status smppi_debug_elementary(int fn, int n, const float* a, const float* b, float* out,
                                    float* ref, void* cuda_stream);

/*
 * Failure-detection self-test (no handle): launches one block of 32 threads on
 * cuda_stream that waits, through the library's bounded device waits, on
 * something nothing completes: which = 0: an mbarrier phase that no thread
 * arrives at (the wait of the bulk-copy staging; gives up after 0.25 s of the
 * global timer); which = 1: a shared-memory counter that no warp advances (the
 * wait of the split merit pass; gives up after 2^24 tries).  The block then ORs
 * SMPPI_DEV_TIMEOUT into *status (DEVICE, one word, not cleared) and returns;
 * the context stays usable.  Asynchronous; SMPPI_ERR_ARG for another `which`
 * or a NULL status.
 */
smppi_status smppi_debug_wait_timeout(int which, uint32_t* status, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SMPPI_H */
