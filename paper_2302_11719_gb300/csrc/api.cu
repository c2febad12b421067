// C ABI of the Shield-MPPI hot path (include/smppi.h): handle, workspace,
// argument checks and the launch sequence of one control update.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bfgs_launch.cuh"
#include "kernels.cuh"

using namespace smppi;

struct smppi_handle {
    smppi_params p;
    DevParams dp;
    cudaStream_t st = nullptr;
    cudaStream_t cap = nullptr;      // private stream for graph capture
    float4* rec = nullptr;           // segment-pair table of the centreline (device.cuh)
    float* S_ws = nullptr;           // [K] rollout costs
    float* blk_min = nullptr;        // [nblk] block minima of S
    float* part_acc = nullptr;       // [UPD_BLK][2T] update-kernel partials
    double* part_eta = nullptr;      // [UPD_BLK]
    int* part_has = nullptr;         // [UPD_BLK]
    unsigned* ticket = nullptr;      // last-block counter of the update launch
    int nblk = 0;
    unsigned* status = nullptr;
    uint32_t* iter_dev = nullptr;
    RepairWs rws{};
    // staging of host-buffer updates, one block each way: x0 (8 floats), V and
    // V_safe (2T floats each), then merit_cap merits; h_io is its pinned mirror
    unsigned char* d_io = nullptr;
    unsigned char* h_io = nullptr;
    int merit_cap = 0;
    cudaGraphExec_t io_exec = nullptr;   // copy in, the update, copy out (host-buffer updates)
    std::string io_key;
    float* kappa = nullptr;          // curvature samples of the curvilinear state
    void* bfgs_ws = nullptr;         // BFGS repair workspace: counter + H slices (grown on use)
    size_t bfgs_ws_bytes = 0;
    int sms = 1;
    cudaGraphExec_t gexec = nullptr;
    std::string graph_key;
    std::string err;
    // per-kernel timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::array<int, 3>> records;   // kind, start event, end event
};

namespace {

// the message of the last failure outside a handle, per host thread
thread_local std::string g_create_err;

smppi_status fail(smppi_handle* h, smppi_status s, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_err = msg;
    return s;
}

#define CU(h, call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail((h), SMPPI_ERR_CUDA,                                               \
                        std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

bool finite_pos(float v) { return std::isfinite(v) && v > 0.0f; }

smppi_status check_params(const smppi_params* p) {
    auto bad = [](const char* m) { return fail(nullptr, SMPPI_ERR_ARG, m); };
    if (!p) return bad("params is NULL");
    if (!finite_pos(p->m) || !finite_pos(p->Iz)) return bad("m and Iz must be > 0");
    if (!(p->lf >= 0) || !(p->lr >= 0) || !(p->lf + p->lr > 0)) return bad("lf, lr must be >= 0, lf + lr > 0");
    if (!std::isfinite(p->B) || !std::isfinite(p->Ct) || !std::isfinite(p->g) || !std::isfinite(p->fx_gain))
        return bad("tyre / gravity / throttle gain must be finite");
    if (!finite_pos(p->dt)) return bad("dt must be > 0");
    if (!(p->sigma[0] >= 0 && p->sigma[1] >= 0) || !std::isfinite(p->sigma[0]) || !std::isfinite(p->sigma[1]))
        return bad("sigma must be finite and >= 0");
    if (!finite_pos(p->lambda)) return bad("lambda must be > 0");
    if (!std::isfinite(p->gamma)) return bad("gamma must be finite");
    if (p->K < 1 || p->K > (1 << 22)) return bad("K must be in [1, 2^22]");
    if (p->T < 1 || p->T > SMPPI_MAX_T) return bad("T must be in [1, SMPPI_MAX_T]");
    if (p->N_r < 0 || p->N_r > p->T) return bad("N_r must be in [0, T]");
    if (!(p->alpha >= 0 && p->alpha <= 1)) return bad("alpha must be in [0, 1]");
    if (!(p->C_cbf >= 0) || !std::isfinite(p->C_cbf)) return bad("C_cbf must be finite and >= 0");
    if (!std::isfinite(p->q_v) || !std::isfinite(p->v_target) || !std::isfinite(p->q_d) || !std::isfinite(p->C_obs))
        return bad("cost weights must be finite");
    for (int j = 0; j < 2; ++j)
        if (!(p->u_min[j] <= p->u_max[j]) || !std::isfinite(p->u_min[j]) || !std::isfinite(p->u_max[j]))
            return bad("u_min <= u_max required");
    if (!finite_pos(p->half_width)) return bad("half_width must be > 0");
    if (!(p->dist_sigma[0] >= 0 && p->dist_sigma[1] >= 0)) return bad("dist_sigma must be >= 0");
    if (!finite_pos(p->ls_s0) || !(p->ls_c >= 0 && p->ls_c < 1)) return bad("ls_s0 > 0, 0 <= ls_c < 1");
    if (p->ls_max_halvings < 1 || p->ls_max_halvings > 64) return bad("ls_max_halvings in [1, 64]");
    if (p->checkpoint < 0 || p->checkpoint > SMPPI_MAX_T) return bad("checkpoint in [0, SMPPI_MAX_T]");
    if (p->max_seq < 1 || p->max_seq > (1 << 20)) return bad("max_seq in [1, 2^20]");
    if (p->n_track < 3 || p->n_track > SMPPI_MAX_TRACK) return bad("n_track in [3, SMPPI_MAX_TRACK]");
    if (!p->track_xy) return bad("track_xy is NULL");
    if (p->state_kind != 0 && p->state_kind != 1) return bad("state_kind must be 0 or 1");
    if (p->state_kind == 1 &&
        !(p->Ct == 1.5f && std::fabs(p->u_min[0]) <= 0.5f && std::fabs(p->u_max[0]) <= 0.5f))
        return bad("state_kind 1 needs Ct = 1.5 and |steer| <= 1/2");
    return SMPPI_OK;
}

// Curvature samples of the curvilinear state (smppi.h, state_kind 1), in
// double: the vertex curvatures (turning angle / mean adjacent segment
// length), linear in arc length between the vertex stations, sampled at n
// uniform stations; sample n repeats sample 0 for the interpolation.  False
// (nothing written) when two consecutive vertices coincide: the turning angle
// and the interpolation are then undefined.
bool curvature_samples(const std::vector<float>& xy, int n, std::vector<float>& out, double& L) {
    std::vector<double> seg(n), station(n + 1, 0.0), kv(n);
    for (int i = 0; i < n; ++i) {
        const int j = (i + 1) % n;
        seg[i] = std::hypot((double)xy[2 * j] - xy[2 * i], (double)xy[2 * j + 1] - xy[2 * i + 1]);
        if (!(seg[i] > 0.0) || !std::isfinite(seg[i])) return false;
        station[i + 1] = station[i] + seg[i];
    }
    L = station[n];
    for (int i = 0; i < n; ++i) {
        const int pv = (i + n - 1) % n, nx = (i + 1) % n;
        const double ux = (double)xy[2 * i] - xy[2 * pv], uy = (double)xy[2 * i + 1] - xy[2 * pv + 1];
        const double wx = (double)xy[2 * nx] - xy[2 * i], wy = (double)xy[2 * nx + 1] - xy[2 * i + 1];
        kv[i] = std::atan2(ux * wy - uy * wx, ux * wx + uy * wy) / (0.5 * (seg[pv] + seg[i]));
    }
    out.assign(n + 1, 0.0f);
    for (int j = 0; j < n; ++j) {
        const double sj = L * j / n;
        int i = (int)(std::upper_bound(station.begin(), station.begin() + n, sj) - station.begin()) - 1;
        i = std::max(0, std::min(n - 1, i));
        const double f = (sj - station[i]) / seg[i];
        out[j] = (float)((1.0 - f) * kv[i] + f * kv[(i + 1) % n]);
    }
    out[n] = out[0];
    return true;
}

DevParams derive(const smppi_params& p) {
    DevParams d{};
    const double m = p.m, lf = p.lf, lr = p.lr, g = p.g;
    d.lf = p.lf; d.lr = p.lr; d.B = p.B; d.Ct = p.Ct;
    d.Fzf = (float)(m * g * lr / (lf + lr));
    d.Fzr = (float)(m * g * lf / (lf + lr));
    d.fx_gain = p.fx_gain;
    d.m_inv = (float)(1.0 / m);
    d.Iz_inv = (float)(1.0 / (double)p.Iz);
    d.dt = p.dt;
    d.sig0 = p.sigma[0]; d.sig1 = p.sigma[1];
    const double s0 = (double)p.sigma[0] * p.sigma[0], s1 = (double)p.sigma[1] * p.sigma[1];
    d.gis0 = (float)(p.gamma == 0.0f ? 0.0 : p.gamma / s0);
    d.gis1 = (float)(p.gamma == 0.0f ? 0.0 : p.gamma / s1);
    d.lam_inv = (float)(1.0 / (double)p.lambda);
    // |eps| <= sigma_max sqrt(-2 ln 2^-24) (smallest uniform of the noise generator)
    const double e_max = std::max(p.sigma[0], p.sigma[1]) * std::sqrt(2.0 * 24.0 * std::log(2.0));
    d.w_skip = e_max > 0.0 ? (float)(1e-8 / ((double)p.K * e_max)) : 3.0e38f;
    d.one_m_alpha = (float)(1.0 - (double)p.alpha);
    d.C_cbf = p.C_cbf;
    d.q_v = p.q_v; d.v_target = p.v_target;
    const double w2 = (double)p.half_width * p.half_width;
    d.qd_w2 = (float)(p.q_d / w2);
    d.C_obs = p.C_obs;
    d.w2 = (float)w2;
    d.umin0 = p.u_min[0]; d.umin1 = p.u_min[1]; d.umax0 = p.u_max[0]; d.umax1 = p.u_max[1];
    d.dsig0 = p.dist_sigma[0]; d.dsig1 = p.dist_sigma[1];
    d.ls_s0 = p.ls_s0; d.ls_c = p.ls_c; d.ls_max = p.ls_max_halvings;
    d.K = p.K; d.T = p.T; d.N_r = p.N_r; d.n_track = p.n_track;
    d.state_kind = p.state_kind;   // the curvature table is set up by smppi_create
    d.key0 = (uint32_t)(p.seed & 0xFFFFFFFFull);
    d.key1 = (uint32_t)(p.seed >> 32);
    for (int i = 0; i < 10; ++i) {
        d.rk0[i] = d.key0 + (uint32_t)i * 0x9E3779B9u;
        d.rk1[i] = d.key1 + (uint32_t)i * 0xBB67AE85u;
    }
    d.tyre15 = (p.Ct == 1.5f) ? 1 : 0;
    d.steer_small = (std::fabs(p.u_min[0]) <= 0.5f && std::fabs(p.u_max[0]) <= 0.5f) ? 1 : 0;
    return d;
}

void free_all(smppi_handle* h) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->io_exec) cudaGraphExecDestroy(h->io_exec);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    void* ptrs[] = {h->rec, h->S_ws, h->blk_min, h->part_acc, h->part_eta, h->part_has,
                    h->ticket,
                    h->status,
                    h->iter_dev,
                    h->rws.tape, h->rws.Vw, h->rws.G, h->rws.seg0, h->d_io,
                    h->bfgs_ws, h->kappa};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (h->h_io) cudaFreeHost(h->h_io);
    if (h->cap) cudaStreamDestroy(h->cap);
}

template <class P>
cudaError_t alloc(P** ptr, size_t bytes) {
    return cudaMalloc(reinterpret_cast<void**>(ptr), bytes < 16 ? 16 : bytes);
}

// Event pair around one launch when timing is on (never inside a graph capture).
int tic(smppi_handle* h, cudaStream_t st) {
    if (!h->timing || st == h->cap) return -1;
    if (h->ev_used + 2 > h->ev_pool.size()) {
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            h->ev_pool.push_back(e);
        }
    }
    const int i0 = (int)h->ev_used;
    h->ev_used += 2;
    cudaEventRecord(h->ev_pool[i0], st);
    return i0;
}

void toc(smppi_handle* h, cudaStream_t st, int kind, int i0) {
    if (i0 < 0) return;
    cudaEventRecord(h->ev_pool[i0 + 1], st);
    h->records.push_back({kind, i0, i0 + 1});
}

smppi_status check_seq_call(smppi_handle* h, int n_seq) {
    if (!h) return fail(nullptr, SMPPI_ERR_ARG, "handle is NULL");
    if (n_seq < 1 || n_seq > h->p.max_seq)
        return fail(h, SMPPI_ERR_ARG, "n_seq must be in [1, max_seq]");
    return SMPPI_OK;
}

smppi_status enqueue_rollout(smppi_handle* h, cudaStream_t st, const float* x0, const float* V,
                             uint32_t iter, uint32_t instance, float* S, float* traj_out,
                             uint32_t* iter_dev) {
    const int ev = tic(h, st);
    if (h->p.state_kind == 1)
        CU(h, launch_rollout_curv(h->dp, h->kappa, traj_out != nullptr, x0, V, iter, instance << 8,
                                  iter_dev, S, traj_out, h->blk_min, h->status, st));
    else
        CU(h, launch_rollout(h->dp, traj_out != nullptr, x0, V, h->rec, iter, instance << 8,
                             iter_dev, S, traj_out, h->blk_min, h->rws.seg0, h->status, st));
    toc(h, st, SMPPI_KERNEL_ROLLOUT, ev);
    return SMPPI_OK;
}

smppi_status enqueue_step(smppi_handle* h, cudaStream_t st, const float* x0, float* V,
                          uint32_t iter, uint32_t instance, float* S_out, float* traj_out,
                          uint32_t* iter_dev) {
    const uint32_t ctr3 = (instance << 8) | 0u;
    float* S = S_out ? S_out : h->S_ws;
    smppi_status s = enqueue_rollout(h, st, x0, V, iter, instance, S, traj_out, iter_dev);
    if (s != SMPPI_OK) return s;
    int ev = tic(h, st);
    CU(h, launch_update(h->dp, S, h->blk_min, rollout_blocks(h->dp), V, iter, ctr3, iter_dev, h->part_acc,
                        h->part_eta, h->part_has, h->ticket, h->status, st));
    toc(h, st, SMPPI_KERNEL_UPDATE, ev);
    return SMPPI_OK;
}

// seg0_known: the nearest segment of x0 is already in the workspace (written
// by the rollout launch of the same update).  ap: optional fused closed loop.
smppi_status enqueue_repair(smppi_handle* h, cudaStream_t st, int n_seq, const float* x0,
                            const float* V_in, float* V_out, int n_iters, int mode, float delta,
                            double* merit_out, int* iters_out, bool seg0_known,
                            const ApplyArgs& ap) {
    int ev;
    const bool curv = h->p.state_kind == 1;
    if (curv && mode != 2) {
        ev = tic(h, st);
        CU(h, launch_repair_curv(h->dp, h->kappa, n_seq, x0, V_in, V_out, n_iters, mode, delta,
                                 merit_out, iters_out, ap, h->status, st));
        toc(h, st, SMPPI_KERNEL_REPAIR, ev);
        return SMPPI_OK;
    }
    if (!curv && !seg0_known && mode == 2) {   // the block repair (modes 0, 1) searches itself
        ev = tic(h, st);
        CU(h, launch_seg0(h->dp, h->rec, n_seq, x0, h->rws.seg0, h->status, st));
        toc(h, st, SMPPI_KERNEL_SEG0, ev);
    }
    if (mode == 2) {
        int wpb = 0;
        const int grid = curv ? curv_bfgs_grid(h->dp, n_seq, h->sms, &wpb)
                              : bfgs_grid(h->dp, n_seq, h->sms, &wpb);
        if (grid < 1) return fail(h, SMPPI_ERR_CUDA, "BFGS repair: no launch shape fits");
        const size_t need = bfgs_ws_bytes(h->dp, grid, wpb);
        if (need > h->bfgs_ws_bytes) {
            if (h->bfgs_ws) {
                CU(h, cudaStreamSynchronize(st));
                cudaFree(h->bfgs_ws);
                h->bfgs_ws = nullptr;
                h->bfgs_ws_bytes = 0;
            }
            const cudaError_t e = cudaMalloc(&h->bfgs_ws, need);
            if (e != cudaSuccess)
                return fail(h, e == cudaErrorMemoryAllocation ? SMPPI_ERR_NOMEM : SMPPI_ERR_CUDA,
                            std::string("BFGS workspace: ") + cudaGetErrorString(e));
            h->bfgs_ws_bytes = need;
        }
        ev = tic(h, st);
        if (curv) {
            CU(h, launch_repair_bfgs_curv(h->dp, h->kappa, n_seq, x0, V_in, V_out, n_iters,
                                          h->bfgs_ws, grid, wpb, merit_out, iters_out, ap,
                                          h->status, st));
        } else {
            CU(h, launch_repair_bfgs(h->dp, h->rec, n_seq, x0, V_in, V_out, n_iters, h->rws.ck,
                                     h->bfgs_ws, grid, wpb, merit_out, iters_out, ap, h->status,
                                     st));
        }
        toc(h, st, SMPPI_KERNEL_REPAIR, ev);
        return SMPPI_OK;
    }
    ev = tic(h, st);
    CU(h, launch_repair(h->dp, h->rec, h->rws, n_seq, x0, V_in, V_out, n_iters, mode,
                        delta, merit_out, iters_out, ap, h->status, st));
    toc(h, st, SMPPI_KERNEL_REPAIR, ev);
    return SMPPI_OK;
}

// One Shield-MPPI control update: the rollout launch, then the update launch
// whose last block also repairs V+ and takes the closed-loop step.
smppi_status enqueue_shield(smppi_handle* h, cudaStream_t st, float* x0, float* V, float* Vs,
                            uint32_t iter, uint32_t instance, int n_repair, double* merit,
                            uint32_t* iter_dev) {
    if (h->p.state_kind == 1) {
        // curvilinear state: the MPPI iteration (V <- V+), then the shield of V+ into
        // Vs, whose block also takes the closed-loop step and shifts V
        smppi_status s = enqueue_step(h, st, x0, V, iter, instance, nullptr, nullptr, iter_dev);
        if (s != SMPPI_OK) return s;
        const ApplyArgs ap{x0, V, iter, (instance << 8) | 1u, iter_dev, h->kappa};
        const int ev = tic(h, st);
        CU(h, launch_repair_curv(h->dp, h->kappa, 1, x0, V, Vs, n_repair, 1, 0.0f, merit, nullptr,
                                 ap, h->status, st));
        toc(h, st, SMPPI_KERNEL_REPAIR, ev);
        return SMPPI_OK;
    }
    if (n_repair > 0 && merge_shield_applies(h->dp)) {
        // rollouts whose blocks each write their min-shifted partial of the update,
        // then one block that merges them into V+ and runs the shield
        const BlockPartials part{h->part_acc, h->part_eta, h->part_has};
        int ev = tic(h, st);
        CU(h, launch_rollout(h->dp, false, x0, V, h->rec, iter, instance << 8, iter_dev, h->S_ws,
                             nullptr, h->blk_min, h->rws.seg0, h->status, st, 0u, part));
        toc(h, st, SMPPI_KERNEL_ROLLOUT, ev);
        ev = tic(h, st);
        CU(h, launch_merge_shield(h->dp, rollout_blocks(h->dp), h->blk_min, part, V, iter,
                                  iter_dev, h->status, h->rec, h->rws.seg0, x0, Vs, n_repair,
                                  h->rws.ck, merit, (instance << 8) | 1u, st));
        toc(h, st, SMPPI_KERNEL_UPDATE_SHIELD, ev);
        return SMPPI_OK;
    }
    if (n_repair > 0) {
        smppi_status s = enqueue_rollout(h, st, x0, V, iter, instance, h->S_ws, nullptr, iter_dev);
        if (s != SMPPI_OK) return s;
        const int ev = tic(h, st);
        CU(h, launch_update_shield(h->dp, h->S_ws, h->blk_min, rollout_blocks(h->dp), V, iter,
                                   instance << 8, iter_dev, h->part_acc, h->part_eta, h->part_has,
                                   h->ticket, h->status, h->rec, h->rws.seg0, x0, Vs, n_repair,
                                   h->rws.ck, merit, (instance << 8) | 1u, st));
        toc(h, st, SMPPI_KERNEL_UPDATE_SHIELD, ev);
        return SMPPI_OK;
    }
    smppi_status s = enqueue_step(h, st, x0, V, iter, instance, nullptr, nullptr, iter_dev);
    if (s != SMPPI_OK) return s;
    const ApplyArgs ap{x0, V, iter, (instance << 8) | 1u, iter_dev, h->kappa};
    CU(h, cudaMemcpyAsync(Vs, V, sizeof(float) * 2 * h->p.T, cudaMemcpyDeviceToDevice, st));
    const int ev = tic(h, st);
    CU(h, launch_apply(h->dp, ap, Vs, st));
    toc(h, st, SMPPI_KERNEL_APPLY, ev);
    return SMPPI_OK;
}

}  // namespace

// Parameter checks and derived constants for entry points without a handle.
namespace smppi {
smppi_status validate_params(const smppi_params* p) { return check_params(p); }
DevParams derive_params(const smppi_params& p) { return derive(p); }
smppi_status report_error(smppi_status s, const char* msg) { return fail(nullptr, s, msg); }
}  // namespace smppi

extern "C" {

void smppi_default_params(smppi_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->m = 21.7f; p->Iz = 1.12f; p->lf = 0.34f; p->lr = 0.23f;
    p->B = 4.0f; p->Ct = 1.5f; p->g = 9.81f; p->fx_gain = 60.0f;
    p->dt = 0.02f;
    p->sigma[0] = 0.15f; p->sigma[1] = 0.3f;
    p->lambda = 1.0f; p->gamma = 1.0f;
    p->K = 256; p->T = 50; p->N_r = 50;
    p->alpha = 0.3f; p->C_cbf = 1000.0f;
    p->q_v = 2.0f; p->v_target = 8.0f; p->q_d = 100.0f; p->C_obs = 0.0f;
    p->u_min[0] = -0.5f; p->u_min[1] = -1.0f; p->u_max[0] = 0.5f; p->u_max[1] = 1.0f;
    p->half_width = 2.0f;
    p->dist_sigma[0] = 0.3f; p->dist_sigma[1] = 0.3f;
    p->ls_s0 = 0.1f; p->ls_c = 1e-4f; p->ls_max_halvings = 20;
    p->checkpoint = 0;
    p->max_seq = 1;
    p->n_track = 0;
    p->track_xy = nullptr;
    p->seed = 0;
    p->state_kind = 0;
}

smppi_status smppi_create(const smppi_params* p, void* cuda_stream, smppi_handle** out) {
    if (!out) return fail(nullptr, SMPPI_ERR_ARG, "out is NULL");
    *out = nullptr;
    smppi_status s = check_params(p);
    if (s != SMPPI_OK) return s;
    const size_t smem = rollout_smem_bytes(p->n_track, p->T);
    if (smem > 200 * 1024)
        return fail(nullptr, SMPPI_ERR_ARG, "n_track and T need more shared memory than a block has");
    smppi_handle* h = new smppi_handle();
    h->p = *p;
    if (h->p.checkpoint == 0) h->p.checkpoint = (int)std::ceil(std::sqrt((double)p->T));
    h->dp = derive(h->p);
    h->st = static_cast<cudaStream_t>(cuda_stream);
    h->nblk = (p->K + ROLL_BLK - 1) / ROLL_BLK;
    const int T = p->T, ms = p->max_seq;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
        if (h->sms < 1) h->sms = 1;
    }
    h->rws.max_seq = ms;
    h->rws.T = T;
    h->rws.ck = h->p.checkpoint;
    h->rws.nslot = T + 2;
    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, bytes)                                                   \
    if (e == cudaSuccess) e = alloc(&(ptr), (bytes));
    ALLOC(h->rec, rec_table_bytes(p->n_track));
    ALLOC(h->S_ws, sizeof(float) * p->K);
    ALLOC(h->blk_min, sizeof(float) * h->nblk);
    // partials of the update kernel's blocks or of the packed rollout blocks
    const size_t n_part = (size_t)std::max(UPD_BLK, (p->K + 2 * ROLL2_BLK - 1) / (2 * ROLL2_BLK));
    ALLOC(h->part_acc, sizeof(float) * 2 * T * n_part);
    ALLOC(h->part_eta, sizeof(double) * n_part);
    ALLOC(h->part_has, sizeof(int) * n_part);
    ALLOC(h->ticket, sizeof(unsigned));
    ALLOC(h->status, sizeof(unsigned));
    ALLOC(h->iter_dev, sizeof(uint32_t));
    ALLOC(h->rws.tape, sizeof(float) * (size_t)h->rws.nslot * NFIELD * ms);
    ALLOC(h->rws.Vw, sizeof(float2) * (size_t)T * ms);
    ALLOC(h->rws.G, sizeof(float2) * (size_t)T * ms);
    ALLOC(h->rws.seg0, sizeof(int) * ms);
#undef ALLOC
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->iter_dev, 0, sizeof(uint32_t), h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->ticket, 0, sizeof(unsigned), h->st);
    if (e == cudaSuccess) e = launch_rec_table(p->track_xy, p->n_track, h->rec, h->st);
    bool track_ok = true;
    if (e == cudaSuccess && p->state_kind == 1) {
        std::vector<float> xy(2 * (size_t)p->n_track), ks;
        double L = 0.0;
        e = cudaMemcpy(xy.data(), p->track_xy, sizeof(float) * xy.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) track_ok = curvature_samples(xy, p->n_track, ks, L);
        if (e == cudaSuccess && track_ok) {
            e = alloc(&h->kappa, sizeof(float) * ks.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(h->kappa, ks.data(), sizeof(float) * ks.size(), cudaMemcpyHostToDevice);
            h->dp.kap_scale = (float)(p->n_track / L);
            h->dp.track_len = (float)L;
            h->dp.inv_len = (float)(1.0 / L);
        }
    }
    // the segment-pair table is complete before any launch of this handle: the
    // merge-and-shield kernel stages it before its wait on the rollout launch
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e == cudaSuccess && !track_ok) {
        free_all(h);
        delete h;
        return fail(nullptr, SMPPI_ERR_ARG,
                    "state_kind 1 needs a track whose consecutive vertices differ (finite curvature)");
    }
    if (e != cudaSuccess) {
        const bool oom = (e == cudaErrorMemoryAllocation);
        fail(nullptr, oom ? SMPPI_ERR_NOMEM : SMPPI_ERR_CUDA,
             std::string("smppi_create: ") + cudaGetErrorString(e));
        free_all(h);
        delete h;
        return oom ? SMPPI_ERR_NOMEM : SMPPI_ERR_CUDA;
    }
    *out = h;
    return SMPPI_OK;
}

smppi_status smppi_destroy(smppi_handle* h) {
    if (!h) return SMPPI_OK;
    cudaStreamSynchronize(h->st);
    free_all(h);
    delete h;
    return SMPPI_OK;
}

const char* smppi_last_error(const smppi_handle* h) {
    return h ? h->err.c_str() : g_create_err.c_str();
}

smppi_status smppi_sync_status(smppi_handle* h, uint32_t* bits_out) {
    if (!h) return fail(nullptr, SMPPI_ERR_ARG, "handle is NULL");
    unsigned bits = 0;
    CU(h, cudaStreamSynchronize(h->st));
    CU(h, cudaMemcpy(&bits, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    CU(h, cudaMemset(h->status, 0, sizeof(unsigned)));
    if (bits_out) *bits_out = bits;
    if (bits & SMPPI_DEV_NUMERIC) return fail(h, SMPPI_ERR_NUMERIC, "NaN/Inf met on the device");
    if (bits & SMPPI_DEV_TIMEOUT) return fail(h, SMPPI_ERR_TIMEOUT, "a device wait gave up");
    if (bits & SMPPI_DEV_STALLED) return fail(h, SMPPI_ERR_STALLED, "repair line search stalled");
    return SMPPI_OK;
}

smppi_status smppi_step(smppi_handle* h, const float* x0, float* V, uint32_t iter,
                        uint32_t instance, float* S_out, float* traj_out) {
    if (!h) return fail(nullptr, SMPPI_ERR_ARG, "handle is NULL");
    if (!x0 || !V) return fail(h, SMPPI_ERR_ARG, "x0 and V must not be NULL");
    if (instance >= (1u << 24)) return fail(h, SMPPI_ERR_ARG, "instance must be < 2^24");
    return enqueue_step(h, h->st, x0, V, iter, instance, S_out, traj_out, nullptr);
}

smppi_status smppi_step_partial(smppi_handle* h, const float* x0, const float* V, uint32_t iter,
                                uint32_t instance, int k_lo, int k_hi, double* partial_out) {
    if (!h) return fail(nullptr, SMPPI_ERR_ARG, "handle is NULL");
    if (!x0 || !V || !partial_out)
        return fail(h, SMPPI_ERR_ARG, "x0, V and partial_out must not be NULL");
    if (instance >= (1u << 24)) return fail(h, SMPPI_ERR_ARG, "instance must be < 2^24");
    if (k_lo < 0 || k_lo >= k_hi || k_hi > h->p.K)
        return fail(h, SMPPI_ERR_ARG, "need 0 <= k_lo < k_hi <= K");
    // the slice's rollouts as a problem of k_hi - k_lo rollouts whose Philox
    // counters start at k_lo; the noise-skip threshold stays the one of all K
    DevParams dp = h->dp;
    dp.K = k_hi - k_lo;
    const uint32_t ctr3 = instance << 8;
    cudaStream_t st = h->st;
    int ev = tic(h, st);
    if (h->p.state_kind == 1)
        CU(h, launch_rollout_curv(dp, h->kappa, false, x0, V, iter, ctr3, nullptr, h->S_ws,
                                  nullptr, h->blk_min, h->status, st, (uint32_t)k_lo));
    else
        CU(h, launch_rollout(dp, false, x0, V, h->rec, iter, ctr3, nullptr, h->S_ws, nullptr,
                             h->blk_min, nullptr, h->status, st, (uint32_t)k_lo));
    toc(h, st, SMPPI_KERNEL_ROLLOUT, ev);
    ev = tic(h, st);
    CU(h, launch_update_partial(dp, h->S_ws, h->blk_min, rollout_blocks(dp), V, iter, ctr3,
                                h->part_acc, h->part_eta, h->part_has, h->ticket, h->status,
                                (uint32_t)k_lo, partial_out, st));
    toc(h, st, SMPPI_KERNEL_UPDATE, ev);
    return SMPPI_OK;
}

smppi_status smppi_merge_partials(smppi_handle* h, int n_parts, const double* partials,
                                  float* V) {
    if (!h) return fail(nullptr, SMPPI_ERR_ARG, "handle is NULL");
    if (!partials || !V) return fail(h, SMPPI_ERR_ARG, "partials and V must not be NULL");
    if (n_parts < 1 || n_parts > MERGE_MAX_PARTS)
        return fail(h, SMPPI_ERR_ARG, "n_parts must be in [1, 1024]");
    const int ev = tic(h, h->st);
    CU(h, launch_merge(h->dp, n_parts, partials, V, h->status, h->st));
    toc(h, h->st, SMPPI_KERNEL_MERGE, ev);
    return SMPPI_OK;
}

smppi_status smppi_update(smppi_handle* h, const float* S, float* V, uint32_t iter,
                          uint32_t instance) {
    if (!h) return fail(nullptr, SMPPI_ERR_ARG, "handle is NULL");
    if (!S || !V) return fail(h, SMPPI_ERR_ARG, "S and V must not be NULL");
    if (instance >= (1u << 24)) return fail(h, SMPPI_ERR_ARG, "instance must be < 2^24");
    const int ev = tic(h, h->st);
    CU(h, launch_update(h->dp, S, nullptr, 0, V, iter, instance << 8, nullptr, h->part_acc,
                        h->part_eta, h->part_has, h->ticket, h->status, h->st));
    toc(h, h->st, SMPPI_KERNEL_UPDATE, ev);
    return SMPPI_OK;
}

smppi_status smppi_cost_grad(smppi_handle* h, int n_seq, const float* x0, const float* V, int N,
                             float w_run, float w_cbf, int checkpoint, double* J_out,
                             float* grad_out) {
    smppi_status s = check_seq_call(h, n_seq);
    if (s != SMPPI_OK) return s;
    if (!x0 || !V || !grad_out) return fail(h, SMPPI_ERR_ARG, "x0, V, grad_out must not be NULL");
    if (N < 0 || N > h->p.T) return fail(h, SMPPI_ERR_ARG, "N must be in [0, T]");
    if (!std::isfinite(w_run) || !std::isfinite(w_cbf)) return fail(h, SMPPI_ERR_ARG, "weights must be finite");
    if (checkpoint > h->p.T) return fail(h, SMPPI_ERR_ARG, "checkpoint must be <= T");
    if (h->p.state_kind == 1) {   // full tape: the checkpoint interval does not apply
        const int ev = tic(h, h->st);
        CU(h, launch_cost_grad_curv(h->dp, h->kappa, n_seq, x0, V, N, w_run, w_cbf, J_out,
                                    grad_out, h->status, h->st));
        toc(h, h->st, SMPPI_KERNEL_COST_GRAD, ev);
        return SMPPI_OK;
    }
    const int ck = checkpoint == 0 ? h->p.checkpoint : (checkpoint < 0 ? 0 : checkpoint);
    int ev = tic(h, h->st);
    CU(h, launch_seg0(h->dp, h->rec, n_seq, x0, h->rws.seg0, h->status, h->st));
    toc(h, h->st, SMPPI_KERNEL_SEG0, ev);
    ev = tic(h, h->st);
    CU(h, launch_cost_grad(h->dp, h->rec, h->rws, n_seq, x0, V, N, w_run, w_cbf, ck, J_out,
                           grad_out, h->status, h->st));
    toc(h, h->st, SMPPI_KERNEL_COST_GRAD, ev);
    return SMPPI_OK;
}

smppi_status smppi_timing(smppi_handle* h, int enable) {
    if (!h) return fail(nullptr, SMPPI_ERR_ARG, "handle is NULL");
    h->timing = enable != 0;
    return SMPPI_OK;
}

smppi_status smppi_timing_read(smppi_handle* h, double* ms_out, int* count_out, int n_kinds) {
    if (!h) return fail(nullptr, SMPPI_ERR_ARG, "handle is NULL");
    if (n_kinds < 0 || (n_kinds > 0 && (!ms_out || !count_out)))
        return fail(h, SMPPI_ERR_ARG, "ms_out and count_out must hold n_kinds values");
    CU(h, cudaStreamSynchronize(h->st));
    for (int k = 0; k < n_kinds; ++k) {
        ms_out[k] = 0.0;
        count_out[k] = 0;
    }
    for (const auto& r : h->records) {
        float ms = 0.0f;
        CU(h, cudaEventElapsedTime(&ms, h->ev_pool[r[1]], h->ev_pool[r[2]]));
        if (r[0] < n_kinds) {
            ms_out[r[0]] += ms;
            count_out[r[0]] += 1;
        }
    }
    h->records.clear();
    h->ev_used = 0;
    return SMPPI_OK;
}

smppi_status smppi_repair(smppi_handle* h, int n_seq, const float* x0, const float* V_in,
                          float* V_out, int n_iters, int mode, float delta, double* merit_out,
                          int* iters_out) {
    smppi_status s = check_seq_call(h, n_seq);
    if (s != SMPPI_OK) return s;
    if (!x0 || !V_in || !V_out) return fail(h, SMPPI_ERR_ARG, "x0, V_in, V_out must not be NULL");
    if (n_iters < 0 || n_iters > 100000) return fail(h, SMPPI_ERR_ARG, "n_iters must be in [0, 1e5]");
    if (mode != 0 && mode != 1 && mode != 2) return fail(h, SMPPI_ERR_ARG, "mode must be 0, 1 or 2");
    if (mode == 0 && !(std::isfinite(delta) && delta >= 0)) return fail(h, SMPPI_ERR_ARG, "delta must be >= 0");
    const ApplyArgs none{nullptr, nullptr, 0u, 0u, nullptr};
    return enqueue_repair(h, h->st, n_seq, x0, V_in, V_out, n_iters, mode, delta, merit_out,
                          iters_out, false, none);
}

smppi_status smppi_apply(smppi_handle* h, float* x0, float* V, const float* V_exec, uint32_t n,
                         uint32_t instance) {
    if (!h) return fail(nullptr, SMPPI_ERR_ARG, "handle is NULL");
    if (!x0 || !V || !V_exec) return fail(h, SMPPI_ERR_ARG, "x0, V, V_exec must not be NULL");
    if (instance >= (1u << 24)) return fail(h, SMPPI_ERR_ARG, "instance must be < 2^24");
    const ApplyArgs ap{x0, V, n, (instance << 8) | 1u, nullptr, h->kappa};
    const int ev = tic(h, h->st);
    CU(h, launch_apply(h->dp, ap, V_exec, h->st));
    toc(h, h->st, SMPPI_KERNEL_APPLY, ev);
    return SMPPI_OK;
}

smppi_status smppi_shield_update(smppi_handle* h, float* x0, float* V, float* V_safe,
                                 uint32_t iter, uint32_t instance, int n_repair,
                                 double* merit_out, int host_buffers) {
    if (!h) return fail(nullptr, SMPPI_ERR_ARG, "handle is NULL");
    if (!x0 || !V || !V_safe) return fail(h, SMPPI_ERR_ARG, "x0, V, V_safe must not be NULL");
    if (n_repair < 0 || n_repair > 100000) return fail(h, SMPPI_ERR_ARG, "n_repair must be in [0, 1e5]");
    if (instance >= (1u << 24)) return fail(h, SMPPI_ERR_ARG, "instance must be < 2^24");
    if (!host_buffers)
        return enqueue_shield(h, h->st, x0, V, V_safe, iter, instance, n_repair, merit_out, nullptr);
    // host state: checked here (the device search for the nearest segment has no
    // answer for a position whose squared distances overflow float32)
    for (int j = 0; j < 6; ++j)
        if (!std::isfinite(x0[j])) return fail(h, SMPPI_ERR_ARG, "x0 must be finite");
    if (std::fabs(x0[3]) > 1e18f || std::fabs(x0[4]) > 1e18f)
        return fail(h, SMPPI_ERR_ARG, "x0 position beyond 1e18 m");
    // one copy in (x0, the iteration, V) and one copy out (x0, V, V_safe, merits)
    // through the handle's staging block and its pinned mirror, the copies and the
    // update's launches replayed from one CUDA graph per (instance, n_repair,
    // merits): the iteration reaches the kernels through the staged word that
    // they read as their device iteration counter
    const size_t vb = sizeof(float) * 2 * h->p.T, off_iter = 24, off_V = 32,
                 off_Vs = off_V + vb, off_m = off_Vs + vb;
    const int n_merit = (merit_out && n_repair > 0) ? n_repair + 1 : 0;
    if (!h->d_io || h->merit_cap < n_merit) {
        if (h->io_exec) cudaGraphExecDestroy(h->io_exec);
        h->io_exec = nullptr;
        if (h->d_io) cudaFree(h->d_io);
        if (h->h_io) cudaFreeHost(h->h_io);
        h->d_io = h->h_io = nullptr;
        h->merit_cap = 0;
        const int cap = std::max(n_merit, 11);
        const size_t bytes = off_m + sizeof(double) * cap;
        CU(h, cudaMalloc(&h->d_io, bytes));
        CU(h, cudaMallocHost(&h->h_io, bytes));
        h->merit_cap = cap;
    }
    char key[64];
    std::snprintf(key, sizeof(key), "%u %d %d", instance, n_repair, n_merit);
    if (!h->io_exec || h->io_key != key) {
        if (h->io_exec) cudaGraphExecDestroy(h->io_exec);
        h->io_exec = nullptr;
        float* dx = reinterpret_cast<float*>(h->d_io);
        float* dV = reinterpret_cast<float*>(h->d_io + off_V);
        float* dVs = reinterpret_cast<float*>(h->d_io + off_Vs);
        double* dm = n_merit ? reinterpret_cast<double*>(h->d_io + off_m) : nullptr;
        uint32_t* di = reinterpret_cast<uint32_t*>(h->d_io + off_iter);
        cudaGraph_t g = nullptr;
        CU(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaMemcpyAsync(h->d_io, h->h_io, off_Vs, cudaMemcpyHostToDevice, h->cap);
        smppi_status s = SMPPI_OK;
        if (e == cudaSuccess)
            s = enqueue_shield(h, h->cap, dx, dV, dVs, 0u, instance, n_repair, dm, di);
        if (e == cudaSuccess && s == SMPPI_OK)
            e = cudaMemcpyAsync(h->h_io, h->d_io, off_m + sizeof(double) * n_merit,
                                cudaMemcpyDeviceToHost, h->cap);
        const cudaError_t e_end = cudaStreamEndCapture(h->cap, &g);
        if (s != SMPPI_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e == cudaSuccess) e = e_end;
        if (e != cudaSuccess && g) cudaGraphDestroy(g);
        CU(h, e);
        e = cudaGraphInstantiate(&h->io_exec, g, 0);
        cudaGraphDestroy(g);
        CU(h, e);
        h->io_key = key;
    }
    std::memcpy(h->h_io, x0, sizeof(float) * 6);
    std::memcpy(h->h_io + off_iter, &iter, sizeof(uint32_t));
    std::memcpy(h->h_io + off_V, V, vb);
    CU(h, cudaGraphLaunch(h->io_exec, h->st));
    CU(h, cudaStreamSynchronize(h->st));
    std::memcpy(x0, h->h_io, sizeof(float) * 6);
    std::memcpy(V, h->h_io + off_V, vb);
    std::memcpy(V_safe, h->h_io + off_Vs, vb);
    if (n_merit) std::memcpy(merit_out, h->h_io + off_m, sizeof(double) * n_merit);
    return SMPPI_OK;
}

smppi_status smppi_shield_loop(smppi_handle* h, float* x0, float* V, float* V_safe,
                               uint32_t iter0, uint32_t instance, int n_repair, int n_updates) {
    if (!h) return fail(nullptr, SMPPI_ERR_ARG, "handle is NULL");
    if (!x0 || !V || !V_safe) return fail(h, SMPPI_ERR_ARG, "x0, V, V_safe must not be NULL");
    if (n_repair < 0 || n_repair > 100000 || n_updates < 0)
        return fail(h, SMPPI_ERR_ARG, "n_repair in [0, 1e5], n_updates >= 0");
    if (instance >= (1u << 24)) return fail(h, SMPPI_ERR_ARG, "instance must be < 2^24");
    char key[256];
    std::snprintf(key, sizeof(key), "%p %p %p %u %u %d", (void*)x0, (void*)V, (void*)V_safe,
                  iter0, instance, n_repair);
    if (!h->gexec || h->graph_key != key) {
        if (h->gexec) {
            cudaGraphExecDestroy(h->gexec);
            h->gexec = nullptr;
        }
        cudaGraph_t g = nullptr;
        CU(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        smppi_status s = enqueue_shield(h, h->cap, x0, V, V_safe, iter0, instance, n_repair,
                                        nullptr, h->iter_dev);
        cudaError_t e = cudaStreamEndCapture(h->cap, &g);
        if (s != SMPPI_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        CU(h, e);
        e = cudaGraphInstantiate(&h->gexec, g, 0);
        cudaGraphDestroy(g);
        CU(h, e);
        h->graph_key = key;
    }
    CU(h, cudaMemsetAsync(h->iter_dev, 0, sizeof(uint32_t), h->st));
    for (int i = 0; i < n_updates; ++i) CU(h, cudaGraphLaunch(h->gexec, h->st));
    return SMPPI_OK;
}

smppi_status smppi_debug_elementary(int fn, int n, const float* a, const float* b, float* out,
                                    float* ref, void* cuda_stream) {
    if (fn < 0 || fn > 9) return fail(nullptr, SMPPI_ERR_ARG, "fn must be in [0, 9]");
    if (n < 0) return fail(nullptr, SMPPI_ERR_ARG, "n must be >= 0");
    if (n == 0) return SMPPI_OK;
    if (!a || !b || !out || !ref) return fail(nullptr, SMPPI_ERR_ARG, "NULL array");
    const cudaError_t e =
        launch_debug_elementary(fn, n, a, b, out, ref, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return fail(nullptr, SMPPI_ERR_CUDA, cudaGetErrorString(e));
    return SMPPI_OK;
}

smppi_status smppi_debug_noise(smppi_handle* h, uint32_t iter, uint32_t instance, int K, int T,
                               float* eps_out, uint32_t* raw_out) {
    if (!h) return fail(nullptr, SMPPI_ERR_ARG, "handle is NULL");
    if (K < 1 || T < 1 || T > SMPPI_MAX_T) return fail(h, SMPPI_ERR_ARG, "K >= 1, 1 <= T <= SMPPI_MAX_T");
    if (!eps_out && !raw_out) return fail(h, SMPPI_ERR_ARG, "no output given");
    if (instance >= (1u << 24)) return fail(h, SMPPI_ERR_ARG, "instance must be < 2^24");
    CU(h, launch_debug_noise(h->dp, iter, instance << 8, K, T, eps_out, raw_out, h->st));
    return SMPPI_OK;
}

}  // extern "C"
