// Launchers shared between the kernel translation units and the C ABI.
#pragma once

#include "device.cuh"

namespace smppi {

constexpr int ROLL_BLK = 128;   // rollouts per block of the single-problem kernel
constexpr int ROLL2_BLK = 128;  // threads per block of the packed kernel (two rollouts each)
constexpr int UPD_BLK = 256;    // threads per block of the update kernel (also its max grid)

// Opt a kernel in to more than 48 KB of dynamic shared memory when needed.
inline cudaError_t ensure_smem(const void* kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Per-block partials of the update (Eq. 10-11 min-shifted by each rollout
// block's own minimum, which blk_min holds) written by the packed rollout
// kernel: acc [blocks][2T], eta [blocks], has [blocks].  All null: none written.
struct BlockPartials {
    float* acc;
    double* eta;
    int* has;
};
// Largest number of rollout blocks the single-block merge takes (2 * ROLL2_BLK
// rollouts each: K <= 2^19).
constexpr int MERGE_MAX_BLOCKS = 2048;

// Dynamic shared memory of the rollout launch (the larger of its two kernels).
size_t rollout_smem_bytes(int n_track, int T);
// Block minima the rollout launch writes (<= ceil(K / ROLL_BLK)).
int rollout_blocks(const DevParams& P);
// Rollouts of the curvilinear state (curv.cu; state_kind 1), same outputs as
// launch_rollout (no nearest segment).
cudaError_t launch_rollout_curv(const DevParams& P, const float* kappa, bool dump, const float* x0,
                                const float* V, uint32_t iter, uint32_t ctr3,
                                const uint32_t* iter_dev, float* S_out, float* traj,
                                float* blk_min, unsigned* status, cudaStream_t st,
                                uint32_t k_off = 0);
// Rollouts: S_out [K] and blk_min [rollout_blocks(P)]; traj (optional dump);
// seg0_out (optional): nearest segment of x0.  rec: segment-pair table of
// launch_rec_table.  The P.K rollouts are rollouts k_off .. k_off + P.K - 1 of
// the problem (their Philox counters); outputs are indexed from 0.
cudaError_t launch_rollout(const DevParams& P, bool dump, const float* x0, const float* V,
                           const float4* rec, uint32_t iter, uint32_t ctr3,
                           const uint32_t* iter_dev, float* S_out, float* traj, float* blk_min,
                           int* seg0_out, unsigned* status, cudaStream_t st, uint32_t k_off = 0,
                           BlockPartials part = BlockPartials{nullptr, nullptr, nullptr});
// True when the rollout launch can write block partials for launch_merge_shield
// (the packed kernel applies and the blocks are few enough).
bool merge_shield_applies(const DevParams& P);
// Segment-pair table of a closed polyline (layout in device.cuh): n + 5
// records of three float4.
__host__ __device__ inline size_t rec_table_bytes(int n) { return (size_t)(n + 5) * 3 * sizeof(float4); }
cudaError_t launch_rec_table(const float* track_xy, int n, float4* rec, cudaStream_t st);
// Grid of the update kernel for K rollouts (<= UPD_BLK blocks).
int update_grid(int K);
// Softmin update V <- clamp(V + sum omega eps / sum omega) from S [K].  blk_min
// (n_min values) may be NULL.  part_acc [grid][2T], part_eta [grid]; ticket:
// a device counter that is 0 on entry and left 0.
cudaError_t launch_update(const DevParams& P, const float* S, const float* blk_min, int n_min,
                          float* V, uint32_t iter, uint32_t ctr3, uint32_t* iter_dev,
                          float* part_acc, double* part_eta, int* part_has, unsigned* ticket,
                          unsigned* status, cudaStream_t st);
// The same update followed, in its last block, by the safety shield on V+
// (n_repair Armijo iterations; V_safe out; merits optional) and the
// closed-loop step on x0 (disturbance counter word ctr3_dist); V ends as
// shift(V+).  seg0: nearest segment of x0 from the rollout launch.  iter_dev
// (graph replays) is advanced by one.
cudaError_t launch_update_shield(const DevParams& P, const float* S, const float* blk_min,
                                 int n_min, float* V, uint32_t iter, uint32_t ctr3,
                                 uint32_t* iter_dev, float* part_acc, double* part_eta,
                                 int* part_has, unsigned* ticket, unsigned* status,
                                 const float4* rec, const int* seg0, float* x0, float* V_safe,
                                 int n_repair, int ck, double* merit_out, uint32_t ctr3_dist,
                                 cudaStream_t st);
// The update over a slice of rollouts (P.K of them, rollouts k_off ..) without
// touching V: partial_out [2T + 2] (float64) = (m, eta, A) with m the slice's
// minimum cost, eta = sum exp(-(S - m)/lambda) and A [2T] = sum exp(-(S - m)
// /lambda) eps over the slice.
cudaError_t launch_update_partial(const DevParams& P, const float* S, const float* blk_min,
                                  int n_min, const float* V, uint32_t iter, uint32_t ctr3,
                                  float* part_acc, double* part_eta, int* part_has,
                                  unsigned* ticket, unsigned* status, uint32_t k_off,
                                  double* partial_out, cudaStream_t st);
// The update from the rollout launch's block partials (one block: the block
// minima, m = min, c_b = exp(-(m_b - m)/lambda), eta = sum c_b eta_b, A = sum
// c_b A_b in float64 in block order), then the shield and the closed-loop step
// as launch_update_shield.  nb = rollout_blocks(P) <= MERGE_MAX_BLOCKS.
cudaError_t launch_merge_shield(const DevParams& P, int nb, const float* blk_min,
                                BlockPartials part, float* V, uint32_t iter, uint32_t* iter_dev,
                                unsigned* status, const float4* rec, const int* seg0, float* x0,
                                float* V_safe, int n_repair, int ck, double* merit_out,
                                uint32_t ctr3_dist, cudaStream_t st);
// V <- clamp(V + A / eta) from n_parts slice partials [n_parts][2T + 2]: with
// m = min_g m_g and c_g = exp(-(m_g - m)/lambda), eta = sum_g c_g eta_g and
// A = sum_g c_g A_g, summed in float64 in slice order.
constexpr int MERGE_MAX_PARTS = 1024;
cudaError_t launch_merge(const DevParams& P, int n_parts, const double* parts, float* V,
                         unsigned* status, cudaStream_t st);
cudaError_t launch_debug_elementary(int fn, int n, const float* a, const float* b, float* out,
                                   float* ref, cudaStream_t st);
cudaError_t launch_debug_noise(const DevParams& P, uint32_t iter, uint32_t ctr3, int K, int T,
                               float* eps, uint32_t* raw, cudaStream_t st);


// Repair / adjoint workspace (device), sized for max_seq sequences of horizon T.
struct RepairWs {
    int max_seq, T, ck;        // capacity, horizon, checkpoint interval
    int nslot;                 // tape slots per sequence
    float* tape;               // [nslot][NFIELD][max_seq]
    float2* Vw;                // [T][max_seq]  working controls
    float2* G;                 // [T][max_seq]  gradient
    int* seg0;                 // [max_seq]     nearest segment of x0
};
constexpr int NFIELD = 11;     // x (6), cos psi, sin psi, segment, h, h of the previous step

// Closed-loop step fused into the tail of the repair of sequence 0.
struct ApplyArgs {
    float* x0;                 // in/out state (NULL: no closed-loop step)
    float* V;                  // in/out: shifted V+
    uint32_t n, ctr3;          // disturbance index and counter word
    uint32_t* iter_dev;        // graph replays: n += *iter_dev, then ++*iter_dev
    const float* kappa;        // curvature samples (state_kind 1)
};

cudaError_t launch_seg0(const DevParams& P, const float4* rec, int n_seq,
                        const float* x0, int* seg0, unsigned* status, cudaStream_t st);
cudaError_t launch_cost_grad(const DevParams& P, const float4* rec,
                             const RepairWs& ws, int n_seq, const float* x0, const float* V, int N,
                             float w_run, float w_cbf, int ck, double* J_out, float* grad_out,
                             unsigned* status, cudaStream_t st);
cudaError_t launch_repair(const DevParams& P, const float4* rec,
                          const RepairWs& ws, int n_seq, const float* x0, const float* V_in,
                          float* V_out, int n_iters, int mode, float delta, double* merit_out,
                          int* iters_out, const ApplyArgs& ap, unsigned* status, cudaStream_t st);
cudaError_t launch_apply(const DevParams& P, const ApplyArgs& ap, const float* V_exec,
                         cudaStream_t st);

// Shield on the curvilinear state (curv_repair.cu; state_kind 1): modes 0 and 1
// of smppi_repair, one block per sequence, optional closed-loop tail (ap).
cudaError_t launch_repair_curv(const DevParams& P, const float* kappa, int n_seq,
                               const float* x0, const float* V_in, float* V_out, int n_iters,
                               int mode, float delta, double* merit_out, int* iters_out,
                               const ApplyArgs& ap, unsigned* status, cudaStream_t st);

// smppi_cost_grad on the curvilinear state (curv_repair.cu): full tape, one warp
// per sequence (the checkpoint interval does not apply).
cudaError_t launch_cost_grad_curv(const DevParams& P, const float* kappa, int n_seq,
                                  const float* x0, const float* V, int N, float w_run, float w_cbf,
                                  double* J_out, float* grad_out, unsigned* status,
                                  cudaStream_t st);

// BFGS repair (bfgs.cu): bfgs_grid() blocks of *wpb warps, one sequence per
// warp at a time; the workspace (bfgs_ws_bytes()) holds a work counter and an
// H slice of (2 N_r)^2 floats per warp slot.
int bfgs_grid(const DevParams& P, int n_seq, int sms, int* wpb);
size_t bfgs_ws_bytes(const DevParams& P, int grid, int wpb);
cudaError_t launch_repair_bfgs(const DevParams& P, const float4* rec, int n_seq, const float* x0,
                               const float* V_in, float* V_out, int n_iters, int ck, void* ws,
                               int grid, int wpb, double* merit_out, int* iters_out,
                               const ApplyArgs& ap, unsigned* status, cudaStream_t st);

// Host helpers of the C ABI for entry points that have no handle: check a
// parameter struct, derive the kernel constants, record the message that
// smppi_last_error(NULL) returns.
smppi_status validate_params(const smppi_params* p);
DevParams derive_params(const smppi_params& p);
smppi_status report_error(smppi_status s, const char* msg);

}  // namespace smppi
