// Launchers shared between the kernel translation units and the C ABI.
#pragma once

#include "device.cuh"

namespace smppi {

enum { MODE_ROLL = 0, MODE_DUMP = 1, MODE_FROM_S = 2 };

// Opt a kernel in to more than 48 KB of dynamic shared memory when needed.
inline cudaError_t ensure_smem(const void* kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
constexpr int ROLL_BLK = 128;   // rollouts per block of the single-problem kernel

size_t rollout_smem_bytes(int n_track, int T);
cudaError_t launch_rollout(const DevParams& P, int mode, const float* x0, const float* V,
                           const float4* seg, const float* inv, uint32_t iter, uint32_t ctr3,
                           const uint32_t* iter_dev, const float* S_in, float* S_out, float* traj, float* part_acc,
                           float2* part_mh, unsigned* status, cudaStream_t st);
cudaError_t launch_merge(const DevParams& P, const float* part_acc, const float2* part_mh,
                         int nblk, float* V, unsigned* status, cudaStream_t st);
cudaError_t launch_debug_noise(const DevParams& P, uint32_t iter, uint32_t ctr3, int K, int T,
                               float* eps, uint32_t* raw, cudaStream_t st);

// Segment table of a closed polyline: seg[i] = (A_i, A_{i+1} - A_i), inv[i] = 1/|D_i|^2.
cudaError_t launch_seg_table(const float* track_xy, int n, float4* seg, float* inv,
                             cudaStream_t st);

// Repair / adjoint workspace (device), sized for max_seq sequences of horizon T.
struct RepairWs {
    int max_seq, T, ck;        // capacity, horizon, checkpoint interval
    int nslot;                 // tape slots per sequence
    float* tape;               // [nslot][NFIELD][max_seq]
    float2* Vw;                // [T][max_seq]  working controls
    float2* G;                 // [T][max_seq]  gradient
    int* seg0;                 // [max_seq]     nearest segment of x0
};
constexpr int NFIELD = 9;      // x (6), segment, h, h of the previous step

cudaError_t launch_seg0(const DevParams& P, const float4* seg, const float* inv, int n_seq,
                        const float* x0, int* seg0, cudaStream_t st);
cudaError_t launch_cost_grad(const DevParams& P, const float4* seg, const float* inv,
                             const RepairWs& ws, int n_seq, const float* x0, const float* V, int N,
                             float w_run, float w_cbf, int ck, double* J_out, float* grad_out,
                             unsigned* status, cudaStream_t st);
cudaError_t launch_repair(const DevParams& P, const float4* seg, const float* inv,
                          const RepairWs& ws, int n_seq, const float* x0, const float* V_in,
                          float* V_out, int n_iters, int mode, float delta, double* merit_out,
                          int* iters_out, unsigned* status, cudaStream_t st);
cudaError_t launch_apply(const DevParams& P, float* x0, float* V, const float* V_exec, uint32_t n,
                         uint32_t ctr3, uint32_t* iter_dev, cudaStream_t st);

}  // namespace smppi
