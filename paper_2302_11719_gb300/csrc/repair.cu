// Safety shield (Alg. 1, Eq. 22): reverse-mode adjoint of the deterministic
// rollout cost with checkpointing, Armijo / fixed-step repair, and the
// closed-loop step (Alg. 2 ExecuteCommand + warm start, Eq. 26).
//
// One thread owns one control sequence.  The forward sweep stores the state
// every `ck` steps (checkpoints, ~sqrt(T) of them); the backward sweep walks
// the checkpoint segments from last to first, recomputes each segment's states
// from its checkpoint and runs the hand-derived adjoint of the Euler step
// through them.  With ck <= 0 the forward sweep stores every state instead
// (full tape, no recomputation).  Per-sequence arrays live in a workspace laid
// out [slot][field][sequence] so that a warp's accesses are coalesced.
#include "shield.cuh"

namespace smppi {

// Global nearest segment of each x0 (one warp per sequence; lowest index on ties).
__global__ void seg0_kernel(DevParams P, const float4* __restrict__ rec, int n_seq,
                            const float* __restrict__ x0, int* __restrict__ seg0,
                            unsigned* __restrict__ status) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= n_seq) return;
    const float X = x0[6 * w + 3], Y = x0[6 * w + 4];
    float bd = 3.0e38f;
    int bi = 0x7fffffff;
    for (int i = lane; i < P.n_track; i += 32) {
        const float d = rec_d2_seg(rec, i, X, Y);
        if (d < bd) { bd = d; bi = i; }
    }
    warp_argmin(bd, bi);
    if (lane == 0) seg0[w] = seg_or_zero(bi, P.n_track, status);
}

constexpr int REP_BLK = 64;

__device__ __forceinline__ void stage_track(const DevParams& P, const float4* __restrict__ recg,
                                            float4* rec) {
    for (int i = threadIdx.x; i < 3 * (P.n_track + 5); i += blockDim.x) rec[i] = recg[i];
    __syncthreads();
}

template <bool FAST>
__global__ void __launch_bounds__(REP_BLK) cost_grad_kernel(
    DevParams P, const float4* __restrict__ recg, RepairWs ws,
    int n_seq, const float* __restrict__ x0g, const float* __restrict__ Vg, int N, float w_run,
    float w_cbf, int ck, double* __restrict__ J_out, float* __restrict__ grad_out,
    unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* rec = reinterpret_cast<float4*>(smem_raw);
    stage_track(P, recg, rec);
    const int q = blockIdx.x * REP_BLK + threadIdx.x;
    if (q >= n_seq) return;
    const int T = P.T, ms = ws.max_seq;
    const float2* Vrow = reinterpret_cast<const float2*>(Vg) + (size_t)q * T;
    for (int t = 0; t < T; ++t) ws.Vw[(size_t)t * ms + q] = Vrow[t];
    const State x0 = make_state(x0g + 6 * q);
    const Tape tape{ws.tape, ms, q};
    const double J = seq_cost_grad<FAST>(P, rec, x0, ws.seg0[q], N, T, ws.Vw, ws.G, ms, q, w_run,
                                         w_cbf, ck, tape);
    if (J_out) J_out[q] = J;
    if (!isfinite(J)) atomicOr(status, SMPPI_DEV_NUMERIC);
    float2* grow = reinterpret_cast<float2*>(grad_out) + (size_t)q * T;
    for (int t = 0; t < T; ++t) grow[t] = ws.G[(size_t)t * ms + q];
}

// Safety shield, one block per sequence, everything in shared memory (track
// table staged by a bulk copy, controls, gradient, the merit pass's buffers and
// the block gradient's workspace); see repair_in_block.  Blocks of sequences
// that finish early free their SM for the next ones, which at 8192 and 65536
// sequences made this form faster than one thread per sequence (5.2 against
// 19.4 ms and 33 against 39 ms for 20 Armijo iterations).
constexpr int REPB_BLK = 128;

template <bool FAST>
__global__ void __launch_bounds__(REPB_BLK) repair_block_kernel(
    DevParams P, const float4* __restrict__ recg, const float* __restrict__ x0g, const float* Vin,
    float* Vout, int n_iters, int mode, float delta, int ck, double* __restrict__ merit_out,
    int* __restrict__ iters_out, ApplyArgs ap, unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = P.T, n = P.n_track;
    float4* rec = reinterpret_cast<float4*>(smem_raw);
    float2* Vw = reinterpret_cast<float2*>(rec + 3 * (n + 5));
    float2* G = Vw + T;
    float* tape_s = reinterpret_cast<float*>(G + T);
    const GradWs gws =
        grad_ws_at(reinterpret_cast<unsigned char*>(tape_s + (size_t)(T + 2) * NFIELD), T);
    __shared__ __align__(8) uint64_t bar;
    __shared__ RepairSmem sm;
    __shared__ float s_red[REPB_BLK / 32];
    __shared__ int s_redi[REPB_BLK / 32];
    __shared__ int s_fail;
    const int tid = threadIdx.x;
    const int q = blockIdx.x;

    // stage the track (bulk copy, bounded wait) and this sequence's controls
    if (tid == 0) {
        s_fail = 0;
        mbar_init(&bar, 1);
        const uint32_t bytes = (uint32_t)rec_table_bytes(n);
        mbar_expect_tx(&bar, bytes);
        bulk_g2s(rec, recg, bytes, &bar);
    }
    const float2* vin = reinterpret_cast<const float2*>(Vin) + (size_t)q * T;
    for (int t = tid; t < T; t += REPB_BLK) Vw[t] = vin[t];
    const State x0 = make_state(x0g + 6 * q);
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0)) s_fail = 1;
    __syncthreads();
    if (s_fail) {
        if (tid == 0) {
            atomicOr(status, SMPPI_DEV_TIMEOUT);
            mbar_wait_bounded(&bar, 0);   // let the copy in flight land before the block exits
        }
        return;
    }
    const int s0 = block_nearest_segment<REPB_BLK>(rec, n, x0.X, x0.Y, s_red, s_redi, nullptr,
                                                   status);
    repair_in_block<REPB_BLK, FAST>(P, rec, x0, s0, Vw, G, tape_s, n_iters, mode, delta, ck,
                              merit_out ? merit_out + (size_t)q * (n_iters + 1) : nullptr,
                              iters_out ? iters_out + q : nullptr, status, sm, NoSide(), &gws);
    float2* vout = reinterpret_cast<float2*>(Vout) + (size_t)q * T;
    for (int t = tid; t < T; t += REPB_BLK) vout[t] = Vw[t];
    if (q == 0 && tid == 0 && ap.x0) closed_loop_step(P, ap, Vw[0]);
}

// Closed-loop step as its own launch (V_exec may alias ap.V: it is read first).
__global__ void apply_kernel(DevParams P, ApplyArgs ap, const float* V_exec) {
    const float2 v = reinterpret_cast<const float2*>(V_exec)[0];
    closed_loop_step(P, ap, v);
}

// ----------------------------------------------------------------------------
cudaError_t launch_seg0(const DevParams& P, const float4* rec, int n_seq, const float* x0,
                        int* seg0, unsigned* status, cudaStream_t st) {
    const int warps_per_block = 4;
    seg0_kernel<<<(n_seq + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(
        P, rec, n_seq, x0, seg0, status);
    return cudaGetLastError();
}

static bool fast_model(const DevParams& P) { return P.tyre15 && P.steer_small; }

cudaError_t launch_cost_grad(const DevParams& P, const float4* rec, const RepairWs& ws, int n_seq,
                             const float* x0, const float* V, int N, float w_run, float w_cbf,
                             int ck, double* J_out, float* grad_out, unsigned* status,
                             cudaStream_t st) {
    const size_t smem = rec_table_bytes(P.n_track);
    auto kern = fast_model(P) ? cost_grad_kernel<true> : cost_grad_kernel<false>;
    cudaError_t e = ensure_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<(n_seq + REP_BLK - 1) / REP_BLK, REP_BLK, smem, st>>>(
        P, rec, ws, n_seq, x0, V, N, w_run, w_cbf, ck, J_out, grad_out, status);
    return cudaGetLastError();
}

cudaError_t launch_repair(const DevParams& P, const float4* rec, const RepairWs& ws, int n_seq,
                          const float* x0, const float* V_in, float* V_out, int n_iters, int mode,
                          float delta, double* merit_out, int* iters_out, const ApplyArgs& ap,
                          unsigned* status, cudaStream_t st) {
    const size_t smem = rec_table_bytes(P.n_track) + (size_t)P.T * 16 +
                        (size_t)(P.T + 2) * NFIELD * 4 + grad_ws_bytes(P.T);
    auto kern = fast_model(P) ? repair_block_kernel<true> : repair_block_kernel<false>;
    cudaError_t e = ensure_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<n_seq, REPB_BLK, smem, st>>>(P, rec, x0, V_in, V_out, n_iters, mode, delta, ws.ck,
                                        merit_out, iters_out, ap, status);
    return cudaGetLastError();
}

cudaError_t launch_apply(const DevParams& P, const ApplyArgs& ap, const float* V_exec,
                         cudaStream_t st) {
    apply_kernel<<<1, 1, 0, st>>>(P, ap, V_exec);
    return cudaGetLastError();
}

}  // namespace smppi
