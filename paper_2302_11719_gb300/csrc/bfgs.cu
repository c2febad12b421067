// BFGS repair on the Cartesian state (smppi_repair mode 2): the solver Sec. IV-B
// names for the local problem of Eq. 22, run for a fixed number of iterations;
// the solver, its variant (box projection, Armijo on the projected path,
// binding coordinates held, gradient-step restarts) and the forms of H are in
// bfgs.cuh.  One WARP per sequence: the warp forms the adjoint gradient (lane 0
// the forward pass into the warp's tape unless the merit or the full step's
// trial left it there, the lanes the coefficients of the steps' adjoint maps,
// lane 0 the recursion: tape_cost_grad), and the lanes evaluate the line-search
// trials in parallel.  A block holds a few warps that share the staged track
// table; warps take sequences from an atomic counter, so the sequences that
// need many iterations do not hold up a fixed share of the others.
#include <algorithm>

#include "bfgs.cuh"
#include "bfgs_launch.cuh"

namespace smppi {
namespace {

// The merit of the Cartesian state from x0 (nearest segment s0): forward_cost
// (the merit and a kept trial leave their trajectory on the warp's full tape),
// and its gradient from that tape by the warp (tape_cost_grad; the C = 1.5,
// small-steer model) or by lane 0 alone (seq_cost_grad, checkpoint interval ck,
// which writes its own tape).
template <bool FAST>
struct CartMerit {
    const float4* rec;
    State x0;
    int s0, ck;
    Tape tape;
    float4* coef;   // 5 float4 per step
    __device__ __forceinline__ double merit(const DevParams& P, const float2* Vw) const {
        return forward_cost<true, false, FAST>(P, rec, x0, s0, P.N_r, Vw, nullptr, 0.0f, 1, 0, 0.0f,
                                               1.0f, 0, tape, nullptr);
    }
    __device__ __forceinline__ void grad(const DevParams& P, const float2* Vw, float2* G,
                                         bool have_tape) const {
        const int lane = threadIdx.x & 31;
        if (FAST)
            tape_cost_grad<FAST>(P, rec, x0, s0, P.N_r, P.T, Vw, G, tape, coef, lane, 32,
                                 []() { __syncwarp(); }, have_tape);
        else if (lane == 0)
            seq_cost_grad<FAST>(P, rec, x0, s0, P.N_r, P.T, Vw, G, 1, 0, 0.0f, 1.0f, ck, tape);
    }
    __device__ __forceinline__ double trial(const DevParams& P, const float2* Vw, const float2* G,
                                            const float2* Dn, float a, double* dec,
                                            bool keep) const {
        return forward_cost<true, true, FAST>(P, rec, x0, s0, P.N_r, Vw, G, a, 1, 0, 0.0f, 1.0f, 0,
                                              keep ? tape : Tape{nullptr, 1, 0}, dec, Dn);
    }
};

}  // namespace

// Bytes of one warp's shared-memory region for horizon T (a multiple of 8, so
// every warp's float2 arrays stay aligned): the solver's arrays, the tape
// padded to 16 bytes, and the gradient's coefficients (5 float4 per step, at the
// next 16-byte boundary).
__host__ __device__ inline size_t bfgs_tape_bytes(int T) {
    return (((size_t)(T + 2) * NFIELD * 4) + 15) & ~size_t(15);
}
__host__ __device__ inline size_t bfgs_warp_bytes(int T) {
    return bfgs_array_bytes(T) + bfgs_tape_bytes(T) + (size_t)T * 80 + 16;
}

template <bool FAST>
__global__ void __launch_bounds__(32 * BFGS_WPB_MAX, 2) repair_bfgs_kernel(
    DevParams P, const float4* __restrict__ recg, const float* __restrict__ x0g, const float* Vin,
    float* Vout, int n_seq, int n_iters, int ck, float* __restrict__ Hws,
    unsigned* __restrict__ next, double* __restrict__ merit_out, int* __restrict__ iters_out,
    ApplyArgs ap, unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = P.T, nt = P.n_track, n = 2 * P.N_r;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    float4* rec = reinterpret_cast<float4*>(smem_raw);
    unsigned char* wbase = smem_raw + rec_table_bytes(nt) + (size_t)warp * bfgs_warp_bytes(T);
    const BfgsArrays a = bfgs_arrays(wbase, T);
    float* tape_s = reinterpret_cast<float*>(wbase + bfgs_array_bytes(T));
    float4* coef = reinterpret_cast<float4*>(
        (reinterpret_cast<uintptr_t>(wbase + bfgs_array_bytes(T) + bfgs_tape_bytes(T)) + 15) &
        ~uintptr_t(15));
    float* H = Hws + ((size_t)blockIdx.x * wpb + warp) * n * n;

    for (int i = threadIdx.x; i < 3 * (nt + 5); i += blockDim.x) rec[i] = recg[i];
    __syncthreads();

    for (;;) {
        int q = 0;
        if (lane == 0) q = (int)atomicAdd(next, 1u);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= n_seq) break;
        const float2* vin = reinterpret_cast<const float2*>(Vin) + (size_t)q * T;
        for (int t = lane; t < T; t += 32) a.Vw[t] = vin[t];
        const State x0 = make_state(x0g + 6 * q);
        // global nearest segment of x0 (lowest index on ties)
        float bd = 3.0e38f;
        int s0 = 0x7fffffff;
        for (int i = lane; i < nt; i += 32) {
            const float d = rec_d2_seg(rec, i, x0.X, x0.Y);
            if (d < bd) { bd = d; s0 = i; }
        }
        warp_argmin(bd, s0);
        s0 = seg_or_zero(s0, nt, lane == 0 ? status : nullptr);
        __syncwarp();
        const CartMerit<FAST> f{rec, x0, s0, ck, Tape{tape_s, 1, 0}, coef};
        double P0;
        bool stalled;
        const int it = bfgs_solve(P, f, a, H, n_iters,
                                  merit_out ? merit_out + (size_t)q * (n_iters + 1) : nullptr, &P0,
                                  &stalled);
        if (lane == 0) {
            if (iters_out) iters_out[q] = it;
            if (stalled) atomicOr(status, SMPPI_DEV_STALLED);
            if (!isfinite(P0)) atomicOr(status, SMPPI_DEV_NUMERIC);
        }
        float2* vout = reinterpret_cast<float2*>(Vout) + (size_t)q * T;
        for (int t = lane; t < T; t += 32) vout[t] = a.Vw[t];
        if (q == 0 && lane == 0 && ap.x0) closed_loop_step(P, ap, a.Vw[0]);
        __syncwarp();   // the warp's shared memory is reused by its next sequence
    }
}

namespace {

const void* bfgs_kernel(const DevParams& P) {
    return (P.tyre15 && P.steer_small) ? (const void*)repair_bfgs_kernel<true>
                                       : (const void*)repair_bfgs_kernel<false>;
}

}  // namespace

int bfgs_shape(const void* kern, size_t fixed_bytes, size_t warp_bytes, int N_r, int n_seq,
               int sms, int* wpb_out) {
    int dev = 0, max_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if ((size_t)max_optin < fixed_bytes + warp_bytes) return 0;
    const int wpb = (int)std::min<size_t>(BFGS_WPB_MAX, ((size_t)max_optin - fixed_bytes) / warp_bytes);
    const size_t smem = fixed_bytes + (size_t)wpb * warp_bytes;
    if (ensure_smem(kern, smem) != cudaSuccess) return 0;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, 32 * wpb, smem) != cudaSuccess)
        return 0;
    const size_t n = 2 * (size_t)N_r;
    const size_t per = std::max<size_t>(1, n * n * sizeof(float));
    const int by_ws = (int)std::max<size_t>(1, BFGS_WS_MAX / per / wpb);
    const int by_seq = (n_seq + wpb - 1) / wpb;
    if (wpb_out) *wpb_out = wpb;
    return std::max(1, std::min({by_seq, std::max(1, bps) * sms, by_ws}));
}

// Launch shape of the BFGS repair: the track table and the warps' regions.
int bfgs_grid(const DevParams& P, int n_seq, int sms, int* wpb_out) {
    return bfgs_shape(bfgs_kernel(P), rec_table_bytes(P.n_track), bfgs_warp_bytes(P.T), P.N_r,
                      n_seq, sms, wpb_out);
}

// Workspace: a 16-byte work counter, then one H slice per warp slot.
size_t bfgs_ws_bytes(const DevParams& P, int grid, int wpb) {
    const size_t n = 2 * (size_t)P.N_r;
    return 16 + (size_t)grid * wpb * n * n * sizeof(float);
}

cudaError_t launch_repair_bfgs(const DevParams& P, const float4* rec, int n_seq, const float* x0,
                               const float* V_in, float* V_out, int n_iters, int ck, void* ws,
                               int grid, int wpb, double* merit_out, int* iters_out,
                               const ApplyArgs& ap, unsigned* status, cudaStream_t st) {
    const size_t smem = rec_table_bytes(P.n_track) + (size_t)wpb * bfgs_warp_bytes(P.T);
    const void* kern = bfgs_kernel(P);
    cudaError_t e = ensure_smem(kern, smem);
    if (e != cudaSuccess) return e;
    unsigned* next = static_cast<unsigned*>(ws);
    float* H = reinterpret_cast<float*>(static_cast<unsigned char*>(ws) + 16);
    e = cudaMemsetAsync(next, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    if (P.tyre15 && P.steer_small)
        repair_bfgs_kernel<true><<<grid, 32 * wpb, smem, st>>>(P, rec, x0, V_in, V_out, n_seq, n_iters,
                                                                ck, H, next, merit_out, iters_out, ap,
                                                                status);
    else
        repair_bfgs_kernel<false><<<grid, 32 * wpb, smem, st>>>(P, rec, x0, V_in, V_out, n_seq, n_iters,
                                                                 ck, H, next, merit_out, iters_out, ap,
                                                                 status);
    return cudaGetLastError();
}

}  // namespace smppi
