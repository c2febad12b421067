// smppi_step_noalloc: one MPPI iteration for callers that cannot allocate
// device memory (hard real-time control loops that forbid allocation after
// start-up, or host runtimes that own every device allocation themselves).
//
// The iteration's scratch (segment-pair table, rollout costs, block minima, the
// update kernel's partials and counters) lives in one file-scope __device__
// array of fixed size, so the call allocates nothing.  Host code cannot use
// the array's name as a device address: its device address is looked up with
// cudaGetSymbolAddress (the first call on a device does this, so that call
// should come before any stream capture; later calls outside a capture look it
// up again) and passed to the kernels.  Every call on a device shares the
// same array and leaves the last call's contents in it; calls whose work
// overlaps on the GPU (different streams, host threads) race on it and must be
// serialised by the caller.
#include <mutex>

#include "kernels.cuh"

using namespace smppi;

namespace {

// Limits of the allocation-free entry point.
constexpr int NA_MAX_K = 65536;
constexpr int NA_MAX_BLK = (NA_MAX_K + ROLL_BLK - 1) / ROLL_BLK;

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t OFF_REC = 0;
constexpr size_t OFF_S = OFF_REC + align256((size_t)(SMPPI_MAX_TRACK + 5) * 3 * sizeof(float4));
constexpr size_t OFF_MIN = OFF_S + align256(sizeof(float) * NA_MAX_K);
constexpr size_t OFF_ACC = OFF_MIN + align256(sizeof(float) * NA_MAX_BLK);
constexpr size_t OFF_ETA = OFF_ACC + align256(sizeof(float) * 2 * SMPPI_MAX_T * UPD_BLK);
constexpr size_t OFF_HAS = OFF_ETA + align256(sizeof(double) * UPD_BLK);
constexpr size_t OFF_TICKET = OFF_HAS + align256(sizeof(int) * UPD_BLK);
constexpr size_t OFF_STATUS = OFF_TICKET + 256;
constexpr size_t SCRATCH_BYTES = OFF_STATUS + 256;   // about 1.4 MB per device

__device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_scratch_dev[MAX_DEVICES] = {};

// Device address of g_scratch on the current device.  Looked up again on
// every call made outside a stream capture (the address does not survive a
// device reset, after which the module is loaded anew); a call inside a
// capture uses the address of the last call on the device.
smppi_status scratch_address(cudaStream_t st, unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report_error(SMPPI_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES)
        return report_error(SMPPI_ERR_ARG, "smppi_step_noalloc: device ordinal out of range");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return report_error(SMPPI_ERR_CUDA, cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev] || cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return report_error(SMPPI_ERR_CUDA, "smppi_step_noalloc: cudaGetSymbolAddress failed");
        g_scratch_dev[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_dev[dev];
    return SMPPI_OK;
}

}  // namespace

extern "C" smppi_status smppi_step_noalloc(const smppi_params* p, const float* x0, float* V,
                                           uint32_t iter, uint32_t instance, float* S_out,
                                           void* cuda_stream) {
    smppi_status s = validate_params(p);
    if (s == SMPPI_OK && p->state_kind != 0)
        return report_error(SMPPI_ERR_ARG, "smppi_step_noalloc: needs state_kind 0");
    if (s != SMPPI_OK) return s;
    if (!x0 || !V) return report_error(SMPPI_ERR_ARG, "smppi_step_noalloc: x0 and V must not be NULL");
    if (p->K > NA_MAX_K)
        return report_error(SMPPI_ERR_ARG, "smppi_step_noalloc: K exceeds its limit of 65536");
    if (instance >= (1u << 24))
        return report_error(SMPPI_ERR_ARG, "smppi_step_noalloc: instance must be < 2^24");
    if (rollout_smem_bytes(p->n_track, p->T) > 200 * 1024)
        return report_error(SMPPI_ERR_ARG, "smppi_step_noalloc: n_track and T exceed shared memory");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned char* base = nullptr;
    s = scratch_address(st, &base);
    if (s != SMPPI_OK) return s;
    const DevParams dp = derive_params(*p);
    float4* rec = reinterpret_cast<float4*>(base + OFF_REC);
    float* S = S_out ? S_out : reinterpret_cast<float*>(base + OFF_S);
    float* blk_min = reinterpret_cast<float*>(base + OFF_MIN);
    float* part_acc = reinterpret_cast<float*>(base + OFF_ACC);
    double* part_eta = reinterpret_cast<double*>(base + OFF_ETA);
    int* part_has = reinterpret_cast<int*>(base + OFF_HAS);
    unsigned* ticket = reinterpret_cast<unsigned*>(base + OFF_TICKET);
    unsigned* status = reinterpret_cast<unsigned*>(base + OFF_STATUS);
    const uint32_t ctr3 = instance << 8;
    // the update's ticket must start at zero (a launch that was cut short can leave it set)
    cudaError_t e = cudaMemsetAsync(base + OFF_TICKET, 0, 512, st);
    if (e == cudaSuccess) e = launch_rec_table(p->track_xy, p->n_track, rec, st);
    if (e == cudaSuccess)
        e = launch_rollout(dp, false, x0, V, rec, iter, ctr3, nullptr, S, nullptr,
                           blk_min, nullptr, status, st);
    if (e == cudaSuccess)
        e = launch_update(dp, S, blk_min, rollout_blocks(dp), V, iter, ctr3, nullptr,
                          part_acc, part_eta, part_has, ticket, status, st);
    if (e != cudaSuccess) return report_error(SMPPI_ERR_CUDA, cudaGetErrorString(e));
    return SMPPI_OK;
}
