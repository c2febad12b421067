// Failure-detection self-test: one block waits, through the library's own
// bounded device waits, on something that nothing completes, so that a caller
// can check on a live GPU that a wait which runs out ends the kernel with
// SMPPI_DEV_TIMEOUT in a status word (and leaves the context usable) instead
// of hanging.  The waits are the ones the kernels use: mbar_wait_bounded (the
// staging of the segment-pair table by bulk copy) and spin_until_geq (the
// progress counters of the split merit pass).
#include "shield.cuh"

namespace smppi {

__global__ void wait_timeout_kernel(int which, unsigned* __restrict__ status) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int counter;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);   // one arrival expected; none comes
        counter = 0;          // nothing advances it
    }
    __syncthreads();
    const bool ok = (which == 0) ? mbar_wait_bounded(&bar, 0u) : spin_until_geq(&counter, 1);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, SMPPI_DEV_TIMEOUT);
}

}  // namespace smppi

using namespace smppi;

extern "C" smppi_status smppi_debug_wait_timeout(int which, uint32_t* status, void* cuda_stream) {
    if (which != 0 && which != 1)
        return report_error(SMPPI_ERR_ARG, "smppi_debug_wait_timeout: which must be 0 or 1");
    if (!status) return report_error(SMPPI_ERR_ARG, "smppi_debug_wait_timeout: status is NULL");
    wait_timeout_kernel<<<1, 32, 0, static_cast<cudaStream_t>(cuda_stream)>>>(which, status);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(SMPPI_ERR_CUDA, cudaGetErrorString(e));
    return SMPPI_OK;
}
