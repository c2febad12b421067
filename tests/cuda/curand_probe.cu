// Test helper: cuRAND's Philox4_32_10 device generator for given counters.
// curand_init(seed, subsequence, offset) starts at counter
// (offset/4 as a 64-bit add to words 0-1, subsequence to words 2-3) with key
// (seed lo, seed hi); curand4 returns the block of the current counter.
#include <curand_kernel.h>

__global__ void probe(unsigned long long seed, const unsigned* ctr, int n, unsigned* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned* c = ctr + 4 * i;
    unsigned long long subseq = (unsigned long long)c[2] | ((unsigned long long)c[3] << 32);
    unsigned long long offset = 4ull * ((unsigned long long)c[0] | ((unsigned long long)c[1] << 32));
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subseq, offset, &st);
    uint4 r = curand4(&st);
    out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
}

extern "C" int curand_probe(unsigned long long seed, const unsigned* ctr_dev, int n,
                            unsigned* out_dev) {
    probe<<<(n + 127) / 128, 128>>>(seed, ctr_dev, n, out_dev);
    return (int)cudaDeviceSynchronize();
}
