// Test helper: evaluates the library's integer-pipe reciprocal and CUDA's
// __drcp_rn on the same inputs (compiled by tests/test_gpu_reciprocal.py).
#include <cstdint>

#include "tinylu_device.cuh"

__global__ void k_rcp_check(const double *in, double *ours, double *ref, int64_t n)
{
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        ours[i] = tl::dev::rcp_rn(in[i]);
        ref[i] = __drcp_rn(in[i]);
    }
}

extern "C" int rcp_check(const double *in, double *ours, double *ref, int64_t n)
{
    k_rcp_check<<<1024, 256>>>(in, ours, ref, n);
    return static_cast<int>(cudaDeviceSynchronize());
}
