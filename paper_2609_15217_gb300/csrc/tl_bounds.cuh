// tl_bounds.cuh -- index checks of the bounds-checked build (-DTL_CHECK_BOUNDS,
// libtinylu_checked.so): the library's stand-in for a memory checker on
// shared GPUs where none may run.
//
// In a checked build TL_SM(M, idx, lim) checks 0 <= idx < lim before the
// shared-memory access M[idx].  A violation is counted in a device word of
// the translation unit and the access goes to M[0] instead, so a wrong
// index never reaches memory outside the system's block: nothing traps,
// asserts or faults.  tl_check_bounds_violations() (tl_api.cu) sums and
// clears the words of every unit.  In the normal build TL_SM(M, idx, lim)
// is M[idx] and costs nothing.
#pragma once
#include <cuda_runtime.h>

#ifndef TL_CHECK_BOUNDS
#define TL_CHECK_BOUNDS 0
#endif

#if TL_CHECK_BOUNDS
namespace tl {
namespace chk {

// Violations counted by the kernels of this translation unit.
static __device__ unsigned long long g_violations;

__device__ __forceinline__ int guard(int idx, int lim)
{
    if (static_cast<unsigned>(idx) >= static_cast<unsigned>(lim)) {
        atomicAdd(&g_violations, 1ULL);
        return 0;
    }
    return idx;
}

// Host side: each unit registers a reader of its word (tl_api.cu keeps the
// list and sums them).
using Reader = unsigned long long (*)();
void register_reader(Reader r);

static unsigned long long read_and_clear()
{
    unsigned long long v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_violations, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return ~0ULL;
    }
    cudaMemcpyToSymbol(g_violations, &zero, sizeof(zero));
    return v;
}

struct ReaderRegistration {
    ReaderRegistration() { register_reader(&read_and_clear); }
};
static const ReaderRegistration reader_registration;

}  // namespace chk
}  // namespace tl
#define TL_SM(M, idx, lim) (M)[tl::chk::guard((idx), (lim))]
#else
#define TL_SM(M, idx, lim) (M)[(idx)]
#endif
