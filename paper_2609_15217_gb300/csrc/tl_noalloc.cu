// tl_noalloc.cu -- tl_lupp_solve_batched_noalloc: the ragged-batch solve for
// callers that must not allocate device memory.
//
// tl_lupp_solve_batched keeps its bucket lists in a workspace that the
// handle grows with cudaMalloc (and, when it grows, a device-wide
// synchronization and cudaFree of the old buffer).  Some callers cannot
// afford either: code that runs under a fixed device-memory budget owned by
// someone else, latency-bound serving loops that must never stall the whole
// device, and code that is not allowed to synchronize other work on the GPU.
// This entry point does the same solve with its scratch in a fixed array
// that is part of the library itself, so a call never allocates or frees.
//
// The array below is created with the library's module on every GPU that
// loads it and stays there until the process exits.  In host code the name
// `g_ragged_scratch` is only a host-side stand-in: its device address is
// looked up once per device with cudaGetSymbolAddress and passed to the
// kernels.
#include <mutex>

#include "tinylu.h"
#include "tl_handle.h"
#include "tl_internal.h"

namespace tl {
namespace {

// The ragged workspace header (per-size counters and the plan of the
// persistent launch), then one int32 system index per system.
constexpr int64_t kNoAllocMaxBatch = TL_NOALLOC_MAX_BATCH;
constexpr size_t kScratchInts = kRaggedHeaderInts + static_cast<size_t>(kNoAllocMaxBatch);

static __device__ __align__(256) int32_t g_ragged_scratch[kScratchInts];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
int32_t *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up on
// the first call made with that device current.
tl_status scratch_address(tl_handle *h, int32_t **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(h, e);
    if (dev < 0 || dev >= kMaxDevices) return TL_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_ragged_scratch);
        if (e != cudaSuccess) return fail_cuda(h, e);
        g_scratch_addr[dev] = static_cast<int32_t *>(p);
    }
    *out = g_scratch_addr[dev];
    return TL_OK;
}

}  // namespace
}  // namespace tl

using namespace tl;

extern "C" tl_status tl_lupp_solve_batched_noalloc(tl_handle *h, int64_t batch, const int32_t *n,
                                                   const int64_t *a_off, const double *A, const int64_t *b_off,
                                                   const double *b, double *x, const int64_t *piv_off,
                                                   int32_t *ipiv, int32_t *info, cudaStream_t stream)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (batch < 0 || batch > kNoAllocMaxBatch) return fail_arg(h, 2);
    if (batch == 0) return TL_OK;
    auto mis = [](const void *p, size_t a) { return !p || (reinterpret_cast<uintptr_t>(p) % a) != 0; };
    if (mis(n, 4)) return fail_arg(h, 3);
    if (mis(a_off, 8)) return fail_arg(h, 4);
    if (mis(A, 8)) return fail_arg(h, 5);
    if (mis(b_off, 8)) return fail_arg(h, 6);
    if (mis(b, 8)) return fail_arg(h, 7);
    if (mis(x, 8)) return fail_arg(h, 8);
    if (mis(piv_off, 8)) return fail_arg(h, 9);
    if (mis(ipiv, 4)) return fail_arg(h, 10);
    if (mis(info, 4)) return fail_arg(h, 11);
    int32_t *ws = nullptr;
    tl_status st = scratch_address(h, &ws);
    if (st != TL_OK) return st;
    // ragged_solve clears the per-size counters on `stream` before using them;
    // the index lists are fully rewritten by every call.
    RaggedArgs r{nullptr, nullptr, a_off, A, b_off, b, x, piv_off, ipiv, info};
    return ragged_solve(h, batch, n, r, ws, stream);
}
