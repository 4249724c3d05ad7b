// tl_handle.h -- the opaque tl_handle of the C ABI (library-internal).
#pragma once
#include <cstddef>
#include <cstdint>
#include <functional>
#include <unordered_map>
#include <unordered_set>
#include <utility>

#include "tinylu.h"
#include "tl_internal.h"

namespace tl {

// Dispatch choice for one (n, layout, op): lanes per system (0 = default
// policy) and block size (0 = occupancy + wave-fill heuristic per launch).
struct Choice {
    int lanes;
    int block;
};

struct PairHash {
    size_t operator()(const std::pair<const void *, int> &p) const
    {
        return std::hash<const void *>()(p.first) ^ (static_cast<size_t>(p.second) * 0x9e3779b97f4a7c15ULL);
    }
};

int default_lanes(int n);
int default_register_lanes(int n);
// Default mixed-precision ragged variant id for n: one thread, then 4 lanes
// per system in registers, then the shared-memory warp kernel.
int default_ir_id(int n);
const Variant *find_variant(int n, int layout, int op, int id);
tl_status fail_arg(tl_handle *h, int pos);
tl_status fail_cuda(tl_handle *h, cudaError_t e);
int pick_block(tl_handle *h, const void *kernel, int64_t threads, int lanes, size_t smem_per_system,
               int smem_limit);
tl_status launch_variant(tl_handle *h, const Variant *v, int n, int block, SolveArgs &args, cudaStream_t stream);
tl_status smem_opt_in(tl_handle *h, const void *kernel, int *limit);
int blocks_per_sm(tl_handle *h, const void *kernel, int block, size_t smem);
// Default ragged variant id for n: register kernels up to n = 16, the
// shared-memory solver (16 lanes, then 32) above.
int default_ragged_id(int n);
tl_status launch_op(tl_handle *h, int n, int layout, int op, SolveArgs &args, cudaStream_t stream);
tl_status ensure_workspace(tl_handle *h, size_t bytes, cudaStream_t stream);
// Buckets `batch` systems by n[s] using the int32 scratch `ws` (3*64 bin
// counters followed by `batch` indices) and launches the per-n kernels.
// With mixed precision the scratch also holds 64 fallback counters and
// `batch` fallback indices (ragged_ws_ints).
tl_status ragged_solve(tl_handle *h, int64_t batch, const int32_t *n, RaggedArgs r, int32_t *ws,
                       cudaStream_t stream, bool mixed = false);
// Mixed precision for size n: true when its systems refine a binary32
// factorization, false when they go straight to the binary64 solve.
bool mixed_refines(const tl_handle *h, int n);
size_t ragged_ws_ints(int64_t batch, bool mixed);
// int32 slots in front of the bucket indices in the ragged workspace: bin
// counts, offsets and cursors (64 each) and the persistent launch's plan.
constexpr int kRaggedHeaderInts = 4 * 64;

}  // namespace tl

struct tl_handle {
    int device = 0;
    int sm_count = 1;
    int max_threads_per_sm = 2048;
    int max_smem_per_block = 48 * 1024;
    int last_cuda_error = 0;
    int last_bad_arg = 0;
    int ragged_mode = TL_RAGGED_PERSISTENT;  // tl_ragged_set_mode
    // mixed precision per n: -1 default rule, 0 refine, 1 solve in binary64
    signed char mixed_route[TL_MAX_N + 1] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
                                             -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
    tl::Choice choice[TL_MAX_N + 1][2][tl::kOps] = {};
    std::unordered_map<std::pair<const void *, int>, int, tl::PairHash> occupancy;
    std::unordered_map<const void *, int> smem_opt_in;  // kernel -> dynamic smem limit set
    // device workspace owned by the handle (grown on demand, never inside a
    // stream capture) and pinned host staging buffers
    void *ws = nullptr;
    size_t ws_bytes = 0;
    void *host_stage[2] = {nullptr, nullptr};
    size_t host_stage_bytes = 0;
};
