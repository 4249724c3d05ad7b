// tl_api.cu -- implementation of the C ABI declared in include/tinylu.h:
// handle, argument checking, the per-n kernel dispatcher ("best X" table of
// the paper's Sec. 4.1 reporting convention) and the launch heuristic that
// picks the block size maximizing occupancy + wave fill (Sec. 4.1, "Kernel
// launch configuration").
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <new>
#include <unordered_map>

#include <vector>

#include "tinylu.h"
#include "tl_handle.h"
#include "tl_internal.h"
#include "tl_smem.cuh"

namespace tl {

#if TL_CHECK_BOUNDS
namespace chk {
// Readers of the violation words of every checked translation unit.
static std::vector<Reader> &readers()
{
    static std::vector<Reader> v;
    return v;
}
void register_reader(Reader r) { readers().push_back(r); }
}  // namespace chk
#endif

// Zero-initialized before any dynamic initializer runs, so the
// instantiation units may register from their static constructors in any
// order.
static VariantList g_registry[TL_MAX_N + 1][2][kOps];

VariantList &registry(int n, int layout, int op) { return g_registry[n][layout][op]; }

void register_variant(int n, int layout, int op, int lanes, const void *kernel, int kind, const void *fixup)
{
    if (n < 1 || n > TL_MAX_N || layout < 0 || layout > 1 || op < 0 || op >= kOps) return;
    VariantList &l = g_registry[n][layout][op];
    for (int i = 0; i < l.count; ++i)
        if (l.v[i].lanes == lanes && l.v[i].kind == kind) return;
    if (l.count < kMaxVariants) l.v[l.count++] = Variant{lanes, kernel, kind, fixup};
}

// Default thread-to-system mapping per n before any autotuning: one thread
// per system while the matrix fits in registers without spilling, then the
// fewest lanes per system that keep a lane's rows in registers.
int default_register_lanes(int n)
{
    if (n <= 9) return 1;
    if (n <= 12) return 2;
    if (n <= 16) return 4;
    if (n <= 24) return 8;
    return 16;
}

// Lanes per system of the mixed-precision ragged kernel before any tuning.
int default_ir_id(int n)
{
    if (n <= 10) return variant_id(1, 0);
    if (n <= 16) return variant_id(4, 0);
    return variant_id(32, 1);
}

int default_ragged_id(int n)
{
    if (n <= 16) return variant_id(default_register_lanes(n), 0);
    return variant_id(n <= 26 ? 16 : 32, 1);
}

// Default gesv/getrf variant id per n before any autotuning: the variant
// tl_autotune found fastest at each n on a GB300 (interleaved batches of
// about 1.6 GFLOP per n).  One thread per system in registers up to n = 9,
// then the two-step element walk in shared memory with 2, 4, 8, 16 and 32
// lanes per system (16 up to n = 30, 32 at n = 31, 32).
int default_lanes(int n)
{
    if (n <= 9) return variant_id(1, 0);
    if (n <= 11) return variant_id(2, 2);
    if (n <= 15) return variant_id(4, 2);
    if (n <= 23) return variant_id(8, 2);
    if (n <= 30) return variant_id(16, 1);
    return variant_id(32, 1);
}

// Variant by id (lanes + 100 * kind); falls back to the register kernel of
// the default lane count, then to anything registered.
const Variant *find_variant(int n, int layout, int op, int id)
{
    const VariantList &l = g_registry[n][layout][op];
    for (int i = 0; i < l.count; ++i)
        if (variant_id(l.v[i].lanes, l.v[i].kind) == id) return &l.v[i];
    const int dflt = default_register_lanes(n);
    for (int i = 0; i < l.count; ++i)
        if (l.v[i].kind == 0 && l.v[i].lanes == dflt) return &l.v[i];
    return l.count ? &l.v[0] : nullptr;
}

tl_status fail_arg(tl_handle *h, int pos)
{
    if (h) h->last_bad_arg = pos;
    return TL_ERR_INVALID_ARG;
}

tl_status fail_cuda(tl_handle *h, cudaError_t e)
{
    if (h) h->last_cuda_error = static_cast<int>(e);
    return TL_ERR_CUDA;
}

// Resident blocks per SM of `kernel` at `block` threads and `smem` bytes of
// dynamic shared memory (cached).
int blocks_per_sm(tl_handle *h, const void *kernel, int block, size_t smem)
{
    auto key = std::make_pair(kernel, block * 1048576 + static_cast<int>(smem / 16));
    auto it = h->occupancy.find(key);
    if (it != h->occupancy.end()) return it->second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, smem) != cudaSuccess) {
        cudaGetLastError();
        nb = 0;
    }
    h->occupancy[key] = nb;
    return nb;
}

// Block size maximizing O + W: O the theoretical occupancy, W the mean fill
// of the waves the grid needs.  For shared-memory kernels (smem_per_lane_group
// > 0) a block of b threads holds b / lanes systems.
int pick_block(tl_handle *h, const void *kernel, int64_t threads, int lanes, size_t smem_per_system, int smem_limit)
{
    static const int cands[] = {32, 64, 128};
    int best = 0;
    double best_score = -1.0;
    for (int b : cands) {
        if (b < lanes) continue;
        const size_t smem = smem_per_system ? (b / lanes) * smem_per_system : 0;
        if (smem > static_cast<size_t>(smem_limit)) continue;
        int nb = blocks_per_sm(h, kernel, b, smem);
        if (nb <= 0) continue;
        double O = static_cast<double>(nb) * b / h->max_threads_per_sm;
        int64_t blocks = (threads + b - 1) / b;
        int64_t per_wave = static_cast<int64_t>(nb) * h->sm_count;
        int64_t waves = (blocks + per_wave - 1) / per_wave;
        double W = static_cast<double>(blocks) / static_cast<double>(waves * per_wave);
        double score = O + W;
        if (score >= best_score - 1e-12) {
            best_score = score;
            best = b;
        }
    }
    if (best == 0) best = lanes > 32 ? lanes : 32;  // nothing resident: smallest block
    return best;
}

// Allow a shared-memory kernel all the opt-in shared memory its static part
// leaves free (once per kernel, before any occupancy query); *limit receives
// the dynamic shared memory a block may use.
tl_status smem_opt_in(tl_handle *h, const void *kernel, int *limit)
{
    auto it = h->smem_opt_in.find(kernel);
    if (it != h->smem_opt_in.end()) {
        *limit = it->second;
        return TL_OK;
    }
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return fail_cuda(h, e);
    const int dyn_limit = h->max_smem_per_block - static_cast<int>(fa.sharedSizeBytes);
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_limit);
    if (e != cudaSuccess) return fail_cuda(h, e);
    h->smem_opt_in[kernel] = dyn_limit;
    *limit = dyn_limit;
    return TL_OK;
}

tl_status launch_variant(tl_handle *h, const Variant *v, int n, int block, SolveArgs &args, cudaStream_t stream)
{
    if (args.batch == 0) return TL_OK;
    const int64_t threads = args.batch * v->lanes;
    const size_t per_sys = v->kind >= 1 ? smem_sys_bytes(n, v->lanes) : 0;
    cudaError_t e;
    int dyn_limit = h->max_smem_per_block;
    if (v->kind >= 1) {
        const tl_status st = smem_opt_in(h, v->kernel, &dyn_limit);
        if (st != TL_OK) return st;
    }
    if (block <= 0) block = pick_block(h, v->kernel, threads, v->lanes, per_sys, dyn_limit);
    const int64_t grid = (threads + block - 1) / block;
    if (grid > INT_MAX) return TL_ERR_UNSUPPORTED;
    if (v->kind >= 1) {
        const size_t smem = (block / v->lanes) * per_sys;
        if (smem > static_cast<size_t>(dyn_limit)) return TL_ERR_UNSUPPORTED;
        int nn = n;
        void *params[] = {&args, &nn};
        e = cudaLaunchKernel(v->kernel, dim3(static_cast<unsigned>(grid)), dim3(block), params, smem, stream);
    } else {
        void *params[] = {&args};
        e = cudaLaunchKernel(v->kernel, dim3(static_cast<unsigned>(grid)), dim3(block), params, 0, stream);
        if (e == cudaSuccess && v->fixup) {
            const int64_t fgrid = (args.batch + 127) / 128;
            e = cudaLaunchKernel(v->fixup, dim3(static_cast<unsigned>(fgrid)), dim3(128), params, 0, stream);
        }
    }
    if (e != cudaSuccess) return fail_cuda(h, e);
    return TL_OK;
}

tl_status launch_op(tl_handle *h, int n, int layout, int op, SolveArgs &args, cudaStream_t stream)
{
    const Choice &c = h->choice[n][layout][op];
    const Variant *v = find_variant(n, layout, op, c.lanes ? c.lanes : default_lanes(n));
    if (!v) return TL_ERR_UNSUPPORTED;
    return launch_variant(h, v, n, c.block, args, stream);
}

static bool misaligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) != 0; }

}  // namespace tl

using namespace tl;

extern "C" {

tl_status tl_create(tl_handle **out)
{
    if (!out) return TL_ERR_INVALID_ARG;
    *out = nullptr;
    tl_handle *h = new (std::nothrow) tl_handle();
    if (!h) return TL_ERR_NO_MEMORY;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&h->max_threads_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, h->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&h->max_smem_per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    if (e != cudaSuccess) {
        delete h;
        return TL_ERR_CUDA;
    }
    *out = h;
    return TL_OK;
}

tl_status tl_destroy(tl_handle *h)
{
    if (!h) return TL_ERR_INVALID_ARG;
    tl_status st = TL_OK;
    if (h->ws) {
        if (cudaDeviceSynchronize() != cudaSuccess) st = TL_ERR_CUDA;
        cudaFree(h->ws);
    }
    for (int i = 0; i < 2; ++i)
        if (h->host_stage[i]) cudaFreeHost(h->host_stage[i]);
    delete h;
    return st;
}

const char *tl_status_string(tl_status s)
{
    switch (s) {
    case TL_OK: return "TL_OK";
    case TL_ERR_INVALID_ARG: return "TL_ERR_INVALID_ARG: an argument was rejected (see tl_last_bad_arg)";
    case TL_ERR_CUDA: return "TL_ERR_CUDA: a CUDA call failed (see tl_last_cuda_error)";
    case TL_ERR_NO_MEMORY: return "TL_ERR_NO_MEMORY: workspace allocation failed";
    case TL_ERR_UNSUPPORTED: return "TL_ERR_UNSUPPORTED: request not supported by the library";
    case TL_ERR_TIMEOUT: return "TL_ERR_TIMEOUT: a bounded device wait gave up";
    }
    return "unknown tl_status";
}

tl_status tl_last_cuda_error(tl_handle *h, int *err)
{
    if (!h || !err) return TL_ERR_INVALID_ARG;
    *err = h->last_cuda_error;
    return TL_OK;
}

int tl_last_bad_arg(tl_handle *h) { return h ? h->last_bad_arg : 0; }

tl_status tl_check_bounds_violations(unsigned long long *count)
{
    if (!count) return TL_ERR_INVALID_ARG;
    *count = 0;
#if TL_CHECK_BOUNDS
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return TL_ERR_CUDA;
    }
    for (chk::Reader r : chk::readers()) {
        const unsigned long long v = r();
        if (v == ~0ULL) return TL_ERR_CUDA;
        *count += v;
    }
    return TL_OK;
#else
    return TL_ERR_UNSUPPORTED;
#endif
}

tl_status tl_getrf_batched(tl_handle *h, int n, double *A, tl_layout layout, int64_t ld_batch,
                           int32_t *ipiv, int32_t *info, int64_t batch, cudaStream_t stream)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (n < 1 || n > TL_MAX_N) return fail_arg(h, 2);
    if (layout != TL_LAYOUT_PER_SYSTEM && layout != TL_LAYOUT_INTERLEAVED) return fail_arg(h, 4);
    if (batch < 0) return fail_arg(h, 8);
    if (layout == TL_LAYOUT_INTERLEAVED && ld_batch < batch) return fail_arg(h, 5);
    if (batch == 0) return TL_OK;
    if (!A || misaligned(A, 8)) return fail_arg(h, 3);
    if (!ipiv || misaligned(ipiv, 4)) return fail_arg(h, 6);
    if (!info || misaligned(info, 4)) return fail_arg(h, 7);
    SolveArgs a{nullptr, A, nullptr, nullptr, ipiv, info, ld_batch, batch, 1};
    return launch_op(h, n, layout, kOpGetrf, a, stream);
}

tl_status tl_getrs_batched(tl_handle *h, int n, int nrhs, const double *LU, const int32_t *ipiv,
                           tl_layout layout, int64_t ld_batch, double *B, int64_t batch,
                           cudaStream_t stream)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (n < 1 || n > TL_MAX_N) return fail_arg(h, 2);
    if (nrhs < 1 || nrhs > TL_MAX_N) return fail_arg(h, 3);
    if (layout != TL_LAYOUT_PER_SYSTEM && layout != TL_LAYOUT_INTERLEAVED) return fail_arg(h, 6);
    if (batch < 0) return fail_arg(h, 9);
    if (layout == TL_LAYOUT_INTERLEAVED && ld_batch < batch) return fail_arg(h, 7);
    if (batch == 0) return TL_OK;
    if (!LU || misaligned(LU, 8)) return fail_arg(h, 4);
    if (!ipiv || misaligned(ipiv, 4)) return fail_arg(h, 5);
    if (!B || misaligned(B, 8)) return fail_arg(h, 8);
    SolveArgs a{LU, nullptr, nullptr, B, const_cast<int32_t *>(ipiv), nullptr, ld_batch, batch, nrhs};
    return launch_op(h, n, layout, kOpGetrs, a, stream);
}

tl_status tl_gesv_batched(tl_handle *h, int n, const double *A, double *LU_out, const double *b,
                          double *x, int32_t *ipiv, int32_t *info, tl_layout layout,
                          int64_t ld_batch, int64_t batch, cudaStream_t stream)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (n < 1 || n > TL_MAX_N) return fail_arg(h, 2);
    if (layout != TL_LAYOUT_PER_SYSTEM && layout != TL_LAYOUT_INTERLEAVED) return fail_arg(h, 9);
    if (batch < 0) return fail_arg(h, 11);
    if (layout == TL_LAYOUT_INTERLEAVED && ld_batch < batch) return fail_arg(h, 10);
    if (batch == 0) return TL_OK;
    if (!A || misaligned(A, 8)) return fail_arg(h, 3);
    if (LU_out && misaligned(LU_out, 8)) return fail_arg(h, 4);
    if (!b || misaligned(b, 8)) return fail_arg(h, 5);
    if (!x || misaligned(x, 8)) return fail_arg(h, 6);
    if (!ipiv || misaligned(ipiv, 4)) return fail_arg(h, 7);
    if (!info || misaligned(info, 4)) return fail_arg(h, 8);
    SolveArgs a{A, LU_out, b, x, ipiv, info, ld_batch, batch, 1};
    return launch_op(h, n, layout, LU_out ? kOpGesvLU : kOpGesv, a, stream);
}

tl_status tl_gesv_batched_tilepiv(tl_handle *h, int n, int tile, double threshold, const double *A,
                                  double *LU_out, const double *b, double *x, int32_t *ipiv, int32_t *info,
                                  tl_layout layout, int64_t ld_batch, int64_t batch, cudaStream_t stream)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (n < 1 || n > TL_MAX_N) return fail_arg(h, 2);
    if (tile < 0) return fail_arg(h, 3);
    if (!(threshold >= 0.0) || !std::isfinite(threshold)) return fail_arg(h, 4);
    if (layout != TL_LAYOUT_PER_SYSTEM && layout != TL_LAYOUT_INTERLEAVED) return fail_arg(h, 11);
    if (batch < 0) return fail_arg(h, 13);
    if (layout == TL_LAYOUT_INTERLEAVED && ld_batch < batch) return fail_arg(h, 12);
    if (batch == 0) return TL_OK;
    if (!A || misaligned(A, 8)) return fail_arg(h, 5);
    if (LU_out && misaligned(LU_out, 8)) return fail_arg(h, 6);
    if (!b || misaligned(b, 8)) return fail_arg(h, 7);
    if (!x || misaligned(x, 8)) return fail_arg(h, 8);
    if (!ipiv || misaligned(ipiv, 4)) return fail_arg(h, 9);
    if (!info || misaligned(info, 4)) return fail_arg(h, 10);
    SolveArgs a{A, LU_out, b, x, ipiv, info, ld_batch, batch, 1};
    a.tile = (tile >= n) ? 0 : tile;
    a.threshold = threshold;
    const int op = LU_out ? kOpGesvLU : kOpGesv;
    if (n == 1) return launch_op(h, n, layout, op, a, stream);  // nothing to pivot
    // the shared-memory kernels (run-time n) carry the tile-local search
    const int lanes = n <= 6 ? 2 : n <= 12 ? 4 : n <= 20 ? 8 : 16;
    const Variant *v = find_variant(n, layout, op, variant_id(lanes, 1));
    if (!v || v->kind != 1) return TL_ERR_UNSUPPORTED;
    return launch_variant(h, v, n, 0, a, stream);
}

}  // extern "C"
