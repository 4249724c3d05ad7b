// tl_ragged.cu -- tl_lupp_solve_batched: a batch whose systems have their
// own sizes n[s] (1..32) and their own places in memory.
//
// The systems are bucketed by n on the device (histogram, exclusive scan,
// block-aggregated scatter of the system indices into the handle's
// workspace), then ONE persistent launch solves every size class
// (tl_persist.cuh: work items laid out largest n first, taken by warps from
// a device counter).  The previous design -- one persistent grid-stride
// launch per n with the per-n kernels of tl_gesv_batched -- stays available
// as a mode (tl_ragged_set_mode), the comparator of the single launch.  No
// host synchronization: the bucket sizes stay on the device and every
// launch reads them there.
#include <climits>

#include "tinylu.h"
#include "tl_handle.h"
#include "tl_internal.h"
#include "tl_ir_smem.cuh"
#include "tl_persist.cuh"
#include "tl_smem.cuh"

namespace tl {
namespace {

constexpr int kSlots = 64;  // per-bin arrays, indices 0..TL_MAX_N+1 used

__global__ void k_bucket_hist(int64_t batch, const int32_t *__restrict__ n, int32_t *__restrict__ counts,
                              int32_t *__restrict__ info, int32_t *__restrict__ refine)
{
    __shared__ int32_t sh[kSlots];
    if (threadIdx.x < kSlots) sh[threadIdx.x] = 0;
    __syncthreads();
    const int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s < batch) {
        const int v = n[s];
        if (v >= 1 && v <= TL_MAX_N) {
            atomicAdd(&sh[v], 1);
        } else {
            info[s] = -2;
            if (refine) refine[s] = -1;
        }
    }
    __syncthreads();
    if (threadIdx.x >= 1 && threadIdx.x <= TL_MAX_N && sh[threadIdx.x] > 0)
        atomicAdd(&counts[threadIdx.x], sh[threadIdx.x]);
}

// offsets[v] = number of systems with size < v (v = 1..TL_MAX_N+1)
__global__ void k_bucket_scan(const int32_t *__restrict__ counts, int32_t *__restrict__ offsets,
                              int32_t *__restrict__ cursor)
{
    if (threadIdx.x != 0) return;
    int32_t acc = 0;
    offsets[0] = 0;
    for (int v = 1; v <= TL_MAX_N + 1; ++v) {
        offsets[v] = acc;
        cursor[v] = acc;
        if (v <= TL_MAX_N) acc += counts[v];
    }
}

// Mixed precision, sizes routed to binary64: their bucket entries become
// their fallback lists as they are (the same positions), their refinement
// counts -1.  `routed` has bit n set for every routed size.
__global__ void k_route_binary64(int64_t batch, const int32_t *__restrict__ n, const int32_t *__restrict__ offsets,
                                 const int32_t *__restrict__ bucket, int32_t *__restrict__ fb_count,
                                 int32_t *__restrict__ fb_list, int32_t *__restrict__ refine, unsigned long long routed)
{
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i0 <= TL_MAX_N && i0 >= 1 && ((routed >> i0) & 1ULL))
        fb_count[i0] = offsets[i0 + 1] - offsets[i0];
    const int64_t total = offsets[TL_MAX_N + 1];
    for (int64_t i = i0; i < total; i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t s = bucket[i];
        if ((routed >> n[s]) & 1ULL) {
            fb_list[i] = s;
            if (refine) refine[s] = -1;
        }
    }
}

__global__ void k_bucket_scatter(int64_t batch, const int32_t *__restrict__ n, int32_t *__restrict__ cursor,
                                 int32_t *__restrict__ bucket)
{
    __shared__ int32_t sh[kSlots];
    __shared__ int32_t base[kSlots];
    if (threadIdx.x < kSlots) sh[threadIdx.x] = 0;
    __syncthreads();
    const int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    int v = 0, rank = 0;
    if (s < batch) {
        v = n[s];
        if (v >= 1 && v <= TL_MAX_N) rank = atomicAdd(&sh[v], 1);
        else v = 0;
    }
    __syncthreads();
    if (threadIdx.x >= 1 && threadIdx.x <= TL_MAX_N && sh[threadIdx.x] > 0)
        base[threadIdx.x] = atomicAdd(&cursor[threadIdx.x], sh[threadIdx.x]);
    __syncthreads();
    if (v > 0) bucket[base[v] + rank] = static_cast<int32_t>(s);
}

}  // namespace

// Grow the handle's device workspace to at least `bytes`.  Never allocates
// while `stream` is being captured into a graph.
tl_status ensure_workspace(tl_handle *h, size_t bytes, cudaStream_t stream)
{
    if (h->ws_bytes >= bytes) return TL_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusNone;
    }
    if (cs != cudaStreamCaptureStatusNone) return TL_ERR_NO_MEMORY;
    if (h->ws) {
        cudaError_t e = cudaDeviceSynchronize();  // earlier calls may still read it
        if (e != cudaSuccess) return fail_cuda(h, e);
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    size_t want = bytes < (size_t(1) << 20) ? (size_t(1) << 20) : bytes;
    if (cudaMalloc(&h->ws, want) != cudaSuccess) {
        cudaGetLastError();
        h->ws = nullptr;
        return TL_ERR_NO_MEMORY;
    }
    h->ws_bytes = want;
    return TL_OK;
}

size_t ragged_ws_ints(int64_t batch, bool mixed)
{
    return kRaggedHeaderInts + static_cast<size_t>(batch) + (mixed ? kSlots + static_cast<size_t>(batch) : 0);
}

// Lanes per system of the single persistent launch for size n when the
// dispatch table names none: the choice tl_autotune_ragged makes on a
// GB300 within the launch's slice of kPersistSliceDoubles (one thread in
// registers up to kPersistRegMaxN, 2 lanes up to n = 10, 4 up to 14, 8 up
// to 22, 16 above).  A choice set through the dispatch table may need a
// larger slice: the launch then takes it, with fewer warps resident.
int default_persist_lanes(int n)
{
    if (n <= kPersistRegMaxN) return 1;
    if (n <= 10) return 2;
    if (n <= 14) return 4;
    if (n <= 22) return 8;
    return 16;
}

// Lanes per system of the single launch for n: the dispatch table's
// shared-memory ragged variant, else the default; widened until one warp's
// systems fit in `limit` bytes of shared memory.
// Sizes that refine by default under TL_PREC_FP32_IR: measured on GB300,
// the binary32 factorization with binary64 refinement beats the binary64
// solve from n = 21 on (1.1x at n = 21, 1.5-1.7x at n = 25..32) and loses
// below, where the FP64 pipe is not the only limit.
constexpr int kMixedMinN = 21;

bool mixed_refines(const tl_handle *h, int n)
{
    const int v = h->mixed_route[n];
    return v < 0 ? n >= kMixedMinN : v == 0;
}

int persist_lanes(const tl_handle *h, int n, int limit)
{
    int T = default_persist_lanes(n);
    const int id = h->choice[n][kPerSystem][kOpRagged].lanes;
    if (id >= 100) {
        const int L = id % 100;
        if ((L == 1 && n <= kPersistRegMaxN) || L == 2 || L == 4 || L == 8 || L == 16 || L == 32) T = L;
    }
    while (T < 32 && static_cast<size_t>(persist_need(n, T)) * sizeof(double) > static_cast<size_t>(limit)) T *= 2;
    return T;
}

namespace {

// Persistent grid for one per-n ragged kernel: enough warps for the whole
// batch (an upper bound on the bucket) but no more than stay resident.
unsigned ragged_grid(tl_handle *h, const Variant *v, int64_t batch, int blk)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, v->kernel, blk, 0) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    const int64_t need = (batch * v->lanes + blk - 1) / blk;
    const int64_t resident = static_cast<int64_t>(nb) * h->sm_count;
    return static_cast<unsigned>(need < resident ? need : resident);
}

// Persistent launch of a shared-memory ragged kernel for size nn with `per`
// bytes of shared memory per system.
tl_status launch_smem_ragged(tl_handle *h, const Variant *v, int nn, int64_t batch, RaggedArgs &r,
                             cudaStream_t stream, size_t per)
{
    int limit = 0;
    tl_status st = smem_opt_in(h, v->kernel, &limit);
    if (st != TL_OK) return st;
    for (int blk : {128, 64, 32}) {
        if (blk < v->lanes) continue;
        const size_t smem = static_cast<size_t>(blk / v->lanes) * per;
        if (smem > static_cast<size_t>(limit)) continue;
        const int nb = blocks_per_sm(h, v->kernel, blk, smem);
        if (nb < 1) continue;
        const int64_t sb = blk / v->lanes;
        const int64_t need = (batch + sb - 1) / sb;
        const int64_t resident = static_cast<int64_t>(nb) * h->sm_count;
        const unsigned g = static_cast<unsigned>(need < resident ? need : resident);
        int n_arg = nn;
        void *params[] = {&r, &n_arg};
        const cudaError_t e = cudaLaunchKernel(v->kernel, dim3(g), dim3(blk), params, smem, stream);
        if (e != cudaSuccess) return fail_cuda(h, e);
        return TL_OK;
    }
    return TL_ERR_UNSUPPORTED;
}

// The single persistent launch (plus its one-thread planning kernel) over
// the lists in r.
tl_status launch_persist(tl_handle *h, RaggedArgs &r, int32_t *plan, cudaStream_t stream)
{
    const void *kern = reinterpret_cast<const void *>(&k_ragged_persist);
    int limit = 0;
    const tl_status st = smem_opt_in(h, kern, &limit);
    if (st != TL_OK) return st;
    PersistPlan P{};
    int need = kPersistSliceDoubles;
    P.lanes[0] = 32;
    for (int n = 1; n <= TL_MAX_N; ++n) {
        const int T = persist_lanes(h, n, limit);
        P.lanes[n] = static_cast<unsigned char>(T);
        const int w = persist_need(n, T);
        need = w > need ? w : need;
    }
    P.warp_doubles = need;
    P.plan = plan;
    k_ragged_plan<<<1, 32, 0, stream>>>(r, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(h, e);
    const size_t smem = static_cast<size_t>(need) * sizeof(double);
    if (smem > static_cast<size_t>(limit)) return TL_ERR_UNSUPPORTED;
    const int nb = blocks_per_sm(h, kern, 32, smem);
    if (nb < 1) return TL_ERR_UNSUPPORTED;
    const unsigned grid = static_cast<unsigned>(nb * h->sm_count);
    void *params[] = {&r, &P};
    e = cudaLaunchKernel(kern, dim3(grid), dim3(32), params, smem, stream);
    if (e != cudaSuccess) return fail_cuda(h, e);
    return TL_OK;
}

// Binary64 ragged kernels for every n over the lists in r (one launch per
// size class, the per-size mode).
tl_status launch_per_size(tl_handle *h, RaggedArgs &r, cudaStream_t stream, int64_t batch)
{
    for (int nn = 1; nn <= TL_MAX_N; ++nn) {
        const Choice &c = h->choice[nn][kPerSystem][kOpRagged];
        const Variant *v = find_variant(nn, kPerSystem, kOpRagged, c.lanes ? c.lanes : default_ragged_id(nn));
        if (!v) return TL_ERR_UNSUPPORTED;
        if (v->kind >= 1) {
            const tl_status st = launch_smem_ragged(h, v, nn, batch, r, stream, smem_sys_bytes(nn, v->lanes));
            if (st != TL_OK) return st;
            continue;
        }
        const int blk = 128;
        const unsigned g = ragged_grid(h, v, batch, blk);
        void *params[] = {&r};
        cudaError_t e = cudaLaunchKernel(v->kernel, dim3(g), dim3(blk), params, 0, stream);
        if (e == cudaSuccess && v->fixup) e = cudaLaunchKernel(v->fixup, dim3(g), dim3(blk), params, 0, stream);
        if (e != cudaSuccess) return fail_cuda(h, e);
    }
    return TL_OK;
}

tl_status launch_binary64(tl_handle *h, int64_t batch, RaggedArgs &r, int32_t *plan, cudaStream_t stream)
{
    if (h->ragged_mode == TL_RAGGED_PER_SIZE) return launch_per_size(h, r, stream, batch);
    return launch_persist(h, r, plan, stream);
}

}  // namespace

// Bucket the batch by size and solve every size class.  `ws` holds the
// kRaggedHeaderInts int32 header (bin counts, offsets, cursors, the
// persistent launch's plan) followed by `batch` int32 indices, and with
// mixed precision kSlots fallback counters and `batch` fallback indices.
tl_status ragged_solve(tl_handle *h, int64_t batch, const int32_t *n, RaggedArgs r, int32_t *ws,
                       cudaStream_t stream, bool mixed)
{
    int32_t *counts = ws;
    int32_t *offsets = ws + kSlots;
    int32_t *cursor = ws + 2 * kSlots;
    int32_t *plan = ws + 3 * kSlots;
    int32_t *bucket = ws + kRaggedHeaderInts;
    cudaError_t e = cudaMemsetAsync(counts, 0, kSlots * sizeof(int32_t), stream);
    if (e == cudaSuccess && mixed) e = cudaMemsetAsync(bucket + batch, 0, kSlots * sizeof(int32_t), stream);
    if (e != cudaSuccess) return fail_cuda(h, e);
    const int block = 256;
    const unsigned grid = static_cast<unsigned>((batch + block - 1) / block);
    k_bucket_hist<<<grid, block, 0, stream>>>(batch, n, counts, r.info, mixed ? r.refine : nullptr);
    k_bucket_scan<<<1, 32, 0, stream>>>(counts, offsets, cursor);
    k_bucket_scatter<<<grid, block, 0, stream>>>(batch, n, cursor, bucket);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(h, e);
    r.bucket = bucket;
    r.offsets = offsets;
    r.counts = nullptr;
    if (!mixed) return launch_binary64(h, batch, r, plan, stream);

    // mixed precision: binary32 factor + binary64 refinement for the sizes
    // that refine, then the binary64 launch over the systems each size
    // handed back and over every system of the sizes routed to binary64
    r.fb_count = bucket + batch;
    r.fb_list = bucket + batch + kSlots;
    unsigned long long routed = 0;
    for (int nn = 1; nn <= TL_MAX_N; ++nn)
        if (!mixed_refines(h, nn)) routed |= 1ULL << nn;
    if (routed) {
        k_route_binary64<<<grid < 1024u ? grid : 1024u, block, 0, stream>>>(batch, n, offsets, bucket, r.fb_count,
                                                                          r.fb_list, r.refine, routed);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(h, e);
    }
    for (int nn = 1; nn <= TL_MAX_N; ++nn) {
        if ((routed >> nn) & 1ULL) continue;
        const Choice &c = h->choice[nn][kPerSystem][kOpRaggedIr];
        const Variant *v =
            find_variant(nn, kPerSystem, kOpRaggedIr, c.lanes ? c.lanes : default_ir_id(nn));
        if (!v) return TL_ERR_UNSUPPORTED;
        if (v->kind >= 1) {
            const tl_status st = launch_smem_ragged(h, v, nn, batch, r, stream, ir_smem_bytes_per_system(nn));
            if (st != TL_OK) return st;
            continue;
        }
        const int blk = 128;
        const unsigned g = ragged_grid(h, v, batch, blk);
        void *params[] = {&r};
        e = cudaLaunchKernel(v->kernel, dim3(g), dim3(blk), params, 0, stream);
        if (e != cudaSuccess) return fail_cuda(h, e);
    }
    RaggedArgs fb = r;
    fb.bucket = r.fb_list;
    fb.counts = r.fb_count;
    return launch_binary64(h, batch, fb, plan, stream);
}

}  // namespace tl

using namespace tl;

extern "C" tl_status tl_lupp_solve_batched(tl_handle *h, int64_t batch, const int32_t *n, const int64_t *a_off,
                                           const double *A, const int64_t *b_off, const double *b, double *x,
                                           const int64_t *piv_off, int32_t *ipiv, int32_t *info,
                                           tl_precision prec, int32_t *refine_steps, cudaStream_t stream)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (batch < 0) return fail_arg(h, 2);
    if (prec != TL_PREC_FP64 && prec != TL_PREC_FP32_IR) return fail_arg(h, 12);
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
    if (refine_steps && (reinterpret_cast<uintptr_t>(refine_steps) & 3)) return fail_arg(h, 13);
    if (batch > INT32_MAX) return TL_ERR_UNSUPPORTED;
    const bool mixed = prec == TL_PREC_FP32_IR;
    const size_t bytes = ragged_ws_ints(batch, mixed) * sizeof(int32_t);
    tl_status st = ensure_workspace(h, bytes, stream);
    if (st != TL_OK) return st;
    RaggedArgs r{nullptr, nullptr, a_off, A, b_off, b, x, piv_off, ipiv, info};
    r.refine = mixed ? refine_steps : nullptr;
    return ragged_solve(h, batch, n, r, static_cast<int32_t *>(h->ws), stream, mixed);
}

extern "C" tl_status tl_ragged_set_mode(tl_handle *h, int mode)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (mode != TL_RAGGED_PERSISTENT && mode != TL_RAGGED_PER_SIZE) return fail_arg(h, 2);
    h->ragged_mode = mode;
    return TL_OK;
}

extern "C" tl_status tl_ragged_dispatch_set(tl_handle *h, int n, int lanes, int mixed_route)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (n < 1 || n > TL_MAX_N) return fail_arg(h, 2);
    if (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32)
        return fail_arg(h, 3);
    if (lanes == 1 && n > kPersistRegMaxN) return fail_arg(h, 3);  // one thread in registers: n <= kPersistRegMaxN
    if (mixed_route < -1 || mixed_route > 1) return fail_arg(h, 4);
    h->choice[n][kPerSystem][kOpRagged] = Choice{lanes ? variant_id(lanes, 1) : 0, 0};
    h->mixed_route[n] = static_cast<signed char>(mixed_route);
    return TL_OK;
}

extern "C" tl_status tl_ragged_dispatch_get(tl_handle *h, int n, int *lanes, int *refines)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (n < 1 || n > TL_MAX_N) return fail_arg(h, 2);
    if (!lanes) return fail_arg(h, 3);
    int limit = h->max_smem_per_block;
    smem_opt_in(h, reinterpret_cast<const void *>(&k_ragged_persist), &limit);
    *lanes = persist_lanes(h, n, limit);
    if (refines) *refines = mixed_refines(h, n) ? 1 : 0;
    return TL_OK;
}
