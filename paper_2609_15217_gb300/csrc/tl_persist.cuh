// tl_persist.cuh -- one persistent launch over a ragged batch (systems of
// mixed n, each at its own offsets), the batched form of Sec. 2.3 with the
// work of every size class in a single kernel.
//
// The bucketing pass (tl_ragged.cu) lists the systems of each size n.
// k_ragged_plan turns the per-size counts into work items -- one item is
// the 32 / T(n) systems a warp solves at once with T(n) lanes per system --
// laid out largest n first, so the longest items start first and the short
// ones fill the tail (longest-processing-time order).  k_ragged_persist is
// launched with as many one-warp blocks as stay resident; each warp takes
// the next item from a counter in device memory (one item ahead, so the
// counter's latency overlaps the current item), loads its systems
// (coalesced, each system is contiguous in memory) into its own slice of
// shared memory, solves them with the element-walk solver (smem_lupp2) and
// stores x, the pivots and info.  Size classes without systems have no
// items; nothing waits on anything (the counter only grows).
#pragma once
#include "tl_persist_sizes.h"
#include "tl_smem.cuh"

namespace tl {

// Layout of the plan block in the ragged workspace (int32 slots): item
// starts of the 32 size classes in order n = 32, 31, ..., 1 and the total,
// then the work counter.
constexpr int kPlanTotal = TL_MAX_N;
constexpr int kPlanCounter = 48;

struct PersistPlan {
    unsigned char lanes[TL_MAX_N + 1];  // lanes per system for each n: 1 (n <= 7), 2, 4, 8, 16 or 32
    int warp_doubles;                   // shared-memory slice of one warp
    int32_t *plan;                      // the plan block (device)
};

// Systems of size n listed for this pass: the bucket, or the first
// counts[n] entries of the list when counts is set.
__device__ __forceinline__ int64_t class_count(const RaggedArgs &r, int n)
{
    const int64_t full = r.offsets[n + 1] - r.offsets[n];
    if (!r.counts) return full;
    const int64_t c = r.counts[n];
    return c < 0 ? 0 : (c < full ? c : full);
}

// One thread: item starts in largest-n-first order and a zero counter.
__global__ void k_ragged_plan(RaggedArgs r, const __grid_constant__ PersistPlan P)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int32_t acc = 0;
    for (int c = 0; c < TL_MAX_N; ++c) {
        const int n = TL_MAX_N - c;
        P.plan[c] = acc;
        const int G = 32 / P.lanes[n];
        acc += static_cast<int32_t>((class_count(r, n) + G - 1) / G);
    }
    P.plan[kPlanTotal] = acc;
    P.plan[kPlanCounter] = 0;
}

// One work item: systems first .. first + G - 1 of size class n.
template <int T>
__device__ __forceinline__ void persist_item(const RaggedArgs &r, int n, int64_t beg, int64_t count, int64_t first,
                                             double *W, int lane)
{
    constexpr int G = 32 / T;
    const int q = lane / T, t = lane % T;
    const int per = smem_sys_doubles(n, T);
    const int RS = smem_row_stride(n);
    const int nn = n * n;
    const unsigned m20 = magic20(n);
    // lane g < G fetches the index and offsets of the item's system g (one
    // latency for the whole item instead of one chain per system)
    int64_t my_s = 0, my_a = 0, my_b = 0, my_p = 0;
    if (lane < G && first + lane < count) {
        my_s = r.bucket[beg + first + lane];
        my_a = r.a_off[my_s];
        my_b = r.b_off[my_s];
        my_p = r.piv_off[my_s];
    }
    // load: the warp copies one system at a time, 32 consecutive entries per
    // access (cp.async, all in flight together); A is column-major, the
    // shared block row-major with b as column n
#pragma unroll 1
    for (int g = 0; g < G; ++g) {
        if (first + g >= count) break;  // warp-uniform
        const double *A = r.A + __shfl_sync(0xffffffffu, my_a, g);
        const double *bv = r.b + __shfl_sync(0xffffffffu, my_b, g);
        double *M = W + g * per;
        for (int e = lane; e < nn; e += 32) {
            const int j = div20(e, m20);
            cp_async8(&TL_SM(M, (e - j * n) * RS + j, per), A + e);
        }
        if (lane < n) cp_async8(&TL_SM(M, lane * RS + n, per), bv + lane);
    }
    cp_async_wait_all();
    __syncwarp();
    double *M = W + q * per;
    // a non-finite entry anywhere in the group's system
    int badv = 0;
    if (first + q < count) {
        for (int e = t; e < nn; e += T) {
            const int j = div20(e, m20);
            badv |= dev::is_nonfinite(M[(e - j * n) * RS + j]) ? 1 : 0;
        }
    }
    const bool bad = group_any_int<T>(badv) != 0;
    int info = smem_lupp2<T, true, false>(M, n, RS, t, 0, 0.0);
    if (bad) info = -1;
    const int64_t s = __shfl_sync(0xffffffffu, my_s, q);
    const int64_t xo = __shfl_sync(0xffffffffu, my_b, q);
    const int64_t po = __shfl_sync(0xffffffffu, my_p, q);
    if (first + q < count) {
        const int *piv = reinterpret_cast<const int *>(M + smem_piv_offset(n));
        double *x = r.x + xo;
        int32_t *ip = r.ipiv + po;
        for (int i = t; i < n; i += T) {
            st_stream(x + i, info != 0 ? dev::nan_value() : M[i * RS + n]);
            st_stream(ip + i, bad ? i + 1 : piv[i] + 1);
        }
        if (t == 0) st_stream(r.info + s, info);
    }
    __syncwarp();  // the next item's loads overwrite the slice
}

// One work item of the one-thread register path (n <= 7): the 32 systems
// are copied into the warp's slice (coalesced, one system after another),
// then lane g loads system g into its registers and solves it with the
// branch-free fast path of the one-thread kernels; a system that meets a
// zero, tiny, huge or non-finite pivot takes the exact general path.
template <int N>
__device__ __forceinline__ void persist_item_reg(const RaggedArgs &r, int64_t beg, int64_t count, int64_t first,
                                                 double *W, int lane)
{
    constexpr int NN = N * N;
    constexpr int STRIDE = persist_reg_stride(N);
    const bool act = first + lane < count;
    int64_t s = 0, ao = 0, bo = 0, po = 0;
    if (act) {
        s = r.bucket[beg + first + lane];
        ao = r.a_off[s];
        bo = r.b_off[s];
        po = r.piv_off[s];
    }
#pragma unroll 1
    for (int g = 0; g < 32; ++g) {
        if (first + g >= count) break;  // warp-uniform
        const double *A = r.A + __shfl_sync(0xffffffffu, ao, g);
        const double *bv = r.b + __shfl_sync(0xffffffffu, bo, g);
        double *M = W + g * STRIDE;
        for (int e = lane; e < NN; e += 32) cp_async8(&TL_SM(M, e, STRIDE), A + e);
        if (lane < N) cp_async8(&TL_SM(M, NN + lane, STRIDE), bv + lane);
    }
    cp_async_wait_all();
    __syncwarp();
    if (act) {
        const double *M = W + lane * STRIDE;
        double a[N][N];
        double b[1][N];
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
            for (int i = 0; i < N; ++i) a[i][j] = TL_SM(M, j * N + i, STRIDE);
#pragma unroll
        for (int i = 0; i < N; ++i) b[0][i] = TL_SM(M, NN + i, STRIDE);
        const bool bad = dev::any_nonfinite<N>(a);
        int piv[N];
        double rcp[N];
        const bool slow = dev::lu_thread_factor_fast<N, false, 1>(a, b, piv, rcp) || bad;
        if (!slow) {
            dev::lu_thread_backsolve_fast<N>(a, b[0], rcp);
#pragma unroll
            for (int i = 0; i < N; ++i) st_stream(r.x + bo + i, b[0][i]);
#pragma unroll
            for (int k = 0; k < N; ++k) st_stream(r.ipiv + po + k, piv[k] + 1);
            st_stream(r.info + s, 0);
        } else {
            slow_ragged_thread<N>(r, s);
        }
    }
    __syncwarp();  // the next item's copies overwrite the slice
}

// One warp per block; dynamic shared memory = P.warp_doubles doubles.
// kPersistWarps blocks per SM (the slice's occupancy) set the register
// limit (170 per thread for 12).
__global__ void __launch_bounds__(32, kPersistWarps) k_ragged_persist(RaggedArgs r, const __grid_constant__ PersistPlan P)
{
    extern __shared__ double smem[];
    __shared__ int32_t s_start[TL_MAX_N + 1];
    __shared__ unsigned char s_lanes[TL_MAX_N + 1];
    const int lane = static_cast<int>(threadIdx.x);
    for (int c = lane; c <= TL_MAX_N; c += 32) {
        s_start[c] = P.plan[c];
        s_lanes[c] = P.lanes[c];
    }
    __syncwarp();
    const int32_t total = s_start[kPlanTotal];
    int c = 0;
    int32_t item = 0;
    if (lane == 0) item = atomicAdd(P.plan + kPlanCounter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    while (item < total) {
        // take the next item now: the counter's latency overlaps this item
        int32_t next = 0;
        if (lane == 0) next = atomicAdd(P.plan + kPlanCounter, 1);
        while (item >= s_start[c + 1]) ++c;  // items only grow: c never goes back
        const int n = TL_MAX_N - c;
        const int T = s_lanes[n];
        const int64_t beg = r.offsets[n];
        const int64_t count = class_count(r, n);
        const int64_t first = static_cast<int64_t>(item - s_start[c]) * (32 / T);
        switch (T) {
        case 1:
            switch (n) {
            case 1: persist_item_reg<1>(r, beg, count, first, smem, lane); break;
            case 2: persist_item_reg<2>(r, beg, count, first, smem, lane); break;
            case 3: persist_item_reg<3>(r, beg, count, first, smem, lane); break;
            case 4: persist_item_reg<4>(r, beg, count, first, smem, lane); break;
            case 5: persist_item_reg<5>(r, beg, count, first, smem, lane); break;
            case 6: persist_item_reg<6>(r, beg, count, first, smem, lane); break;
            default: persist_item_reg<kPersistRegMaxN>(r, beg, count, first, smem, lane); break;
            }
            break;
        case 2: persist_item<2>(r, n, beg, count, first, smem, lane); break;
        case 4: persist_item<4>(r, n, beg, count, first, smem, lane); break;
        case 8: persist_item<8>(r, n, beg, count, first, smem, lane); break;
        case 16: persist_item<16>(r, n, beg, count, first, smem, lane); break;
        default: persist_item<32>(r, n, beg, count, first, smem, lane); break;
        }
        item = __shfl_sync(0xffffffffu, next, 0);
    }
}

}  // namespace tl
