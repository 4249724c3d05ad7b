// tl_kernels.cuh -- batched LUpp kernels (gesv / getrf / getrs) built on the
// device-callable solvers of tinylu_device.cuh, for the two storage layouts of
// the C ABI.  Instantiated per system size N in tl_inst_*.cu.
#pragma once
#include "tinylu_device.cuh"
#include "tl_internal.h"

namespace tl {

// Element offsets in the two layouts (include/tinylu.h).
template <int N, int LAYOUT>
struct Idx {
    __device__ __forceinline__ static int64_t a(int64_t s, int i, int j, int64_t ld)
    {
        return LAYOUT == kInterleaved ? static_cast<int64_t>(j * N + i) * ld + s
                                      : s * (N * N) + (j * N + i);
    }
    __device__ __forceinline__ static int64_t v(int64_t s, int i, int64_t ld)
    {
        return LAYOUT == kInterleaved ? static_cast<int64_t>(i) * ld + s : s * N + i;
    }
    // right-hand side r of a multi-RHS block
    __device__ __forceinline__ static int64_t rhs(int64_t s, int i, int r, int nrhs, int64_t ld)
    {
        return LAYOUT == kInterleaved ? static_cast<int64_t>(r * N + i) * ld + s
                                      : s * (static_cast<int64_t>(N) * nrhs) + (r * N + i);
    }
};

// info value the fast one-thread kernels leave for a system that must be
// redone by the exact general path; the fixup kernel that runs right after
// them on the same stream replaces it, so callers never see it.
constexpr int32_t kInfoSlow = -2147483000;

// Streaming loads/stores: every input is read once and every output written
// once, so keep them out of the way of the L2 lines that are reused.
__device__ __forceinline__ double ld_stream(const double *p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(double *p, double v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(int32_t *p, int32_t v) { __stcs(p, v); }

// Asynchronous 8-byte global -> shared copy (cp.async, no register staging):
// every copy a thread issues is in flight at once, where a load-then-store
// loop waits for each element's memory latency in turn.
__device__ __forceinline__ void cp_async8(double *smem_dst, const double *gsrc)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}

// Wait for every cp.async the calling thread issued (the caller then
// synchronizes the threads that read the data).
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;\n" ::: "memory");
}

// ceil(2^20 / c): floor(x / c) == (x * magic20(c)) >> 20 for 0 <= x < 1024
// and 1 <= c <= 32 (the error x (m - 2^20/c) / 2^20 stays below 1/c).
__host__ __device__ constexpr unsigned magic20(int c) { return (1048576u + static_cast<unsigned>(c) - 1u) / c; }
__device__ __forceinline__ int div20(int x, unsigned m) { return static_cast<int>((static_cast<unsigned>(x) * m) >> 20); }

// ---------------------------------------------------------------------------
// One thread per system.
// MODE: kGesv (A const, LU_out optional via KEEP), kGetrf (A in place).
// ---------------------------------------------------------------------------
// Exact general path for one system (zero, tiny, huge or non-finite pivots
// or inputs): loads the system again, factors it with lu_thread_factor and
// stores every output.
template <int N, int LAYOUT, int MODE, bool KEEP>
__device__ __forceinline__ void slow_factor_thread(SolveArgs args, int64_t s)
{
    using I = Idx<N, LAYOUT>;
    const double *A = (MODE == kGetrf) ? args.LU : args.A;
    double a[N][N];
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
        for (int i = 0; i < N; ++i) a[i][j] = A[I::a(s, i, j, args.ld)];
    double b[1][N];
    if (MODE == kGesv) {
#pragma unroll
        for (int i = 0; i < N; ++i) b[0][i] = args.b[I::v(s, i, args.ld)];
    }
    const bool bad = dev::any_nonfinite<N>(a);
    int piv[N];
    double rcp[N];
    bool tiny = false;
    int info = dev::lu_thread_factor<N, KEEP, (MODE == kGesv) ? 1 : 0>(a, b, piv, rcp, tiny);
    if (MODE == kGesv) dev::lu_thread_backsolve<N>(a, b[0], rcp, tiny);
    if (bad) info = -1;
    if (MODE == kGesv) {
#pragma unroll
        for (int i = 0; i < N; ++i) args.x[I::v(s, i, args.ld)] = info != 0 ? dev::nan_value() : b[0][i];
    }
    if (KEEP) {
        // info = -1: nothing is factored; the factors output keeps A.
        if (!bad) {
            dev::lu_thread_unnegate_L<N>(a);
#pragma unroll
            for (int j = 0; j < N; ++j)
#pragma unroll
                for (int i = 0; i < N; ++i) args.LU[I::a(s, i, j, args.ld)] = a[i][j];
        } else if (MODE == kGesv) {
            for (int j = 0; j < N; ++j)
                for (int i = 0; i < N; ++i) args.LU[I::a(s, i, j, args.ld)] = args.A[I::a(s, i, j, args.ld)];
        }
    }
#pragma unroll
    for (int k = 0; k < N; ++k) args.ipiv[I::v(s, k, args.ld)] = bad ? k + 1 : piv[k] + 1;
    args.info[s] = info;
}

template <int N, int LAYOUT, int MODE, bool KEEP>
__global__ void __launch_bounds__(128) k_factor_thread(SolveArgs args)
{
    const int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= args.batch) return;
    using I = Idx<N, LAYOUT>;
    const double *A = (MODE == kGetrf) ? args.LU : args.A;
    double a[N][N];
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
        for (int i = 0; i < N; ++i) a[i][j] = (MODE == kGetrf) ? A[I::a(s, i, j, args.ld)]
                                                                 : ld_stream(A + I::a(s, i, j, args.ld));
    double b[1][N];
    if (MODE == kGesv) {
#pragma unroll
        for (int i = 0; i < N; ++i) b[0][i] = ld_stream(args.b + I::v(s, i, args.ld));
    }
    // Branch-free fast path; a system with a zero, tiny, huge or non-finite
    // pivot (or input) is redone from its input by the exact general path.
    const bool bad = dev::any_nonfinite<N>(a);
    int piv[N];
    double rcp[N];
    const bool slow = dev::lu_thread_factor_fast<N, KEEP, (MODE == kGesv) ? 1 : 0>(a, b, piv, rcp) || bad;
    if (!slow) {
        if (MODE == kGesv) {
            dev::lu_thread_backsolve_fast<N>(a, b[0], rcp);
#pragma unroll
            for (int i = 0; i < N; ++i) st_stream(args.x + I::v(s, i, args.ld), b[0][i]);
        }
        if (KEEP) {
            dev::lu_thread_unnegate_L<N>(a);
#pragma unroll
            for (int j = 0; j < N; ++j)
#pragma unroll
                for (int i = 0; i < N; ++i) st_stream(args.LU + I::a(s, i, j, args.ld), a[i][j]);
        }
#pragma unroll
        for (int k = 0; k < N; ++k) st_stream(args.ipiv + I::v(s, k, args.ld), piv[k] + 1);
        st_stream(args.info + s, 0);
    } else {
        args.info[s] = kInfoSlow;  // redone by k_fixup_thread
    }
}

// Second pass after k_factor_thread: the systems it flagged go through the
// exact general path.  A separate kernel so that the general path's registers
// never weigh on the fast kernel.
template <int N, int LAYOUT, int MODE, bool KEEP>
__global__ void __launch_bounds__(128) k_fixup_thread(SolveArgs args)
{
    const int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= args.batch) return;
    if (args.info[s] != kInfoSlow) return;
    slow_factor_thread<N, LAYOUT, MODE, KEEP>(args, s);
}

// One thread per system: solve with given factors, nrhs right-hand sides.
template <int N, int LAYOUT>
__global__ void __launch_bounds__(128) k_getrs_thread(SolveArgs args)
{
    const int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= args.batch) return;
    using I = Idx<N, LAYOUT>;
    double a[N][N];
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
        for (int i = 0; i < N; ++i) a[i][j] = args.A[I::a(s, i, j, args.ld)];
    int piv[N];
#pragma unroll
    for (int k = 0; k < N; ++k) piv[k] = args.ipiv[I::v(s, k, args.ld)] - 1;
    double rcp[N];
    unsigned long long smallest = ~0ULL;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        rcp[i] = dev::rcp_rn(a[i][i]);
        unsigned long long m = dev::mag_bits(a[i][i]);
        smallest = m < smallest ? m : smallest;
    }
    const bool tiny = smallest < dev::kDblMinBits;
    for (int r = 0; r < args.nrhs; ++r) {
        double y[N];
#pragma unroll
        for (int i = 0; i < N; ++i) y[i] = args.x[I::rhs(s, i, r, args.nrhs, args.ld)];
        dev::lu_thread_forward<N>(a, piv, y);
        dev::lu_thread_backsolve<N>(a, y, rcp, tiny);
#pragma unroll
        for (int i = 0; i < N; ++i) args.x[I::rhs(s, i, r, args.nrhs, args.ld)] = y[i];
    }
}

// ---------------------------------------------------------------------------
// T lanes per system (row-cyclic).  Whole warps stay resident until the end
// because every lane takes part in the shuffles; lanes of groups past the
// batch end compute on zeros and store nothing.
// ---------------------------------------------------------------------------

// OR of a predicate over the T lanes of a group.
template <int T>
__device__ __forceinline__ bool group_any(bool v)
{
    int x = v ? 1 : 0;
#pragma unroll
    for (int off = T / 2; off >= 1; off >>= 1) x |= __shfl_xor_sync(0xffffffffu, x, off);
    return x != 0;
}

template <int N, int T, int LAYOUT, int MODE, bool KEEP>
__global__ void __launch_bounds__(128) k_factor_group(SolveArgs args)
{
    constexpr int K = dev::Group<N, T>::K;
    const int lane = threadIdx.x & 31;
    const int t = lane % T;
    const int lane0 = lane - t;
    const int64_t s = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / T;
    const int64_t warp_first = ((static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) & ~31LL) / T;
    if (warp_first >= args.batch) return;  // the whole warp is past the end
    const bool active = s < args.batch;
    using I = Idx<N, LAYOUT>;
    const double *A = (MODE == kGetrf) ? args.LU : args.A;

    double a[K][N];
    double b[K];
#pragma unroll
    for (int sl = 0; sl < K; ++sl) {
        const int i = t + sl * T;
        const bool ok = active && i < N;
#pragma unroll
        for (int j = 0; j < N; ++j) a[sl][j] = ok ? A[I::a(s, i, j, args.ld)] : 0.0;
        b[sl] = (MODE == kGesv && ok) ? ld_stream(args.b + I::v(s, i, args.ld)) : 0.0;
    }
    bool mybad = false;
#pragma unroll
    for (int sl = 0; sl < K; ++sl)
#pragma unroll
        for (int j = 0; j < N; ++j) mybad |= dev::is_nonfinite(a[sl][j]);
    const bool bad = group_any<T>(mybad);

    int pivk[K];
    double rcp[K];
    bool tiny = false;
    int info = dev::lu_group_factor<N, T, KEEP, (MODE == kGesv) ? 1 : 0>(a, b, pivk, rcp, t, lane0, tiny);
    if (MODE == kGesv) dev::lu_group_backsolve<N, T>(a, b, rcp, t, lane0, tiny);
    if (bad) info = -1;
    if (!active) return;

#pragma unroll
    for (int sl = 0; sl < K; ++sl) {
        const int i = t + sl * T;
        if (i < N) {
            if (MODE == kGesv) st_stream(args.x + I::v(s, i, args.ld), info != 0 ? dev::nan_value() : b[sl]);
            st_stream(args.ipiv + I::v(s, i, args.ld), bad ? i + 1 : pivk[sl] + 1);
            if (KEEP && !bad) {
#pragma unroll
                for (int j = 0; j < N; ++j)
                    st_stream(args.LU + I::a(s, i, j, args.ld), j < i ? dev::neg(a[sl][j]) : a[sl][j]);
            } else if (KEEP && MODE == kGesv) {
                for (int j = 0; j < N; ++j) args.LU[I::a(s, i, j, args.ld)] = args.A[I::a(s, i, j, args.ld)];
            }
        }
    }
    if (t == 0) st_stream(args.info + s, info);
}

// T lanes per system: solve with given factors, nrhs right-hand sides.
template <int N, int T, int LAYOUT>
__global__ void __launch_bounds__(128) k_getrs_group(SolveArgs args)
{
    constexpr int K = dev::Group<N, T>::K;
    const int lane = threadIdx.x & 31;
    const int t = lane % T;
    const int lane0 = lane - t;
    const int64_t s = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / T;
    const int64_t warp_first = ((static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) & ~31LL) / T;
    if (warp_first >= args.batch) return;
    const bool active = s < args.batch;
    using I = Idx<N, LAYOUT>;

    double a[K][N];
    int pivk[K];
    double rcp[K];
    bool tiny = false;
#pragma unroll
    for (int sl = 0; sl < K; ++sl) {
        const int i = t + sl * T;
        const bool ok = active && i < N;
#pragma unroll
        for (int j = 0; j < N; ++j) a[sl][j] = ok ? args.A[I::a(s, i, j, args.ld)] : 0.0;
        pivk[sl] = ok ? args.ipiv[I::v(s, i, args.ld)] - 1 : i;
    }
    // The diagonal entry of row i sits in column i, a run-time index here;
    // re-read it with a select chain so the register array stays static.
#pragma unroll
    for (int sl = 0; sl < K; ++sl) {
        const int i = t + sl * T;
        double d = 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j) d = dev::sel(j == i, a[sl][j], d);
        const bool ok = active && i < N;
        rcp[sl] = dev::rcp_rn(d);
        tiny = tiny || (ok && dev::mag_bits(d) < dev::kDblMinBits);
    }
    for (int r = 0; r < args.nrhs; ++r) {
        double y[K];
#pragma unroll
        for (int sl = 0; sl < K; ++sl) {
            const int i = t + sl * T;
            y[sl] = (active && i < N) ? args.x[I::rhs(s, i, r, args.nrhs, args.ld)] : 0.0;
        }
        // interchanges in order k = 0..N-1 (pivot of step k broadcast by its owner)
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int owner_k = k % T, slot_k = k / T;
            const int p = __shfl_sync(0xffffffffu, pivk[slot_k], lane0 + owner_k);
            const int owner_p = p % T, slot_p = p / T;
            double vp = 0.0;
#pragma unroll
            for (int sl = 0; sl < K; ++sl) vp = dev::sel(sl == slot_p, y[sl], vp);
            const double new_k = __shfl_sync(0xffffffffu, vp, lane0 + owner_p);
            const double new_p = __shfl_sync(0xffffffffu, y[slot_k], lane0 + owner_k);
#pragma unroll
            for (int sl = 0; sl < K; ++sl) y[sl] = dev::sel(t == owner_p && sl == slot_p, new_p, y[sl]);
            if (t == owner_k) y[slot_k] = new_k;
        }
        // forward: y_i -= l_ik y_k for i > k, k increasing
#pragma unroll
        for (int k = 0; k < N - 1; ++k) {
            const double nyk = dev::neg(__shfl_sync(0xffffffffu, y[k / T], lane0 + k % T));
#pragma unroll
            for (int sl = 0; sl < K; ++sl) {
                if (dev::Group<N, T>::slot_alive(sl, k)) {
                    const int i = t + sl * T;
                    if (i > k && i < N) y[sl] = __fma_rn(a[sl][k], nyk, y[sl]);
                }
            }
        }
        dev::lu_group_backsolve<N, T>(a, y, rcp, t, lane0, tiny);
        if (active) {
#pragma unroll
            for (int sl = 0; sl < K; ++sl) {
                const int i = t + sl * T;
                if (i < N) args.x[I::rhs(s, i, r, args.nrhs, args.ld)] = y[sl];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Ragged batches (tl_lupp_solve_batched): persistent grid-stride kernels over
// the bucket of systems of size N, each system at its own offsets.
// ---------------------------------------------------------------------------
// Number of systems of size N to process: the whole bucket, or the first
// counts[N] entries of the list when counts is set (never more than the
// bucket holds).
template <int N>
__device__ __forceinline__ int64_t ragged_count(const RaggedArgs &r, int64_t beg)
{
    const int64_t full = r.offsets[N + 1] - beg;
    if (!r.counts) return full;
    const int64_t c = r.counts[N];
    return c < 0 ? 0 : (c < full ? c : full);
}

// Exact general path of one ragged system (see slow_factor_thread).
template <int N>
__device__ __forceinline__ void slow_ragged_thread(RaggedArgs r, int64_t s)
{
    const double *A = r.A + r.a_off[s];
    const double *bv = r.b + r.b_off[s];
    double a[N][N];
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
        for (int i = 0; i < N; ++i) a[i][j] = A[j * N + i];
    double b[1][N];
#pragma unroll
    for (int i = 0; i < N; ++i) b[0][i] = bv[i];
    const bool bad = dev::any_nonfinite<N>(a);
    int piv[N];
    double rcp[N];
    bool tiny = false;
    int info = dev::lu_thread_factor<N, false, 1>(a, b, piv, rcp, tiny);
    dev::lu_thread_backsolve<N>(a, b[0], rcp, tiny);
    if (bad) info = -1;
    double *x = r.x + r.b_off[s];
    int32_t *ip = r.ipiv + r.piv_off[s];
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = info != 0 ? dev::nan_value() : b[0][i];
#pragma unroll
    for (int k = 0; k < N; ++k) ip[k] = bad ? k + 1 : piv[k] + 1;
    r.info[s] = info;
}

template <int N>
__global__ void __launch_bounds__(128) k_ragged_thread(RaggedArgs r)
{
    const int64_t beg = r.offsets[N];
    const int64_t count = ragged_count<N>(r, beg);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < count; q += stride) {
        const int64_t s = r.bucket[beg + q];
        const double *A = r.A + r.a_off[s];
        const double *bv = r.b + r.b_off[s];
        double a[N][N];
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
            for (int i = 0; i < N; ++i) a[i][j] = ld_stream(A + (j * N + i));
        double b[1][N];
#pragma unroll
        for (int i = 0; i < N; ++i) b[0][i] = ld_stream(bv + i);
        const bool bad = dev::any_nonfinite<N>(a);
        int piv[N];
        double rcp[N];
        const bool slow = dev::lu_thread_factor_fast<N, false, 1>(a, b, piv, rcp) || bad;
        if (!slow) {
            dev::lu_thread_backsolve_fast<N>(a, b[0], rcp);
            double *x = r.x + r.b_off[s];
            int32_t *ip = r.ipiv + r.piv_off[s];
#pragma unroll
            for (int i = 0; i < N; ++i) st_stream(x + i, b[0][i]);
#pragma unroll
            for (int k = 0; k < N; ++k) st_stream(ip + k, piv[k] + 1);
            st_stream(r.info + s, 0);
        } else {
            r.info[s] = kInfoSlow;  // redone by k_ragged_fixup
        }
    }
}

template <int N>
__global__ void __launch_bounds__(128) k_ragged_fixup(RaggedArgs r)
{
    const int64_t beg = r.offsets[N];
    const int64_t count = ragged_count<N>(r, beg);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < count; q += stride) {
        const int64_t s = r.bucket[beg + q];
        if (r.info[s] == kInfoSlow) slow_ragged_thread<N>(r, s);
    }
}

template <int N, int T>
__global__ void __launch_bounds__(128) k_ragged_group(RaggedArgs r)
{
    constexpr int K = dev::Group<N, T>::K;
    constexpr int G = 32 / T;  // systems per warp
    const int lane = threadIdx.x & 31;
    const int t = lane % T;
    const int lane0 = lane - t;
    const int64_t beg = r.offsets[N];
    const int64_t count = ragged_count<N>(r, beg);
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t q0 = warp * G; q0 < count; q0 += nwarps * G) {  // warp-uniform loop
        const int64_t q = q0 + lane / T;
        const bool active = q < count;
        const int64_t s = active ? r.bucket[beg + q] : 0;
        const double *A = r.A + (active ? r.a_off[s] : 0);
        double a[K][N];
        double b[K];
#pragma unroll
        for (int sl = 0; sl < K; ++sl) {
            const int i = t + sl * T;
            const bool ok = active && i < N;
#pragma unroll
            for (int j = 0; j < N; ++j) a[sl][j] = ok ? A[j * N + i] : 0.0;
            b[sl] = ok ? ld_stream(r.b + r.b_off[s] + i) : 0.0;
        }
        bool mybad = false;
#pragma unroll
        for (int sl = 0; sl < K; ++sl)
#pragma unroll
            for (int j = 0; j < N; ++j) mybad |= dev::is_nonfinite(a[sl][j]);
        const bool bad = group_any<T>(mybad);
        int pivk[K];
        double rcp[K];
        bool tiny = false;
        int info = dev::lu_group_factor<N, T, false, 1>(a, b, pivk, rcp, t, lane0, tiny);
        dev::lu_group_backsolve<N, T>(a, b, rcp, t, lane0, tiny);
        if (bad) info = -1;
        if (active) {
            double *x = r.x + r.b_off[s];
            int32_t *ip = r.ipiv + r.piv_off[s];
#pragma unroll
            for (int sl = 0; sl < K; ++sl) {
                const int i = t + sl * T;
                if (i < N) {
                    st_stream(x + i, info != 0 ? dev::nan_value() : b[sl]);
                    st_stream(ip + i, bad ? i + 1 : pivk[sl] + 1);
                }
            }
            if (t == 0) st_stream(r.info + s, info);
        }
    }
}

}  // namespace tl
