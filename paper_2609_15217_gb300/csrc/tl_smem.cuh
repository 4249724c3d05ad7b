// tl_smem.cuh -- LUpp with the matrices in shared memory, T lanes per
// system, run-time n (<= 32).
//
// Each system is an augmented n x (n+1) row-major block in shared memory
// (column n holds b, then y, then x).  Rows are never moved: a position ->
// row table `perm` implements the physical interchanges of Sec. 2.2 (swapping
// two table entries swaps two whole rows, L part included), and a pivot
// candidate at position i is the row perm[i], so the first-maximum rule sees
// exactly the row order of the sequential algorithm.
//
// Work split: at elimination step k the m = n-k-1 live rows and the n-k live
// columns (b included) form one flattened block of m(n-k) updates that the T
// lanes share element by element, so every FP64 instruction issued at a step
// is useful except for the last partial round of each lane: the lane
// efficiency stays near 1 at every step, unlike a row-cyclic split whose
// dead rows keep their slots issued.  All loops run at run time, so the code
// is small and stays in the instruction cache whatever n is.
//
// Arithmetic is the same as the register solvers of tl_device.cuh (negated
// multipliers a_ik * (-RN(1/a_kk)), one FMA per update in increasing k, the
// back substitution by RN(1/u_ii)); LU and pivots are bit-identical to the
// sequential elimination.
#pragma once
#include "tinylu.h"
#include "tl_kernels.cuh"

namespace tl {

// Shared-memory footprint of one system in doubles: the n x (n+1) block,
// 32 reciprocals, 32 + 32 ints (row table, pivots).  Padded so that the
// systems of one half-warp (16 lanes of 8-byte accesses) start T banks apart
// and their lanes do not collide on the same bank.
__host__ __device__ constexpr int smem_sys_doubles(int n, int T = 16)
{
    const int base = n * (n + 1) + 32 + 32;
    const int want = (T < 16) ? T : 0;
    return base + ((want - base % 16) % 16 + 16) % 16;
}
__host__ __device__ constexpr size_t smem_sys_bytes(int n, int T = 16)
{
    return static_cast<size_t>(smem_sys_doubles(n, T)) * 8;
}

template <int T>
__device__ __forceinline__ int group_any_int(int v)
{
#pragma unroll
    for (int off = T / 2; off >= 1; off >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// MODE: kGesv (A const, b -> x, LU optional by KEEP) or kGetrf (A in place).
template <int T, int LAYOUT, int MODE, bool KEEP>
__global__ void __launch_bounds__(128) k_smem_group(SolveArgs args, int n)
{
    extern __shared__ double smem[];
    const int SB = blockDim.x / T;                 // systems per block
    const int per = smem_sys_doubles(n, T);
    const int RS = n + 1;                          // row stride
    const int64_t s0 = static_cast<int64_t>(blockIdx.x) * SB;
    const double *Ag = (MODE == kGetrf) ? args.LU : args.A;
    const int nn = n * n;
    __shared__ int s_bad[128];

    // ---- load: thread (q = tid % SB, t' = tid / SB) copies elements
    //      e = t', t'+T, ... of system s0+q (coalesced over q) ----
    {
        const int q = threadIdx.x % SB;
        const int tp = threadIdx.x / SB;
        const int64_t s = s0 + q;
        double *M = smem + q * per;
        int bad = 0;
        if (s < args.batch) {
            if (LAYOUT == kInterleaved) {
                int i = tp % n, j = tp / n;
                for (int e = tp; e < nn; e += T) {
                    const double v = ld_stream(Ag + static_cast<int64_t>(e) * args.ld + s);
                    bad |= dev::is_nonfinite(v);
                    M[i * RS + j] = v;
                    i += T;
                    while (i >= n) { i -= n; ++j; }
                }
                if (MODE == kGesv)
                    for (int i2 = tp; i2 < n; i2 += T) M[i2 * RS + n] = ld_stream(args.b + static_cast<int64_t>(i2) * args.ld + s);
            } else {
                const double *src = Ag + s * nn;
                int i = tp % n, j = tp / n;
                for (int e = tp; e < nn; e += T) {
                    const double v = ld_stream(src + e);
                    bad |= dev::is_nonfinite(v);
                    M[i * RS + j] = v;
                    i += T;
                    while (i >= n) { i -= n; ++j; }
                }
                if (MODE == kGesv)
                    for (int i2 = tp; i2 < n; i2 += T) M[i2 * RS + n] = ld_stream(args.b + s * n + i2);
            }
        }
        s_bad[threadIdx.x] = bad;
    }
    __syncthreads();

    // ---- compute: lanes t = lane % T of a group own system q ----
    const int lane = threadIdx.x & 31;
    const int t = lane % T;
    const int q = threadIdx.x / T;
    const int64_t s = s0 + q;
    const bool active = s < args.batch;
    double *M = smem + q * per;
    double *rcp = M + n * RS;                              // 32 doubles
    int *perm = reinterpret_cast<int *>(rcp + 32);         // 32 ints
    int *piv = perm + 32;                                  // 32 ints
    // non-finite entries anywhere in this system (loaded by threads q + SB*t')
    int badv = 0;
    for (int tp = t; tp < T; tp += T) badv |= s_bad[q + SB * tp];
    const bool bad = group_any_int<T>(badv) != 0;
    for (int i = t; i < n; i += T) perm[i] = i;
    __syncwarp();

    int info = 0;
    bool tiny = false;
    const int wcols = n + (MODE == kGesv ? 1 : 0);         // columns incl. b
    for (int k = 0; k < n; ++k) {
        // a2: first maximum of |a_ik| over positions k..hi-1: the whole
        // column, or with tile-local pivoting the diagonal tile first and
        // the positions below it only when the tile's best magnitude is
        // under the threshold (the first maximum over k..n-1 then)
        int hi = n;
        if (args.tile > 0 && args.tile < n) hi = min(n, (k / args.tile + 1) * args.tile);
        double cv = 0.0;
        int cpos = n;
        for (int i = k + t; i < hi; i += T) {
            const double v = M[perm[i] * RS + k];
            if (cpos == n || dev::mag_bits(v) > dev::mag_bits(cv)) { cv = v; cpos = i; }
        }
        dev::group_argmax<T>(cv, cpos);
        if (hi < n) {
            const bool below = dev::mag_bits(cv) < dev::mag_bits(args.threshold);
            if (below) {
                for (int i = hi + ((t - hi) % T + T) % T; i < n; i += T) {
                    const double v = M[perm[i] * RS + k];
                    if (dev::mag_bits(v) > dev::mag_bits(cv)) { cv = v; cpos = i; }
                }
            }
            if (__any_sync(0xffffffffu, below)) dev::group_argmax<T>(cv, cpos);
        }
        const int p = cpos;
        const bool zero = dev::mag_bits(cv) == 0ULL;
        if (zero && info == 0) info = k + 1;
        if (t == 0) piv[k] = p;
        __syncwarp();
        // a3: interchange positions k and p (whole rows, L part included)
        if (t == 0 && p != k) {
            const int tmp = perm[k];
            perm[k] = perm[p];
            perm[p] = tmp;
        }
        __syncwarp();
        const int rk = perm[k];
        // a4: reciprocal and negated multipliers
        const bool small = !zero && dev::mag_bits(cv) < dev::kDblMinBits;
        const double r = dev::rcp_rn(cv);
        if (t == 0) rcp[k] = r;
        tiny = tiny || small;
        const double nr = dev::neg(r);
        if (!__any_sync(0xffffffffu, small)) {
            for (int i = k + 1 + t; i < n; i += T) {
                double *a = &M[perm[i] * RS + k];
                *a = zero ? dev::neg(*a) : __dmul_rn(*a, nr);
            }
        } else {
            const double ncv = dev::neg(cv);
            for (int i = k + 1 + t; i < n; i += T) {
                double *a = &M[perm[i] * RS + k];
                *a = zero ? dev::neg(*a) : (small ? __ddiv_rn(*a, ncv) : __dmul_rn(*a, nr));
            }
        }
        __syncwarp();
        // a5 (+ forward part of a6 through column n): a_ij += (-l_ik) u_kj
        if (!zero) {
            const int m = n - k - 1;
            const int w = wcols - k - 1;
            const int total = m * w;
            if (total > 0) {
                // each lane walks elements e = t, t+T, ... of the flattened
                // m x w block, four at a time: all loads of a group are issued
                // before its FMAs (the four elements are distinct, so the
                // reordering is exact; the compiler cannot prove it alone)
                int ii = t / w, jj = t % w;
                const double *urow = M + rk * RS + k + 1;
                for (int e = t; e < total; e += 4 * T) {
                    int off[4];
                    double l[4], u[4], a[4];
#pragma unroll
                    for (int q2 = 0; q2 < 4; ++q2) {
                        const bool ok = e + q2 * T < total;
                        const int row = ok ? perm[k + 1 + ii] : rk;
                        off[q2] = ok ? row * RS + k + 1 + jj : -1;
                        l[q2] = ok ? M[row * RS + k] : 0.0;
                        u[q2] = ok ? urow[jj] : 0.0;
                        jj += T;
                        while (jj >= w) { jj -= w; ++ii; }
                    }
#pragma unroll
                    for (int q2 = 0; q2 < 4; ++q2) a[q2] = off[q2] >= 0 ? M[off[q2]] : 0.0;
#pragma unroll
                    for (int q2 = 0; q2 < 4; ++q2)
                        if (off[q2] >= 0) M[off[q2]] = __fma_rn(l[q2], u[q2], a[q2]);
                }
            }
        }
        __syncwarp();
    }

    // a6 (back part): x_i = y_i * RN(1/u_ii), then y_r -= u_ri x_i for r < i
    if (MODE == kGesv) {
        const bool any_tiny = __any_sync(0xffffffffu, tiny);
        for (int i = n - 1; i >= 0; --i) {
            const int ri = perm[i];
            if (t == 0) {
                const double y = M[ri * RS + n];
                double xi;
                if (!any_tiny) xi = __dmul_rn(y, rcp[i]);
                else xi = tiny ? __ddiv_rn(y, M[ri * RS + i]) : __dmul_rn(y, rcp[i]);
                M[ri * RS + n] = xi;
            }
            __syncwarp();
            const double nxi = dev::neg(M[ri * RS + n]);
            for (int r2 = t; r2 < i; r2 += T) {
                const int rr = perm[r2];
                M[rr * RS + n] = __fma_rn(M[rr * RS + i], nxi, M[rr * RS + n]);
            }
            __syncwarp();
        }
    }
    if (bad) info = -1;

    // a7: store
    if (active) {
        for (int i = t; i < n; i += T) {
            const int64_t vi = (LAYOUT == kInterleaved) ? static_cast<int64_t>(i) * args.ld + s : s * n + i;
            if (MODE == kGesv) st_stream(args.x + vi, info != 0 ? dev::nan_value() : M[perm[i] * RS + n]);
            st_stream(args.ipiv + vi, bad ? i + 1 : piv[i] + 1);
        }
        if (t == 0) st_stream(args.info + s, info);
        if (KEEP) {
            // element e = j*n + i of the factors: row at position i, column j
            for (int e = t; e < nn; e += T) {
                const int i = e % n, j = e / n;
                const int64_t ai = (LAYOUT == kInterleaved) ? static_cast<int64_t>(e) * args.ld + s : s * nn + e;
                if (!bad) {
                    const double v = M[perm[i] * RS + j];
                    st_stream(args.LU + ai, j < i ? dev::neg(v) : v);
                } else if (MODE == kGesv) {
                    args.LU[ai] = args.A[ai];
                }
            }
        }
    }
}

}  // namespace tl
