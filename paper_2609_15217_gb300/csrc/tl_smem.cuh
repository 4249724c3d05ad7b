// tl_smem.cuh -- LUpp with the matrices in shared memory, T lanes per
// system, run-time n (<= 32).
//
// Each system is an augmented n x (n+1) row-major block in shared memory
// (column n holds b, then y, then x), rows RS doubles apart (RS odd), then
// n reciprocals and n pivot rows.  The interchanges of Sec. 2.2 swap whole
// rows in place, the T lanes sharing the columns.
//
// Two eliminations share this layout:
//   * smem_lupp2 (the fast path): the trailing block is walked element by
//     element, lane t taking every T-th element row-major, and the updates
//     of two elimination steps are applied in one pass; see its comment.
//   * smem_lupp: one step per pass on a TR x TC tile of lanes (lane (tr, tc)
//     keeps its columns of the pivot row in registers and walks its rows)
//     or an element walk; kept for the lane-tile variants.
// The kernels: k_smem_group (fixed-size batches, both layouts; loads into
// shared memory by cp.async for 2..8 lanes and by register-staged streaming
// loads for 16 and 32 lanes, the faster choice measured for each) and
// k_smem_ragged (one size of a ragged batch, the per-size mode).
//
// Arithmetic is the same as the register solvers of tinylu_device.cuh (negated
// multipliers a_ik * (-RN(1/a_kk)), one FMA per update in increasing k, the
// back substitution by RN(1/u_ii)); LU and pivots are bit-identical to the
// sequential elimination.
#pragma once
#include "tinylu.h"
#include "tl_bounds.cuh"
#include "tl_kernels.cuh"

// Unroll factor of the row loop of the lane-tile trailing update (2
// measured 5-10% slower than 1).
#ifndef TL_SMEM_ROW_UNROLL
#define TL_SMEM_ROW_UNROLL 1
#endif

namespace tl {

constexpr int kSmemRowUnroll = TL_SMEM_ROW_UNROLL;

// Row stride of a system's n x (n+1) block: the smallest odd number of
// doubles >= n+1, so that a column walked by consecutive lanes hits distinct
// banks and the block stays small (shared memory bounds the warps resident
// per SM).
__host__ __device__ constexpr int smem_row_stride(int n) { return (n + 1) | 1; }

// Offsets (in doubles) of the n reciprocals RN(1/u_kk) and of the n pivot
// rows (int32, two per double) behind a system's n x RS block.
__host__ __device__ constexpr int smem_rcp_offset(int n) { return n * smem_row_stride(n); }
__host__ __device__ constexpr int smem_piv_offset(int n) { return n * smem_row_stride(n) + n; }

// Shared-memory footprint of one system in doubles: the n x RS block, n
// reciprocals, n pivots.  Padded so that consecutive systems start T slots
// apart modulo 16 (the systems of one half-warp then do not collide on a
// bank).
__host__ __device__ constexpr int smem_sys_doubles(int n, int T = 16)
{
    const int base = smem_piv_offset(n) + (n + 1) / 2;
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

// Elimination of one system held by the T lanes of a group: the augmented
// n x (n+1) block M (row stride RS; column n = b when SOLVE), followed by
// n reciprocals and n pivot rows.  LUpp with the arithmetic of the
// register solvers (negated multipliers a_ik * (-RN(1/a_kk)), one FMA per
// update in increasing k, b carried as column n, back substitution by
// RN(1/u_ii)); on return M holds L (negated, below the diagonal) and U, and
// column n holds x when SOLVE.  Returns info.  Every lane of the warp must
// call it together (shuffles and votes inside).
//
// Trailing updates either walk the trailing block element by element (WALK:
// lane t takes every T-th element, row-major) or use a TR x TC tile of
// lanes: lane (tr, tc) updates rows k+1+tr, k+1+tr+TR, ... and columns
// k+1+tc, k+1+tc+TC, ..., keeping its columns of the pivot row in registers.
template <int T, bool SOLVE, bool WALK = (T >= 16)>
__device__ __forceinline__ int smem_lupp(double *M, int n, int RS, int t, int tile, double threshold)
{
    constexpr int MODE = SOLVE ? kGesv : kGetrf;
    constexpr int TC = WALK ? 1 : (T >= 4) ? 4 : T;  // lane tile (when not walking elements)
    constexpr int TR = T / TC;
    constexpr int MAXC = TL_MAX_N / TC;  // whole column chunks per lane (at most 32 live columns)
    static_assert(WALK || MAXC <= 16, "the chunk switch below covers 16 chunks");
    static_assert(T >= 1 && T <= 32 && (32 % T) == 0, "T must divide 32");
    const int tr = t / TC, tc = t % TC;
    double *rcp = M + n * RS;                              // n doubles
    int *piv = reinterpret_cast<int *>(rcp + n);           // n ints
    int info = 0;
    bool tiny = false;
    const int wcols = n + (MODE == kGesv ? 1 : 0);         // columns incl. b
    for (int k = 0; k < n; ++k) {
        // a2: first maximum of |a_ik| over rows k..hi-1: the whole column,
        // or with tile-local pivoting the diagonal tile first and the rows
        // below it only when the tile's best magnitude is under the
        // threshold (the first maximum over k..n-1 then)
        int hi = n;
        if (tile > 0 && tile < n) hi = min(n, (k / tile + 1) * tile);
        double cv = 0.0;
        int cpos = n;
        for (int i = k + t; i < hi; i += T) {
            const double v = M[i * RS + k];
            if (cpos == n || dev::mag_bits(v) > dev::mag_bits(cv)) { cv = v; cpos = i; }
        }
        dev::group_argmax<T>(cv, cpos);
        if (hi < n) {
            const bool below = dev::mag_bits(cv) < dev::mag_bits(threshold);
            if (below) {
                for (int i = hi + ((t - hi) % T + T) % T; i < n; i += T) {
                    const double v = M[i * RS + k];
                    if (dev::mag_bits(v) > dev::mag_bits(cv)) { cv = v; cpos = i; }
                }
            }
            if (__any_sync(0xffffffffu, below)) dev::group_argmax<T>(cv, cpos);
        }
        const int p = cpos;
        const bool zero = dev::mag_bits(cv) == 0ULL;
        if (zero && info == 0) info = k + 1;
        if (t == 0) piv[k] = p;
        // a3: physical interchange of rows k and p (L part and b included)
        if (p != k) {
            for (int j = t; j < wcols; j += T) {
                const double tmp = M[k * RS + j];
                M[k * RS + j] = M[p * RS + j];
                M[p * RS + j] = tmp;
            }
        }
        __syncwarp();
        // a4: reciprocal and negated multipliers
        const bool small = !zero && dev::mag_bits(cv) < dev::kDblMinBits;
        const double r = dev::rcp_rn(cv);
        if (t == 0) rcp[k] = r;
        tiny = tiny || small;
        const double nr = dev::neg(r);
        if (!__any_sync(0xffffffffu, small)) {
            for (int i = k + 1 + t; i < n; i += T) {
                double *a = &M[i * RS + k];
                *a = zero ? dev::neg(*a) : __dmul_rn(*a, nr);
            }
        } else {
            const double ncv = dev::neg(cv);
            for (int i = k + 1 + t; i < n; i += T) {
                double *a = &M[i * RS + k];
                *a = zero ? dev::neg(*a) : (small ? __ddiv_rn(*a, ncv) : __dmul_rn(*a, nr));
            }
        }
        __syncwarp();
        // a5 (+ forward part of a6 through column n): a_ij += (-l_ik) u_kj.
        if (!zero && WALK) {
            // element walk: the R x C trailing block (R = n-k-1
            // rows, C live columns) is walked row-major, lane t taking the
            // elements t, t+T, t+2T, ...; every lane issues ceil(R C / T)
            // FMAs, the least any split can (a TR x TC lane tile issues
            // ceil(R/TR) ceil(C/TC)).  l_i and u_j come from shared memory.
            const int ncols = wcols - (k + 1);
            const int nrows = n - (k + 1);
            const int nel = nrows * ncols;
            if (nel > 0) {
                const int q = T / ncols, rq = T % ncols;  // (row, column) advance per stride
                int ei = t / ncols, ej = t % ncols;        // element t: row k+1+ei, column k+1+ej
                const double *urow = M + k * RS + k + 1;
                for (int e = t; e < nel; e += T) {
                    double *Mi = M + (k + 1 + ei) * RS;
                    const double l = Mi[k];
                    Mi[k + 1 + ej] = __fma_rn(l, urow[ej], Mi[k + 1 + ej]);
                    ej += rq;
                    ei += q;
                    if (ej >= ncols) {
                        ej -= ncols;
                        ++ei;
                    }
                }
            }
        } else if (!zero) {
            // fewer lanes: lane (tr, tc) owns columns k+1+tc + c*TC: nfull
            // whole chunks (the same count on every lane of the warp) and
            // possibly one tail column; the chunks are a straight-line
            // fall-through block entered once per row, with immediate
            // offsets from the row pointer
            const int ncols = wcols - (k + 1);
            const int nfull = ncols / TC;
            const bool has_tail = tc < ncols - nfull * TC;
            const double *urow = M + k * RS + k + 1 + tc;
            double u[MAXC];
#pragma unroll
            for (int c = 0; c < MAXC; ++c) u[c] = c < nfull ? urow[c * TC] : 0.0;
            const double ut = has_tail ? urow[nfull * TC] : 0.0;
#pragma unroll kSmemRowUnroll
            for (int i = k + 1 + tr; i < n; i += TR) {
                double *Mi = M + i * RS;
                const double l = Mi[k];
                double *Mr = Mi + k + 1 + tc;
                switch (nfull) {
#define TL_SMEM_CHUNK(c)                                                                \
    case (c) + 1:                                                                       \
        if ((c) < MAXC) Mr[(c) * TC] = __fma_rn(l, u[(c) < MAXC ? (c) : 0], Mr[(c) * TC]); \
        [[fallthrough]];
                    TL_SMEM_CHUNK(15)
                    TL_SMEM_CHUNK(14)
                    TL_SMEM_CHUNK(13)
                    TL_SMEM_CHUNK(12)
                    TL_SMEM_CHUNK(11)
                    TL_SMEM_CHUNK(10)
                    TL_SMEM_CHUNK(9)
                    TL_SMEM_CHUNK(8)
                    TL_SMEM_CHUNK(7)
                    TL_SMEM_CHUNK(6)
                    TL_SMEM_CHUNK(5)
                    TL_SMEM_CHUNK(4)
                    TL_SMEM_CHUNK(3)
                    TL_SMEM_CHUNK(2)
                    TL_SMEM_CHUNK(1)
                    TL_SMEM_CHUNK(0)
#undef TL_SMEM_CHUNK
                default: break;
                }
                if (has_tail) Mr[nfull * TC] = __fma_rn(l, ut, Mr[nfull * TC]);
            }
        }
        __syncwarp();
    }

    // a6 (back part): x_i = y_i * RN(1/u_ii), then y_r -= u_ri x_i for r < i
    if (MODE == kGesv) {
        const bool any_tiny = __any_sync(0xffffffffu, tiny);
        for (int i = n - 1; i >= 0; --i) {
            if (t == 0) {
                const double y = M[i * RS + n];
                double xi;
                if (!any_tiny) xi = __dmul_rn(y, rcp[i]);
                else xi = tiny ? __ddiv_rn(y, M[i * RS + i]) : __dmul_rn(y, rcp[i]);
                M[i * RS + n] = xi;
            }
            __syncwarp();
            const double nxi = dev::neg(M[i * RS + n]);
            for (int r2 = t; r2 < i; r2 += T) M[r2 * RS + n] = __fma_rn(M[r2 * RS + i], nxi, M[r2 * RS + n]);
            __syncwarp();
        }
    }
    return info;
}

// ---------------------------------------------------------------------------
// Element-walk elimination with the trailing update of two steps per pass.
//
// Same result as smem_lupp<T, SOLVE, true> bit for bit (every element still
// receives fma(-l_ik, u_kj, a_ij) in increasing k with the same operands),
// organized to issue fewer instructions per FMA, which measured as the
// bottleneck of the one-step walk (about 50 warp instructions per FP64
// instruction, the FP64 pipe 67-77% busy):
//   * steps k and k+1 are paired: after the pivot of step k (search, row
//     interchange, multipliers, column k+1 updated in the same pass), the
//     pivot of step k+1 is found, row k+1 receives its step-k update and
//     column k+1 its multipliers; then one walk over the block below and to
//     the right of (k+1, k+1) applies both steps' updates to each element
//     (one load, two FMAs in order, one store).  Rows interchanged at step
//     k+1 still carry their pending step-k update and their own -l_ik, so
//     the interchange covers column k as well.
//   * with a full warp per system the pivot search is three warp reductions
//     (redux.sync) on the high and low words of the magnitude and on the row;
//   * element walk indices come from a multiply-shift instead of run-time
//     divisions;
//   * the back substitution keeps y in registers (lane t holds rows
//     t, t+T, ...) and broadcasts each x_i with a shuffle.
// KEEPL: interchange whole rows, L part included (getrf output); without it
// only the columns the remaining elimination reads are interchanged.
// ---------------------------------------------------------------------------

// ceil(2^16 / c): floor(x / c) == (x * kDivMagic[c]) >> 16 for 0 <= x < 64.
struct DivMagic {
    unsigned short m[65];
    constexpr DivMagic() : m()
    {
        for (int c = 1; c <= 64; ++c) m[c] = static_cast<unsigned short>((65536 + c - 1) / c == 65536 ? 0 : (65536 + c - 1) / c);
    }
};
static __constant__ const DivMagic kDivMagic{};

// floor(x / c) for 0 <= x < 64, 1 <= c <= 64.
__device__ __forceinline__ int div_small(int x, int c)
{
    return c == 1 ? x : static_cast<int>((static_cast<unsigned>(x) * kDivMagic.m[c]) >> 16);
}

// First maximum of |M[i*RS + k]| over candidate rows i in [lo, hi) of the
// group; every lane of the group receives the pivot row and value.  lim is
// the size of the system's block (checked builds, see tl_bounds.cuh).
template <int T>
__device__ __forceinline__ void smem_pivot_search(const double *M, int RS, int k, int lo, int hi, int t, int lim,
                                                  double &cv, int &cpos)
{
    if constexpr (T == 32) {
        // one candidate per lane (n <= 32): reduce the high word, the low
        // word among the lanes holding the largest high word, then the row
        const int i = lo + t;
        const bool cand = i < hi;
        const unsigned long long m = cand ? dev::mag_bits(TL_SM(M, i * RS + k, lim)) : 0ULL;
        const unsigned mh = static_cast<unsigned>(m >> 32), ml = static_cast<unsigned>(m);
        const unsigned maxh = __reduce_max_sync(0xffffffffu, cand ? mh : 0u);
        const bool c2 = cand && mh == maxh;
        const unsigned maxl = __reduce_max_sync(0xffffffffu, c2 ? ml : 0u);
        const bool c3 = c2 && ml == maxl;
        cpos = static_cast<int>(__reduce_min_sync(0xffffffffu, c3 ? static_cast<unsigned>(i) : 0xffffffffu));
        cv = TL_SM(M, cpos * RS + k, lim);
    } else if constexpr (T == 16 || T == 8) {
        // 32 / T systems per warp: each lane's first maximum over its rows,
        // then the same three reductions once per group (the lanes of the
        // other groups contribute the neutral value).  Measured against the
        // shuffle butterfly below: 2.4-4.4% faster at n = 24..28 with 16
        // lanes, 0.4-1.6% at n = 18..21 with 8
        constexpr int G = 32 / T;
        unsigned long long best = 0;
        int row = hi;
        for (int i = lo + t; i < hi; i += T) {
            const unsigned long long m = dev::mag_bits(TL_SM(M, i * RS + k, lim));
            if (row == hi || m > best) {
                best = m;
                row = i;
            }
        }
        const int grp = static_cast<int>(threadIdx.x & 31u) / T;
        const bool cand = row < hi;
        const unsigned mh = static_cast<unsigned>(best >> 32), ml = static_cast<unsigned>(best);
        unsigned maxh = 0;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const unsigned v = __reduce_max_sync(0xffffffffu, grp == g && cand ? mh : 0u);
            maxh = grp == g ? v : maxh;
        }
        const bool c2 = cand && mh == maxh;
        unsigned maxl = 0;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const unsigned v = __reduce_max_sync(0xffffffffu, grp == g && c2 ? ml : 0u);
            maxl = grp == g ? v : maxl;
        }
        const bool c3 = c2 && ml == maxl;
        unsigned rmin = 0;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const unsigned v =
                __reduce_min_sync(0xffffffffu, grp == g && c3 ? static_cast<unsigned>(row) : 0xffffffffu);
            rmin = grp == g ? v : rmin;
        }
        cpos = static_cast<int>(rmin);
        cv = TL_SM(M, cpos * RS + k, lim);
    } else {
        unsigned long long best = 0;
        int row = hi;
        for (int i = lo + t; i < hi; i += T) {
            const unsigned long long m = dev::mag_bits(TL_SM(M, i * RS + k, lim));
            if (row == hi || m > best) {
                best = m;
                row = i;
            }
        }
        // butterfly over the T lanes of the group: largest magnitude, ties
        // (and lanes without a candidate) to the smallest row
#pragma unroll
        for (int off = T / 2; off >= 1; off >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, off);
            const int orow = __shfl_xor_sync(0xffffffffu, row, off);
            const bool take = (orow < hi) && (row >= hi || ob > best || (ob == best && orow < row));
            best = take ? ob : best;
            row = take ? orow : row;
        }
        cpos = row;
        cv = TL_SM(M, row * RS + k, lim);
    }
}

// Pivot of step k: search (whole column, or the tile-local rule), record
// pivot and info, interchange rows k and p over columns [jlo, wcols).
template <int T>
__device__ __forceinline__ void smem_pivot_step(double *M, int n, int RS, int k, int t, int lim, int jlo, int wcols,
                                                int tile, double threshold, int *piv, double &cv, int &info)
{
    int hi = n;
    if (tile > 0 && tile < n) hi = min(n, (k / tile + 1) * tile);
    int p;
    smem_pivot_search<T>(M, RS, k, k, hi, t, lim, cv, p);
    if (hi < n && __any_sync(0xffffffffu, dev::mag_bits(cv) < dev::mag_bits(threshold))) {
        // tile-local pivoting: the in-tile best is below the threshold (in
        // some group of the warp): the first maximum over the whole column
        double cv2;
        int p2;
        smem_pivot_search<T>(M, RS, k, k, n, t, lim, cv2, p2);
        const bool below = dev::mag_bits(cv) < dev::mag_bits(threshold);
        cv = below ? cv2 : cv;
        p = below ? p2 : p;
    }
    if (dev::mag_bits(cv) == 0ULL && info == 0) info = k + 1;
    if (t == 0) TL_SM(piv, k, n) = p;
    if (p != k) {
        for (int j = jlo + t; j < wcols; j += T) {
            const double tmp = TL_SM(M, k * RS + j, lim);
            TL_SM(M, k * RS + j, lim) = TL_SM(M, p * RS + j, lim);
            TL_SM(M, p * RS + j, lim) = tmp;
        }
    }
}

// Negated multipliers of column k below row k (quotient for a pivot below
// DBL_MIN, a sign flip for a zero column); with UPD the same lane also
// applies step k to the entry of column k+1 of its row.
template <int T, bool UPD>
__device__ __forceinline__ void smem_multipliers(double *M, int n, int RS, int k, int t, int lim, double cv,
                                                 double nr, bool zero, bool small)
{
    const double ukk1 = UPD ? TL_SM(M, k * RS + k + 1, lim) : 0.0;
    if (!__any_sync(0xffffffffu, small)) {
        for (int i = k + 1 + t; i < n; i += T) {
            const double l = zero ? dev::neg(TL_SM(M, i * RS + k, lim)) : __dmul_rn(TL_SM(M, i * RS + k, lim), nr);
            TL_SM(M, i * RS + k, lim) = l;
            if (UPD && !zero) TL_SM(M, i * RS + k + 1, lim) = __fma_rn(l, ukk1, TL_SM(M, i * RS + k + 1, lim));
        }
    } else {
        const double ncv = dev::neg(cv);
        for (int i = k + 1 + t; i < n; i += T) {
            const double a = TL_SM(M, i * RS + k, lim);
            const double l = zero ? dev::neg(a) : (small ? __ddiv_rn(a, ncv) : __dmul_rn(a, nr));
            TL_SM(M, i * RS + k, lim) = l;
            if (UPD && !zero) TL_SM(M, i * RS + k + 1, lim) = __fma_rn(l, ukk1, TL_SM(M, i * RS + k + 1, lim));
        }
    }
}

template <int T, bool SOLVE, bool KEEPL>
__device__ __forceinline__ int smem_lupp2(double *M, int n, int RS, int t, int tile, double threshold)
{
    static_assert(T >= 1 && T <= 32 && (32 % T) == 0, "T must divide 32");
    const int lane0 = (static_cast<int>(threadIdx.x) & 31) - t;
    const int lim = smem_piv_offset(n) + (n + 1) / 2;  // doubles in the system's block
    double *rcp = M + n * RS;                           // n doubles
    int *piv = reinterpret_cast<int *>(rcp + n);        // n ints
    int info = 0;
    bool tiny = false;
    const int wcols = n + (SOLVE ? 1 : 0);              // columns incl. b
    int k = 0;
    for (; k + 1 < n; k += 2) {
        // ---- step k: pivot, interchange, multipliers, column k+1 ----
        double cv;
        smem_pivot_step<T>(M, n, RS, k, t, lim, KEEPL ? 0 : k, wcols, tile, threshold, piv, cv, info);
        const bool z0 = dev::mag_bits(cv) == 0ULL;
        const bool s0 = !z0 && dev::mag_bits(cv) < dev::kDblMinBits;
        const double r0 = dev::rcp_rn(cv);
        if (t == 0) TL_SM(rcp, k, n) = r0;
        tiny = tiny || s0;
        __syncwarp();
        smem_multipliers<T, true>(M, n, RS, k, t, lim, cv, dev::neg(r0), z0, s0);
        __syncwarp();
        // ---- step k+1: pivot (column k+1 is up to date), interchange rows
        //      that still carry step k's pending update and -l_ik ----
        const int k1 = k + 1;
        double cv1;
        smem_pivot_step<T>(M, n, RS, k1, t, lim, KEEPL ? 0 : k, wcols, tile, threshold, piv, cv1, info);
        const bool z1 = dev::mag_bits(cv1) == 0ULL;
        const bool s1 = !z1 && dev::mag_bits(cv1) < dev::kDblMinBits;
        const double r1 = dev::rcp_rn(cv1);
        if (t == 0) TL_SM(rcp, k1, n) = r1;
        tiny = tiny || s1;
        __syncwarp();
        // row k+1 receives step k (columns k+2..); column k+1 its multipliers
        if (!z0) {
            const double l = TL_SM(M, k1 * RS + k, lim);
            for (int j = k + 2 + t; j < wcols; j += T)
                TL_SM(M, k1 * RS + j, lim) = __fma_rn(l, TL_SM(M, k * RS + j, lim), TL_SM(M, k1 * RS + j, lim));
        }
        smem_multipliers<T, false>(M, n, RS, k1, t, lim, cv1, dev::neg(r1), z1, s1);
        __syncwarp();
        // ---- both updates of the block rows k+2.., columns k+2.. ----
        const int ncols = wcols - (k + 2);
        const int nrows = n - (k + 2);
        const int nel = nrows * ncols;
        if (nel > 0) {
            const int q = div_small(T, ncols), rq = T - q * ncols;   // (row, column) advance per stride
            int ei = div_small(t, ncols);
            int ej = t - ei * ncols;                                 // element t: row k+2+ei, column k+2+ej
            const int u0 = k * RS + k + 2;                          // rows k and k+1 from column k+2
            const int u1 = k1 * RS + k + 2;
            if (!__any_sync(0xffffffffu, z0 || z1)) {
                for (int e = t; e < nel; e += T) {
                    const int ri = (k + 2 + ei) * RS;
                    double a = TL_SM(M, ri + k + 2 + ej, lim);
                    a = __fma_rn(TL_SM(M, ri + k, lim), TL_SM(M, u0 + ej, lim), a);
                    a = __fma_rn(TL_SM(M, ri + k1, lim), TL_SM(M, u1 + ej, lim), a);
                    TL_SM(M, ri + k + 2 + ej, lim) = a;
                    ej += rq;
                    ei += q;
                    if (ej >= ncols) {
                        ej -= ncols;
                        ++ei;
                    }
                }
            } else {  // a zero pivot in some group: that step leaves the block as it is
                for (int e = t; e < nel; e += T) {
                    const int ri = (k + 2 + ei) * RS;
                    double a = TL_SM(M, ri + k + 2 + ej, lim);
                    if (!z0) a = __fma_rn(TL_SM(M, ri + k, lim), TL_SM(M, u0 + ej, lim), a);
                    if (!z1) a = __fma_rn(TL_SM(M, ri + k1, lim), TL_SM(M, u1 + ej, lim), a);
                    TL_SM(M, ri + k + 2 + ej, lim) = a;
                    ej += rq;
                    ei += q;
                    if (ej >= ncols) {
                        ej -= ncols;
                        ++ei;
                    }
                }
            }
        }
        __syncwarp();
    }
    if (k < n) {  // odd n: the last step (one row: its pivot and reciprocal)
        double cv;
        smem_pivot_step<T>(M, n, RS, k, t, lim, KEEPL ? 0 : k, wcols, tile, threshold, piv, cv, info);
        const bool s0 = dev::mag_bits(cv) != 0ULL && dev::mag_bits(cv) < dev::kDblMinBits;
        const double r0 = dev::rcp_rn(cv);
        if (t == 0) TL_SM(rcp, k, n) = r0;
        tiny = tiny || s0;
        __syncwarp();
    }

    // a6 (back part): x_i = y_i * RN(1/u_ii) (y_i / u_ii when a pivot was
    // below DBL_MIN), then y_r -= u_ri x_i for r < i
    if (SOLVE) {
        const bool any_tiny = __any_sync(0xffffffffu, tiny);
        if constexpr (T >= 4) {
            constexpr int KM = TL_MAX_N / T;  // row slots per lane
            double y[KM];
#pragma unroll
            for (int s = 0; s < KM; ++s) {
                const int r = t + s * T;
                y[s] = r < n ? TL_SM(M, r * RS + n, lim) : 0.0;
            }
            for (int i = n - 1; i >= 0; --i) {
                const int owner = i % T, slot = i / T;
                double yi = y[0];
#pragma unroll
                for (int s = 1; s < KM; ++s) yi = dev::sel(s == slot, y[s], yi);
                double xi;
                if (!any_tiny) xi = __dmul_rn(yi, TL_SM(rcp, i, n));
                else xi = tiny ? __ddiv_rn(yi, TL_SM(M, i * RS + i, lim)) : __dmul_rn(yi, TL_SM(rcp, i, n));
                xi = __shfl_sync(0xffffffffu, xi, lane0 + owner);
#pragma unroll
                for (int s = 0; s < KM; ++s) y[s] = dev::sel(t == owner && s == slot, xi, y[s]);
                const double nxi = dev::neg(xi);
#pragma unroll
                for (int s = 0; s < KM; ++s) {
                    if (s * T >= i) break;  // no row of this slot lies above row i
                    const int r = t + s * T;
                    if (r < i) y[s] = __fma_rn(TL_SM(M, r * RS + i, lim), nxi, y[s]);
                }
            }
#pragma unroll
            for (int s = 0; s < KM; ++s) {
                const int r = t + s * T;
                if (r < n) TL_SM(M, r * RS + n, lim) = y[s];
            }
            __syncwarp();
        } else {
            for (int i = n - 1; i >= 0; --i) {
                if (t == 0) {
                    const double y = TL_SM(M, i * RS + n, lim);
                    double xi;
                    if (!any_tiny) xi = __dmul_rn(y, TL_SM(rcp, i, n));
                    else xi = tiny ? __ddiv_rn(y, TL_SM(M, i * RS + i, lim)) : __dmul_rn(y, TL_SM(rcp, i, n));
                    TL_SM(M, i * RS + n, lim) = xi;
                }
                __syncwarp();
                const double nxi = dev::neg(TL_SM(M, i * RS + n, lim));
                for (int r2 = t; r2 < i; r2 += T)
                    TL_SM(M, r2 * RS + n, lim) = __fma_rn(TL_SM(M, r2 * RS + i, lim), nxi, TL_SM(M, r2 * RS + n, lim));
                __syncwarp();
            }
        }
    }
    return info;
}

// MODE: kGesv (A const, b -> x, LU optional by KEEP) or kGetrf (A in place).
// WALK: element walk of the trailing update instead of the lane tile.
template <int T, int LAYOUT, int MODE, bool KEEP, bool WALK = (T >= 16), bool ASYNC_LOAD = (T < 16)>
__global__ void __launch_bounds__(128) k_smem_group(SolveArgs args, int n)
{
    extern __shared__ double smem[];
    const int SB = blockDim.x / T;                 // systems per block
    const int per = smem_sys_doubles(n, T);
    const int RS = smem_row_stride(n);            // row stride
    const int64_t s0 = static_cast<int64_t>(blockIdx.x) * SB;
    const double *Ag = (MODE == kGetrf) ? args.LU : args.A;
    const int nn = n * n;
    const unsigned m20 = magic20(n);

    // ---- load: thread (q = tid % SB, t' = tid / SB) copies elements
    //      e = t', t'+T, ... of system s0+q (coalesced over q): cp.async,
    //      or register-staged streaming loads (ASYNC_LOAD false) ----
    {
        const int q = threadIdx.x % SB;
        const int tp = threadIdx.x / SB;
        const int64_t s = s0 + q;
        double *M = smem + q * per;
        if (!ASYNC_LOAD && s < args.batch) {
            const double *src = Ag + (LAYOUT == kInterleaved ? s : s * nn);
            const int64_t es = LAYOUT == kInterleaved ? args.ld : 1;
#pragma unroll 4
            for (int e = tp; e < nn; e += T) {
                const int j = div20(e, m20);
                TL_SM(M, (e - j * n) * RS + j, per) = ld_stream(src + e * es);
            }
            if (MODE == kGesv) {
                const double *bs = args.b + (LAYOUT == kInterleaved ? s : s * n);
                for (int i2 = tp; i2 < n; i2 += T) TL_SM(M, i2 * RS + n, per) = ld_stream(bs + i2 * es);
            }
        } else if (s < args.batch) {
            if (LAYOUT == kInterleaved) {
                for (int e = tp; e < nn; e += T) {
                    const int j = div20(e, m20);
                    cp_async8(&TL_SM(M, (e - j * n) * RS + j, per), Ag + static_cast<int64_t>(e) * args.ld + s);
                }
                if (MODE == kGesv)
                    for (int i2 = tp; i2 < n; i2 += T)
                        cp_async8(&TL_SM(M, i2 * RS + n, per), args.b + static_cast<int64_t>(i2) * args.ld + s);
            } else {
                const double *src = Ag + s * nn;
                for (int e = tp; e < nn; e += T) {
                    const int j = div20(e, m20);
                    cp_async8(&TL_SM(M, (e - j * n) * RS + j, per), src + e);
                }
                if (MODE == kGesv)
                    for (int i2 = tp; i2 < n; i2 += T) cp_async8(&TL_SM(M, i2 * RS + n, per), args.b + s * n + i2);
            }
        }
        cp_async_wait_all();
    }
    __syncthreads();

    // ---- compute: lanes t = lane % T of a group own system q ----
    const int lane = threadIdx.x & 31;
    const int t = lane % T;
    const int q = threadIdx.x / T;
    const int64_t s = s0 + q;
    const bool active = s < args.batch;
    double *M = smem + q * per;
    const int *piv = reinterpret_cast<const int *>(M + smem_piv_offset(n));  // pivots (after n reciprocals)
    // non-finite entries anywhere in this system
    int badv = 0;
    if (active) {
        for (int e = t; e < nn; e += T) {
            const int j = div20(e, m20);
            badv |= dev::is_nonfinite(M[(e - j * n) * RS + j]) ? 1 : 0;
        }
    }
    const bool bad = group_any_int<T>(badv) != 0;

    int info0;
    if constexpr (WALK)
        info0 = smem_lupp2<T, MODE == kGesv, KEEP || MODE == kGetrf>(M, n, RS, t, args.tile, args.threshold);
    else
        info0 = smem_lupp<T, MODE == kGesv, false>(M, n, RS, t, args.tile, args.threshold);
    int info = info0;
    if (bad) info = -1;

    // a7: store
    if (active) {
        for (int i = t; i < n; i += T) {
            const int64_t vi = (LAYOUT == kInterleaved) ? static_cast<int64_t>(i) * args.ld + s : s * n + i;
            if (MODE == kGesv) st_stream(args.x + vi, info != 0 ? dev::nan_value() : M[i * RS + n]);
            st_stream(args.ipiv + vi, bad ? i + 1 : piv[i] + 1);
        }
        if (t == 0) st_stream(args.info + s, info);
        if (KEEP) {
            // element e = j*n + i of the factors
            for (int e = t; e < nn; e += T) {
                const int i = e % n, j = e / n;
                const int64_t ai = (LAYOUT == kInterleaved) ? static_cast<int64_t>(e) * args.ld + s : s * nn + e;
                if (!bad) {
                    const double v = M[i * RS + j];
                    st_stream(args.LU + ai, j < i ? dev::neg(v) : v);
                } else if (MODE == kGesv) {
                    args.LU[ai] = args.A[ai];
                }
            }
        }
    }
}

// Ragged batches (tl_lupp_solve_batched): persistent over the bucket of
// systems of size n (run-time), SB = blockDim/T systems per block and trip;
// each system at its own offsets in per-system column-major storage.  Same
// elimination as k_smem_group (smem_lupp), binary64.
template <int T>
__global__ void __launch_bounds__(128) k_smem_ragged(RaggedArgs r, int n)
{
    extern __shared__ double smem[];
    const int SB = blockDim.x / T;
    const int per = smem_sys_doubles(n, T);
    const int RS = smem_row_stride(n);
    const int nn = n * n;
    const unsigned m20 = magic20(n);
    const int64_t beg = r.offsets[n];
    const int64_t full = r.offsets[n + 1] - beg;
    int64_t count = full;
    if (r.counts) {
        const int64_t c = r.counts[n];
        count = c < 0 ? 0 : (c < full ? c : full);
    }
    const int lane = threadIdx.x & 31;
    const int t = lane % T;
    const int q = threadIdx.x / T;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * SB; base < count;
         base += static_cast<int64_t>(gridDim.x) * SB) {           // block-uniform trip
        // load: thread (qL = tid % SB, tp = tid / SB) copies elements
        // e = tp, tp+T, ... of system base+qL (cp.async)
        {
            const int qL = threadIdx.x % SB;
            const int tp = threadIdx.x / SB;
            double *M = smem + qL * per;
            if (base + qL < count) {
                const int64_t sidx = r.bucket[beg + base + qL];
                const double *A = r.A + r.a_off[sidx];
                for (int e = tp; e < nn; e += T) {
                    const int j = div20(e, m20);
                    cp_async8(&TL_SM(M, (e - j * n) * RS + j, per), A + e);
                }
                const double *bv = r.b + r.b_off[sidx];
                for (int i2 = tp; i2 < n; i2 += T) cp_async8(&TL_SM(M, i2 * RS + n, per), bv + i2);
            }
            cp_async_wait_all();
        }
        __syncthreads();
        const bool active = base + q < count;
        double *M = smem + q * per;
        int badv = 0;
        if (active) {
            for (int e = t; e < nn; e += T) {
                const int j = div20(e, m20);
                badv |= dev::is_nonfinite(M[(e - j * n) * RS + j]) ? 1 : 0;
            }
        }
        const bool bad = group_any_int<T>(badv) != 0;
        int info = smem_lupp2<T, true, false>(M, n, RS, t, 0, 0.0);
        if (bad) info = -1;
        if (active) {
            const int64_t sidx = r.bucket[beg + base + q];
            const int *piv = reinterpret_cast<const int *>(M + smem_piv_offset(n));
            double *x = r.x + r.b_off[sidx];
            int32_t *ip = r.ipiv + r.piv_off[sidx];
            for (int i = t; i < n; i += T) {
                st_stream(x + i, info != 0 ? dev::nan_value() : M[i * RS + n]);
                st_stream(ip + i, bad ? i + 1 : piv[i] + 1);
            }
            if (t == 0) st_stream(r.info + sidx, info);
        }
        __syncthreads();  // the next trip's loads overwrite the blocks
    }
}

}  // namespace tl
