// tinylu_device.cuh -- device-callable tiny LUpp solvers for sm_103a: the
// public header for user kernels (the tl::lupp_solve* entry points at the
// end of this file) and the code the library's batched and fused Newton
// kernels are built on.  Self-contained: include it alone in a .cu file.
//
// Two thread-to-system mappings (paper Sec. 2.3, "thread-to-system mapping"):
//
//   * lu_thread_*  -- one thread owns one system; the whole matrix lives in
//     that thread's registers (single-threaded family of Sec. 3.2.2).  All
//     loops are unrolled at compile time for the system size N, so every
//     FP64 instruction issued does useful work on all 32 lanes.
//
//   * lu_group_*   -- T consecutive lanes own one system, lane t holding the
//     rows i = t, t+T, t+2T, ... (K = ceil(N/T) row slots, round-robin so a
//     column access stays coalesced, Sec. 3.2.1); slots past N are phantom
//     rows skipped at compile time.  The pivot search is a butterfly
//     __shfl_xor arg-max, the pivot row is broadcast with __shfl, and the
//     physical row interchange is a register permutation between the two
//     owning lanes.
//
// Arithmetic (identical in both mappings, and identical to the sequential
// right-looking elimination of Sec. 2.2):
//   pivot    p = first row i >= k of largest |a_ik|.  The magnitude compare is
//            an integer compare of the IEEE bit pattern with the sign cleared,
//            which orders finite values exactly as |x| does and keeps the
//            search off the FP64 pipe.
//   zero     a_pk == 0: info = k+1 (first), the step does nothing else.
//   scale    l_ik = a_ik * RN(1/a_kk) (a_ik / a_kk when |a_kk| < DBL_MIN).
//   update   a_ij = fma(-l_ik, a_kj, a_ij), every element updated once per
//            step in increasing k, so the order of rounding is fixed.
// Every FP64 operation is an explicit round-to-nearest intrinsic, so the
// compiler cannot contract or reorder any of them.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

// Reciprocal of the one-thread fast path of the batched solvers: the
// integer-pipe sequence up to this n, the FP64 instruction above it.
// Measured on GB300: the integer sequence wins for n <= 5 (0.64-0.72 of the
// FP64 peak at n = 4, 5 against 0.47-0.56) and loses for n = 6..9, where
// its registers cost more than the FP64 slots it saves.  The Newton kernels,
// whose FP64 pipe is saturated by the law, always take the integer
// sequence (+10% points/s).
#ifndef TL_THREAD_RCP_INT_MAX_N
#define TL_THREAD_RCP_INT_MAX_N 5
#endif
// Reciprocal of the sub-warp group solvers (same choice).
#ifndef TL_GROUP_RCP_INT
#define TL_GROUP_RCP_INT 0
#endif

namespace tl {
namespace dev {

constexpr unsigned long long kMagMask = 0x7fffffffffffffffULL;
constexpr unsigned long long kDblMinBits = 0x0010000000000000ULL;  // DBL_MIN
constexpr unsigned long long kInfBits = 0x7ff0000000000000ULL;      // +Inf

// |v| as its IEEE bit pattern (an unsigned integer that orders like |v| for
// every non-NaN value).  Written as inline PTX on the high word: in plain C++
// the compiler recognizes the mask as fabs() and issues it on the FP64 pipe,
// which costs as much as an FMA on this GPU.
__device__ __forceinline__ unsigned long long mag_bits(double v)
{
    unsigned long long r;
    asm("{\n\t.reg .b32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\tand.b32 hi, hi, 0x7fffffff;\n\t"
        "mov.b64 %0, {lo, hi};\n\t}"
        : "=l"(r)
        : "d"(v));
    return r;
}

__device__ __forceinline__ bool is_nonfinite(double v) { return mag_bits(v) >= kInfBits; }

__device__ __forceinline__ double nan_value() { return __longlong_as_double(0x7ff8000000000000LL); }

// -x by flipping the sign bit on the integer pipe.  The FP64 pipe is the
// scarce unit on this GPU (one warp-wide DFMA per 64 clocks per SM
// sub-partition), and a negated operand reused by several FMAs would
// otherwise be materialized by an FP64 instruction.  Inline PTX keeps the
// compiler from turning the XOR back into a floating-point negation.
__device__ __forceinline__ double neg(double x)
{
    double r;
    asm("{\n\t.reg .b32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\txor.b32 hi, hi, 0x80000000;\n\t"
        "mov.b64 %0, {lo, hi};\n\t}"
        : "=d"(r)
        : "d"(x));
    return r;
}

// RN(1/a), IEEE binary64 round to nearest even, computed with integer and
// FP32 instructions only, so the reciprocal of every elimination step costs
// no FP64 pipe time (the FP64 pipe is the bottleneck; the integer pipes are
// mostly idle).  The published method followed: Newton-Raphson iteration
// for the reciprocal from a low-precision seed, then correct rounding by an
// exact remainder (Markstein, IBM J. Res. Dev. 34(1), 1990; Muller et al.,
// Handbook of Floating-Point Arithmetic, 2nd ed., 2018, ch. 5), here carried
// out in integer fixed point.  Method: a = X * 2^(e-1075) with the 53-bit integer
// significand X; the result significand is Q = RN(2^105 / X):
//   1. seed  Y0 = RN32(1 / (X >> 29)) * 2^76         (~22 correct bits)
//   2. two Newton steps in fixed point, Y += Y * (2^105 - X Y) / 2^105
//      (the first with a 128-bit residual, the second with its exact low
//      64 bits)                                       (Y within +-2 of 2^105/X)
//   3. exact remainder R = 2^105 - X Y (low 64 bits of the product), Y
//      adjusted until 0 <= R < X, then Y += (2R > X)   (2R == X is impossible
//      for X > 2^52: 2^106 / X would have to be an odd integer).
// A power-of-two significand gives Y = 2^53, which the final packing carries
// into the exponent.  Inputs whose reciprocal would be subnormal or that are
// zero, subnormal, Inf or NaN take __drcp_rn, behind a warp-uniform branch so
// that the common path issues no FP64 instruction at all.
// Integer-pipe core of RN(1/a): exact for normal |a| in [DBL_MIN, 2^1021)
// (biased exponent 1..2044); any other input returns an unspecified value.
// Straight-line code without a branch, so the compiler can interleave it
// with independent FMAs.
__device__ __forceinline__ double rcp_rn_fast(double a)
{
    unsigned long long bits;
    asm("mov.b64 %0, %1;" : "=l"(bits) : "d"(a));  // opaque: no FP pattern matching
    const int eb = static_cast<int>((bits >> 52) & 0x7ff);
    const unsigned long long sign = bits & 0x8000000000000000ULL;
    const unsigned long long X = (bits & 0x000fffffffffffffULL) | 0x0010000000000000ULL;
    // 1. seed from the FP32 reciprocal of the top 24 bits (exact as a float)
    const unsigned xh = static_cast<unsigned>(X >> 29);
    const float xf = __uint_as_float((150u << 23) | (xh & 0x7fffffu));
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(xf));
    const unsigned rb = __float_as_uint(rf);
    unsigned long long Y = static_cast<unsigned long long>((rb & 0x7fffffu) | 0x800000u) << ((rb >> 23) - 74);
    // 2a. D = 2^105 - X Y as a 128-bit value, |D| < 2^84; Y += Y D / 2^105
    {
        const unsigned long long plo = X * Y;
        const unsigned long long phi = __umul64hi(X, Y);
        const unsigned long long dlo = 0ULL - plo;
        const unsigned long long dhi = (1ULL << 41) - phi - (plo != 0ULL ? 1ULL : 0ULL);
        const long long dsh = static_cast<long long>((dhi << 24) | (dlo >> 40));  // D >> 40
        Y = static_cast<unsigned long long>(static_cast<long long>(Y) + (__mul64hi(static_cast<long long>(Y), dsh) >> 1));
    }
    // 2b. |D| < 2^63 now: its low 64 bits are exact
    {
        const long long d1 = static_cast<long long>(0ULL - X * Y);
        Y = static_cast<unsigned long long>(static_cast<long long>(Y) + (__mul64hi(static_cast<long long>(Y), d1) >> 41));
    }
    // 3. exact remainder and rounding
    long long R = static_cast<long long>(0ULL - X * Y);
    const long long Xs = static_cast<long long>(X);
#pragma unroll
    for (int it = 0; it < 3; ++it) {
        const bool lo = R < 0;
        Y = lo ? Y - 1 : Y;
        R = lo ? R + Xs : R;
    }
#pragma unroll
    for (int it = 0; it < 3; ++it) {
        const bool hi = R >= Xs;
        Y = hi ? Y + 1 : Y;
        R = hi ? R - Xs : R;
    }
    Y += (2 * R > Xs) ? 1ULL : 0ULL;
    // a power-of-two significand gives Y = 2^53, carried into the exponent
    return __longlong_as_double(static_cast<long long>(sign | ((static_cast<unsigned long long>(2045 - eb) << 52) +
                                                               (Y - 0x0010000000000000ULL))));
}

// True when rcp_rn_fast is exact for a value of magnitude bits m.
__device__ __forceinline__ bool rcp_fast_ok(unsigned long long m)
{
    return m >= 0x0010000000000000ULL && m < 0x7fd0000000000000ULL;
}

// Out-of-line so that the compiler cannot if-convert the rare fallback into
// predicated FP64 instructions that every call would then issue.
static __device__ __noinline__ double rcp_rn_fallback(double a) { return __drcp_rn(a); }

// RN(1/a) for every input (IEEE binary64, round to nearest even):
// rcp_rn_fast where it is exact, __drcp_rn otherwise behind a warp-uniform
// branch.  The method of rcp_rn_fast: a = X * 2^(e-1075) with the 53-bit
// integer significand X; the result significand is Q = RN(2^105 / X):
//   1. seed  Y0 = RN32(1 / (X >> 29)) * 2^76         (~22 correct bits)
//   2. two Newton steps in fixed point, Y += Y * (2^105 - X Y) / 2^105
//      (the first with a 128-bit residual, the second with its exact low
//      64 bits)                                       (Y within +-2 of 2^105/X)
//   3. exact remainder R = 2^105 - X Y (low 64 bits of the product), Y
//      adjusted until 0 <= R < X, then Y += (2R > X)   (2R == X is impossible
//      for X > 2^52: 2^106 / X would have to be an odd integer).
__device__ __forceinline__ double rcp_rn(double a)
{
    const unsigned long long m = mag_bits(a);
    double res = rcp_rn_fast(a);
    const bool special = !rcp_fast_ok(m);
    if (__any_sync(__activemask(), special)) {
        if (special) res = rcp_rn_fallback(a);
    }
    return res;
}

// 64-bit select done on the integer pipe (two 32-bit selects).
__device__ __forceinline__ double sel(bool c, double a, double b)
{
    long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    return __longlong_as_double(c ? ia : ib);
}

// ---------------------------------------------------------------------------
// One thread per system, everything in registers.
// ---------------------------------------------------------------------------

// Returns true when any entry is NaN or +-Inf.
template <int N>
__device__ __forceinline__ bool any_nonfinite(const double (&a)[N][N])
{
    unsigned long long worst = 0;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            unsigned long long m = mag_bits(a[i][j]);
            worst = m > worst ? m : worst;
        }
    return worst >= kInfBits;
}

// In-register LUpp of a[i][j] (row i, column j).
//   KEEP_L : also permute the already-computed multipliers (getrf output);
//            without it the L part is left in elimination order, which is
//            all a fused solve needs.
//   NB     : number of right-hand-side columns eliminated along with A
//            (forward substitution fused into the factorization).
// piv[k] receives the 0-based pivot row, rcp[k] = RN(1/u_kk) (valid when
// `tiny` stays false).  Returns info (0 or first zero pivot step + 1).
// Below the diagonal a holds -l_ik (see lu_thread_unnegate_L).
template <int N, bool KEEP_L, int NB>
__device__ __forceinline__ int lu_thread_factor(double (&a)[N][N], double (&b)[NB > 0 ? NB : 1][N],
                                                int (&piv)[N], double (&rcp)[N], bool &tiny)
{
    // Look-ahead: step k updates column k+1 first, then searches its pivot
    // and forms the next reciprocal, and only then updates the remaining
    // columns, so the integer search and reciprocal of step k+1 overlap the
    // FMAs of step k.  Every element still receives its updates in
    // increasing k, so the rounding sequence is unchanged.
    int info = 0;
    // pivot search of column k (first maximum of the magnitude bits)
    auto search = [&](int k, int &p, unsigned long long &best, double &pv) {
        best = mag_bits(a[k][k]);
        p = k;
        pv = a[k][k];
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const unsigned long long m = mag_bits(a[i][k]);
            const bool gt = m > best;
            best = gt ? m : best;
            p = gt ? i : p;
            pv = sel(gt, a[i][k], pv);
        }
    };
    int p_next;
    unsigned long long best_next;
    double pv_next;
    search(0, p_next, best_next, pv_next);
    double r_next = rcp_rn(pv_next);
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const int p = p_next;
        const unsigned long long best = best_next;
        const double pv = pv_next;
        const double r = r_next;
        piv[k] = p;
        rcp[k] = 0.0;
        const bool zero = (best == 0ULL);
        if (zero) {
            if (info == 0) info = k + 1;
            // the column below is zero; store it in the negated convention
            // too so that the final sign flip restores it bit for bit
#pragma unroll
            for (int i = k + 1; i < N; ++i) a[i][k] = neg(a[i][k]);
        } else {
            // a3: physical row interchange k <-> p as a register permutation.
            const int j0 = KEEP_L ? 0 : k;
#pragma unroll
            for (int i = k + 1; i < N; ++i) {
                const bool s = (p == i);
#pragma unroll
                for (int j = j0; j < N; ++j) {
                    double t = a[k][j];
                    a[k][j] = sel(s, a[i][j], t);
                    a[i][j] = sel(s, t, a[i][j]);
                }
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    double t = b[c][k];
                    b[c][k] = sel(s, b[c][i], t);
                    b[c][i] = sel(s, t, b[c][i]);
                }
            }
            // a4: multipliers, kept NEGATED: -l_ik = RN(a_ik * (-r)); the
            // quotient path for |pivot| < DBL_MIN is a warp-uniform branch.
            const bool small = best < kDblMinBits;
            if (!__any_sync(__activemask(), small)) {
                rcp[k] = r;
                const double nr = neg(r);
#pragma unroll
                for (int i = k + 1; i < N; ++i) a[i][k] = __dmul_rn(a[i][k], nr);
            } else {
                rcp[k] = r;
                const double nr = neg(r);
                const double npv = neg(pv);
                tiny = tiny || small;
#pragma unroll
                for (int i = k + 1; i < N; ++i)
                    a[i][k] = small ? __ddiv_rn(a[i][k], npv) : __dmul_rn(a[i][k], nr);
            }
            // a5 part 1: column k+1 of the Schur update
            if (k + 1 < N) {
#pragma unroll
                for (int i = k + 1; i < N; ++i) a[i][k + 1] = __fma_rn(a[i][k], a[k][k + 1], a[i][k + 1]);
            }
        }
        // look-ahead: pivot and reciprocal of step k+1
        if (k + 1 < N) {
            search(k + 1, p_next, best_next, pv_next);
            r_next = rcp_rn(pv_next);
        }
        if (!zero) {
            // a5 part 2: the remaining columns; a6 (forward part): b follows
            // as extra columns.
#pragma unroll
            for (int j = k + 2; j < N; ++j)
#pragma unroll
                for (int i = k + 1; i < N; ++i) a[i][j] = __fma_rn(a[i][k], a[k][j], a[i][j]);
#pragma unroll
            for (int c = 0; c < NB; ++c)
#pragma unroll
                for (int i = k + 1; i < N; ++i) b[c][i] = __fma_rn(a[i][k], b[c][k], b[c][i]);
        }
    }
    return info;
}

// Branch-free fast path of lu_thread_factor for the common case: every
// pivot normal and below 2^1021 in magnitude.  The same arithmetic, the same
// look-ahead, no data-dependent branch at all (so the compiler can schedule
// each step as one block), and the reciprocal entirely on the integer pipe.
// Returns true when the system needs the exact general path instead (a zero,
// subnormal, huge or non-finite pivot was met): the caller then restarts the
// system from its input with lu_thread_factor.
template <int N, bool KEEP_L, int NB, bool RCP_INT = (N <= TL_THREAD_RCP_INT_MAX_N)>
__device__ __forceinline__ bool lu_thread_factor_fast(double (&a)[N][N], double (&b)[NB > 0 ? NB : 1][N],
                                                      int (&piv)[N], double (&rcp)[N])
{
    // The whole factorization is one straight-line block (every loop is
    // unrolled and there is no data-dependent branch), so the instruction
    // scheduler is free to overlap the integer pivot search and reciprocal
    // of a step with the FMAs still in flight from the previous one.
    bool slow = false;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        // a2: pivot search (first maximum of the magnitude bits)
        unsigned long long best = mag_bits(a[k][k]);
        int p = k;
        double pv = a[k][k];
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const unsigned long long m = mag_bits(a[i][k]);
            const bool gt = m > best;
            best = gt ? m : best;
            p = gt ? i : p;
            pv = sel(gt, a[i][k], pv);
        }
        slow = slow || !rcp_fast_ok(best);
        piv[k] = p;
        const double r = RCP_INT ? rcp_rn_fast(pv) : __drcp_rn(pv);
        rcp[k] = r;
        // a3: interchange as a register permutation
        const int j0 = KEEP_L ? 0 : k;
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const bool s = (p == i);
#pragma unroll
            for (int j = j0; j < N; ++j) {
                double t = a[k][j];
                a[k][j] = sel(s, a[i][j], t);
                a[i][j] = sel(s, t, a[i][j]);
            }
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                double t = b[c][k];
                b[c][k] = sel(s, b[c][i], t);
                b[c][i] = sel(s, t, b[c][i]);
            }
        }
        // a4: negated multipliers; a5 + forward part of a6
        const double nr = neg(r);
#pragma unroll
        for (int i = k + 1; i < N; ++i) a[i][k] = __dmul_rn(a[i][k], nr);
#pragma unroll
        for (int j = k + 1; j < N; ++j)
#pragma unroll
            for (int i = k + 1; i < N; ++i) a[i][j] = __fma_rn(a[i][k], a[k][j], a[i][j]);
#pragma unroll
        for (int c = 0; c < NB; ++c)
#pragma unroll
            for (int i = k + 1; i < N; ++i) b[c][i] = __fma_rn(a[i][k], b[c][k], b[c][i]);
    }
    return slow;
}

// Back substitution of the fast path (all pivots normal): x_i = s * RN(1/u_ii).
template <int N>
__device__ __forceinline__ void lu_thread_backsolve_fast(const double (&a)[N][N], double (&y)[N],
                                                         const double (&rcp)[N])
{
    double nx[N];
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        double s = y[i];
#pragma unroll
        for (int j = N - 1; j > i; --j) s = __fma_rn(a[i][j], nx[j], s);
        y[i] = __dmul_rn(s, rcp[i]);
        nx[i] = neg(y[i]);
    }
}

// lu_thread_factor leaves -l_ik below the diagonal; flip them back to the
// LAPACK storage of L (integer sign flips only).
template <int N>
__device__ __forceinline__ void lu_thread_unnegate_L(double (&a)[N][N])
{
#pragma unroll
    for (int i = 1; i < N; ++i)
#pragma unroll
        for (int j = 0; j < i; ++j) a[i][j] = neg(a[i][j]);
}

// a6 (back part): x_i = (y_i - sum_{j>i} u_ij x_j) * RN(1/u_ii), the sum
// accumulated in decreasing j.  y is overwritten by x.  When a pivot was
// below DBL_MIN the reciprocal may overflow, so that case divides.
template <int N>
__device__ __forceinline__ void lu_thread_backsolve(const double (&a)[N][N], double (&y)[N],
                                                    const double (&rcp)[N], bool tiny)
{
    // nx[j] = -x_j (integer sign flip) so that each step is fma(u_ij, -x_j, s).
    double nx[N];
    if (!__any_sync(__activemask(), tiny)) {
#pragma unroll
        for (int i = N - 1; i >= 0; --i) {
            double s = y[i];
#pragma unroll
            for (int j = N - 1; j > i; --j) s = __fma_rn(a[i][j], nx[j], s);
            y[i] = __dmul_rn(s, rcp[i]);
            nx[i] = neg(y[i]);
        }
    } else {
#pragma unroll
        for (int i = N - 1; i >= 0; --i) {
            double s = y[i];
#pragma unroll
            for (int j = N - 1; j > i; --j) s = __fma_rn(a[i][j], nx[j], s);
            y[i] = tiny ? __ddiv_rn(s, a[i][i]) : __dmul_rn(s, rcp[i]);
            nx[i] = neg(y[i]);
        }
    }
}

// Forward substitution with the factors of lu_thread_factor<N, true, 0>:
// apply the interchanges to y in order, then y_i -= l_ij y_j (increasing j).
template <int N>
__device__ __forceinline__ void lu_thread_forward(const double (&a)[N][N], const int (&piv)[N],
                                                  double (&y)[N])
{
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const int p = piv[k];
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const bool s = (p == i);
            double t = y[k];
            y[k] = sel(s, y[i], t);
            y[i] = sel(s, t, y[i]);
        }
    }
    double ny[N];
    ny[0] = neg(y[0]);
#pragma unroll
    for (int i = 1; i < N; ++i) {
        double s = y[i];
#pragma unroll
        for (int j = 0; j < i; ++j) s = __fma_rn(a[i][j], ny[j], s);
        y[i] = s;
        ny[i] = neg(s);
    }
}

// Device-callable fused solve for one system held by the calling thread:
// A (destroyed) x = b (overwritten by x).  Returns info; x is NaN on
// info != 0.  The exact general path (zero, tiny, huge or non-finite pivots).
template <int N>
__device__ __forceinline__ int lupp_solve(double (&a)[N][N], double (&b)[N], int (&piv)[N])
{
    if (any_nonfinite<N>(a)) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            piv[k] = k;
            b[k] = nan_value();
        }
        return -1;
    }
    double rcp[N];
    bool tiny = false;
    double (&bb)[1][N] = *reinterpret_cast<double (*)[1][N]>(&b);
    int info = lu_thread_factor<N, false, 1>(a, bb, piv, rcp, tiny);
    lu_thread_backsolve<N>(a, b, rcp, tiny);
    if (info != 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) b[i] = nan_value();
    }
    return info;
}

// The fast solve: returns false when it cannot vouch for the result (the
// system met a zero, tiny, huge or non-finite pivot or input); the caller must
// then restore a and b and use lupp_solve.  Same arithmetic otherwise.
template <int N, bool RCP_INT = (N <= TL_THREAD_RCP_INT_MAX_N)>
__device__ __forceinline__ bool lupp_solve_fast(double (&a)[N][N], double (&b)[N], int (&piv)[N])
{
    const bool bad = any_nonfinite<N>(a);
    double rcp[N];
    double (&bb)[1][N] = *reinterpret_cast<double (*)[1][N]>(&b);
    const bool slow = lu_thread_factor_fast<N, false, 1, RCP_INT>(a, bb, piv, rcp);
    lu_thread_backsolve_fast<N>(a, b, rcp);
    return !(slow || bad);
}

// ---------------------------------------------------------------------------
// T lanes per system (row-cyclic ownership), everything in registers.
// ---------------------------------------------------------------------------

template <int N, int T>
struct Group {
    static constexpr int K = (N + T - 1) / T;  // row slots per lane
    static_assert(T >= 1 && T <= 32 && (32 % T) == 0, "T must divide 32");
    // A slot is live at step k when some lane's row in it is still below the
    // pivot row: (T-1) + s*T > k, and the slot is not entirely phantom.
    __host__ __device__ static constexpr bool slot_alive(int s, int k)
    {
        return s * T < N && (T - 1) + s * T > k;
    }
};

// Butterfly arg-max over the T lanes of a group.  Each lane proposes
// (value bits, row); the winner has the largest magnitude, ties to the
// smallest row.  All lanes of the warp must call this together.
template <int T>
__device__ __forceinline__ void group_argmax(double &v, int &row)
{
#pragma unroll
    for (int off = T / 2; off >= 1; off >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, off);
        int orow = __shfl_xor_sync(0xffffffffu, row, off);
        unsigned long long m = mag_bits(v), om = mag_bits(ov);
        bool take = (om > m) || (om == m && orow < row);
        v = sel(take, ov, v);
        row = take ? orow : row;
    }
}

// Group LUpp.  Lane t (0..T-1) of the group holds rows t + s*T in a[s][*]
// and, for NB = 1, the matching entries of the right-hand side in b[s].
// `lane0` is the warp lane of the group's first lane.  `active` is false for
// groups past the end of the batch (they compute on zeros but must still
// take part in the warp shuffles).
// On return: pivk[s] = 0-based pivot row of step k = t + s*T (for this
// lane's steps), rcp[s] = RN(1/u_ii) of this lane's rows, info as usual.
// The multipliers are left NEGATED below the diagonal (-l_ik); the owner of
// row i flips columns j < i back when the factors are stored.
template <int N, int T, bool KEEP_L, int NB>
__device__ __forceinline__ int lu_group_factor(double (&a)[Group<N, T>::K][N],
                                               double (&b)[Group<N, T>::K],
                                               int (&pivk)[Group<N, T>::K],
                                               double (&rcp)[Group<N, T>::K], int t, int lane0,
                                               bool &tiny)
{
    constexpr int K = Group<N, T>::K;
    int info = 0;
    // a2: this lane's candidate in column k, then the butterfly across the
    // group (first maximum: ties go to the smaller row).
    auto search = [&](int k, double &cv, int &crow) {
        cv = 0.0;
        crow = N;  // sentinel: no candidate
#pragma unroll
        for (int s = 0; s < K; ++s) {
            if (s * T < N && (T - 1) + s * T >= k) {
                const int i = t + s * T;
                const bool cand = (i >= k) && (i < N);
                const unsigned long long m = mag_bits(a[s][k]);
                const bool take = cand && (crow == N || m > mag_bits(cv));
                cv = sel(take, a[s][k], cv);
                crow = take ? i : crow;
            }
        }
        group_argmax<T>(cv, crow);
    };
    // Look-ahead as in lu_thread_factor: column k+1 is updated first, the
    // search and reciprocal of step k+1 are issued, then the other columns.
    auto group_rcp = [](double v) {
#if TL_GROUP_RCP_INT
        return rcp_rn(v);
#else
        return __drcp_rn(v);
#endif
    };
    double cv_next;
    int crow_next;
    search(0, cv_next, crow_next);
    double r_next = group_rcp(cv_next);
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const int owner_k = k % T;   // lane (in group) holding row k
        const int slot_k = k / T;
        const double cv = cv_next;
        const int p = crow_next;
        const double r = r_next;
        const bool zero = (mag_bits(cv) == 0ULL);
        if (t == owner_k) pivk[slot_k] = p;
        if (zero && info == 0) info = k + 1;

        // a3: interchange rows k and p between their owning lanes.  The
        // shuffle that brings row p to row k reaches every lane of the
        // group, so it is also the broadcast of the pivot row u_kj.
        const int owner_p = p % T;
        const int slot_p = p / T;
        const int j0 = KEEP_L ? 0 : k;
        double uk[N + 1];
#pragma unroll
        for (int j = j0; j < N + NB; ++j) {
            double vk, vp = 0.0;
            if (j < N) {
                vk = a[slot_k][j];
#pragma unroll
                for (int s = 0; s < K; ++s) vp = sel(s == slot_p, a[s][j], vp);
            } else {
                vk = b[slot_k];
#pragma unroll
                for (int s = 0; s < K; ++s) vp = sel(s == slot_p, b[s], vp);
            }
            const double new_k = __shfl_sync(0xffffffffu, vp, lane0 + owner_p);
            const double new_p = __shfl_sync(0xffffffffu, vk, lane0 + owner_k);
            if (j > k) uk[j] = new_k;
            if (j < N) {
#pragma unroll
                for (int s = 0; s < K; ++s)
                    a[s][j] = sel(t == owner_p && s == slot_p, new_p, a[s][j]);
                if (t == owner_k) a[slot_k][j] = new_k;
            } else {
#pragma unroll
                for (int s = 0; s < K; ++s) b[s] = sel(t == owner_p && s == slot_p, new_p, b[s]);
                if (t == owner_k) b[slot_k] = new_k;
            }
        }

        // a4: reciprocal (formed by the look-ahead; the butterfly left the
        // pivot value in cv on every lane) and this lane's multipliers, kept
        // negated (see lu_thread_factor); a zero column is flipped as well so
        // the final sign flip restores it bit for bit.
        const bool small = !zero && mag_bits(cv) < kDblMinBits;
        if (t == owner_k) rcp[slot_k] = r;
        tiny = tiny || small;
        const double nr = neg(r);
#pragma unroll
        for (int s = 0; s < K; ++s) {
            if (Group<N, T>::slot_alive(s, k)) {
                const int i = t + s * T;
                if (zero && i > k && i < N) a[s][k] = neg(a[s][k]);
            }
        }
        if (!__any_sync(0xffffffffu, small)) {
#pragma unroll
            for (int s = 0; s < K; ++s) {
                if (Group<N, T>::slot_alive(s, k)) {
                    const int i = t + s * T;
                    const bool live = !zero && i > k && i < N;
                    if (live) a[s][k] = __dmul_rn(a[s][k], nr);
                }
            }
        } else {  // some group of the warp has a pivot below DBL_MIN
            const double ncv = neg(cv);
#pragma unroll
            for (int s = 0; s < K; ++s) {
                if (Group<N, T>::slot_alive(s, k)) {
                    const int i = t + s * T;
                    const bool live = !zero && i > k && i < N;
                    if (live) a[s][k] = small ? __ddiv_rn(a[s][k], ncv) : __dmul_rn(a[s][k], nr);
                }
            }
        }
        // a5 part 1: column k+1
        if (k + 1 < N) {
#pragma unroll
            for (int s = 0; s < K; ++s) {
                if (Group<N, T>::slot_alive(s, k)) {
                    const int i = t + s * T;
                    if (!zero && i > k && i < N) a[s][k + 1] = __fma_rn(a[s][k], uk[k + 1], a[s][k + 1]);
                }
            }
            // look-ahead: pivot and reciprocal of step k+1
            search(k + 1, cv_next, crow_next);
            r_next = group_rcp(cv_next);
        }
        // a5 part 2: the other columns, and b (forward part of a6)
#pragma unroll
        for (int s = 0; s < K; ++s) {
            if (Group<N, T>::slot_alive(s, k)) {
                const int i = t + s * T;
                const bool live = !zero && i > k && i < N;
                if (live) {
#pragma unroll
                    for (int j = k + 2; j < N; ++j) a[s][j] = __fma_rn(a[s][k], uk[j], a[s][j]);
                    if (NB > 0) b[s] = __fma_rn(a[s][k], uk[N], b[s]);
                }
            }
        }
    }
    return info;
}

// Group back substitution for one right-hand side: lane t holds y of its rows
// in b[s]; on return b[s] holds x of its rows.  x_i is formed by the owner of
// row i (times RN(1/u_ii), or a division on the tiny path) and broadcast.
template <int N, int T>
__device__ __forceinline__ void lu_group_backsolve(const double (&a)[Group<N, T>::K][N],
                                                   double (&b)[Group<N, T>::K],
                                                   const double (&rcp)[Group<N, T>::K], int t,
                                                   int lane0, bool tiny)
{
    constexpr int K = Group<N, T>::K;
    const bool any_tiny = __any_sync(0xffffffffu, tiny);
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        const int owner = i % T;
        const int slot = i / T;
        double xi;
        if (!any_tiny) {
            xi = __dmul_rn(b[slot], rcp[slot]);
        } else {
            xi = tiny ? __ddiv_rn(b[slot], a[slot][i]) : __dmul_rn(b[slot], rcp[slot]);
        }
        xi = __shfl_sync(0xffffffffu, xi, lane0 + owner);
        if (t == owner) b[slot] = xi;
        const double nxi = neg(xi);
#pragma unroll
        for (int s = 0; s < K; ++s) {
            if (s * T < i) {  // some lane of this slot has a row below i
                const int r = t + s * T;
                if (r < i) b[s] = __fma_rn(a[s][i], nxi, b[s]);
            }
        }
    }
}

}  // namespace dev
}  // namespace tl

// ===========================================================================
// Public device-callable API: the LUpp solve of Sec. 2.2 called per system
// from a user's own kernel (the device-callable form of Sec. 2.3, used the
// same way inside the fused Newton loop of Algorithm 2).  Arithmetic: first
// maximum of |a_ik| as pivot, l_ik = a_ik * RN(1/a_kk) (a quotient when
// |a_kk| < DBL_MIN), one fma per update in increasing k, then
// x_i = y_i * RN(1/u_ii); the pivots and info equal those of the textbook
// elimination in this arithmetic bit for bit.
// ===========================================================================
namespace tl {

// One system per calling thread, held in its registers (N <= 9 keeps the
// matrix in registers without spilling).
//   a     a[i][j] = A_ij on entry; destroyed.
//   b     the right-hand side on entry, x on return (NaN when info != 0).
//   ipiv  on return ipiv[k] = the 1-based row interchanged with row k at
//         step k (LAPACK convention).
// Returns info: 0; k + 1 when the pivot of step k is exactly zero (the first
// such k; the factorization completes); -1 when A holds a NaN or an
// infinity (nothing factored, ipiv the identity).
template <int N>
__device__ __forceinline__ int lupp_solve(double (&a)[N][N], double (&b)[N], int (&ipiv)[N])
{
    int piv[N];
    const int info = dev::lupp_solve<N>(a, b, piv);
#pragma unroll
    for (int k = 0; k < N; ++k) ipiv[k] = piv[k] + 1;
    return info;
}

// T consecutive lanes per system (T = 2, 4, 8, 16 or 32; the 32 / T groups
// of a warp each solve their own system).  Lane t of a group holds the rows
// t, t + T, t + 2T, ...: a[s][j] = A_{t+sT, j} and b[s] = b_{t+sT}; slots of
// rows past N are ignored.  On return b[s] = x_{t+sT} (NaN when
// info != 0) and ipiv[s] = the 1-based row interchanged at step t + sT.
// Returns info (as lupp_solve) on every lane of the group.  Every lane of
// the warp must call it together (the pivot search and the row interchanges
// are shuffles); a group without a system of its own passes any finite
// values and ignores the result.
template <int N, int T>
__device__ __forceinline__ int lupp_solve_subwarp(double (&a)[dev::Group<N, T>::K][N],
                                                  double (&b)[dev::Group<N, T>::K],
                                                  int (&ipiv)[dev::Group<N, T>::K])
{
    constexpr int K = dev::Group<N, T>::K;
    const int lane = static_cast<int>(threadIdx.x) & 31;
    const int t = lane % T;
    const int lane0 = lane - t;
    int bad = 0;
#pragma unroll
    for (int s = 0; s < K; ++s) {
        const bool row = t + s * T < N;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            if (!row) a[s][j] = 0.0;
            bad |= dev::is_nonfinite(a[s][j]) ? 1 : 0;
        }
        if (!row) b[s] = 0.0;
    }
#pragma unroll
    for (int off = T / 2; off >= 1; off >>= 1) bad |= __shfl_xor_sync(0xffffffffu, bad, off);
    int pivk[K];
    double rcp[K];
    bool tiny = false;
    int info = dev::lu_group_factor<N, T, false, 1>(a, b, pivk, rcp, t, lane0, tiny);
    dev::lu_group_backsolve<N, T>(a, b, rcp, t, lane0, tiny);
    if (bad) info = -1;
#pragma unroll
    for (int s = 0; s < K; ++s) {
        ipiv[s] = (bad ? t + s * T : pivk[s]) + 1;
        if (info != 0) b[s] = dev::nan_value();
    }
    return info;
}

}  // namespace tl
