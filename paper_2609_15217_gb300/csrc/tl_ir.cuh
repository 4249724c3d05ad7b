// tl_ir.cuh -- mixed-precision ragged solve (TL_PREC_FP32_IR of
// tl_lupp_solve_batched): factor a binary32 copy of A, solve in binary32,
// then refine the binary64 solution with binary64 residuals and binary32
// correction solves (the iterative-refinement scheme of Langou et al. 2006,
// as in LAPACK's dsgesv).  The paper itself factors in binary64 only; on
// this GPU binary32 FMAs are ~60x cheaper than binary64 ones, so the O(n^3)
// factorization moves off the FP64 pipe and only the O(n^2) residuals stay
// on it.
//
// Arithmetic, fixed operation by operation (every step one IEEE
// round-to-nearest operation in the stated format and order):
//   input    A finite; every nonzero a_ij rounds to a binary32 value in
//            [FLT_MIN, FLT_MAX]: a32_ij = RN32(a_ij).
//   norm     anrm = max over rows of the binary32 sum, j increasing, of
//            |a32_ij| (finite); cte = RN64(anrm * RN64(sqrt(n) * 2^-53)).
//   factor   binary32 LUpp with the steps of the binary64 one (first maximum
//            of the magnitude bits, l_ik = a_ik * RN32(1/a_kk), a_ij =
//            fmaf(-l_ik, a_kj, a_ij)); a pivot outside [FLT_MIN, Inf) stops.
//   solve    interchanges and unit-L forward substitution, then
//            x_i = (y_i - sum u_ij x_j) * RN32(1/u_ii), j decreasing; the
//            result must be finite.
//   refine   x = widen(solve(RN32(b))); then for it = 0..3:
//            r_i = b_i, r_i = fma(-a_ij, x_j, r_i) for j = 0..n-1;
//            stop (steps = it) when max|r_i| <= RN64(max|x_i| * cte);
//            at it = 3 give up; else x_i = RN64(x_i + widen(solve(RN32(r)))_i).
// Any failure hands the system to the binary64 LUpp (steps = -1): the kernel
// appends it to a per-size fallback list that the binary64 ragged kernels
// then process.
//
// Mapping: T consecutive lanes per system, lane t holding the rows
// t + s*T (T = 1: one thread per system, everything in its registers), as
// the binary64 group kernels.  L is kept in elimination order (only the
// trailing columns are interchanged); the solves interleave the
// interchanges with the forward elimination, which applies the same
// operations in the same order as permuting the right-hand side first.
#pragma once
#include "tl_kernels.cuh"

namespace tl {
namespace ir {

constexpr unsigned kF32MinBits = 0x00800000u;  // FLT_MIN
constexpr unsigned kF32InfBits = 0x7f800000u;  // +Inf
constexpr int kMaxCorrections = 3;

__device__ __forceinline__ unsigned magf(float v) { return __float_as_uint(v) & 0x7fffffffu; }

template <int T, typename V>
__device__ __forceinline__ V gshfl(V v, int src)
{
    if constexpr (T == 1) return v;
    else return __shfl_sync(0xffffffffu, v, src);
}

template <int T>
__device__ __forceinline__ bool gany(bool v)
{
    if constexpr (T == 1) return v;
    else return group_any<T>(v);
}

template <int T>
__device__ __forceinline__ unsigned long long gmax64(unsigned long long v)
{
#pragma unroll
    for (int off = T / 2; off >= 1; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
        v = o > v ? o : v;
    }
    return v;
}

template <int T>
__device__ __forceinline__ unsigned gmax32(unsigned v)
{
#pragma unroll
    for (int off = T / 2; off >= 1; off >>= 1) {
        const unsigned o = __shfl_xor_sync(0xffffffffu, v, off);
        v = o > v ? o : v;
    }
    return v;
}

// Binary32 LUpp of the group's rows; returns true (on every lane of the
// group) when a pivot is outside [FLT_MIN, Inf).  pivk[s] / rcp[s] receive
// the pivot row and RN32(1/u_ii) of the steps k = t + s*T this lane owns.
template <int N, int T>
__device__ __forceinline__ bool factor32(float (&a)[dev::Group<N, T>::K][N], int (&pivk)[dev::Group<N, T>::K],
                                         float (&rcp)[dev::Group<N, T>::K], int t, int lane0)
{
    constexpr int K = dev::Group<N, T>::K;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        // pivot search: this lane's first maximum, then the group butterfly
        // (ties to the smaller row)
        unsigned cb = 0u;
        int crow = N;
#pragma unroll
        for (int s = 0; s < K; ++s) {
            if (s * T < N && (T - 1) + s * T >= k) {
                const int i = t + s * T;
                const unsigned bits = __float_as_uint(a[s][k]);
                const bool take = (i >= k) && (i < N) && (crow == N || (bits & 0x7fffffffu) > (cb & 0x7fffffffu));
                cb = take ? bits : cb;
                crow = take ? i : crow;
            }
        }
#pragma unroll
        for (int off = T / 2; off >= 1; off >>= 1) {
            const unsigned ob = __shfl_xor_sync(0xffffffffu, cb, off);
            const int orow = __shfl_xor_sync(0xffffffffu, crow, off);
            const unsigned m = cb & 0x7fffffffu, om = ob & 0x7fffffffu;
            const bool take = (om > m) || (om == m && orow < crow);
            cb = take ? ob : cb;
            crow = take ? orow : crow;
        }
        const int p = crow;
        const unsigned pm = cb & 0x7fffffffu;
        bad = bad || !(pm >= kF32MinBits && pm < kF32InfBits);
        const float r = __frcp_rn(__uint_as_float(cb));
        const int owner_k = k % T, slot_k = k / T;
        if (t == owner_k) {
            pivk[slot_k] = p;
            rcp[slot_k] = r;
        }
        // interchange rows k and p over the trailing columns; the shuffle
        // that brings row p to row k broadcasts u_kj to the group
        const int owner_p = p % T, slot_p = p / T;
        float uk[N];
#pragma unroll
        for (int j = k; j < N; ++j) {
            const float vk = a[slot_k][j];
            float vp = 0.0f;
#pragma unroll
            for (int s = 0; s < K; ++s) vp = (s == slot_p) ? a[s][j] : vp;
            const float new_k = gshfl<T>(vp, lane0 + owner_p);
            const float new_p = gshfl<T>(vk, lane0 + owner_k);
            uk[j] = new_k;
#pragma unroll
            for (int s = 0; s < K; ++s) a[s][j] = (t == owner_p && s == slot_p) ? new_p : a[s][j];
            if (t == owner_k) a[slot_k][j] = new_k;
        }
        // multipliers and the Schur update of this lane's rows below k
#pragma unroll
        for (int s = 0; s < K; ++s) {
            if (dev::Group<N, T>::slot_alive(s, k)) {
                const int i = t + s * T;
                if (i > k && i < N) {
                    const float l = __fmul_rn(a[s][k], r);
                    a[s][k] = l;
#pragma unroll
                    for (int j = k + 1; j < N; ++j) a[s][j] = __fmaf_rn(-l, uk[j], a[s][j]);
                }
            }
        }
    }
    return bad;
}

// Binary32 solve with the factors of factor32, in place on y (lane t holds
// the entries t + s*T; on entry in the original row order, on return the
// solution).  All lanes of the warp must call it together.
template <int N, int T>
__device__ __forceinline__ void solve32(const float (&a)[dev::Group<N, T>::K][N],
                                        const int (&pivk)[dev::Group<N, T>::K],
                                        const float (&rcp)[dev::Group<N, T>::K], float (&y)[dev::Group<N, T>::K],
                                        int t, int lane0)
{
    constexpr int K = dev::Group<N, T>::K;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const int owner_k = k % T, slot_k = k / T;
        const int p = gshfl<T>(pivk[slot_k], lane0 + owner_k);
        const int owner_p = p % T, slot_p = p / T;
        float vp = 0.0f;
#pragma unroll
        for (int s = 0; s < K; ++s) vp = (s == slot_p) ? y[s] : vp;
        const float new_k = gshfl<T>(vp, lane0 + owner_p);
        const float new_p = gshfl<T>(y[slot_k], lane0 + owner_k);
#pragma unroll
        for (int s = 0; s < K; ++s) y[s] = (t == owner_p && s == slot_p) ? new_p : y[s];
        if (t == owner_k) y[slot_k] = new_k;
        if (k + 1 < N) {
            const float yk = new_k;  // every lane received row p's old entry = new y_k
#pragma unroll
            for (int s = 0; s < K; ++s) {
                if (dev::Group<N, T>::slot_alive(s, k)) {
                    const int i = t + s * T;
                    if (i > k && i < N) y[s] = __fmaf_rn(-a[s][k], yk, y[s]);
                }
            }
        }
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        const int owner = i % T, slot = i / T;
        const float xi = gshfl<T>(__fmul_rn(y[slot], rcp[slot]), lane0 + owner);
        if (t == owner) y[slot] = xi;
#pragma unroll
        for (int s = 0; s < K; ++s) {
            if (s * T < i) {
                const int rr = t + s * T;
                if (rr < i) y[s] = __fmaf_rn(-a[s][i], xi, y[s]);
            }
        }
    }
}

template <int N, int T>
__device__ __forceinline__ bool any_nonfinite32(const float (&y)[dev::Group<N, T>::K], int t)
{
    constexpr int K = dev::Group<N, T>::K;
    bool bad = false;
#pragma unroll
    for (int s = 0; s < K; ++s)
        if (t + s * T < N) bad = bad || magf(y[s]) >= kF32InfBits;
    return gany<T>(bad);
}

}  // namespace ir

// One persistent launch per size N over the bucket of systems of size N:
// warp-uniform loop, 32/T systems per warp and trip.
template <int N, int T>
__global__ void __launch_bounds__(128) k_ragged_ir(RaggedArgs r)
{
    constexpr int K = dev::Group<N, T>::K;
    constexpr int G = 32 / T;
    const int lane = threadIdx.x & 31;
    const int t = lane % T;
    const int lane0 = lane - t;
    const int64_t beg = r.offsets[N];
    const int64_t count = r.offsets[N + 1] - beg;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const double cte_n = sqrt(static_cast<double>(N)) * 0x1p-53;
    for (int64_t q0 = warp * G; q0 < count; q0 += nwarps * G) {
        const int64_t q = q0 + lane / T;
        const bool active = q < count;
        const int64_t s_idx = active ? r.bucket[beg + q] : 0;
        const double *A = r.A + (active ? r.a_off[s_idx] : 0);
        const double *bv = r.b + (active ? r.b_off[s_idx] : 0);

        // load: binary32 copy, range checks, row sums of |a32|
        float a[K][N];
        double bd[K];
        bool bad = false;
        unsigned anrm_bits = 0u;
#pragma unroll
        for (int sl = 0; sl < K; ++sl) {
            const int i = t + sl * T;
            const bool ok = active && i < N;
            float rs = 0.0f;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const double v = ok ? A[j * N + i] : 0.0;
                const unsigned long long m = dev::mag_bits(v);
                const float f = __double2float_rn(v);
                bad = bad || m >= dev::kInfBits || (m != 0ULL && !(ir::magf(f) >= ir::kF32MinBits && ir::magf(f) < ir::kF32InfBits));
                a[sl][j] = f;
                rs = __fadd_rn(rs, __uint_as_float(ir::magf(f)));
            }
            anrm_bits = ir::magf(rs) > anrm_bits ? ir::magf(rs) : anrm_bits;
            bd[sl] = ok ? ld_stream(bv + i) : 0.0;
        }
        anrm_bits = ir::gmax32<T>(anrm_bits);
        bad = ir::gany<T>(bad) || anrm_bits >= ir::kF32InfBits;
        const double cte = __dmul_rn(static_cast<double>(__uint_as_float(anrm_bits)), cte_n);

        int pivk[K];
        float rcp[K];
        bad = ir::factor32<N, T>(a, pivk, rcp, t, lane0) || bad;

        // x0 = widen(solve(RN32(b)))
        float y[K];
#pragma unroll
        for (int sl = 0; sl < K; ++sl) y[sl] = __double2float_rn(bd[sl]);
        ir::solve32<N, T>(a, pivk, rcp, y, t, lane0);
        // (every lane must reach the group vote: no short-circuit)
        const bool ybad = ir::any_nonfinite32<N, T>(y, t);
        bad = bad || ybad;
        double xd[K];
#pragma unroll
        for (int sl = 0; sl < K; ++sl) xd[sl] = static_cast<double>(y[sl]);

        bool fail = bad || !active;
        bool done = fail;
        int steps = -1;
#pragma unroll 1
        for (int it = 0; it <= ir::kMaxCorrections; ++it) {
            if (!__any_sync(0xffffffffu, !done)) break;
            // binary64 residual of this lane's rows (original order)
            double rr[K];
#pragma unroll
            for (int sl = 0; sl < K; ++sl) rr[sl] = bd[sl];
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const double nxj = dev::neg(ir::gshfl<T>(xd[j / T], lane0 + j % T));
#pragma unroll
                for (int sl = 0; sl < K; ++sl) {
                    const int i = t + sl * T;
                    if (sl * T < N && i < N && !done) rr[sl] = __fma_rn(A[j * N + i], nxj, rr[sl]);
                }
            }
            unsigned long long rm = 0ULL, xm = 0ULL;
#pragma unroll
            for (int sl = 0; sl < K; ++sl) {
                if (t + sl * T < N) {
                    const unsigned long long a1 = dev::mag_bits(rr[sl]), a2 = dev::mag_bits(xd[sl]);
                    rm = a1 > rm ? a1 : rm;
                    xm = a2 > xm ? a2 : xm;
                }
            }
            rm = ir::gmax64<T>(rm);
            xm = ir::gmax64<T>(xm);
            const bool conv = __longlong_as_double(static_cast<long long>(rm)) <=
                              __dmul_rn(__longlong_as_double(static_cast<long long>(xm)), cte);
            if (!done) {
                if (conv) {
                    done = true;
                    steps = it;
                } else if (it == ir::kMaxCorrections) {
                    done = true;
                    fail = true;
                }
            }
            // correction (every lane takes part in the shuffles)
#pragma unroll
            for (int sl = 0; sl < K; ++sl) y[sl] = __double2float_rn(rr[sl]);
            ir::solve32<N, T>(a, pivk, rcp, y, t, lane0);
            const bool dbad = ir::any_nonfinite32<N, T>(y, t);
            if (!done) {
                if (dbad) {
                    done = true;
                    fail = true;
                } else {
#pragma unroll
                    for (int sl = 0; sl < K; ++sl) xd[sl] = __dadd_rn(xd[sl], static_cast<double>(y[sl]));
                }
            }
        }

        if (active && !fail) {
            double *x = r.x + r.b_off[s_idx];
            int32_t *ip = r.ipiv + r.piv_off[s_idx];
#pragma unroll
            for (int sl = 0; sl < K; ++sl) {
                const int i = t + sl * T;
                if (i < N) {
                    st_stream(x + i, xd[sl]);
                    st_stream(ip + i, pivk[sl] + 1);
                }
            }
            if (t == 0) {
                st_stream(r.info + s_idx, 0);
                if (r.refine) st_stream(r.refine + s_idx, steps);
            }
        }
        // systems that failed go to the binary64 fallback list (one
        // atomic per warp)
        const bool lead_fail = active && fail && t == 0;
        const unsigned m = __ballot_sync(0xffffffffu, lead_fail);
        if (m) {
            int base = 0;
            if (lane == 0) base = atomicAdd(r.fb_count + N, __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (lead_fail) {
                const int64_t slot = base + __popc(m & ((1u << lane) - 1u));
                if (slot < count) r.fb_list[beg + slot] = static_cast<int32_t>(s_idx);
                if (r.refine) r.refine[s_idx] = -1;
            }
        }
    }
}

}  // namespace tl
