// tl_ir_smem.cuh -- the mixed-precision ragged solve (binary32 factor,
// binary64 refinement: the scheme and the operation order stated in
// tl_ir.cuh) with one system per warp, compiled for one n.  The binary32
// copy of the system lives in shared memory and is factored in place with
// its pivots and reciprocals; the binary64 A stays in global memory (the
// residuals re-read it from L2, which keeps the shared memory per system
// small and the occupancy high).  The binary32 elimination works on an
// 8 x 4 lane tile (lane (tr, tc) keeps its columns of the pivot row in
// registers and walks the rows tr, tr + 8, ...); the pivot search, the
// solves and the residuals keep row i in lane i.  Rows are interchanged
// physically, so the solves apply the whole permutation first (one
// shuffle) and then the column-oriented substitutions: per entry the same
// operations in the same order as the register kernels, hence the same
// bits.  n is known at compile time: every loop but the factorization's
// step loop is unrolled, with immediate shared-memory offsets.
#pragma once
#include "tl_ir.cuh"

namespace tl {

// Row stride of the binary32 block: >= n and 4 modulo 8, so that the 32
// accesses of the 8 x 4 lane tile fall in 32 distinct banks.
__host__ __device__ constexpr int ir_row_stride32(int n) { return n + ((4 - n % 8) + 8) % 8; }

// Shared memory of one system in 4-byte words: A32 (n rows of
// ir_row_stride32(n) floats), 32 reciprocals, 32 pivots.
__host__ __device__ constexpr int ir_smem_words(int n) { return n * ir_row_stride32(n) + 64; }
inline size_t ir_smem_bytes_per_system(int n) { return static_cast<size_t>(ir_smem_words(n)) * 4; }

namespace irs {

// Binary32 solve with the factors whose row `lane` starts at Mrow (rows in
// pivoted order, L unit lower below the diagonal, U above it, rcp_own =
// RN32(1/u_ii) of this lane's row) of the right-hand side whose original
// row `src` this lane reads from y.  Lane i returns x_i.
template <int N>
__device__ __forceinline__ float solve32(const float *Mrow, float rcp_own, int lane, int src, float y)
{
    y = __shfl_sync(0xffffffffu, y, src);
#pragma unroll
    for (int j = 0; j + 1 < N; ++j) {
        const float yj = __shfl_sync(0xffffffffu, y, j);
        if (lane > j && lane < N) y = __fmaf_rn(-Mrow[j], yj, y);
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        const float xi = __shfl_sync(0xffffffffu, __fmul_rn(y, rcp_own), i);
        if (lane == i) y = xi;
        if (lane < i) y = __fmaf_rn(-Mrow[i], xi, y);
    }
    return y;
}

__device__ __forceinline__ bool any_nonfinite(float y, bool row_lane)
{
    return __any_sync(0xffffffffu, row_lane && ir::magf(y) >= ir::kF32InfBits);
}

}  // namespace irs

// One persistent launch over the bucket of systems of size N; every warp
// takes systems warp, warp + nwarps, ... on its own (no block barrier).
// 8 blocks per SM (64 registers; a few bytes of spill at n = 20..28):
// measured 1-3% faster than 7 blocks at 72 registers for n = 17..28.
// The int argument (the size, passed by the shared-memory launcher) is N.
template <int N>
__global__ void __launch_bounds__(128, 8) k_smem_ir(RaggedArgs r, int)
{
    constexpr int R32 = ir_row_stride32(N);
    constexpr int TC = 4, TR = 8;  // lane tile
    extern __shared__ float smem32[];
    const int lane = threadIdx.x & 31;
    const int tr = lane / TC, tc = lane % TC;
    const bool row_lane = lane < N;
    const int64_t beg = r.offsets[N];
    const int64_t count = r.offsets[N + 1] - beg;
    const double cte_n = sqrt(static_cast<double>(N)) * 0x1p-53;
    float *M32 = smem32 + (threadIdx.x >> 5) * ir_smem_words(N);
    float *rcp = M32 + N * R32;
    int *piv = reinterpret_cast<int *>(rcp + 32);
    float *Mrow = M32 + lane * R32;         // row `lane` (lane < N)
    float *Mtile = M32 + tr * R32 + tc;     // + (k + 1) (R32 + 1): row k + 1 + tr, column k + 1 + tc
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;

    for (int64_t q = warp; q < count; q += nwarps) {                      // warp-uniform trip
        const int64_t sidx = r.bucket[beg + q];
        const double *Acol = r.A + r.a_off[sidx] + lane;  // a_ij at Acol[j * N] for i = lane
        // load column by column (coalesced over the column-major source)
        // with the range checks of the binary32 copy, and the binary32 row
        // sum of |a32_ij| in increasing j
        unsigned badv = 0u;
        float rs = 0.0f;
        if (row_lane) {
#pragma unroll 8
            for (int j = 0; j < N; ++j) {
                const double v = Acol[j * N];
                const unsigned long long m = dev::mag_bits(v);
                const float f = __double2float_rn(v);
                const unsigned fm = ir::magf(f);
                badv |= static_cast<unsigned>(m >= dev::kInfBits) |
                        (static_cast<unsigned>(m != 0ULL) & static_cast<unsigned>(fm - ir::kF32MinBits >=
                                                                               ir::kF32InfBits - ir::kF32MinBits));
                Mrow[j] = f;
                rs = __fadd_rn(rs, __uint_as_float(fm));
            }
        }
        const double bi = row_lane ? ld_stream(r.b + r.b_off[sidx] + lane) : 0.0;
        const unsigned rsb = __reduce_max_sync(0xffffffffu, ir::magf(rs));      // anrm
        bool bad = __any_sync(0xffffffffu, badv != 0u) || rsb >= ir::kF32InfBits;
        const double cte = __dmul_rn(static_cast<double>(__uint_as_float(rsb)), cte_n);
        __syncwarp();

        // binary32 LUpp in place: first maximum of the magnitude bits (the
        // largest magnitude, then the smallest row), l_ik = a_ik * RN32(1/p),
        // a_ij = fmaf(-l_ik, u_kj, a_ij)
        // a rolled loop: the unrolled body of n = 32 outgrows the
        // instruction cache (measured: the same speed, 8 registers fewer)
#pragma unroll 1
        for (int k = 0; k < N; ++k) {
            const bool cand = row_lane && lane >= k;
            const float ak = cand ? Mrow[k] : 0.0f;
            const unsigned mag = ir::magf(ak);
            const unsigned mmax = __reduce_max_sync(0xffffffffu, mag);
            const int p = static_cast<int>(
                __reduce_min_sync(0xffffffffu, cand && mag == mmax ? static_cast<unsigned>(lane) : 32u));
            const float pv = __shfl_sync(0xffffffffu, ak, p);
            bad = bad || !(mmax >= ir::kF32MinBits && mmax < ir::kF32InfBits);
            if (p != k && row_lane) {
                const float t = M32[k * R32 + lane];
                M32[k * R32 + lane] = M32[p * R32 + lane];
                M32[p * R32 + lane] = t;
            }
            const float rk = __frcp_rn(pv);
            if (lane == 0) {
                piv[k] = p;
                rcp[k] = rk;
            }
            __syncwarp();
            const int ncols = N - 1 - k;
            if (ncols > 0) {
                const int nfull = ncols / TC, rem = ncols % TC;
                const float *urow = M32 + k * R32 + (k + 1) + tc;
                float u[(N + TC - 1) / TC];
#pragma unroll
                for (int c = 0; c < (N + TC - 1) / TC; ++c) u[c] = c < nfull ? urow[c * TC] : 0.0f;
                const float ut = tc < rem ? urow[nfull * TC] : 0.0f;
                float *base = Mtile + (k + 1) * (R32 + 1);
                // row i = k + 1 + tr + 8 m: lane tc = 0 forms l_ik and hands it
                // to the three other lanes of the row
#pragma unroll
                for (int m = 0; m < (N + TR - 2) / TR; ++m) {
                    if (m * TR >= ncols) break;  // warp-uniform
                    const bool valid = k + 1 + tr + m * TR < N;
                    float *Mr = base + m * TR * R32;                    // column k + 1 + tc
                    float l = 0.0f;
                    if (valid && tc == 0) l = __fmul_rn(Mr[-1], rk);
                    l = __shfl_sync(0xffffffffu, l, lane & ~(TC - 1));
                    if (valid) {
                        const float nl = -l;
#pragma unroll
                        for (int c = 0; c < (N + TC - 1) / TC; ++c)
                            if (c < nfull) Mr[c * TC] = __fmaf_rn(nl, u[c], Mr[c * TC]);
                        if (tc < rem) Mr[nfull * TC] = __fmaf_rn(nl, ut, Mr[nfull * TC]);
                        if (tc == 0) Mr[-1] = l;
                    }
                }
            }
            __syncwarp();
        }
        // where row `lane` of the pivoted order comes from: the interchanges
        // k = 0, 1, ... applied to the original rows, traced backwards
        int src = lane;
#pragma unroll
        for (int k = N - 1; k >= 0; --k) {
            const int p = piv[k];
            src = src == k ? p : (src == p ? k : src);
        }
        const float rcp_own = row_lane ? rcp[lane] : 1.0f;

        // x0 = widen(solve(RN32(b))), then up to kMaxCorrections corrections
        // from binary64 residuals r_i = b_i - sum_j a_ij x_j (j increasing)
        float y = irs::solve32<N>(Mrow, rcp_own, lane, src, __double2float_rn(bi));
        bad = bad || irs::any_nonfinite(y, row_lane);
        double xi = static_cast<double>(y);
        int steps = -1;
        for (int it = 0; !bad; ++it) {                                    // warp-uniform
            double ri = bi;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const double nxj = dev::neg(__shfl_sync(0xffffffffu, xi, j));
                if (row_lane) ri = __fma_rn(Acol[j * N], nxj, ri);
            }
            const unsigned long long rm = ir::gmax64<32>(row_lane ? dev::mag_bits(ri) : 0ULL);
            const unsigned long long xm = ir::gmax64<32>(row_lane ? dev::mag_bits(xi) : 0ULL);
            if (__longlong_as_double(static_cast<long long>(rm)) <=
                __dmul_rn(__longlong_as_double(static_cast<long long>(xm)), cte)) {
                steps = it;
                break;
            }
            if (it == ir::kMaxCorrections) {
                bad = true;
                break;
            }
            y = irs::solve32<N>(Mrow, rcp_own, lane, src, __double2float_rn(ri));
            bad = irs::any_nonfinite(y, row_lane);
            if (!bad) xi = __dadd_rn(xi, static_cast<double>(y));
        }
        if (!bad) {
            if (row_lane) {
                st_stream(r.x + r.b_off[sidx] + lane, xi);
                st_stream(r.ipiv + r.piv_off[sidx] + lane, piv[lane] + 1);
            }
            if (lane == 0) {
                st_stream(r.info + sidx, 0);
                if (r.refine) st_stream(r.refine + sidx, steps);
            }
        } else if (lane == 0) {
            // hand the system to the binary64 kernels
            const int slot = atomicAdd(r.fb_count + N, 1);
            if (slot < count) r.fb_list[beg + slot] = static_cast<int32_t>(sidx);
            if (r.refine) r.refine[sidx] = -1;
        }
        __syncwarp();
    }
}

}  // namespace tl
