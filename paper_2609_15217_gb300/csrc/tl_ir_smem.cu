// tl_ir_smem.cu -- the mixed-precision ragged solve (binary32 factor,
// binary64 refinement: the scheme and the operation order stated in
// tl_ir.cuh) with one system per warp and the binary32 copy of the system
// in shared memory, factored in place with its pivots and reciprocals.  The
// binary64 A stays in global memory (the residuals re-read it from L2, which
// keeps the shared memory per system small and the occupancy high).  The
// binary32 elimination works on an 8 x 4 lane tile (lane (tr, tc) keeps its
// columns of the pivot row in registers and walks the rows tr, tr + 8, ...);
// the pivot search, the solves and the residuals keep row i in lane i.  Rows
// are interchanged physically, so the solves apply the whole permutation
// first (one shuffle) and then the column-oriented substitutions: per entry
// the same operations in the same order as the register kernels, hence the
// same bits.
#include <cmath>

#include "tinylu.h"
#include "tl_handle.h"
#include "tl_internal.h"
#include "tl_ir.cuh"
#include "tl_smem.cuh"

namespace tl {
namespace {

// Row stride of the binary32 block: >= n and 4 modulo 8, so that the 32
// accesses of the 8 x 4 lane tile fall in 32 distinct banks.
__host__ __device__ constexpr int ir_row_stride32(int n) { return n + ((4 - n % 8) + 8) % 8; }

// Shared memory of one system in 4-byte words: A32 (n rows of
// ir_row_stride32(n) floats), 32 reciprocals, 32 pivots.
__host__ __device__ constexpr int ir_smem_words(int n) { return n * ir_row_stride32(n) + 64; }

// Binary32 solve with the factors in F (rows in pivoted order, L unit lower
// below the diagonal, U on and above it) of the right-hand side whose
// entry `src` (row src of the original order) this lane reads from y.
// Lane i returns x_i.
__device__ __forceinline__ float ir_solve32(const float *F, int R32, const float *rcp, int n, int lane, int src,
                                            float y)
{
    y = __shfl_sync(0xffffffffu, y, src);
    const float *Fi = F + lane * R32;
    for (int j = 0; j + 1 < n; ++j) {
        const float yj = __shfl_sync(0xffffffffu, y, j);
        if (lane > j && lane < n) y = __fmaf_rn(-Fi[j], yj, y);
    }
    for (int i = n - 1; i >= 0; --i) {
        const float xi = __shfl_sync(0xffffffffu, __fmul_rn(y, rcp[i]), i);
        if (lane == i) y = xi;
        if (lane < i) y = __fmaf_rn(-Fi[i], xi, y);
    }
    return y;
}

__device__ __forceinline__ bool warp_any_nonfinite(float y, int lane, int n)
{
    return __any_sync(0xffffffffu, lane < n && ir::magf(y) >= ir::kF32InfBits);
}

// One persistent launch per size n over the bucket of systems of size n;
// every warp takes systems warp, warp + nwarps, ... on its own (no block
// barrier).
__global__ void __launch_bounds__(128) k_smem_ir(RaggedArgs r, int n)
{
    extern __shared__ float smem32[];
    const int lane = threadIdx.x & 31;
    const int R32 = ir_row_stride32(n);
    const int64_t beg = r.offsets[n];
    const int64_t count = r.offsets[n + 1] - beg;
    const double cte_n = sqrt(static_cast<double>(n)) * 0x1p-53;
    float *M32 = smem32 + (threadIdx.x >> 5) * ir_smem_words(n);
    float *rcp = M32 + n * R32;
    int *piv = reinterpret_cast<int *>(rcp + 32);
    float *Mrow = M32 + lane * R32;  // this lane's row (lane < n)
    constexpr int TC = 4, TR = 8, MAXC = 8;  // lane tile; MAXC * TC >= TL_MAX_N
    const int tr = lane / TC, tc = lane % TC;
    const bool row_lane = lane < n;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;

    for (int64_t q = warp; q < count; q += nwarps) {                      // warp-uniform trip
        const int64_t sidx = r.bucket[beg + q];
        const double *Acol = r.A + r.a_off[sidx] + lane;  // a_ij at Acol[j * n] for i = lane
        // load column by column (coalesced over the column-major source)
        // with the range checks of the binary32 copy, and the binary32 row
        // sum of |a32_ij| in increasing j
        bool bad = false;
        float rs = 0.0f;
        if (row_lane) {
            for (int j = 0; j < n; ++j) {
                const double v = Acol[j * n];
                const unsigned long long m = dev::mag_bits(v);
                const float f = __double2float_rn(v);
                const unsigned fm = ir::magf(f);
                bad = bad || m >= dev::kInfBits || (m != 0ULL && !(fm >= ir::kF32MinBits && fm < ir::kF32InfBits));
                Mrow[j] = f;
                rs = __fadd_rn(rs, __uint_as_float(fm));
            }
        }
        const double bi = row_lane ? ld_stream(r.b + r.b_off[sidx] + lane) : 0.0;
        const unsigned rsb = __reduce_max_sync(0xffffffffu, ir::magf(rs));      // anrm
        bad = __any_sync(0xffffffffu, bad) || rsb >= ir::kF32InfBits;
        const double cte = __dmul_rn(static_cast<double>(__uint_as_float(rsb)), cte_n);
        __syncwarp();

        // binary32 LUpp in place: first maximum of the magnitude bits (the
        // largest magnitude, then the smallest row), l_ik = a_ik * RN32(1/p),
        // a_ij = fmaf(-l_ik, u_kj, a_ij)
        for (int k = 0; k < n; ++k) {
            const bool cand = lane >= k && row_lane;
            const float ak = cand ? Mrow[k] : 0.0f;
            const unsigned mag = ir::magf(ak);
            const unsigned mmax = __reduce_max_sync(0xffffffffu, mag);
            const int p = static_cast<int>(__reduce_min_sync(0xffffffffu, cand && mag == mmax ? lane : 32u));
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
            // lane tc = 0 of each row computes the multiplier, hands it to the
            // other three lanes of the row and stores it
            const int ncols = n - (k + 1);
            const int nfull = ncols / TC;
            const bool has_tail = tc < ncols - nfull * TC;
            const float *urow = M32 + k * R32 + k + 1 + tc;
            float u[MAXC];
#pragma unroll
            for (int c = 0; c < MAXC; ++c) u[c] = c < nfull ? urow[c * TC] : 0.0f;
            const float ut = has_tail ? urow[nfull * TC] : 0.0f;
            for (int i = k + 1 + tr; i < n; i += TR) {
                float *Mi = M32 + i * R32;
                float l = 0.0f;
                if (tc == 0) l = __fmul_rn(Mi[k], rk);
                l = __shfl_sync(0xfu << (lane & ~3), l, lane & ~3);
                const float nl = -l;
                float *Mr = Mi + k + 1 + tc;
                switch (nfull) {
#define TL_IR_CHUNK(c) \
    case (c) + 1: Mr[(c) * TC] = __fmaf_rn(nl, u[c], Mr[(c) * TC]); [[fallthrough]];
                    TL_IR_CHUNK(7)
                    TL_IR_CHUNK(6)
                    TL_IR_CHUNK(5)
                    TL_IR_CHUNK(4)
                    TL_IR_CHUNK(3)
                    TL_IR_CHUNK(2)
                    TL_IR_CHUNK(1)
                    TL_IR_CHUNK(0)
#undef TL_IR_CHUNK
                default: break;
                }
                if (has_tail) Mr[nfull * TC] = __fmaf_rn(nl, ut, Mr[nfull * TC]);
                if (tc == 0) Mi[k] = l;
            }
            __syncwarp();
        }
        // where row `lane` of the pivoted order comes from: the interchanges
        // k = 0, 1, ... applied to the original rows, traced backwards
        int src = lane;
        for (int k = n - 1; k >= 0; --k) {
            const int p = piv[k];
            src = src == k ? p : (src == p ? k : src);
        }

        // x0 = widen(solve(RN32(b))), then up to kMaxCorrections corrections
        // from binary64 residuals r_i = b_i - sum_j a_ij x_j (j increasing)
        float y = ir_solve32(M32, R32, rcp, n, lane, src, __double2float_rn(bi));
        bad = bad || warp_any_nonfinite(y, lane, n);
        double xi = static_cast<double>(y);
        int steps = -1;
        for (int it = 0; !bad; ++it) {                                    // warp-uniform
            double ri = bi;
#pragma unroll 4
            for (int j = 0; j < n; ++j) {
                const double nxj = dev::neg(__shfl_sync(0xffffffffu, xi, j));
                if (row_lane) ri = __fma_rn(Acol[j * n], nxj, ri);
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
            y = ir_solve32(M32, R32, rcp, n, lane, src, __double2float_rn(ri));
            bad = warp_any_nonfinite(y, lane, n);
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
            const int slot = atomicAdd(r.fb_count + n, 1);
            if (slot < count) r.fb_list[beg + slot] = static_cast<int32_t>(sidx);
            if (r.refine) r.refine[sidx] = -1;
        }
        __syncwarp();
    }
}

struct RegistrarIrSmem {
    RegistrarIrSmem()
    {
        for (int n = 2; n <= TL_MAX_N; ++n)
            register_variant(n, kPerSystem, kOpRaggedIr, 32, reinterpret_cast<const void *>(&k_smem_ir), 1);
    }
};
const RegistrarIrSmem registrar_ir_smem_instance;

}  // namespace

size_t ir_smem_bytes_per_system(int n) { return static_cast<size_t>(ir_smem_words(n)) * 4; }

}  // namespace tl
