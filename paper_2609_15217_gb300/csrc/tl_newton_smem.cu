// tl_newton_smem.cu -- fused per-point Newton integration of the tanh law
// (Algorithm 2) for 25 <= n <= 32 with the Jacobian in shared memory: one
// point per warp, the LUpp of the shared-memory solver (smem_lupp, 32 lanes,
// run-time n).  Per iteration lane i assembles row i of F and J
// (F_i = sum_j a_ij x_j + c_i tanh(x_i) - b_i with the sum as fma in
// increasing j; J = A + diag(c .* (1 - tanh^2 x))) into the augmented block
// [J | -F], the warp factors it and solves for dx, and lane i updates x_i.
// ||F||_2 is a warp sum of F_i^2.  Persistent: a warp that finishes a point
// stores it and takes the next one.
#include <cmath>

#include "tinylu.h"
#include "tl_handle.h"
#include "tl_internal.h"
#include "tl_newton.cuh"
#include "tl_smem.cuh"

namespace tl {
namespace {

constexpr int kWarpsPerBlock = 4;

// Smallest n run by this kernel (the sub-warp register kernels take the
// sizes below it: measured faster up to n = 24, where their 8-lane groups
// keep eight points per warp; at n = 32 this kernel is 1.23x faster than
// 16-lane groups).
#ifndef TL_NEWTON_SMEM_MIN_N
#define TL_NEWTON_SMEM_MIN_N 25
#endif

// Shared memory per point: the solver's block plus 32 doubles of x.
__host__ __device__ constexpr int newton_smem_doubles(int n) { return smem_sys_doubles(n, 32) + 32; }

__global__ void __launch_bounds__(128) k_newton_tanh_smem(NewtonBatch B, int n)
{
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    double *M = smem + w * newton_smem_doubles(n);
    double *xs = M + smem_sys_doubles(n, 32);
    const int RS = smem_row_stride(n);
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * kWarpsPerBlock;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * kWarpsPerBlock + w; g < B.total; g += nwarps) {
        const NewtonJob jb = load_job(B, g);
        const double *in = jb.in;
        const int64_t np = jb.npoints, p = g - jb.start;
        const bool mine = lane < n;
        if (mine) xs[lane] = 0.0;
        const double ci = mine ? in[(n * n + lane) * np + p] : 0.0;
        const double bi = mine ? in[(n * n + n + lane) * np + p] : 0.0;
        __syncwarp();
        double r0 = 0.0;
        int k = 0, st = -1;
        for (bool fresh = true;; fresh = false) {
            // assemble row `lane` of [J | -F]
            double acc = 0.0;
            const double xi = mine ? xs[lane] : 0.0;
            const double ti = mine ? tanh(xi) : 0.0;
            for (int j = 0; j < n; ++j) {
                const double aij = mine ? in[(j * n + lane) * np + p] : 0.0;
                acc = fma(aij, xs[j], acc);
                if (mine) M[lane * RS + j] = (j == lane) ? fma(ci, fma(-ti, ti, 1.0), aij) : aij;
            }
            const double Fi = mine ? fma(ci, ti, acc) - bi : 0.0;
            if (mine) M[lane * RS + n] = dev::neg(Fi);
            double ss = Fi * Fi;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
            const double r = sqrt(ss);
            if (fresh) r0 = r;
            st = newton_decide<32>(r, r0, k, B.rtol, B.max_iter);
            if (st >= 0) break;                        // warp-uniform: r is the same on every lane
            __syncwarp();
            const int info = smem_lupp2<32, true, false>(M, n, RS, lane, 0, 0.0);
            if (info != 0) {
                st = TL_NEWTON_SINGULAR;
                break;
            }
            if (mine) xs[lane] = xi + M[lane * RS + n];
            ++k;
            __syncwarp();
        }
        if (mine) jb.x[lane * np + p] = xs[lane];
        if (lane == 0) {
            jb.iters[p] = k;
            jb.status[p] = st;
        }
        __syncwarp();
    }
}

}  // namespace

// Shared-memory tanh Newton for n in TL_NEWTON_SMEM_MIN_N..32 (false when n
// is outside).
bool newton_tanh_smem_launch(tl_handle *h, int n, const NewtonBatch &B, cudaStream_t stream, tl_status *out)
{
    if (n < TL_NEWTON_SMEM_MIN_N || n > TL_MAX_N) return false;
    const void *kern = reinterpret_cast<const void *>(&k_newton_tanh_smem);
    int limit = 0;
    tl_status st = smem_opt_in(h, kern, &limit);
    if (st != TL_OK) {
        *out = st;
        return true;
    }
    const size_t smem = static_cast<size_t>(kWarpsPerBlock) * newton_smem_doubles(n) * 8;
    if (smem > static_cast<size_t>(limit)) {
        *out = TL_ERR_UNSUPPORTED;
        return true;
    }
    const int nb = blocks_per_sm(h, kern, 32 * kWarpsPerBlock, smem);
    const int64_t need = (B.total + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int64_t resident = static_cast<int64_t>(nb < 1 ? 1 : nb) * h->sm_count;
    const unsigned grid = static_cast<unsigned>(need < resident ? need : resident);
    NewtonBatch arg = B;
    int n_arg = n;
    void *params[] = {&arg, &n_arg};
    const cudaError_t e = cudaLaunchKernel(kern, dim3(grid), dim3(32 * kWarpsPerBlock), params, smem, stream);
    *out = e == cudaSuccess ? TL_OK : fail_cuda(h, e);
    return true;
}

}  // namespace tl
