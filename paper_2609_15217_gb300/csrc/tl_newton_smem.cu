// tl_newton_smem.cu -- fused per-point Newton integration of the tanh law
// (Algorithm 2) for 11 <= n <= 32 with the Jacobian in shared memory: T
// lanes per point, 32 / T points per warp, the two-step element-walk LUpp
// of the shared-memory solver (smem_lupp2, run-time n).  Per iteration
// lane t of a point's group assembles rows t, t + T, ... of F and J
// (F_i = sum_j a_ij x_j + c_i tanh(x_i) - b_i with the sum as fma in
// increasing j; J = A + diag(c .* (1 - tanh^2 x))) into the augmented block
// [J | -F], the warp factors every group's block and solves for dx, and
// the group updates x.  ||F||_2: each lane's fma sum over its rows, then a
// butterfly over the group.  Persistent: a group whose point stops stores
// it and takes the next one of its stride.
#include <cmath>

#include "tinylu.h"
#include "tl_handle.h"
#include "tl_internal.h"
#include "tl_newton.cuh"
#include "tl_smem.cuh"

namespace tl {
namespace {

// Warps per block: 2 keeps 14 instead of 12 warps resident at n = 19..20
// (+6%); within +-2% of 1 and 4 warps elsewhere (measured at n = 10..32).
constexpr int kWarpsPerBlock = 2;

// Lanes per point of the shared-memory kernel for the tanh law at size n;
// 0 where the sub-warp register kernel runs (n = 10; n <= 9 runs one
// thread per point).  Measured on GB300 (points/s over n = 10..32 for
// every lane count and the register kernels): 4 lanes win at n = 11..14,
// 8 at 15..22, 16 at 23..28, 32 from 29; 9-56% over the register kernels.
int newton_smem_lanes(int n)
{
    if (n <= 10 || n > TL_MAX_N) return 0;
    if (n <= 14) return 4;
    if (n <= 22) return 8;
    if (n <= 28) return 16;
    return 32;
}

// Shared memory per point: the solver's block plus 32 doubles of x.
__host__ __device__ constexpr int newton_smem_doubles(int n, int T) { return smem_sys_doubles(n, T) + 32; }

// T lanes per point, 32 / T points per warp.  Every trip of the loop each
// group with a live point assembles [J | -F] of its point (lane t the rows
// t, t + T, ...), the warp factors every group's block with the shared-
// memory solver (warp-synchronous, so groups without a point factor a
// stale block and ignore it), and each group updates x, decides, and on a
// stop stores the point and takes the next one of its stride.
template <int T>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) k_newton_tanh_smem(NewtonBatch B, int n)
{
    extern __shared__ double smem[];
    constexpr int KM = TL_MAX_N / T;  // row slots per lane
    const int lane = threadIdx.x & 31;
    const int t = lane % T;
    const int per = newton_smem_doubles(n, T);
    double *M = smem + (threadIdx.x / T) * per;
    double *xs = M + smem_sys_doubles(n, T);
    const int RS = smem_row_stride(n);
    const int64_t ngroups = (static_cast<int64_t>(gridDim.x) * blockDim.x) / T;
    int64_t g = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / T;
    bool have = g < B.total;
    const double *in = nullptr;
    int64_t np = 1, p = 0;
    double r0 = 0.0;
    int k = 0;
    bool fresh = true;
    while (__any_sync(0xffffffffu, have)) {
        if (have && fresh) {
            const NewtonJob jb = load_job(B, g);
            in = jb.in;
            np = jb.npoints;
            p = g - jb.start;
            for (int i = t; i < n; i += T) xs[i] = 0.0;
            k = 0;
        }
        __syncwarp();
        // assemble this lane's rows of [J | -F]
        double ss = 0.0;
#pragma unroll
        for (int s = 0; s < KM; ++s) {
            const int i = t + s * T;
            if (have && i < n) {
                const double xi = xs[i];
                const double ti = tanh(xi);
                const double ci = in[(n * n + i) * np + p];
                const double bi = in[(n * n + n + i) * np + p];
                double acc = 0.0;
                for (int j = 0; j < n; ++j) {
                    const double aij = in[(j * n + i) * np + p];
                    acc = fma(aij, xs[j], acc);
                    M[i * RS + j] = (j == i) ? fma(ci, fma(-ti, ti, 1.0), aij) : aij;
                }
                const double Fi = fma(ci, ti, acc) - bi;
                M[i * RS + n] = dev::neg(Fi);
                ss = fma(Fi, Fi, ss);
            }
        }
#pragma unroll
        for (int off = T / 2; off >= 1; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
        const double r = sqrt(ss);
        if (have && fresh) r0 = r;
        fresh = false;
        int st = have ? newton_decide<32>(r, r0, k, B.rtol, B.max_iter) : 0;
        const bool need = have && st < 0;
        __syncwarp();
        if (__any_sync(0xffffffffu, need)) {
            const int info = smem_lupp2<T, true, false>(M, n, RS, t, 0, 0.0);
            if (need) {
                if (info != 0) {
                    st = TL_NEWTON_SINGULAR;
                } else {
                    for (int i = t; i < n; i += T) xs[i] += M[i * RS + n];
                    ++k;
                }
            }
        }
        __syncwarp();
        if (have && st >= 0) {
            const NewtonJob jb = load_job(B, g);
            for (int i = t; i < n; i += T) jb.x[i * np + p] = xs[i];
            if (t == 0) {
                jb.iters[p] = k;
                jb.status[p] = st;
            }
            g += ngroups;
            have = g < B.total;
            fresh = true;
        }
    }
}

template <int T>
tl_status launch_smem_newton(tl_handle *h, int n, const NewtonBatch &B, cudaStream_t stream)
{
    const void *kern = reinterpret_cast<const void *>(&k_newton_tanh_smem<T>);
    int limit = 0;
    const tl_status st = smem_opt_in(h, kern, &limit);
    if (st != TL_OK) return st;
    const size_t smem = static_cast<size_t>(32 * kWarpsPerBlock / T) * newton_smem_doubles(n, T) * 8;
    if (smem > static_cast<size_t>(limit)) return TL_ERR_UNSUPPORTED;
    const int nb = blocks_per_sm(h, kern, 32 * kWarpsPerBlock, smem);
    const int64_t per_block = 32 * kWarpsPerBlock / T;
    const int64_t need = (B.total + per_block - 1) / per_block;
    const int64_t resident = static_cast<int64_t>(nb < 1 ? 1 : nb) * h->sm_count;
    const unsigned grid = static_cast<unsigned>(need < resident ? need : resident);
    NewtonBatch arg = B;
    int n_arg = n;
    void *params[] = {&arg, &n_arg};
    const cudaError_t e = cudaLaunchKernel(kern, dim3(grid), dim3(32 * kWarpsPerBlock), params, smem, stream);
    return e == cudaSuccess ? TL_OK : fail_cuda(h, e);
}

}  // namespace

// Shared-memory tanh Newton for the sizes newton_smem_lanes names (false
// for the others).
bool newton_tanh_smem_launch(tl_handle *h, int n, const NewtonBatch &B, cudaStream_t stream, tl_status *out)
{
    switch (newton_smem_lanes(n)) {
    case 4: *out = launch_smem_newton<4>(h, n, B, stream); return true;
    case 8: *out = launch_smem_newton<8>(h, n, B, stream); return true;
    case 16: *out = launch_smem_newton<16>(h, n, B, stream); return true;
    case 32: *out = launch_smem_newton<32>(h, n, B, stream); return true;
    default: return false;
    }
}

}  // namespace tl
