// tl_newton_cpu_driven.cu -- the batched, CPU-driven evaluation of
// Algorithm 1 of the paper, kept as the comparator of the fused kernel:
// every Newton iteration is three launches -- assemble F and J for every
// point, one batched LUpp solve (tl_gesv_batched) over ALL points, update --
// followed by a device-to-host copy of the number of points still iterating
// that the host waits for before deciding to loop (Sec. 2.4: converged points
// keep being dragged through the batched solve until the last one stops).
//
// Per point the arithmetic is that of tl_newton_integrate: the same law code,
// the same convergence test and update, and an LUpp whose pivots and factors
// are bit-identical to the fused kernel's.
#include <cmath>

#include "tinylu.h"
#include "tinylu_device.cuh"
#include "tl_handle.h"
#include "tl_internal.h"
#include "tl_norton.cuh"

namespace tl {
namespace {

constexpr int kActive = -1;

// Step A: assemble at x for the points still iterating, run the convergence
// test, and lay J and -F out for the batched solve (interleaved, ld = ldj).
__global__ void k_cd_assemble(NortonParams P, int64_t npoints, const double *__restrict__ in,
                              double *__restrict__ x, double *__restrict__ sigout, int32_t *__restrict__ iters,
                              int32_t *__restrict__ status, double *__restrict__ r0buf, double *__restrict__ J,
                              double *__restrict__ rhs, int64_t ldj, double rtol, int max_iter, int first,
                              unsigned long long *__restrict__ active_count)
{
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    bool still = false;
    if (p < npoints) {
        int st = first ? kActive : status[p];
        if (st == kActive) {
            double sig0[6], deps[6], xv[7], F[7], Jm[7][7], sig[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) sig0[i] = in[i * npoints + p];
#pragma unroll
            for (int i = 0; i < 6; ++i) deps[i] = in[(6 + i) * npoints + p];
            if (first) {
#pragma unroll
                for (int i = 0; i < 6; ++i) xv[i] = deps[i];
                xv[6] = 0.0;
                iters[p] = 0;
            } else {
#pragma unroll
                for (int i = 0; i < 7; ++i) xv[i] = x[i * npoints + p];
            }
            norton_eval(P, sig0, deps, xv, F, Jm, sig);
            const double r = norm2<7>(F);
            if (first) r0buf[p] = r;
            const double r0 = first ? r : r0buf[p];
            const int k = first ? 0 : iters[p];
            if (!isfinite(r)) st = TL_NEWTON_NONFINITE;
            else if (r <= rtol * r0 || r0 == 0.0) st = TL_NEWTON_CONVERGED;
            else if (k >= max_iter) st = TL_NEWTON_MAX_ITER;
            if (st == kActive) {
                still = true;
#pragma unroll
                for (int j = 0; j < 7; ++j)
#pragma unroll
                    for (int i = 0; i < 7; ++i) J[static_cast<int64_t>(j * 7 + i) * ldj + p] = Jm[i][j];
#pragma unroll
                for (int i = 0; i < 7; ++i) rhs[static_cast<int64_t>(i) * ldj + p] = dev::neg(F[i]);
            } else {
                // stopped: keep dragging a well-defined system through the
                // batched solve
#pragma unroll
                for (int j = 0; j < 7; ++j)
#pragma unroll
                    for (int i = 0; i < 7; ++i) J[static_cast<int64_t>(j * 7 + i) * ldj + p] = (i == j) ? 1.0 : 0.0;
#pragma unroll
                for (int i = 0; i < 7; ++i) rhs[static_cast<int64_t>(i) * ldj + p] = 0.0;
            }
            // x in memory is the current iterate from here on (the update
            // kernel adds dx to it); the stress is that of the current
            // iterate, so it is final whenever the point stops, including
            // a singular solve found by the update kernel
            if (first) {
#pragma unroll
                for (int i = 0; i < 7; ++i) x[i * npoints + p] = xv[i];
            }
            if (sigout) {
#pragma unroll
                for (int i = 0; i < 6; ++i) sigout[i * npoints + p] = sig[i];
            }
            status[p] = st;
        }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, still);
    if ((threadIdx.x & 31) == 0 && mask) atomicAdd(active_count, static_cast<unsigned long long>(__popc(mask)));
}

// Step C: x += dx for the points still iterating (singular -> status 2).
__global__ void k_cd_update(int64_t npoints, double *__restrict__ x, const double *__restrict__ dx, int64_t ldj,
                            const int32_t *__restrict__ info, int32_t *__restrict__ iters,
                            int32_t *__restrict__ status)
{
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= npoints || status[p] != kActive) return;
    if (info[p] != 0) {
        status[p] = TL_NEWTON_SINGULAR;
        return;
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) x[i * npoints + p] += dx[static_cast<int64_t>(i) * ldj + p];
    iters[p] += 1;
}

}  // namespace
}  // namespace tl

using namespace tl;

extern "C" tl_status tl_newton_integrate_cpu_driven(tl_handle *h, const tl_law *law, int64_t npoints,
                                                    const double *inputs, double *x, double *outputs,
                                                    int32_t *iterations, int32_t *status, double rtol,
                                                    int max_iter, cudaStream_t stream)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (!law) return fail_arg(h, 2);
    if (law->id == TL_LAW_TANH) return TL_ERR_UNSUPPORTED;
    NortonParams P;
    if (!norton_params_from_law(*law, &P)) return fail_arg(h, 2);
    if (npoints < 0) return fail_arg(h, 3);
    if (!(rtol >= 0.0)) return fail_arg(h, 9);
    if (max_iter < 0) return fail_arg(h, 10);
    if (npoints == 0) return TL_OK;
    if (!inputs || (reinterpret_cast<uintptr_t>(inputs) & 7)) return fail_arg(h, 4);
    if (!x || (reinterpret_cast<uintptr_t>(x) & 7)) return fail_arg(h, 5);
    if (outputs && (reinterpret_cast<uintptr_t>(outputs) & 7)) return fail_arg(h, 6);
    if (!iterations || (reinterpret_cast<uintptr_t>(iterations) & 3)) return fail_arg(h, 7);
    if (!status || (reinterpret_cast<uintptr_t>(status) & 3)) return fail_arg(h, 8);

    // workspace: J (49 ld), rhs (7 ld), dx (7 ld), r0 (npoints), ipiv (7 ld),
    // info (npoints), counter
    const int64_t ld = (npoints + 31) / 32 * 32;
    const size_t nJ = 49 * ld, nv = 7 * ld;
    const size_t bytes = (nJ + 2 * nv + npoints) * sizeof(double) + (nv + npoints) * sizeof(int32_t) + 256;
    tl_status st = ensure_workspace(h, bytes, stream);
    if (st != TL_OK) return st;
    double *J = static_cast<double *>(h->ws);
    double *rhs = J + nJ;
    double *dx = rhs + nv;
    double *r0 = dx + nv;
    int32_t *ipiv = reinterpret_cast<int32_t *>(r0 + npoints);
    int32_t *info = ipiv + nv;
    unsigned long long *counter =
        reinterpret_cast<unsigned long long *>((reinterpret_cast<uintptr_t>(info + npoints) + 255) & ~uintptr_t(255));
    if (!h->host_stage[0]) {
        if (cudaMallocHost(&h->host_stage[0], 256) != cudaSuccess) {
            cudaGetLastError();
            return TL_ERR_NO_MEMORY;
        }
    }
    unsigned long long *host_count = static_cast<unsigned long long *>(h->host_stage[0]);

    const int block = 128;
    const unsigned grid = static_cast<unsigned>((npoints + block - 1) / block);
    for (int it = 0;; ++it) {
        cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream);
        if (e != cudaSuccess) return fail_cuda(h, e);
        k_cd_assemble<<<grid, block, 0, stream>>>(P, npoints, inputs, x, outputs, iterations, status, r0, J, rhs,
                                                  ld, rtol, max_iter, it == 0 ? 1 : 0, counter);
        // Algorithm 1: the convergence information goes back to the host
        e = cudaMemcpyAsync(host_count, counter, sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return fail_cuda(h, e);
        if (*host_count == 0) break;
        st = tl_gesv_batched(h, 7, J, nullptr, rhs, dx, ipiv, info, TL_LAYOUT_INTERLEAVED, ld, npoints, stream);
        if (st != TL_OK) return st;
        k_cd_update<<<grid, block, 0, stream>>>(npoints, x, dx, ld, info, iterations, status);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(h, e);
    }
    return TL_OK;
}
