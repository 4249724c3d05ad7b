// tl_newton.cu -- fused per-point Newton integration (Algorithm 2 of the
// paper: one kernel in which every integration point runs its own loop
// assemble F, J -> LUpp solve J dx = -F -> x += dx -> convergence test,
// Eqs. 1-3 of Sec. 2.1), and the C ABI entry tl_newton_integrate.
//
// Mapping: one thread per point, the 7x7 Jacobian and its LUpp in registers
// (lupp_solve<7> of tl_device.cuh).  Threads are persistent: when a point
// stops (converged, iteration cap, singular, non-finite) its thread stores
// the results and takes the next point of its stride, so a lane idles for one
// solve per point instead of waiting for the slowest point of its warp (the
// divergence the paper attributes to the device-callable paradigm, Sec. 2.4).
#include <cmath>

#include "tinylu.h"
#include "tl_device.cuh"
#include "tl_handle.h"
#include "tl_internal.h"
#include "tl_norton.cuh"

namespace tl {
namespace {

struct NortonState {
    double sig0[6], deps[6], x[7];
};
struct Solve7 {
    double dx[7];
    int info;
};

// Exact general path of one Newton solve (a zero, tiny, huge or non-finite
// pivot met by the fast path): rebuild F and J at x and solve with the
// general LUpp.  Out of line so that it does not weigh on the fast path.
static __device__ __noinline__ Solve7 slow_norton_solve(NortonParams P, NortonState st)
{
    double F[7], J[7][7], sig[6], rhs[7];
    norton_eval(P, st.sig0, st.deps, st.x, F, J, sig);
#pragma unroll
    for (int i = 0; i < 7; ++i) rhs[i] = dev::neg(F[i]);
    int piv[7];
    Solve7 out;
    out.info = dev::lupp_solve<7>(J, rhs, piv);
#pragma unroll
    for (int i = 0; i < 7; ++i) out.dx[i] = rhs[i];
    return out;
}


__global__ void __launch_bounds__(128) k_newton_norton(NortonParams P, int64_t npoints, const double *__restrict__ in,
                                                       double *__restrict__ xout, double *__restrict__ sigout,
                                                       int32_t *__restrict__ iters, int32_t *__restrict__ status,
                                                       double rtol, int max_iter)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= npoints) return;

    double sig0[6], deps[6], x[7], F[7], J[7][7], sig[6];
    double r0 = 0.0;
    int k = 0;
    bool fresh = true;
    for (;;) {
        if (fresh) {
#pragma unroll
            for (int i = 0; i < 6; ++i) sig0[i] = in[i * npoints + p];
#pragma unroll
            for (int i = 0; i < 6; ++i) deps[i] = in[(6 + i) * npoints + p];
#pragma unroll
            for (int i = 0; i < 6; ++i) x[i] = deps[i];
            x[6] = 0.0;
            k = 0;
        }
        norton_eval(P, sig0, deps, x, F, J, sig);
        const double r = norm2<7>(F);
        if (fresh) r0 = r;
        fresh = false;

        int st = -1;
        if (!isfinite(r)) st = TL_NEWTON_NONFINITE;
        else if (r <= rtol * r0 || r0 == 0.0) st = TL_NEWTON_CONVERGED;
        else if (k >= max_iter) st = TL_NEWTON_MAX_ITER;
        if (st < 0) {
            double rhs[7];
#pragma unroll
            for (int i = 0; i < 7; ++i) rhs[i] = dev::neg(F[i]);
            int piv[7];
            int info = 0;
            if (!dev::lupp_solve_fast<7>(J, rhs, piv)) {
                NortonState ns;
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    ns.sig0[i] = sig0[i];
                    ns.deps[i] = deps[i];
                }
#pragma unroll
                for (int i = 0; i < 7; ++i) ns.x[i] = x[i];
                const Solve7 o = slow_norton_solve(P, ns);
                info = o.info;
#pragma unroll
                for (int i = 0; i < 7; ++i) rhs[i] = o.dx[i];
            }
            if (info != 0) {
                st = TL_NEWTON_SINGULAR;
            } else {
#pragma unroll
                for (int i = 0; i < 7; ++i) x[i] += rhs[i];
                ++k;
                continue;
            }
        }
        // this point is done: store and move on to the next point
#pragma unroll
        for (int i = 0; i < 7; ++i) xout[i * npoints + p] = x[i];
        if (sigout) {
#pragma unroll
            for (int i = 0; i < 6; ++i) sigout[i * npoints + p] = sig[i];
        }
        iters[p] = k;
        status[p] = st;
        p += stride;
        if (p >= npoints) break;
        fresh = true;
    }
}

// Synthetic law F(x) = A x + c .* tanh(x) - b, J = A + diag(c .* (1 - tanh^2 x)),
// x0 = 0; one thread per point for n <= kTanhThreadMaxN.  A is re-read from
// memory (L1/L2-resident) at every iteration because the factorization
// overwrites the Jacobian in registers.
constexpr int kTanhThreadMaxN = 9;

template <int N>
struct VecN {
    double v[N];
};
template <int N>
struct SolveN {
    double dx[N];
    int info;
};

// Exact general path of one tanh-law solve (see slow_norton_solve).
template <int N>
static __device__ __noinline__ SolveN<N> slow_tanh_solve(const double *__restrict__ in, int64_t npoints, int64_t p,
                                                         VecN<N> x)
{
    double J[N][N], rhs[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const double ti = tanh(x.v[i]);
        const double ci = in[(N * N + i) * npoints + p];
        const double bi = in[(N * N + N + i) * npoints + p];
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const double aij = in[(j * N + i) * npoints + p];
            acc = fma(aij, x.v[j], acc);
            J[i][j] = aij;
        }
        rhs[i] = dev::neg(fma(ci, ti, acc) - bi);
        J[i][i] = fma(ci, fma(-ti, ti, 1.0), J[i][i]);
    }
    int piv[N];
    SolveN<N> out;
    out.info = dev::lupp_solve<N>(J, rhs, piv);
#pragma unroll
    for (int i = 0; i < N; ++i) out.dx[i] = rhs[i];
    return out;
}

template <int N>
__global__ void __launch_bounds__(128) k_newton_tanh(int64_t npoints, const double *__restrict__ in,
                                                     double *__restrict__ xout, int32_t *__restrict__ iters,
                                                     int32_t *__restrict__ status, double rtol, int max_iter)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= npoints) return;
    double x[N], F[N], J[N][N];
    double r0 = 0.0;
    int k = 0;
    bool fresh = true;
    for (;;) {
        if (fresh) {
#pragma unroll
            for (int i = 0; i < N; ++i) x[i] = 0.0;
            k = 0;
        }
        // assemble F and J at x
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const double ti = tanh(x[i]);
            const double ci = in[(N * N + i) * npoints + p];
            const double bi = in[(N * N + N + i) * npoints + p];
            double acc = 0.0;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const double aij = in[(j * N + i) * npoints + p];
                acc = fma(aij, x[j], acc);
                J[i][j] = aij;
            }
            F[i] = fma(ci, ti, acc) - bi;
            J[i][i] = fma(ci, fma(-ti, ti, 1.0), J[i][i]);
        }
        const double r = norm2<N>(F);
        if (fresh) r0 = r;
        fresh = false;
        int st = -1;
        if (!isfinite(r)) st = TL_NEWTON_NONFINITE;
        else if (r <= rtol * r0 || r0 == 0.0) st = TL_NEWTON_CONVERGED;
        else if (k >= max_iter) st = TL_NEWTON_MAX_ITER;
        if (st < 0) {
            double rhs[N];
#pragma unroll
            for (int i = 0; i < N; ++i) rhs[i] = dev::neg(F[i]);
            int piv[N];
            int info = 0;
            if (!dev::lupp_solve_fast<N>(J, rhs, piv)) {
                VecN<N> xv;
#pragma unroll
                for (int i = 0; i < N; ++i) xv.v[i] = x[i];
                const SolveN<N> o = slow_tanh_solve<N>(in, npoints, p, xv);
                info = o.info;
#pragma unroll
                for (int i = 0; i < N; ++i) rhs[i] = o.dx[i];
            }
            if (info != 0) {
                st = TL_NEWTON_SINGULAR;
            } else {
#pragma unroll
                for (int i = 0; i < N; ++i) x[i] += rhs[i];
                ++k;
                continue;
            }
        }
#pragma unroll
        for (int i = 0; i < N; ++i) xout[i * npoints + p] = x[i];
        iters[p] = k;
        status[p] = st;
        p += stride;
        if (p >= npoints) break;
        fresh = true;
    }
}

template <int N>
tl_status launch_tanh_n(tl_handle *h, int64_t npoints, const double *in, double *x, int32_t *it, int32_t *st,
                        double rtol, int max_iter, cudaStream_t stream)
{
    const void *kern = reinterpret_cast<const void *>(&k_newton_tanh<N>);
    const int block = 128;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, block, 0) != cudaSuccess || nb < 1) nb = 1;
    const int64_t want = (npoints + block - 1) / block;
    const int64_t resident = static_cast<int64_t>(nb) * h->sm_count;
    const int64_t grid = want < resident ? want : resident;
    k_newton_tanh<N><<<static_cast<unsigned>(grid), block, 0, stream>>>(npoints, in, x, it, st, rtol, max_iter);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(h, e);
    return TL_OK;
}

tl_status tl_newton_tanh_launch(tl_handle *h, int n, int64_t npoints, const double *in, double *x, int32_t *it,
                                int32_t *st, double rtol, int max_iter, cudaStream_t stream)
{
    if (npoints == 0) return TL_OK;
    if (!in || (reinterpret_cast<uintptr_t>(in) & 7)) return fail_arg(h, 4);
    if (!x || (reinterpret_cast<uintptr_t>(x) & 7)) return fail_arg(h, 5);
    if (!it || (reinterpret_cast<uintptr_t>(it) & 3)) return fail_arg(h, 7);
    if (!st || (reinterpret_cast<uintptr_t>(st) & 3)) return fail_arg(h, 8);
    switch (n) {
    case 1: return launch_tanh_n<1>(h, npoints, in, x, it, st, rtol, max_iter, stream);
    case 2: return launch_tanh_n<2>(h, npoints, in, x, it, st, rtol, max_iter, stream);
    case 3: return launch_tanh_n<3>(h, npoints, in, x, it, st, rtol, max_iter, stream);
    case 4: return launch_tanh_n<4>(h, npoints, in, x, it, st, rtol, max_iter, stream);
    case 5: return launch_tanh_n<5>(h, npoints, in, x, it, st, rtol, max_iter, stream);
    case 6: return launch_tanh_n<6>(h, npoints, in, x, it, st, rtol, max_iter, stream);
    case 7: return launch_tanh_n<7>(h, npoints, in, x, it, st, rtol, max_iter, stream);
    case 8: return launch_tanh_n<8>(h, npoints, in, x, it, st, rtol, max_iter, stream);
    case 9: return launch_tanh_n<9>(h, npoints, in, x, it, st, rtol, max_iter, stream);
    default: return TL_ERR_UNSUPPORTED;
    }
}

}  // namespace
}  // namespace tl

using namespace tl;

extern "C" tl_status tl_newton_integrate(tl_handle *h, const tl_law *law, int64_t npoints,
                                         const double *inputs, double *x, double *outputs,
                                         int32_t *iterations, int32_t *status, double rtol, int max_iter,
                                         cudaStream_t stream)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (!law) return fail_arg(h, 2);
    if (npoints < 0) return fail_arg(h, 3);
    if (!(rtol >= 0.0)) return fail_arg(h, 9);
    if (max_iter < 0) return fail_arg(h, 10);
    if (law->id == TL_LAW_NORTON) {
        NortonParams P;
        if (!norton_params_from_law(*law, &P)) return fail_arg(h, 2);
        if (npoints == 0) return TL_OK;
        if (!inputs || (reinterpret_cast<uintptr_t>(inputs) & 7)) return fail_arg(h, 4);
        if (!x || (reinterpret_cast<uintptr_t>(x) & 7)) return fail_arg(h, 5);
        if (outputs && (reinterpret_cast<uintptr_t>(outputs) & 7)) return fail_arg(h, 6);
        if (!iterations || (reinterpret_cast<uintptr_t>(iterations) & 3)) return fail_arg(h, 7);
        if (!status || (reinterpret_cast<uintptr_t>(status) & 3)) return fail_arg(h, 8);
        const void *kern = reinterpret_cast<const void *>(&k_newton_norton);
        const int block = 128;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, block, 0) != cudaSuccess || nb < 1) nb = 1;
        int64_t want = (npoints + block - 1) / block;
        int64_t resident = static_cast<int64_t>(nb) * h->sm_count;
        int64_t grid = want < resident ? want : resident;
        k_newton_norton<<<static_cast<unsigned>(grid), block, 0, stream>>>(P, npoints, inputs, x, outputs, iterations,
                                                                         status, rtol, max_iter);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail_cuda(h, e);
        return TL_OK;
    }
    if (law->id == TL_LAW_TANH) {
        if (law->n < 1 || law->n > TL_MAX_N) return fail_arg(h, 2);
        return tl_newton_tanh_launch(h, law->n, npoints, inputs, x, iterations, status, rtol, max_iter, stream);
    }
    return fail_arg(h, 2);
}
