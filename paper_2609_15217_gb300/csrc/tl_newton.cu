// tl_newton.cu -- launches of the fused per-point Newton kernels of
// tl_newton.cuh (Algorithm 2 of the paper) and the C ABI entry
// tl_newton_integrate.  The Norton kernel and the one-thread tanh kernels
// (n <= 9) are instantiated here; the sub-warp tanh kernels (n >= 10) come
// from the instantiation units tl_inst_newton.cu through the registry.
#include <cmath>

#include "tinylu.h"
#include "tl_handle.h"
#include "tl_internal.h"
#include "tl_newton.cuh"

namespace tl {
namespace {

// Persistent grid: enough threads for every point (lanes per point each),
// at most what stays resident.
tl_status launch_persistent(tl_handle *h, const void *kern, int lanes, const NewtonBatch &B, cudaStream_t stream)
{
    const int block = 128;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, block, 0) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    const int64_t want = (B.total * lanes + block - 1) / block;
    const int64_t resident = static_cast<int64_t>(nb) * h->sm_count;
    const int64_t grid = want < resident ? want : resident;
    NewtonBatch arg = B;
    void *params[] = {&arg};
    cudaError_t e = cudaLaunchKernel(kern, dim3(static_cast<unsigned>(grid)), dim3(block), params, 0, stream);
    if (e != cudaSuccess) return fail_cuda(h, e);
    return TL_OK;
}

const void *tanh_thread_kernel(int n)
{
    switch (n) {
    case 1: return reinterpret_cast<const void *>(&k_newton_tanh<1>);
    case 2: return reinterpret_cast<const void *>(&k_newton_tanh<2>);
    case 3: return reinterpret_cast<const void *>(&k_newton_tanh<3>);
    case 4: return reinterpret_cast<const void *>(&k_newton_tanh<4>);
    case 5: return reinterpret_cast<const void *>(&k_newton_tanh<5>);
    case 6: return reinterpret_cast<const void *>(&k_newton_tanh<6>);
    case 7: return reinterpret_cast<const void *>(&k_newton_tanh<7>);
    case 8: return reinterpret_cast<const void *>(&k_newton_tanh<8>);
    case 9: return reinterpret_cast<const void *>(&k_newton_tanh<9>);
    default: return nullptr;
    }
}

}  // namespace

tl_status newton_launch(tl_handle *h, int law_id, int n, const NewtonBatch &B, cudaStream_t stream)
{
    if (B.total == 0) return TL_OK;
    if (law_id == TL_LAW_NORTON) return launch_persistent(h, reinterpret_cast<const void *>(&k_newton_norton), 1, B, stream);
    if (law_id != TL_LAW_TANH || n < 1 || n > TL_MAX_N) return TL_ERR_UNSUPPORTED;
    if (n <= kTanhThreadMaxN) return launch_persistent(h, tanh_thread_kernel(n), 1, B, stream);
    tl_status st = TL_OK;
    if (newton_tanh_smem_launch(h, n, B, stream, &st)) return st;
    const VariantList &l = registry(n, kPerSystem, kOpNewtonTanh);
    if (l.count == 0) return TL_ERR_UNSUPPORTED;
    return launch_persistent(h, l.v[0].kernel, l.v[0].lanes, B, stream);
}

bool law_params(const tl_law &law, NewtonJob *jb)
{
    if (law.id == TL_LAW_NORTON) return norton_params_from_law(law, &jb->P);
    if (law.id == TL_LAW_TANH) {
        jb->P = NortonParams{};
        return law.n >= 1 && law.n <= TL_MAX_N;
    }
    return false;
}

}  // namespace tl

using namespace tl;

namespace {

tl_status integrate(tl_handle *h, const tl_law *law, int64_t npoints, const double *inputs, double *x,
                    double *outputs, double *tangent, int32_t *iterations, int32_t *status, double rtol,
                    int max_iter, cudaStream_t stream)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (!law) return fail_arg(h, 2);
    if (npoints < 0) return fail_arg(h, 3);
    if (!(rtol >= 0.0)) return fail_arg(h, 9);
    if (max_iter < 0) return fail_arg(h, 10);
    NewtonBatch B{};
    if (!law_params(*law, &B.one)) return fail_arg(h, 2);
    if (npoints == 0) return TL_OK;
    if (!inputs || (reinterpret_cast<uintptr_t>(inputs) & 7)) return fail_arg(h, 4);
    if (!x || (reinterpret_cast<uintptr_t>(x) & 7)) return fail_arg(h, 5);
    if (outputs && (reinterpret_cast<uintptr_t>(outputs) & 7)) return fail_arg(h, 6);
    if (!iterations || (reinterpret_cast<uintptr_t>(iterations) & 3)) return fail_arg(h, 7);
    if (!status || (reinterpret_cast<uintptr_t>(status) & 3)) return fail_arg(h, 8);
    B.jobs = nullptr;
    B.one.in = inputs;
    B.one.x = x;
    B.one.out = law->id == TL_LAW_NORTON ? outputs : nullptr;
    B.one.tangent = tangent;
    B.one.iters = iterations;
    B.one.status = status;
    B.one.npoints = npoints;
    B.one.start = 0;
    B.njobs = 1;
    B.total = npoints;
    B.rtol = rtol;
    B.max_iter = max_iter;
    return newton_launch(h, law->id, law->n, B, stream);
}

}  // namespace

extern "C" tl_status tl_newton_integrate(tl_handle *h, const tl_law *law, int64_t npoints,
                                         const double *inputs, double *x, double *outputs,
                                         int32_t *iterations, int32_t *status, double rtol, int max_iter,
                                         cudaStream_t stream)
{
    return integrate(h, law, npoints, inputs, x, outputs, nullptr, iterations, status, rtol, max_iter, stream);
}

extern "C" tl_status tl_newton_integrate_tangent(tl_handle *h, const tl_law *law, int64_t npoints,
                                                 const double *inputs, double *x, double *outputs, double *tangent,
                                                 int32_t *iterations, int32_t *status, double rtol, int max_iter,
                                                 cudaStream_t stream)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (!law) return fail_arg(h, 2);
    if (law->id != TL_LAW_NORTON) return TL_ERR_UNSUPPORTED;
    if (npoints > 0 && (!tangent || (reinterpret_cast<uintptr_t>(tangent) & 7))) return fail_arg(h, 7);
    return integrate(h, law, npoints, inputs, x, outputs, tangent, iterations, status, rtol, max_iter, stream);
}
