// tl_newton.cuh -- fused per-point Newton integration (Algorithm 2 of the
// paper: one kernel in which every integration point runs its own loop
// assemble F, J -> LUpp solve J dx = -F -> x += dx -> convergence test,
// Eqs. 1-3 of Sec. 2.1).
//
// The kernels take a table of jobs (one job = one request's points, with its
// own arrays and law parameters) and run over the concatenation of their
// points, so the same kernel integrates one request (tl_newton_integrate)
// or a continuous batch of many (the request server): a point's arithmetic
// does not depend on which other points share the launch.
//
// Mappings:
//   k_newton_norton        one thread per point, the 7x7 Jacobian and its
//                          LUpp in registers;
//   k_newton_tanh<N>       the same for the tanh law, N <= 9;
//   k_newton_tanh_group<N,T>  T lanes per point (row-cyclic rows, the
//                          sub-warp LUpp of tinylu_device.cuh), N = 10;
//   k_newton_tanh_smem<T>  (tl_newton_smem.cu) T lanes per point with the
//                          Jacobian in shared memory, n = 11..32.
// All are persistent: when a point stops (converged, iteration cap,
// singular, non-finite) its thread (group) stores the results and takes the
// next point of its stride, so a lane idles for one solve per point instead
// of waiting for the slowest point of its warp (the divergence the paper
// attributes to the device-callable paradigm, Sec. 2.4).
#pragma once
#include <cmath>

#include "tinylu.h"
#include "tinylu_device.cuh"
#include "tl_internal.h"
#include "tl_kernels.cuh"
#include "tl_newton_types.h"
#include "tl_norton.cuh"

namespace tl {

__device__ __forceinline__ NewtonJob load_job(const NewtonBatch &B, int64_t g)
{
    if (B.jobs == nullptr) return B.one;
    int lo = 0, hi = B.njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.jobs[mid].start <= g) lo = mid;
        else hi = mid - 1;
    }
    return B.jobs[lo];
}

template <int N>
__device__ __forceinline__ int newton_decide(double r, double r0, int k, double rtol, int max_iter)
{
    if (!isfinite(r)) return TL_NEWTON_NONFINITE;
    if (r <= rtol * r0 || r0 == 0.0) return TL_NEWTON_CONVERGED;
    if (k >= max_iter) return TL_NEWTON_MAX_ITER;
    return -1;
}

// ---------------------------------------------------------------------------
// Norton law, n = 7, one thread per point
// ---------------------------------------------------------------------------

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

// Consistent tangent at a converged state (Sec. 4.3: one multi-RHS solve
// after convergence): J X = [I_6; 0] with the six right-hand sides carried
// through one elimination, then dsig/ddeps = C X[0..5] (Mandel elasticity
// C = lambda 1 (x) 1 + 2 mu I).  Stores tangent[(i + 6 j) np + p]; NaN when
// the Jacobian is singular or not finite.  Out of line: it runs once per
// point and must not weigh on the Newton loop's registers.
static __device__ __noinline__ void norton_tangent_store(NortonParams P, NortonState st, double *tangent, int64_t np,
                                                         int64_t p)
{
    double F[7], J[7][7], sig[6], X[6][7];
    norton_eval(P, st.sig0, st.deps, st.x, F, J, sig);
    const bool bad = dev::any_nonfinite<7>(J);
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int i = 0; i < 7; ++i) X[c][i] = (i == c) ? 1.0 : 0.0;
    int piv[7];
    double rcp[7];
    bool tiny = false;
    const int info = dev::lu_thread_factor<7, false, 6>(J, X, piv, rcp, tiny);
#pragma unroll
    for (int c = 0; c < 6; ++c) dev::lu_thread_backsolve<7>(J, X[c], rcp, tiny);
    const bool ok = info == 0 && !bad;
    const double two_mu = 2.0 * P.mu;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const double tr = X[j][0] + X[j][1] + X[j][2];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const double d = (i < 3) ? fma(P.lambda, tr, two_mu * X[j][i]) : two_mu * X[j][i];
            tangent[(i + 6 * j) * np + p] = ok ? d : dev::nan_value();
        }
    }
}

static __global__ void __launch_bounds__(128) k_newton_norton(NewtonBatch B)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= B.total) return;

    double sig0[6], deps[6], x[7], F[7], J[7][7], sig[6];
    NortonParams P;
    double r0 = 0.0;
    int k = 0;
    bool fresh = true;
    for (;;) {
        if (fresh) {
            const NewtonJob jb = load_job(B, g);
            const int64_t p = g - jb.start, np = jb.npoints;
            P = jb.P;
#pragma unroll
            for (int i = 0; i < 6; ++i) sig0[i] = jb.in[i * np + p];
#pragma unroll
            for (int i = 0; i < 6; ++i) deps[i] = jb.in[(6 + i) * np + p];
#pragma unroll
            for (int i = 0; i < 6; ++i) x[i] = deps[i];
            x[6] = 0.0;
            k = 0;
        }
        norton_eval(P, sig0, deps, x, F, J, sig);
        const double r = norm2<7>(F);
        if (fresh) r0 = r;
        fresh = false;

        int st = newton_decide<7>(r, r0, k, B.rtol, B.max_iter);
        if (st < 0) {
            double rhs[7];
#pragma unroll
            for (int i = 0; i < 7; ++i) rhs[i] = dev::neg(F[i]);
            int piv[7];
            int info = 0;
            if (!dev::lupp_solve_fast<7, true>(J, rhs, piv)) {
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
        const NewtonJob jb = load_job(B, g);
        const int64_t p = g - jb.start, np = jb.npoints;
#pragma unroll
        for (int i = 0; i < 7; ++i) jb.x[i * np + p] = x[i];
        if (jb.out) {
#pragma unroll
            for (int i = 0; i < 6; ++i) jb.out[i * np + p] = sig[i];
        }
        if (jb.tangent) {
            if (st == TL_NEWTON_CONVERGED) {
                NortonState ns;
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    ns.sig0[i] = sig0[i];
                    ns.deps[i] = deps[i];
                }
#pragma unroll
                for (int i = 0; i < 7; ++i) ns.x[i] = x[i];
                norton_tangent_store(P, ns, jb.tangent, np, p);
            } else {
                for (int i = 0; i < 36; ++i) jb.tangent[i * np + p] = dev::nan_value();
            }
        }
        jb.iters[p] = k;
        jb.status[p] = st;
        g += stride;
        if (g >= B.total) break;
        fresh = true;
    }
}

// ---------------------------------------------------------------------------
// Synthetic law F(x) = A x + c .* tanh(x) - b, J = A + diag(c .* (1 - tanh^2 x)),
// x0 = 0.  A is re-read from memory (L1/L2-resident) at every iteration
// because the factorization overwrites the Jacobian in registers.
// ---------------------------------------------------------------------------

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

// F_i and row i of J at x (one thread holds the whole point).
template <int N>
__device__ __forceinline__ void tanh_assemble(const double *__restrict__ in, int64_t np, int64_t p,
                                              const double (&x)[N], double (&F)[N], double (&J)[N][N])
{
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const double ti = tanh(x[i]);
        const double ci = in[(N * N + i) * np + p];
        const double bi = in[(N * N + N + i) * np + p];
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const double aij = in[(j * N + i) * np + p];
            acc = fma(aij, x[j], acc);
            J[i][j] = aij;
        }
        F[i] = fma(ci, ti, acc) - bi;
        J[i][i] = fma(ci, fma(-ti, ti, 1.0), J[i][i]);
    }
}

template <int N>
static __device__ __noinline__ SolveN<N> slow_tanh_solve(const double *__restrict__ in, int64_t np, int64_t p,
                                                         VecN<N> xv)
{
    double F[N], J[N][N], rhs[N];
    tanh_assemble<N>(in, np, p, xv.v, F, J);
#pragma unroll
    for (int i = 0; i < N; ++i) rhs[i] = dev::neg(F[i]);
    int piv[N];
    SolveN<N> out;
    out.info = dev::lupp_solve<N>(J, rhs, piv);
#pragma unroll
    for (int i = 0; i < N; ++i) out.dx[i] = rhs[i];
    return out;
}

template <int N>
__global__ void __launch_bounds__(128) k_newton_tanh(NewtonBatch B)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= B.total) return;
    double x[N], F[N], J[N][N];
    const double *in = nullptr;
    int64_t np = 0, p = 0;
    double r0 = 0.0;
    int k = 0;
    bool fresh = true;
    for (;;) {
        if (fresh) {
            const NewtonJob jb = load_job(B, g);
            in = jb.in;
            np = jb.npoints;
            p = g - jb.start;
#pragma unroll
            for (int i = 0; i < N; ++i) x[i] = 0.0;
            k = 0;
        }
        tanh_assemble<N>(in, np, p, x, F, J);
        const double r = norm2<N>(F);
        if (fresh) r0 = r;
        fresh = false;
        int st = newton_decide<N>(r, r0, k, B.rtol, B.max_iter);
        if (st < 0) {
            double rhs[N];
#pragma unroll
            for (int i = 0; i < N; ++i) rhs[i] = dev::neg(F[i]);
            int piv[N];
            int info = 0;
            if (!dev::lupp_solve_fast<N, true>(J, rhs, piv)) {
                VecN<N> xv;
#pragma unroll
                for (int i = 0; i < N; ++i) xv.v[i] = x[i];
                const SolveN<N> o = slow_tanh_solve<N>(in, np, p, xv);
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
        const NewtonJob jb = load_job(B, g);
#pragma unroll
        for (int i = 0; i < N; ++i) jb.x[i * np + p] = x[i];
        jb.iters[p] = k;
        jb.status[p] = st;
        g += stride;
        if (g >= B.total) break;
        fresh = true;
    }
}

// T lanes per point (N >= 10): lane t holds rows and unknowns t + s*T.  The
// warp runs one Newton step of each of its 32/T points per trip (a
// warp-uniform loop, since the LUpp shuffles across the group); a group
// whose point stops stores it and starts its next point on the next trip.
// F_i = sum_j a_ij x_j (fma, j increasing) + c_i tanh(x_i) - b_i as in the
// one-thread kernel; ||F||_2 is summed per lane and then across the group.
template <int N, int T>
__global__ void __launch_bounds__(128) k_newton_tanh_group(NewtonBatch B)
{
    constexpr int K = dev::Group<N, T>::K;
    const int lane = threadIdx.x & 31;
    const int t = lane % T;
    const int lane0 = lane - t;
    const int64_t ngroups = (static_cast<int64_t>(gridDim.x) * blockDim.x) / T;
    int64_t g = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / T;
    bool have = g < B.total;
    double x[K];
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
#pragma unroll
            for (int s = 0; s < K; ++s) x[s] = 0.0;
            k = 0;
        }
        // assemble this lane's rows of F and J
        double a[K][N], rhs[K];
        double ti[K], ci[K], bi[K], acc[K];
#pragma unroll
        for (int s = 0; s < K; ++s) {
            const int i = t + s * T;
            const bool live = have && i < N;
            ti[s] = live ? tanh(x[s]) : 0.0;
            ci[s] = live ? in[(N * N + i) * np + p] : 0.0;
            bi[s] = live ? in[(N * N + N + i) * np + p] : 0.0;
            acc[s] = 0.0;
        }
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const double xj = __shfl_sync(0xffffffffu, x[j / T], lane0 + j % T);
#pragma unroll
            for (int s = 0; s < K; ++s) {
                const int i = t + s * T;
                const bool live = have && i < N;
                const double aij = live ? in[(j * N + i) * np + p] : 0.0;
                acc[s] = fma(aij, xj, acc[s]);
                a[s][j] = aij;
            }
        }
        double ss = 0.0;
#pragma unroll
        for (int s = 0; s < K; ++s) {
            const int i = t + s * T;
            const double Fi = fma(ci[s], ti[s], acc[s]) - bi[s];
            ss = fma(Fi, Fi, ss);
            rhs[s] = dev::neg(Fi);
#pragma unroll
            for (int j = 0; j < N; ++j)
                if (j == i) a[s][j] = fma(ci[s], fma(-ti[s], ti[s], 1.0), a[s][j]);
        }
#pragma unroll
        for (int off = T / 2; off >= 1; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
        const double r = sqrt(ss);
        if (have && fresh) r0 = r;
        fresh = false;
        int st = have ? newton_decide<N>(r, r0, k, B.rtol, B.max_iter) : 0;
        const bool need = have && st < 0;
        if (__any_sync(0xffffffffu, need)) {
            int pivk[K];
            double rcp[K];
            bool tiny = false;
            const int info = dev::lu_group_factor<N, T, false, 1>(a, rhs, pivk, rcp, t, lane0, tiny);
            dev::lu_group_backsolve<N, T>(a, rhs, rcp, t, lane0, tiny);
            if (need) {
                if (info != 0) {
                    st = TL_NEWTON_SINGULAR;
                } else {
#pragma unroll
                    for (int s = 0; s < K; ++s) x[s] += rhs[s];
                    ++k;
                }
            }
        }
        if (have && st >= 0) {
            const NewtonJob jb = load_job(B, g);
#pragma unroll
            for (int s = 0; s < K; ++s) {
                const int i = t + s * T;
                if (i < N) jb.x[i * np + p] = x[s];
            }
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

}  // namespace tl
