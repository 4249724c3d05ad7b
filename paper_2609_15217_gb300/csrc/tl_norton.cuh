// tl_norton.cuh -- the implicit Norton viscoplastic law of the Newton
// kernels (the law class of Sec. 4.3), shared by the fused per-point kernel
// (Algorithm 2) and the batched, CPU-driven loop (Algorithm 1).
#pragma once
#include <cmath>

#include "tinylu.h"

namespace tl {

struct NortonParams {
    double lambda, mu, Acoef, dt;
    int m;
};

// Implicit Norton law at one point (J2 flow, isotropic elasticity, Mandel
// notation: xx, yy, zz, sqrt2*xy, sqrt2*xz, sqrt2*yz; theta = 1):
//   sig  = sig0 + lambda tr(de) 1 + 2 mu de,  s = dev sig,
//   seq  = sqrt(3/2 s:s), n = 3/2 s / seq,
//   F_el = de - deps + dp n,  F_p = dp - dt A seq^m,
//   dF_el/dde = I + dp (2 mu / seq)(3/2 K - n n^T),  dF_el/ddp = n,
//   (assembled as one FMA per entry around its constant part),
//   dF_p/dde  = -dt A m seq^(m-1) 2 mu n^T,          dF_p/ddp = 1.
__device__ __forceinline__ void norton_eval(const NortonParams &P, const double (&sig0)[6],
                                            const double (&deps)[6], const double (&x)[7],
                                            double (&F)[7], double (&J)[7][7], double (&sig)[6])
{
    const double tr = x[0] + x[1] + x[2];
    const double two_mu = 2.0 * P.mu;
#pragma unroll
    for (int i = 0; i < 6; ++i) sig[i] = sig0[i] + two_mu * x[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) sig[i] += P.lambda * tr;
    const double p3 = (sig[0] + sig[1] + sig[2]) * (1.0 / 3.0);
    double s[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) s[i] = (i < 3) ? sig[i] - p3 : sig[i];
    double ss = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) ss = fma(s[i], s[i], ss);
    const double seq = sqrt(1.5 * ss);
    const double inv = seq > 0.0 ? 1.0 / seq : 0.0;
    double n[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) n[i] = 1.5 * s[i] * inv;
    double pw_m1 = 1.0;
    for (int i = 0; i < P.m - 1; ++i) pw_m1 *= seq;
    const double pw_m = pw_m1 * seq;
    const double dp = x[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) F[i] = fma(dp, n[i], x[i] - deps[i]);
    F[6] = dp - P.dt * P.Acoef * pw_m;

    // dF_el/dde = I + c (3/2 K - n n^T) = C_ij - (c n_i) n_j with the
    // constant part C_ij = delta_ij + 3/2 c K_ij: 1 + c on the normal
    // diagonal, -c/2 between normal components, 1 + 3/2 c on the shear
    // diagonal, 0 elsewhere; one FMA per entry
    const double c = dp * two_mu * inv;
    const double c_nn = 1.0 + c, c_no = -0.5 * c, c_ss = fma(1.5, c, 1.0);
    double cn[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) cn[i] = c * n[i];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const double cij = (i < 3 && j < 3) ? (i == j ? c_nn : c_no) : (i == j ? c_ss : 0.0);
            J[i][j] = fma(-cn[i], n[j], cij);
        }
#pragma unroll
    for (int i = 0; i < 6; ++i) J[i][6] = n[i];
    const double g = -P.dt * P.Acoef * P.m * pw_m1 * two_mu;
#pragma unroll
    for (int j = 0; j < 6; ++j) J[6][j] = g * n[j];
    J[6][6] = 1.0;
}

// Lame constants and step data from a TL_LAW_NORTON descriptor; false when
// the descriptor is invalid (n != 7, E <= 0, nu outside (-1, 1/2), m not an
// integer in 1..64, A or dt not finite).
inline bool norton_params_from_law(const tl_law &law, NortonParams *P)
{
    if (law.id != TL_LAW_NORTON || law.n != 7) return false;
    const double E = law.params[0], nu = law.params[1], Acoef = law.params[2], m = law.params[3],
                 dt = law.params[4];
    if (!(E > 0.0) || !(nu > -1.0 && nu < 0.5) || !(m >= 1.0 && m <= 64.0) || m != std::floor(m) ||
        !std::isfinite(Acoef) || !std::isfinite(dt))
        return false;
    P->lambda = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    P->mu = E / (2.0 * (1.0 + nu));
    P->Acoef = Acoef;
    P->dt = dt;
    P->m = static_cast<int>(m);
    return true;
}

template <int N>
__device__ __forceinline__ double norm2(const double (&F)[N])
{
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) s = fma(F[i], F[i], s);
    return sqrt(s);
}

}  // namespace tl
