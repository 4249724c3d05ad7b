/*
 * tinylu_oracle.c -- plain, slow, obviously-correct CPU oracle for batched
 * tiny LU with partial pivoting (LUpp) and the per-point Newton loop.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or execute this file: only the tests, the smoke check and the timed
 * CPU baseline of the benchmark use it.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Arithmetic: IEEE-754 binary64, round to nearest, compiled with
 * -ffp-contract=off so that every fused multiply-add is the explicit fma()
 * written below and nothing else is contracted (the paper computes in double
 * precision without fast-math, Sec. 4.1 "Software stack").
 *
 * Storage: every matrix is one system, column-major, leading dimension n
 * (LAPACK convention used by all batched solvers of Sec. 3.1): entry (i,j)
 * sits at a[i + j*n].  Pivots are LAPACK 1-based sequential interchanges.
 *
 * Functions and the passages they follow:
 *   orc_getrf   -- Gaussian elimination with partial pivoting, PA = LU,
 *                  right-looking, one column per step (Sec. 2.2).
 *   orc_getrs   -- Ly = Pb then Ux = y (Sec. 2.2).
 *   orc_getrf_tiled -- the same elimination with tile-local pivoting
 *                  (Sec. 3.2, Tiled solvers; acceptance threshold).
 *   orc_gesv    -- getrf + getrs, fused (Sec. 3.1, MAGMA gesv).
 *   orc_newton_* -- Newton-Raphson, Eqs. (1)-(3) of Sec. 2.1, driven per
 *                  point as in Algorithm 2.
 *   orc_norton_eval -- implicit (theta = 1) Norton viscoplastic law used as
 *                  the per-point constitutive law (Sec. 4.3 names a Norton
 *                  law; its equations are not printed, the standard J2 +
 *                  Norton form is used, see the module docstring of the
 *                  Python wrapper for the reading).
 *   orc_tanh_eval -- synthetic law F(x) = A x + c .* tanh(x) - b.
 *   orc_norton_tangent -- consistent tangent of the Norton law at a
 *                  converged state (Sec. 4.3, the multi-RHS solve after
 *                  convergence).
 *   orc_sgetrf / orc_sgetrs / orc_ir_solve -- binary32 factorization with
 *                  binary64 iterative refinement (not in the paper; the
 *                  published scheme of Langou et al. 2006, see below).
 *
 * Readings where the paper is silent (pivot tie-break, multiplier arithmetic,
 * zero and non-finite pivots, pivot base) are listed beside each function.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define AT(a, n, i, j) ((a)[(size_t)(i) + (size_t)(j) * (size_t)(n)])

/* |a| > |b| with NaN ranked above every number and +-Inf above every finite
 * value.  For finite operands this is exactly fabs(a) > fabs(b). */
static int mag_greater(double a, double b)
{
    if (isnan(a)) return !isnan(b);
    if (isnan(b)) return 0;
    return fabs(a) > fabs(b);
}

/*
 * orc_getrf: PA = LU by textbook right-looking Doolittle elimination with
 * physical row swaps (Sec. 2.2: eliminate column by column, pivot row chosen
 * as the entry of largest magnitude; the row interchanges form P).
 *
 * For k = 0 .. n-1:
 *   1. p = smallest i >= k with |a_ik| maximal (first maximum, as LAPACK's
 *      idamax; the paper does not state a tie-break).
 *   2. ipiv[k] = p + 1.
 *   3. a_pk == 0: info = k+1 if no earlier zero pivot; nothing else is done
 *      for this step (the column below is already zero).
 *   4. swap rows k and p over all n columns (L part included).
 *   5. |a_kk| >= DBL_MIN: r = 1/a_kk, l_ik = a_ik * r; otherwise
 *      l_ik = a_ik / a_kk (LAPACK dgetf2's guard against an overflowing
 *      reciprocal).
 *   6. a_ij = fma(-l_ik, a_kj, a_ij) for i, j > k.
 *
 * If any input entry is NaN or +-Inf the matrix is not factored: info = -1,
 * ipiv = identity, a left unchanged.
 *
 * min_gap (nullable): smallest relative separation over all steps between
 * the chosen pivot magnitude and the next largest candidate,
 * (|a_pk| - second)/|a_pk|; +Inf when no step had two candidates.  Used to
 * flag near-ties.
 *
 * Returns info.
 */
static int getrf_core(int n, double *a, int32_t *ipiv, double *min_gap, int tile, double threshold,
                      int *out_of_tile)
{
    int info = 0, outside = 0;
    double gap = INFINITY;
    if (out_of_tile) *out_of_tile = 0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
            if (!isfinite(AT(a, n, i, j))) {
                for (int k = 0; k < n; ++k) ipiv[k] = k + 1;
                if (min_gap) *min_gap = INFINITY;
                return -1;
            }

    for (int k = 0; k < n; ++k) {
        /* candidate rows: k .. hi-1 (the diagonal tile), all rows below k
         * when the tile's best is under the threshold */
        int hi = n;
        if (tile > 0 && tile < n) {
            hi = (k / tile + 1) * tile;
            if (hi > n) hi = n;
        }
        int p = k;
        for (int i = k + 1; i < hi; ++i)
            if (mag_greater(AT(a, n, i, k), AT(a, n, p, k))) p = i;
        if (hi < n && fabs(AT(a, n, p, k)) < threshold) {
            ++outside;
            for (int i = hi; i < n; ++i)
                if (mag_greater(AT(a, n, i, k), AT(a, n, p, k))) p = i;
        }
        ipiv[k] = p + 1;

        if (k + 1 < n && AT(a, n, p, k) != 0.0) {
            double second = 0.0;
            for (int i = k; i < n; ++i)
                if (i != p && fabs(AT(a, n, i, k)) > second) second = fabs(AT(a, n, i, k));
            double g = (fabs(AT(a, n, p, k)) - second) / fabs(AT(a, n, p, k));
            if (g < gap) gap = g;
        }

        if (AT(a, n, p, k) == 0.0) {
            if (info == 0) info = k + 1;
            continue;
        }
        if (p != k)
            for (int j = 0; j < n; ++j) {
                double t = AT(a, n, k, j);
                AT(a, n, k, j) = AT(a, n, p, j);
                AT(a, n, p, j) = t;
            }
        double akk = AT(a, n, k, k);
        if (fabs(akk) >= DBL_MIN) {
            double r = 1.0 / akk;
            for (int i = k + 1; i < n; ++i) AT(a, n, i, k) = AT(a, n, i, k) * r;
        } else {
            for (int i = k + 1; i < n; ++i) AT(a, n, i, k) = AT(a, n, i, k) / akk;
        }
        for (int j = k + 1; j < n; ++j)
            for (int i = k + 1; i < n; ++i)
                AT(a, n, i, j) = fma(-AT(a, n, i, k), AT(a, n, k, j), AT(a, n, i, j));
    }
    if (min_gap) *min_gap = gap;
    if (out_of_tile) *out_of_tile = outside;
    return info;
}

int orc_getrf(int n, double *a, int32_t *ipiv, double *min_gap)
{
    return getrf_core(n, a, ipiv, min_gap, 0, 0.0, NULL);
}

/*
 * orc_getrf_tiled: LU with tile-local pivoting (Sec. 3.2, the Tiled solvers:
 * the pivot row is sought inside the diagonal tile, and rows below it are
 * considered only when the best in-tile candidate falls below an acceptance
 * threshold).  Reading taken: the matrix is cut into tiles of `tile` rows;
 * at step k the candidates are the rows k .. min(n, (k/tile + 1) tile) - 1
 * of the diagonal tile, first maximum as orc_getrf; if that maximum is
 * below `threshold` in magnitude (absolute), the candidates are all rows
 * k .. n-1 instead (first maximum over them).  Everything else is
 * orc_getrf: zero pivots, row swaps, multipliers, updates, non-finite input.
 * tile <= 0 or tile >= n is textbook partial pivoting (orc_getrf is
 * getrf_core with no tile).  *out_of_tile (nullable) counts the steps that
 * looked below the tile.  Returns info.
 */
int orc_getrf_tiled(int n, double *a, int32_t *ipiv, int tile, double threshold, int *out_of_tile)
{
    return getrf_core(n, a, ipiv, NULL, tile, threshold, out_of_tile);
}

/* Batched tile-local factor (one system per s, as orc_getrf_batch). */
void orc_getrf_tiled_batch(int n, int64_t batch, double *A, int32_t *ipiv, int32_t *info, int32_t *out_of_tile,
                           int tile, double threshold, int nthreads)
{
    const size_t nn = (size_t)n * (size_t)n;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int64_t s = 0; s < batch; ++s) {
        int o = 0;
        info[s] = orc_getrf_tiled(n, A + (size_t)s * nn, ipiv + (size_t)s * n, tile, threshold, &o);
        out_of_tile[s] = o;
    }
    (void)nthreads;
}

/*
 * orc_getrs: solve A x = b from the factors of orc_getrf (Sec. 2.2,
 * "Ly = b and Ux = y", with b first permuted by P).
 *   - the interchanges are applied to b in order k = 0 .. n-1;
 *   - forward: y_i = b_i - sum_{j<i} l_ij y_j, fma-accumulated in increasing j
 *     (L has a unit diagonal);
 *   - back: x_i = (y_i - sum_{j>i} u_ij x_j) / u_ii, fma-accumulated in
 *     decreasing j, then one true division.
 * b is overwritten by x.
 */
void orc_getrs(int n, const double *lu, const int32_t *ipiv, double *b)
{
    for (int k = 0; k < n; ++k) {
        int p = ipiv[k] - 1;
        if (p != k) {
            double t = b[k];
            b[k] = b[p];
            b[p] = t;
        }
    }
    for (int i = 1; i < n; ++i) {
        double s = b[i];
        for (int j = 0; j < i; ++j) s = fma(-AT(lu, n, i, j), b[j], s);
        b[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = n - 1; j > i; --j) s = fma(-AT(lu, n, i, j), b[j], s);
        b[i] = s / AT(lu, n, i, i);
    }
}

/*
 * orc_gesv: factor a copy of A and solve for one right-hand side.
 * lu_out (nullable) receives the factors.  When info != 0 (zero pivot or
 * non-finite input) no solve is attempted and x is filled with NaN.
 * work must hold n*n doubles when lu_out is NULL.
 */
int orc_gesv(int n, const double *a, const double *b, double *x, int32_t *ipiv,
             double *lu_out, double *work, double *min_gap)
{
    double *lu = lu_out ? lu_out : work;
    memcpy(lu, a, sizeof(double) * (size_t)n * (size_t)n);
    int info = orc_getrf(n, lu, ipiv, min_gap);
    if (info != 0) {
        for (int i = 0; i < n; ++i) x[i] = NAN;
        return info;
    }
    memcpy(x, b, sizeof(double) * (size_t)n);
    orc_getrs(n, lu, ipiv, x);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Batched drivers.  Systems are contiguous: system s starts at s*n*n in A  */
/* and s*n in b, x and ipiv.  nthreads <= 0 means "all available".         */
/* ---------------------------------------------------------------------- */

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_gesv_batch(int n, int64_t batch, const double *A, const double *b, double *x,
                    int32_t *ipiv, int32_t *info, double *lu_out, double *min_gap,
                    int nthreads)
{
    const size_t nn = (size_t)n * (size_t)n;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        double *work = (double *)malloc(sizeof(double) * (nn ? nn : 1));
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t s = 0; s < batch; ++s) {
            info[s] = orc_gesv(n, A + (size_t)s * nn, b + (size_t)s * n, x + (size_t)s * n,
                               ipiv + (size_t)s * n, lu_out ? lu_out + (size_t)s * nn : NULL,
                               work, min_gap ? min_gap + s : NULL);
        }
        free(work);
    }
    (void)nthreads;
}

void orc_getrf_batch(int n, int64_t batch, double *A, int32_t *ipiv, int32_t *info,
                     double *min_gap, int nthreads)
{
    const size_t nn = (size_t)n * (size_t)n;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int64_t s = 0; s < batch; ++s)
        info[s] = orc_getrf(n, A + (size_t)s * nn, ipiv + (size_t)s * n,
                            min_gap ? min_gap + s : NULL);
    (void)nthreads;
}

void orc_getrs_batch(int n, int64_t batch, const double *LU, const int32_t *ipiv, double *B,
                     int nthreads)
{
    const size_t nn = (size_t)n * (size_t)n;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int64_t s = 0; s < batch; ++s)
        orc_getrs(n, LU + (size_t)s * nn, ipiv + (size_t)s * n, B + (size_t)s * n);
    (void)nthreads;
}

/* ---------------------------------------------------------------------- */
/* Mixed precision: binary32 factorization, binary64 refinement            */
/* ---------------------------------------------------------------------- */
/*
 * The paper factors in binary64 only.  The mixed-precision variant follows
 * the published iterative-refinement scheme of Langou et al. (2006), the
 * one of LAPACK's dsgesv: factor a binary32 copy of A, solve in binary32,
 * then correct the binary64 solution with binary64 residuals and binary32
 * correction solves, falling back to the binary64 LUpp when refinement does
 * not converge.  Every operation below is a single IEEE round-to-nearest
 * operation in the stated format, in the stated order, so that a GPU
 * implementation can reproduce each result bit for bit.
 */

/* |a| > |b| for binary32 with NaN ranked above every number (as mag_greater). */
static int mag_greater_f(float a, float b)
{
    if (isnan(a)) return !isnan(b);
    if (isnan(b)) return 0;
    return fabsf(a) > fabsf(b);
}

/* FLT_MIN <= |v| < Inf (a usable binary32 pivot). */
static int usable_f(float v) { return fabsf(v) >= FLT_MIN && fabsf(v) < INFINITY; }

/*
 * orc_sgetrf: binary32 PA = LU with the steps of orc_getrf (first maximum,
 * full row swaps, l_ik = a_ik * RN32(1/a_kk), a_ij = fmaf(-l_ik, a_kj, a_ij)).
 * No sfmin branch and no zero-pivot continuation: a pivot that is not in
 * [FLT_MIN, Inf) (zero, subnormal, Inf or NaN) stops the factorization and
 * returns 1 -- the caller then solves in binary64.  Returns 0 otherwise.
 */
int orc_sgetrf(int n, float *a, int32_t *ipiv)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (mag_greater_f(AT(a, n, i, k), AT(a, n, p, k))) p = i;
        ipiv[k] = p + 1;
        if (!usable_f(AT(a, n, p, k))) return 1;
        if (p != k)
            for (int j = 0; j < n; ++j) {
                float t = AT(a, n, k, j);
                AT(a, n, k, j) = AT(a, n, p, j);
                AT(a, n, p, j) = t;
            }
        float r = 1.0f / AT(a, n, k, k);
        for (int i = k + 1; i < n; ++i) AT(a, n, i, k) = AT(a, n, i, k) * r;
        for (int j = k + 1; j < n; ++j)
            for (int i = k + 1; i < n; ++i)
                AT(a, n, i, j) = fmaf(-AT(a, n, i, k), AT(a, n, k, j), AT(a, n, i, j));
    }
    return 0;
}

/*
 * orc_sgetrs: binary32 solve with the factors of orc_sgetrf: interchanges in
 * order k = 0..n-1, forward y_i = fmaf(-l_ij, y_j, y_i) in increasing j, back
 * s = fmaf(-u_ij, y_j, s) in decreasing j, then y_i = s * RN32(1/u_ii) (a
 * multiplication by the rounded reciprocal, not a division).  Returns 1 if a
 * result is NaN or +-Inf, else 0.
 */
int orc_sgetrs(int n, const float *lu, const int32_t *ipiv, float *y)
{
    for (int k = 0; k < n; ++k) {
        int p = ipiv[k] - 1;
        if (p != k) {
            float t = y[k];
            y[k] = y[p];
            y[p] = t;
        }
    }
    for (int i = 1; i < n; ++i) {
        float s = y[i];
        for (int j = 0; j < i; ++j) s = fmaf(-AT(lu, n, i, j), y[j], s);
        y[i] = s;
    }
    int bad = 0;
    for (int i = n - 1; i >= 0; --i) {
        float s = y[i];
        for (int j = n - 1; j > i; --j) s = fmaf(-AT(lu, n, i, j), y[j], s);
        y[i] = s * (1.0f / AT(lu, n, i, i));
        if (!isfinite(y[i])) bad = 1;
    }
    return bad;
}

/*
 * orc_ir_solve: the mixed-precision solve of one system.
 *   1. A must be finite, and every nonzero a_ij must round to a binary32
 *      value in [FLT_MIN, FLT_MAX]: a32_ij = RN32(a_ij).
 *   2. anrm = max_i of the binary32 sum, in increasing j, of |a32_ij|; it
 *      must be finite.  cte = RN64(anrm * RN64(sqrt(n) * 2^-53)).
 *   3. orc_sgetrf(a32) must succeed.
 *   4. x = widen(orc_sgetrs(RN32(b))), which must be finite.
 *   5. for it = 0, 1, ...:
 *        r_i = b_i, then r_i = fma(-a_ij, x_j, r_i) for j = 0..n-1 (binary64);
 *        converged when max_i |r_i| <= RN64(max_i |x_i| * cte): steps = it;
 *        at it = 3 without convergence, stop (binary64 fallback);
 *        d = orc_sgetrs(RN32(r)), which must be finite;
 *        x_i = RN64(x_i + widen(d_i)).
 * Returns 0 with x, ipiv (the binary32 pivots, 1-based) and *steps set, or
 * 1 when any condition fails: the caller then solves with orc_gesv.
 * wf holds n*n + n floats.
 */
int orc_ir_solve(int n, const double *a, const double *b, double *x, int32_t *ipiv, int *steps,
                 float *wf)
{
    float *a32 = wf;
    float *y = wf + (size_t)n * (size_t)n;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            const double v = AT(a, n, i, j);
            if (!isfinite(v)) return 1;
            const float f = (float)v;
            if (v != 0.0 && !(fabsf(f) >= FLT_MIN && fabsf(f) <= FLT_MAX)) return 1;
            AT(a32, n, i, j) = f;
        }
    float anrm = 0.0f;
    for (int i = 0; i < n; ++i) {
        float rs = 0.0f;
        for (int j = 0; j < n; ++j) rs = rs + fabsf(AT(a32, n, i, j));
        if (rs > anrm) anrm = rs;
    }
    if (!isfinite(anrm)) return 1;
    const double cte = (double)anrm * (sqrt((double)n) * 0x1p-53);
    if (orc_sgetrf(n, a32, ipiv)) return 1;
    for (int i = 0; i < n; ++i) y[i] = (float)b[i];
    if (orc_sgetrs(n, a32, ipiv, y)) return 1;
    for (int i = 0; i < n; ++i) x[i] = (double)y[i];
    for (int it = 0;; ++it) {
        double rnrm = 0.0, xnrm = 0.0;
        for (int i = 0; i < n; ++i) {
            double r = b[i];
            for (int j = 0; j < n; ++j) r = fma(-AT(a, n, i, j), x[j], r);
            y[i] = (float)r;
            if (isnan(r) || isnan(rnrm)) rnrm = NAN;
            else if (fabs(r) > rnrm) rnrm = fabs(r);
            if (fabs(x[i]) > xnrm) xnrm = fabs(x[i]);
        }
        if (rnrm <= xnrm * cte) {
            *steps = it;
            return 0;
        }
        if (it == 3) return 1;
        if (orc_sgetrs(n, a32, ipiv, y)) return 1;
        for (int i = 0; i < n; ++i) x[i] = x[i] + (double)y[i];
    }
}

/*
 * Batched mixed-precision solve: steps[s] in 0..3 for a refined system
 * (info 0, ipiv from the binary32 factor), -1 for a system solved by
 * orc_gesv instead (ipiv, info and x as orc_gesv gives them).
 */
void orc_ir_gesv_batch(int n, int64_t batch, const double *A, const double *b, double *x,
                       int32_t *ipiv, int32_t *info, int32_t *steps, int nthreads)
{
    const size_t nn = (size_t)n * (size_t)n;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        float *wf = (float *)malloc(sizeof(float) * (nn + (size_t)n + 1));
        double *work = (double *)malloc(sizeof(double) * (nn ? nn : 1));
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t s = 0; s < batch; ++s) {
            const double *as = A + (size_t)s * nn;
            const double *bs = b + (size_t)s * n;
            int st = 0;
            if (orc_ir_solve(n, as, bs, x + (size_t)s * n, ipiv + (size_t)s * n, &st, wf) == 0) {
                steps[s] = st;
                info[s] = 0;
            } else {
                steps[s] = -1;
                info[s] = orc_gesv(n, as, bs, x + (size_t)s * n, ipiv + (size_t)s * n, NULL, work, NULL);
            }
        }
        free(wf);
        free(work);
    }
    (void)nthreads;
}

/* ---------------------------------------------------------------------- */
/* Constitutive laws                                                       */
/* ---------------------------------------------------------------------- */

/*
 * Norton viscoplastic law, implicit Euler (theta = 1), small strain,
 * isotropic elasticity, J2 flow.  Tensors use Mandel notation
 * (xx, yy, zz, sqrt2*xy, sqrt2*xz, sqrt2*yz) so that the double contraction
 * is the plain dot product.
 *
 * Unknowns x = (de_el[0..5], dp).  Inputs per point: sig0[6] (stress at the
 * start of the step), deps[6] (total strain increment).
 * Parameters: E, nu, A, m (integer >= 1), dt.
 *
 *   lambda = E nu / ((1+nu)(1-2nu)),  mu = E / (2(1+nu))
 *   sig   = sig0 + lambda tr(de_el) 1 + 2 mu de_el      (stress at step end)
 *   s     = sig - tr(sig)/3 1,  seq = sqrt(3/2 s:s)
 *   nrm   = 3/2 s / seq   (0 when seq == 0)
 *   f_el  = de_el - deps + dp nrm
 *   f_p   = dp - dt A seq^m,  seq^m as ((seq*seq)*seq)... (m-1 products)
 * Jacobian (rows f_el then f_p, columns de_el then dp):
 *   d f_el / d de_el = I + dp (2 mu / seq) (3/2 K - nrm (x) nrm)
 *   d f_el / d dp    = nrm
 *   d f_p  / d de_el = -dt A m seq^(m-1) 2 mu nrm^T
 *   d f_p  / d dp    = 1
 * with K the deviatoric projector; the seq-dependent terms vanish when
 * seq == 0.  J is written column-major 7x7 (J[i + 7 j]); F has 7 entries.
 * Optional sig_out receives sig.
 */
void orc_norton_eval(const double *prm, const double *sig0, const double *deps,
                     const double *x, double *F, double *J, double *sig_out)
{
    const double E = prm[0], nu = prm[1], Acoef = prm[2], dt = prm[4];
    const int m = (int)prm[3];
    const double lambda = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double mu = E / (2.0 * (1.0 + nu));
    const double *de = x;
    const double dp = x[6];

    double tr_de = de[0] + de[1] + de[2];
    double sig[6];
    for (int i = 0; i < 6; ++i) sig[i] = sig0[i] + 2.0 * mu * de[i];
    for (int i = 0; i < 3; ++i) sig[i] = sig[i] + lambda * tr_de;

    double p3 = (sig[0] + sig[1] + sig[2]) / 3.0;
    double s[6];
    for (int i = 0; i < 6; ++i) s[i] = sig[i];
    for (int i = 0; i < 3; ++i) s[i] = s[i] - p3;
    double ss = 0.0;
    for (int i = 0; i < 6; ++i) ss = ss + s[i] * s[i];
    double seq = sqrt(1.5 * ss);

    double nrm[6];
    for (int i = 0; i < 6; ++i) nrm[i] = (seq > 0.0) ? 1.5 * s[i] / seq : 0.0;

    double pw_m1 = 1.0;                       /* seq^(m-1) */
    for (int i = 0; i < m - 1; ++i) pw_m1 = pw_m1 * seq;
    double pw_m = pw_m1 * seq;                /* seq^m */

    for (int i = 0; i < 6; ++i) F[i] = de[i] - deps[i] + dp * nrm[i];
    F[6] = dp - dt * Acoef * pw_m;

    if (J) {
        double c = (seq > 0.0) ? dp * 2.0 * mu / seq : 0.0;
        for (int j = 0; j < 6; ++j)
            for (int i = 0; i < 6; ++i) {
                double kij = (i == j ? 1.0 : 0.0) - ((i < 3 && j < 3) ? 1.0 / 3.0 : 0.0);
                double v = 1.5 * kij - nrm[i] * nrm[j];
                J[i + 7 * j] = (i == j ? 1.0 : 0.0) + c * v;
            }
        for (int i = 0; i < 6; ++i) J[i + 7 * 6] = nrm[i];
        double g = -dt * Acoef * (double)m * pw_m1 * 2.0 * mu;
        for (int j = 0; j < 6; ++j) J[6 + 7 * j] = g * nrm[j];
        J[6 + 7 * 6] = 1.0;
    }
    if (sig_out)
        for (int i = 0; i < 6; ++i) sig_out[i] = sig[i];
}

/*
 * Synthetic law F(x) = A x + c .* tanh(x) - b, J = A + diag(c .* (1 - tanh(x)^2)).
 * A is column-major n x n.  Sums run in increasing j with plain adds.
 */
void orc_tanh_eval(int n, const double *A, const double *c, const double *b, const double *x,
                   double *F, double *J)
{
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s = s + AT(A, n, i, j) * x[j];
        double t = tanh(x[i]);
        F[i] = s + c[i] * t - b[i];
    }
    if (J) {
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) AT(J, n, i, j) = AT(A, n, i, j);
        for (int i = 0; i < n; ++i) {
            double t = tanh(x[i]);
            AT(J, n, i, i) = AT(J, n, i, i) + c[i] * (1.0 - t * t);
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Newton driver (Sec. 2.1, Eqs. 1-3; one point at a time as Algorithm 2)  */
/* ---------------------------------------------------------------------- */

static double norm2(int n, const double *v)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = s + v[i] * v[i];
    return sqrt(s);
}

enum { ORC_CONVERGED = 0, ORC_MAXITER = 1, ORC_SINGULAR = 2, ORC_NONFINITE = 3 };

/*
 * Generic per-point Newton loop.  eval(ctx, x, F, J) fills the residual and
 * the Jacobian.  k counts linear solves.
 *   r0 = ||F(x0)||_2
 *   loop: r = ||F(x_k)||_2
 *         r not finite            -> status 3
 *         r <= rtol*r0 or r0 == 0 -> status 0 (converged), iterations = k
 *         k == max_iter           -> status 1
 *         solve J dx = -F by orc_gesv; info != 0 -> status 2
 *         x += dx; k += 1
 * rmin_ratio (nullable) receives min over the tests of |r/(rtol r0) - 1|,
 * which flags points whose stopping decision sits at the threshold.
 */
typedef void (*orc_eval_fn)(const void *ctx, const double *x, double *F, double *J);

static int newton_point(int n, orc_eval_fn eval, const void *ctx, double *x, double rtol,
                        int max_iter, int32_t *iterations, double *rmin_ratio)
{
    double F[32], J[32 * 32], LU[32 * 32], dx[32], rhs[32];
    int32_t piv[32];
    eval(ctx, x, F, J);
    double r0 = norm2(n, F);
    double closest = INFINITY;
    int k = 0, status;
    for (;;) {
        double r = (k == 0) ? r0 : norm2(n, F);
        if (!isfinite(r)) { status = ORC_NONFINITE; break; }
        if (r0 > 0.0) {
            double q = fabs(r / (rtol * r0) - 1.0);
            if (q < closest) closest = q;
        }
        if (r <= rtol * r0 || r0 == 0.0) { status = ORC_CONVERGED; break; }
        if (k == max_iter) { status = ORC_MAXITER; break; }
        for (int i = 0; i < n; ++i) rhs[i] = -F[i];
        int info = orc_gesv(n, J, rhs, dx, piv, LU, NULL, NULL);
        if (info != 0) { status = ORC_SINGULAR; break; }
        for (int i = 0; i < n; ++i) x[i] = x[i] + dx[i];
        ++k;
        eval(ctx, x, F, J);
    }
    *iterations = k;
    if (rmin_ratio) *rmin_ratio = closest;
    return status;
}

typedef struct {
    const double *prm, *sig0, *deps;
} norton_ctx;

static void norton_eval_cb(const void *c, const double *x, double *F, double *J)
{
    const norton_ctx *ctx = (const norton_ctx *)c;
    orc_norton_eval(ctx->prm, ctx->sig0, ctx->deps, x, F, J, NULL);
}

typedef struct {
    int n;
    const double *A, *c, *b;
} tanh_ctx;

static void tanh_eval_cb(const void *cc, const double *x, double *F, double *J)
{
    const tanh_ctx *ctx = (const tanh_ctx *)cc;
    orc_tanh_eval(ctx->n, ctx->A, ctx->c, ctx->b, x, F, J);
}

/*
 * orc_norton_tangent: consistent tangent operator of the implicit Norton
 * law at a converged state x (Sec. 4.3: one multi-right-hand-side solve
 * after convergence).  Differentiating F(x(deps); deps) = 0 gives
 * J dx/ddeps = -dF/ddeps = [I_6; 0] (f_el = de_el - deps + dp n, f_p does
 * not involve deps), so X = J^{-1} [I_6; 0] (7x6, six solves with the
 * factors of one orc_getrf) and dsig/ddeps = C X[0..5][.], with the Mandel
 * elasticity C = lambda 1 (x) 1 + 2 mu I.  D receives the 6x6 tangent
 * column-major (D[i + 6 j] = dsig_i / ddeps_j).  Returns the info of the
 * factorization (D is NaN when it is not 0).
 */
int orc_norton_tangent(const double *prm, const double *sig0, const double *deps, const double *x, double *D)
{
    const double E = prm[0], nu = prm[1];
    const double lambda = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double mu = E / (2.0 * (1.0 + nu));
    double F[7], J[49], X[7];
    int32_t piv[7];
    orc_norton_eval(prm, sig0, deps, x, F, J, NULL);
    int info = orc_getrf(7, J, piv, NULL);
    if (info != 0) {
        for (int i = 0; i < 36; ++i) D[i] = NAN;
        return info;
    }
    for (int j = 0; j < 6; ++j) {
        for (int i = 0; i < 7; ++i) X[i] = (i == j) ? 1.0 : 0.0;
        orc_getrs(7, J, piv, X);
        const double tr = X[0] + X[1] + X[2];
        for (int i = 0; i < 6; ++i) D[i + 6 * j] = 2.0 * mu * X[i] + (i < 3 ? lambda * tr : 0.0);
    }
    return 0;
}

/*
 * Norton Newton over a batch of points (point p: sig0 at 6p, deps at 6p,
 * x at 7p).  x_init_default != 0: x0 = (deps, 0), the elastic predictor;
 * otherwise x holds x0 on entry.  sig_out (nullable) receives the stress at
 * the converged state.
 */
void orc_newton_norton_batch(const double *prm, int64_t npoints, const double *sig0,
                             const double *deps, double *x, int x_init_default,
                             int32_t *iterations, int32_t *status, double *sig_out,
                             double *rmin_ratio, double rtol, int max_iter, int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int64_t p = 0; p < npoints; ++p) {
        norton_ctx ctx = {prm, sig0 + 6 * p, deps + 6 * p};
        double *xp = x + 7 * p;
        if (x_init_default) {
            for (int i = 0; i < 6; ++i) xp[i] = ctx.deps[i];
            xp[6] = 0.0;
        }
        status[p] = newton_point(7, norton_eval_cb, &ctx, xp, rtol, max_iter, iterations + p,
                                 rmin_ratio ? rmin_ratio + p : NULL);
        if (sig_out) {
            double F[7];
            orc_norton_eval(prm, ctx.sig0, ctx.deps, xp, F, NULL, sig_out + 6 * p);
        }
    }
    (void)nthreads;
}

/*
 * tanh-law Newton over a batch of points of one size n (point p: A at p*n*n,
 * c, b and x at p*n).  x_init_default != 0: x0 = 0.
 */
void orc_newton_tanh_batch(int n, int64_t npoints, const double *A, const double *c,
                           const double *b, double *x, int x_init_default, int32_t *iterations,
                           int32_t *status, double *rmin_ratio, double rtol, int max_iter,
                           int nthreads)
{
    const size_t nn = (size_t)n * (size_t)n;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int64_t p = 0; p < npoints; ++p) {
        tanh_ctx ctx = {n, A + (size_t)p * nn, c + (size_t)p * n, b + (size_t)p * n};
        double *xp = x + (size_t)p * n;
        if (x_init_default)
            for (int i = 0; i < n; ++i) xp[i] = 0.0;
        status[p] = newton_point(n, tanh_eval_cb, &ctx, xp, rtol, max_iter, iterations + p,
                                 rmin_ratio ? rmin_ratio + p : NULL);
    }
    (void)nthreads;
}
