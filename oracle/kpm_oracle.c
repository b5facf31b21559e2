/*
 * kpm_oracle.c -- plain, slow, obviously-correct FP64 reference of the
 * KPM-DOS hot path of Kreutzer et al., "Performance Engineering of the
 * Kernel Polynomial Method on Large-Scale CPU-GPU Systems" (IPDPS 2015).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  The product library never
 * links, loads or calls it, and the two share no code, header or table.
 *
 * Conventions
 *   - complex double precision throughout (C99 double complex);
 *   - the sparse matrix H is CSR: row_ptr[n+1] (int64), col[nnz] (int32),
 *     val_ri[2*nnz] (interleaved re, im);
 *   - vectors are complex[n] as interleaved (re, im) doubles;
 *   - one random vector at a time; every sum runs in ascending row order;
 *   - the rescaling H~ = a (H - b 1) is applied with the raw (a, b) at every
 *     step, never folded into the matrix.
 *
 * Every function returns 0 on success and a negative value on bad input.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

/* ---------------------------------------------------------------------
 * SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the state advances by the
 * odd constant GOLDEN and each output is mix(state).  The k-th output of a
 * generator started at s0 is therefore mix(s0 + k*GOLDEN).
 *   key(seed, stream)       = mix(seed + (stream+1)*GOLDEN)
 *   u(seed, stream, index)  = (mix(key + (index+1)*GOLDEN) >> 11) * 2^-53
 * The paper only says "rand()" for the start vectors (Figs. 3-5).
 * ------------------------------------------------------------------- */
static const uint64_t GOLDEN = 0x9E3779B97F4A7C15ULL;

static uint64_t splitmix64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double oracle_uniform(uint64_t seed, uint64_t stream, uint64_t index)
{
    uint64_t key = splitmix64_mix(seed + (stream + 1) * GOLDEN);
    uint64_t x = splitmix64_mix(key + (index + 1) * GOLDEN);
    return (double)(x >> 11) * 0x1.0p-53;
}

/* Random-phase start vector r of length n: entry i is exp(2 pi i u) with
 * u = u(seed, 1, r*n + i).  Unit modulus, so <v|v> = n. */
int oracle_random_phase_vector(uint64_t seed, int64_t n, int64_t r, double *v_ri)
{
    if (n < 0 || r < 0 || (n > 0 && !v_ri))
        return ORACLE_EINVAL;
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t i = 0; i < n; i++) {
        double u = oracle_uniform(seed, 1, (uint64_t)r * (uint64_t)n + (uint64_t)i);
        v_ri[2 * i] = cos(two_pi * u);
        v_ri[2 * i + 1] = sin(two_pi * u);
    }
    return 0;
}

/* ---------------------------------------------------------------------
 * CSR sanity check shared by the entry points of this file.
 * ------------------------------------------------------------------- */
static int check_csr(int64_t n, const int64_t *row_ptr, const int32_t *col,
                     const double *val_ri)
{
    if (n < 0 || !row_ptr)
        return ORACLE_EINVAL;
    if (row_ptr[0] != 0)
        return ORACLE_EINVAL;
    for (int64_t i = 0; i < n; i++) {
        if (row_ptr[i + 1] < row_ptr[i])
            return ORACLE_EINVAL;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++)
            if (col[k] < 0 || col[k] >= n)
                return ORACLE_EINVAL;
    }
    if (row_ptr[n] > 0 && (!col || !val_ri))
        return ORACLE_EINVAL;
    return 0;
}

/* ---------------------------------------------------------------------
 * Spectral bounds by Gershgorin's circle theorem (the paper determines the
 * rescaling a, b "with Gershgorin's circle theorem or a few Lanczos sweeps",
 * Sec. "Problem Description").  For Hermitian H every eigenvalue lies in
 * some interval [Re h_ii - r_i, Re h_ii + r_i], r_i = sum_{j != i} |h_ij|.
 * ------------------------------------------------------------------- */
int oracle_gershgorin(int64_t n, const int64_t *row_ptr, const int32_t *col,
                      const double *val_ri, double *emin, double *emax)
{
    if (check_csr(n, row_ptr, col, val_ri) || n < 1 || !emin || !emax)
        return ORACLE_EINVAL;
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < n; i++) {
        double centre = 0.0, radius = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
            double complex h = val_ri[2 * k] + I * val_ri[2 * k + 1];
            if (col[k] == i)
                centre += creal(h);
            else
                radius += cabs(h);
        }
        if (centre - radius < lo)
            lo = centre - radius;
        if (centre + radius > hi)
            hi = centre + radius;
    }
    *emin = lo;
    *emax = hi;
    return 0;
}

/* Rescaling H~ = a (H - b 1) that maps [emin, emax] into [-(1-eps), 1-eps]. */
int oracle_scale_from_bounds(double emin, double emax, double eps, double *a, double *b)
{
    if (!(emax > emin) || !(eps >= 0.0 && eps < 1.0) || !a || !b)
        return ORACLE_EINVAL;
    *b = 0.5 * (emax + emin);
    *a = (1.0 - eps) * 2.0 / (emax - emin);
    return 0;
}

/* ---------------------------------------------------------------------
 * y = H x  (plain CSR sparse matrix-vector product, row order).
 * ------------------------------------------------------------------- */
static void csr_matvec(int64_t n, const int64_t *row_ptr, const int32_t *col,
                       const double *val_ri, const double complex *x, double complex *y)
{
    for (int64_t i = 0; i < n; i++) {
        double complex acc = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
            double complex h = val_ri[2 * k] + I * val_ri[2 * k + 1];
            acc += h * x[col[k]];
        }
        y[i] = acc;
    }
}

/* <x|y> = sum_i conj(x_i) y_i, conjugate-linear in the bra. */
static double complex inner(int64_t n, const double complex *x, const double complex *y)
{
    double complex s = 0.0;
    for (int64_t i = 0; i < n; i++)
        s += conj(x[i]) * y[i];
    return s;
}

/* ---------------------------------------------------------------------
 * One augmented step (the fused operation of Figs. 4 and 5):
 *     w <- 2a (H - b 1) v - w,   eta_even = <v|v>,   eta_odd = <w|v>
 * with w the updated vector.  eta_out = {<v|v>, Re<w|v>, Im<w|v>}.
 * v_ri, w_ri: complex[n] interleaved; w is overwritten.
 * ------------------------------------------------------------------- */
int oracle_aug_spmv(int64_t n, const int64_t *row_ptr, const int32_t *col,
                    const double *val_ri, double a, double b,
                    const double *v_ri, double *w_ri, double *eta_out)
{
    if (check_csr(n, row_ptr, col, val_ri) || !v_ri || !w_ri || !eta_out)
        return ORACLE_EINVAL;
    double complex *v = malloc(sizeof(double complex) * (size_t)(n ? n : 1));
    double complex *w = malloc(sizeof(double complex) * (size_t)(n ? n : 1));
    double complex *u = malloc(sizeof(double complex) * (size_t)(n ? n : 1));
    if (!v || !w || !u) {
        free(v); free(w); free(u);
        return ORACLE_ENOMEM;
    }
    for (int64_t i = 0; i < n; i++) {
        v[i] = v_ri[2 * i] + I * v_ri[2 * i + 1];
        w[i] = w_ri[2 * i] + I * w_ri[2 * i + 1];
    }
    csr_matvec(n, row_ptr, col, val_ri, v, u);            /* u = H v        */
    for (int64_t i = 0; i < n; i++)
        w[i] = 2.0 * a * (u[i] - b * v[i]) - w[i];         /* w = 2a(u-bv)-w */
    double complex vv = inner(n, v, v);
    double complex wv = inner(n, w, v);
    eta_out[0] = creal(vv);
    eta_out[1] = creal(wv);
    eta_out[2] = cimag(wv);
    for (int64_t i = 0; i < n; i++) {
        w_ri[2 * i] = creal(w[i]);
        w_ri[2 * i + 1] = cimag(w[i]);
    }
    free(v); free(w); free(u);
    return 0;
}

/* ---------------------------------------------------------------------
 * KPM-DOS for one start vector (Eq. 3 and the scalar products that follow
 * it; Figs. 3-5 with one column):
 *     nu_0 = v0
 *     nu_1 = H~ nu_0,                        H~ = a (H - b 1)
 *     nu_{m+1} = 2 H~ nu_m - nu_{m-1}
 *     eta_{2m} = <nu_m|nu_m>,  eta_{2m+1} = <nu_{m+1}|nu_m>
 * M even, M >= 2: one initial application (eta_0, eta_1) plus M/2 - 1
 * recurrence steps give eta_0 .. eta_{M-1}, i.e. M moments from M/2
 * applications of the matrix (the count behind Eq. 4).
 * eta_re[M] gets the real parts; eta_im[M] (may be NULL) the imaginary parts,
 * which vanish in exact arithmetic for Hermitian H.
 * ------------------------------------------------------------------- */
int oracle_kpm_vector(int64_t n, const int64_t *row_ptr, const int32_t *col,
                      const double *val_ri, double a, double b, int32_t M,
                      const double *v0_ri, double *eta_re, double *eta_im)
{
    if (check_csr(n, row_ptr, col, val_ri) || M < 2 || (M % 2) != 0 || !v0_ri || !eta_re)
        return ORACLE_EINVAL;
    size_t bytes = sizeof(double complex) * (size_t)(n ? n : 1);
    double complex *prev = malloc(bytes);   /* nu_{m-1} */
    double complex *cur = malloc(bytes);    /* nu_m     */
    double complex *next = malloc(bytes);   /* nu_{m+1} */
    double complex *hx = malloc(bytes);
    if (!prev || !cur || !next || !hx) {
        free(prev); free(cur); free(next); free(hx);
        return ORACLE_ENOMEM;
    }
    for (int64_t i = 0; i < n; i++)
        cur[i] = v0_ri[2 * i] + I * v0_ri[2 * i + 1];

    /* initial step: nu_1 = a (H nu_0 - b nu_0); eta_0, eta_1 */
    csr_matvec(n, row_ptr, col, val_ri, cur, hx);
    for (int64_t i = 0; i < n; i++)
        next[i] = a * (hx[i] - b * cur[i]);
    double complex e0 = inner(n, cur, cur);
    double complex e1 = inner(n, next, cur);
    eta_re[0] = creal(e0);
    eta_re[1] = creal(e1);
    if (eta_im) {
        eta_im[0] = cimag(e0);
        eta_im[1] = cimag(e1);
    }

    for (int32_t m = 1; m < M / 2; m++) {
        /* shift: prev <- nu_{m-1}, cur <- nu_m */
        double complex *tmp = prev;
        prev = cur;
        cur = next;
        next = tmp;
        csr_matvec(n, row_ptr, col, val_ri, cur, hx);
        for (int64_t i = 0; i < n; i++)
            next[i] = 2.0 * a * (hx[i] - b * cur[i]) - prev[i];
        double complex ee = inner(n, cur, cur);    /* eta_{2m}   = <nu_m|nu_m>     */
        double complex eo = inner(n, next, cur);   /* eta_{2m+1} = <nu_{m+1}|nu_m> */
        eta_re[2 * m] = creal(ee);
        eta_re[2 * m + 1] = creal(eo);
        if (eta_im) {
            eta_im[2 * m] = cimag(ee);
            eta_im[2 * m + 1] = cimag(eo);
        }
    }
    free(prev); free(cur); free(next); free(hx);
    return 0;
}

/* KPM-DOS for random-phase start vector number r drawn from seed. */
int oracle_kpm_random_vector(int64_t n, const int64_t *row_ptr, const int32_t *col,
                             const double *val_ri, double a, double b, int32_t M,
                             uint64_t seed, int64_t r, double *eta_re, double *eta_im)
{
    if (n < 0 || r < 0)
        return ORACLE_EINVAL;
    double *v0 = malloc(sizeof(double) * 2 * (size_t)(n ? n : 1));
    if (!v0)
        return ORACLE_ENOMEM;
    int rc = oracle_random_phase_vector(seed, n, r, v0);
    if (rc == 0)
        rc = oracle_kpm_vector(n, row_ptr, col, val_ri, a, b, M, v0, eta_re, eta_im);
    free(v0);
    return rc;
}

/* ---------------------------------------------------------------------
 * Reconstruction (the paper's "second computationally inexpensive step",
 * Sec. "Problem Description", which it does not spell out).
 *
 * Moments of one vector: c_n = <nu_0|T_n(H~)|nu_0>.  From
 * T_{2k} = 2 T_k T_k - T_0 and T_{2k+1} = 2 T_{k+1} T_k - T_1 (Hermitian
 * T_k): c_{2k} = 2 eta_{2k} - eta_0, c_{2k+1} = 2 eta_{2k+1} - eta_1.
 * Stochastic trace over R vectors, normalised so that mu_0 = 1:
 *     mu_n = sum_r c_n^(r) / sum_r eta_0^(r).
 * eta is [R][M] (row r holds the M moments of vector r).
 * ------------------------------------------------------------------- */
int oracle_eta_to_mu(const double *eta, int32_t M, int32_t R, double *mu)
{
    if (!eta || !mu || M < 2 || (M % 2) != 0 || R < 1)
        return ORACLE_EINVAL;
    double norm = 0.0;
    for (int32_t r = 0; r < R; r++)
        norm += eta[(size_t)r * M + 0];
    if (!(norm > 0.0))
        return ORACLE_EINVAL;
    for (int32_t k = 0; k < M; k++) {
        double s = 0.0;
        for (int32_t r = 0; r < R; r++) {
            const double *e = eta + (size_t)r * M;
            double c;
            if (k == 0)
                c = e[0];
            else if (k == 1)
                c = e[1];
            else if (k % 2 == 0)
                c = 2.0 * e[k] - e[0];
            else
                c = 2.0 * e[k] - e[1];
            s += c;
        }
        mu[k] = s / norm;
    }
    return 0;
}

/* Jackson damping factors g_n, n = 0..M-1, for an expansion of M moments:
 * g_n = [(M-n+1) cos(pi n/(M+1)) + sin(pi n/(M+1)) cot(pi/(M+1))] / (M+1). */
int oracle_jackson(int32_t M, double *g)
{
    if (M < 1 || !g)
        return ORACLE_EINVAL;
    const double pi = 3.14159265358979323846264338327950288;
    double q = pi / (double)(M + 1);
    for (int32_t k = 0; k < M; k++)
        g[k] = ((double)(M - k + 1) * cos(q * k) + sin(q * k) * cos(q) / sin(q)) / (double)(M + 1);
    return 0;
}

/* Jackson-damped Chebyshev density on K Chebyshev nodes
 *     x_k = cos(pi (k + 1/2) / K),   k = 0..K-1,
 *     rho~(x) = [g_0 mu_0 + 2 sum_{n>=1} g_n mu_n T_n(x)] / (pi sqrt(1-x^2)),
 * with T_n(x_k) = cos(n theta_k), theta_k = pi (k+1/2)/K.  In the original
 * energy variable E = x/a + b the density is rho(E) = a rho~(x); it
 * integrates to mu_0 (= 1), i.e. this is Eq. 2 divided by N. */
int oracle_dos(const double *mu, int32_t M, int32_t K, double a, double b,
               double *energy, double *rho)
{
    if (!mu || M < 1 || K < 1 || !(a > 0.0) || !energy || !rho)
        return ORACLE_EINVAL;
    const double pi = 3.14159265358979323846264338327950288;
    double *g = malloc(sizeof(double) * (size_t)M);
    if (!g)
        return ORACLE_ENOMEM;
    oracle_jackson(M, g);
    for (int32_t k = 0; k < K; k++) {
        double theta = pi * ((double)k + 0.5) / (double)K;
        double x = cos(theta);
        double s = g[0] * mu[0];
        for (int32_t n = 1; n < M; n++)
            s += 2.0 * g[n] * mu[n] * cos((double)n * theta);
        energy[k] = x / a + b;
        rho[k] = a * s / (pi * sin(theta));
    }
    free(g);
    return 0;
}
