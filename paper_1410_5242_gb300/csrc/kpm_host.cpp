// Host-only parts of libkpm: input validation, Gershgorin bounds, the
// rescaling, the CSR -> SELL-C-sigma converter, and the reconstruction
// eta -> mu -> Jackson DOS.  None of these needs a GPU.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <thread>
#include <vector>

#include "kpm_internal.h"

namespace kpm {

// Host threads for the conversions of large inputs: KPM_HOST_THREADS if set
// (>= 1), else the hardware concurrency, at most kMaxHostThreads.
constexpr int kMaxHostThreads = 64;

int host_threads()
{
    const char *env = std::getenv("KPM_HOST_THREADS");
    if (env && *env) {
        const long v = std::strtol(env, nullptr, 10);
        if (v >= 1)
            return (int)std::min<long>(v, kMaxHostThreads);
    }
    const unsigned hw = std::thread::hardware_concurrency();
    return hw ? (int)std::min<unsigned>(hw, kMaxHostThreads) : 1;
}

// Calls f(begin, end, part) on contiguous parts of [0, n), part p covering
// the p-th range in order, on up to host_threads() threads with at least
// `grain` items each; the calling thread takes part 0.  Returns the number
// of parts.  If a thread cannot be started its part runs on the caller.
template <typename F>
int parallel_parts(int64_t n, int64_t grain, F &&f)
{
    const int64_t want = grain > 0 ? (n + grain - 1) / grain : 1;
    const int parts = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), want));
    auto range = [&](int p, int64_t &b, int64_t &e) {
        b = n * p / parts;
        e = n * (p + 1) / parts;
    };
    std::vector<std::thread> pool;
    std::vector<int> inline_parts;
    for (int p = 1; p < parts; p++) {
        int64_t b, e;
        range(p, b, e);
        try {
            pool.emplace_back([&f, b, e, p]() { f(b, e, p); });
        } catch (...) {
            inline_parts.push_back(p);
        }
    }
    int64_t b0, e0;
    range(0, b0, e0);
    f(b0, e0, 0);
    for (int p : inline_parts) {
        int64_t b, e;
        range(p, b, e);
        f(b, e, p);
    }
    for (std::thread &t : pool)
        t.join();
    return parts;
}

int validate_csr(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val_ri)
{
    return validate_csr_rect(n, n, row_ptr, col, val_ri);
}

int validate_csr_rect(int64_t n, int64_t n_cols, const int64_t *row_ptr, const int32_t *col,
                      const double *val_ri)
{
    if (n < 1 || n > INT32_MAX || n_cols < n || n_cols > INT32_MAX || !row_ptr)
        return KPM_EINVAL;
    if (row_ptr[0] != 0)
        return KPM_EINVAL;
    std::atomic<bool> bad(false);
    parallel_parts(n, 1 << 16, [&](int64_t b, int64_t e, int) {
        for (int64_t i = b; i < e; i++)
            if (row_ptr[i + 1] < row_ptr[i]) {
                bad = true;
                return;
            }
    });
    if (bad)
        return KPM_EINVAL;
    const int64_t nnz = row_ptr[n];
    if (nnz > 0 && (!col || !val_ri))
        return KPM_EINVAL;
    parallel_parts(n, 1 << 14, [&](int64_t b, int64_t e, int) {
        for (int64_t i = b; i < e; i++) {
            int64_t prev = -1;
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
                if (col[k] < 0 || col[k] >= n_cols || col[k] <= prev) {
                    bad = true;
                    return;
                }
                prev = col[k];
            }
        }
    });
    if (bad)
        return KPM_EINVAL;
    parallel_parts(2 * nnz, 1 << 18, [&](int64_t b, int64_t e, int) {
        for (int64_t k = b; k < e; k++)
            if (!std::isfinite(val_ri[k])) {
                bad = true;
                return;
            }
    });
    return bad ? KPM_EINVAL : KPM_OK;
}

int check_hermitian(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val_ri,
                    double rel_tol)
{
    double vmax = 0.0;
    for (int64_t k = 0; k < row_ptr[n]; k++)
        vmax = std::max(vmax, std::hypot(val_ri[2 * k], val_ri[2 * k + 1]));
    const double tol = rel_tol * (vmax > 0 ? vmax : 1.0);
    for (int64_t i = 0; i < n; i++) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
            const int32_t j = col[k];
            const double re = val_ri[2 * k], im = val_ri[2 * k + 1];
            const int32_t *b = col + row_ptr[j], *e = col + row_ptr[j + 1];
            const int32_t *f = std::lower_bound(b, e, (int32_t)i);
            double tre = 0.0, tim = 0.0;
            if (f != e && *f == i) {
                const int64_t kk = f - col;
                tre = val_ri[2 * kk];
                tim = val_ri[2 * kk + 1];
            }
            // h_ji must equal conj(h_ij)
            if (std::fabs(tre - re) > tol || std::fabs(tim + im) > tol)
                return KPM_ENOTHERMITIAN;
        }
    }
    return KPM_OK;
}

}  // namespace kpm

using namespace kpm;

extern "C" {

void kpm_default_options(kpm_options *opt)
{
    if (!opt)
        return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = KPM_PREC_FP64;
    opt->chunk_height = 32;
    opt->sigma = 256;
}

const char *kpm_status_string(int status)
{
    switch (status) {
    case KPM_OK: return "KPM_OK";
    case KPM_EINVAL: return "KPM_EINVAL: invalid argument";
    case KPM_ENOTHERMITIAN: return "KPM_ENOTHERMITIAN: matrix is not Hermitian";
    case KPM_ENOMEM: return "KPM_ENOMEM: out of memory";
    case KPM_ECUDA: return "KPM_ECUDA: CUDA runtime error";
    case KPM_ETIMEOUT: return "KPM_ETIMEOUT: bounded device wait expired";
    case KPM_EUNSUPPORTED: return "KPM_EUNSUPPORTED: unsupported request";
    default: return "unknown KPM status";
    }
}

int kpm_gershgorin(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val_ri,
                   double *emin, double *emax)
{
    if (!emin || !emax)
        return KPM_EINVAL;
    int rc = validate_csr(n, row_ptr, col, val_ri);
    if (rc)
        return rc;
    // rows are independent and min/max do not depend on the order: each
    // part reduces its rows, the parts are reduced at the end
    std::vector<double> part_lo(kMaxHostThreads, INFINITY), part_hi(kMaxHostThreads, -INFINITY);
    const int parts = parallel_parts(n, 1 << 14, [&](int64_t b, int64_t e, int part) {
        double lo = INFINITY, hi = -INFINITY;
        for (int64_t i = b; i < e; i++) {
            double centre = 0.0, radius = 0.0;
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
                if (col[k] == i)
                    centre = val_ri[2 * k];
                else
                    radius += std::hypot(val_ri[2 * k], val_ri[2 * k + 1]);
            }
            lo = std::min(lo, centre - radius);
            hi = std::max(hi, centre + radius);
        }
        part_lo[part] = lo;
        part_hi[part] = hi;
    });
    double lo = INFINITY, hi = -INFINITY;
    for (int p = 0; p < parts; p++) {
        lo = std::min(lo, part_lo[p]);
        hi = std::max(hi, part_hi[p]);
    }
    *emin = lo;
    *emax = hi;
    return KPM_OK;
}

int kpm_scale_from_bounds(double emin, double emax, double eps, double *a, double *b)
{
    if (!a || !b || !std::isfinite(emin) || !std::isfinite(emax) || !(emax > emin) ||
        !(eps >= 0.0 && eps < 1.0))
        return KPM_EINVAL;
    *b = 0.5 * (emax + emin);
    *a = (1.0 - eps) * 2.0 / (emax - emin);
    return KPM_OK;
}

int kpm_eta_to_mu(const double *eta, int32_t M, int32_t R, double *mu)
{
    if (!eta || !mu || M < 2 || (M & 1) || R < 1)
        return KPM_EINVAL;
    double norm = 0.0;
    for (int32_t r = 0; r < R; r++)
        norm += eta[(size_t)r * M];
    if (!(norm > 0.0))
        return KPM_EINVAL;
    // Sum the per-vector terms 2*eta_n over r first, then subtract the
    // parity term R-summed: c_n = 2 eta_n - eta_{n mod 2} for n >= 2.
    double e0 = 0.0, e1 = 0.0;
    for (int32_t r = 0; r < R; r++) {
        e0 += eta[(size_t)r * M];
        e1 += eta[(size_t)r * M + 1];
    }
    mu[0] = e0 / norm;
    mu[1] = e1 / norm;
    for (int32_t k = 2; k < M; k++) {
        double s = 0.0;
        for (int32_t r = 0; r < R; r++)
            s += eta[(size_t)r * M + k];
        mu[k] = (2.0 * s - ((k & 1) ? e1 : e0)) / norm;
    }
    return KPM_OK;
}

int kpm_dos(const double *mu, int32_t M, int32_t K, double a, double b, double *energy,
            double *rho)
{
    if (!mu || !energy || !rho || M < 1 || K < 1 || !(a > 0.0) || !std::isfinite(b))
        return KPM_EINVAL;
    const double pi = 3.14159265358979323846;
    std::vector<double> gm(M);
    const double q = pi / (double)(M + 1);
    const double cotq = std::cos(q) / std::sin(q);
    for (int32_t n = 0; n < M; n++)
        gm[n] = (((double)(M - n + 1)) * std::cos(q * n) + std::sin(q * n) * cotq) /
                (double)(M + 1) * mu[n];
    // Evaluate the damped series at each node with the three-term
    // recurrence T_n = 2x T_{n-1} - T_{n-2}.
    for (int32_t k = 0; k < K; k++) {
        const double theta = pi * ((double)k + 0.5) / (double)K;
        const double x = std::cos(theta);
        double t0 = 1.0, t1 = x;
        double s = gm[0];
        if (M > 1)
            s += 2.0 * gm[1] * t1;
        for (int32_t n = 2; n < M; n++) {
            const double t2 = 2.0 * x * t1 - t0;
            s += 2.0 * gm[n] * t2;
            t0 = t1;
            t1 = t2;
        }
        energy[k] = x / a + b;
        rho[k] = a * s / (pi * std::sin(theta));
    }
    return KPM_OK;
}

// Eigenvalues and the last components of the eigenvectors of the symmetric
// tridiagonal matrix (alpha on the diagonal, beta off it), by Jacobi
// rotations (k is small: a few dozen Lanczos steps).
static void tridiag_eig(const std::vector<double> &alpha, const std::vector<double> &beta,
                        std::vector<double> &theta, std::vector<double> &last)
{
    const int k = (int)alpha.size();
    std::vector<double> A((size_t)k * k, 0.0), Q((size_t)k * k, 0.0);
    for (int i = 0; i < k; i++) {
        A[(size_t)i * k + i] = alpha[i];
        Q[(size_t)i * k + i] = 1.0;
        if (i + 1 < k)
            A[(size_t)i * k + i + 1] = A[(size_t)(i + 1) * k + i] = beta[i];
    }
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int p = 0; p < k; p++)
            for (int q = p + 1; q < k; q++)
                off += A[(size_t)p * k + q] * A[(size_t)p * k + q];
        if (off < 1e-30)
            break;
        for (int p = 0; p < k; p++)
            for (int q = p + 1; q < k; q++) {
                const double apq = A[(size_t)p * k + q];
                if (std::fabs(apq) < 1e-300)
                    continue;
                const double tau = (A[(size_t)q * k + q] - A[(size_t)p * k + p]) / (2.0 * apq);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int r = 0; r < k; r++) {  // A <- J^T A J, Q <- Q J
                    const double arp = A[(size_t)r * k + p], arq = A[(size_t)r * k + q];
                    A[(size_t)r * k + p] = c * arp - s * arq;
                    A[(size_t)r * k + q] = s * arp + c * arq;
                }
                for (int r = 0; r < k; r++) {
                    const double apr = A[(size_t)p * k + r], aqr = A[(size_t)q * k + r];
                    A[(size_t)p * k + r] = c * apr - s * aqr;
                    A[(size_t)q * k + r] = s * apr + c * aqr;
                }
                for (int r = 0; r < k; r++) {
                    const double qrp = Q[(size_t)r * k + p], qrq = Q[(size_t)r * k + q];
                    Q[(size_t)r * k + p] = c * qrp - s * qrq;
                    Q[(size_t)r * k + q] = s * qrp + c * qrq;
                }
            }
    }
    theta.resize(k);
    last.resize(k);
    for (int i = 0; i < k; i++) {
        theta[i] = A[(size_t)i * k + i];
        last[i] = Q[(size_t)(k - 1) * k + i];
    }
}

int kpm_lanczos_bounds(int64_t n, const int64_t *row_ptr, const int32_t *col,
                       const double *val_ri, int32_t steps, uint64_t seed, double *emin,
                       double *emax)
{
    if (!emin || !emax || steps < 2)
        return KPM_EINVAL;
    int rc = validate_csr(n, row_ptr, col, val_ri);
    if (rc)
        return rc;
    double glo, ghi;
    rc = kpm_gershgorin(n, row_ptr, col, val_ri, &glo, &ghi);
    if (rc)
        return rc;
    const int k = (int)std::min<int64_t>(steps, n);
    // complex vectors as interleaved doubles; q1 = random phases / sqrt(n)
    std::vector<double> qprev(2 * n, 0.0), q(2 * n), w(2 * n);
    const uint64_t G = 0x9E3779B97F4A7C15ULL;
    auto mix = [](uint64_t z) {
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    };
    const uint64_t key = mix(seed + 4 * G);  // stream 3
    const double inv = 1.0 / std::sqrt((double)n);
    for (int64_t i = 0; i < n; i++) {
        const double u = (double)(mix(key + ((uint64_t)i + 1) * G) >> 11) * 0x1.0p-53;
        q[2 * i] = std::cos(6.283185307179586 * u) * inv;
        q[2 * i + 1] = std::sin(6.283185307179586 * u) * inv;
    }
    std::vector<double> alpha, beta;
    double b_prev = 0.0;
    for (int j = 0; j < k; j++) {
        // w = H q - b_prev q_prev
        for (int64_t i = 0; i < n; i++) {
            double re = 0.0, im = 0.0;
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
                const double hr = val_ri[2 * e], hi = val_ri[2 * e + 1];
                const double xr = q[2 * (int64_t)col[e]], xi = q[2 * (int64_t)col[e] + 1];
                re += hr * xr - hi * xi;
                im += hr * xi + hi * xr;
            }
            w[2 * i] = re - b_prev * qprev[2 * i];
            w[2 * i + 1] = im - b_prev * qprev[2 * i + 1];
        }
        double a = 0.0;  // Re <q|w> (real for Hermitian H)
        for (int64_t i = 0; i < 2 * n; i++)
            a += q[i] * w[i];
        for (int64_t i = 0; i < 2 * n; i++)
            w[i] -= a * q[i];
        double bn = 0.0;
        for (int64_t i = 0; i < 2 * n; i++)
            bn += w[i] * w[i];
        bn = std::sqrt(bn);
        alpha.push_back(a);
        beta.push_back(bn);
        if (bn < 1e-12 * (std::fabs(ghi) + std::fabs(glo)) || j == k - 1)
            break;
        for (int64_t i = 0; i < 2 * n; i++) {
            qprev[i] = q[i];
            q[i] = w[i] / bn;
        }
        b_prev = bn;
    }
    std::vector<double> theta, last;
    tridiag_eig(alpha, std::vector<double>(beta.begin(), beta.end() - 1), theta, last);
    // Ritz values lie inside [lambda_min, lambda_max] and each theta_i is
    // within |beta_k s_{k,i}| of an eigenvalue; the extreme ones converge to
    // the extreme eigenvalues first, so they are widened by their own
    // residuals (interior values, ghosts included, play no part), and the
    // result is never wider than Gershgorin.
    const double bk = beta.back();
    size_t imin = 0, imax = 0;
    for (size_t i = 1; i < theta.size(); i++) {
        if (theta[i] < theta[imin])
            imin = i;
        if (theta[i] > theta[imax])
            imax = i;
    }
    *emin = std::max(theta[imin] - std::fabs(bk * last[imin]), glo);
    *emax = std::min(theta[imax] + std::fabs(bk * last[imax]), ghi);
    return KPM_OK;
}

int kpm_sell_build(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val_ri,
                   double a, double b, int32_t C, int32_t sigma, const int32_t *row_order,
                   kpm_sell *out)
{
    return kpm::sell_build_rect(n, 0, row_ptr, col, val_ri, a, b, C, sigma, row_order, out);
}

}  // extern "C"

int kpm::sell_build_rect(int64_t n, int64_t n_halo, const int64_t *row_ptr, const int32_t *col,
                         const double *val_ri, double a, double b, int32_t C, int32_t sigma,
                         const int32_t *row_order, kpm_sell *out)
{
    if (!out)
        return KPM_EINVAL;
    std::memset(out, 0, sizeof(*out));
    if (C < 1 || C > 1024 || (C & (C - 1)) || sigma < 1 || !(a > 0.0) || !std::isfinite(a) ||
        !std::isfinite(b) || n_halo < 0)
        return KPM_EINVAL;
    int rc = validate_csr_rect(n, n + n_halo, row_ptr, col, val_ri);
    if (rc)
        return rc;

    // Fold H' = 2a (H - b 1): row lengths after adding missing diagonals.
    std::vector<int32_t> len(n);
    std::vector<uint8_t> has_diag(n, 0);
    parallel_parts(n, 1 << 14, [&](int64_t lo, int64_t hi, int) {
        for (int64_t i = lo; i < hi; i++) {
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++)
                if (col[k] == i)
                    has_diag[i] = 1;
            len[i] = (int32_t)(row_ptr[i + 1] - row_ptr[i]) + ((!has_diag[i] && b != 0.0) ? 1 : 0);
        }
    });

    const int64_t n_chunks = (n + C - 1) / C;
    const int64_t n_pad = n_chunks * C;
    // sigma-window sort by descending row length (stable)
    std::vector<int32_t> perm(n_pad);
    std::iota(perm.begin(), perm.end(), 0);
    if (row_order) {
        // caller's ordering first (must be a permutation of 0..n-1)
        std::vector<uint8_t> seen(n, 0);
        for (int64_t p = 0; p < n; p++) {
            const int32_t i = row_order[p];
            if (i < 0 || i >= n || seen[i])
                return KPM_EINVAL;
            seen[i] = 1;
            perm[p] = i;
        }
    }
    if (sigma > 1) {
        // windows are sorted independently: split them among the threads
        const int64_t n_win = (n + sigma - 1) / sigma;
        parallel_parts(n_win, std::max<int64_t>(1, (1 << 14) / sigma), [&](int64_t lo, int64_t hi,
                                                                          int) {
            for (int64_t wi = lo; wi < hi; wi++) {
                const int64_t w = wi * sigma;
                const int64_t e = std::min<int64_t>(n, w + sigma);
                std::stable_sort(perm.begin() + w, perm.begin() + e,
                                 [&](int32_t x, int32_t y) { return len[x] > len[y]; });
            }
        });
    }
    std::vector<int32_t> iperm(n);
    parallel_parts(n, 1 << 16, [&](int64_t lo, int64_t hi, int) {
        for (int64_t p = lo; p < hi; p++)
            iperm[perm[p]] = (int32_t)p;
    });

    int64_t *chunk_ptr = (int64_t *)std::malloc(sizeof(int64_t) * (n_chunks + 1));
    int32_t *chunk_len = (int32_t *)std::malloc(sizeof(int32_t) * (n_chunks ? n_chunks : 1));
    int32_t *perm_out = (int32_t *)std::malloc(sizeof(int32_t) * n_pad);
    if (!chunk_ptr || !chunk_len || !perm_out) {
        std::free(chunk_ptr); std::free(chunk_len); std::free(perm_out);
        return KPM_ENOMEM;
    }
    chunk_ptr[0] = 0;
    parallel_parts(n_chunks, 1 << 10, [&](int64_t lo, int64_t hi, int) {
        for (int64_t c = lo; c < hi; c++) {
            int32_t m = 0;
            for (int64_t r = 0; r < C; r++) {
                const int64_t p = c * C + r;
                if (p < n)
                    m = std::max(m, len[perm[p]]);
            }
            chunk_len[c] = m;
        }
    });
    int64_t nnz = 0;
    for (int64_t i = 0; i < n; i++)
        nnz += len[i];
    for (int64_t c = 0; c < n_chunks; c++)
        chunk_ptr[c + 1] = chunk_ptr[c] + (int64_t)chunk_len[c] * C;
    const int64_t n_stored = chunk_ptr[n_chunks];
    int32_t *scol = (int32_t *)std::malloc(sizeof(int32_t) * (n_stored ? n_stored : 1));
    double *sval = (double *)std::malloc(sizeof(double) * 2 * (n_stored ? n_stored : 1));
    if (!scol || !sval) {
        std::free(chunk_ptr); std::free(chunk_len); std::free(perm_out);
        std::free(scol); std::free(sval);
        return KPM_ENOMEM;
    }
    const double two_a = 2.0 * a;
    // every chunk writes its own entries [chunk_ptr[c], chunk_ptr[c+1])
    parallel_parts(n_chunks, 1 << 9, [&](int64_t lo_c, int64_t hi_c, int) {
        for (int64_t c = lo_c; c < hi_c; c++) {
            const int64_t base = chunk_ptr[c];
            const int32_t clen = chunk_len[c];
            for (int64_t r = 0; r < C; r++) {
                const int64_t p = c * C + r;
                int32_t j = 0;
                auto put = [&](int32_t newcol, double re, double im) {
                    const int64_t e = base + (int64_t)j * C + r;
                    scol[e] = newcol;
                    sval[2 * e] = re;
                    sval[2 * e + 1] = im;
                    j++;
                };
                if (p < n) {
                    const int64_t i = perm[p];
                    bool diag_done = has_diag[i] || b == 0.0;
                    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
                        if (!diag_done && col[k] > i) {
                            put((int32_t)p, -two_a * b, 0.0);
                            diag_done = true;
                        }
                        double re = val_ri[2 * k], im = val_ri[2 * k + 1];
                        if (col[k] == i)
                            re = two_a * (re - b), im = two_a * im;
                        else
                            re = two_a * re, im = two_a * im;
                        // a halo column (>= n) reads the vector row after the
                        // padded local rows
                        put(col[k] < n ? iperm[col[k]] : (int32_t)(n_pad + (col[k] - n)), re, im);
                    }
                    if (!diag_done)
                        put((int32_t)p, -two_a * b, 0.0);
                }
                // padding: zero value, the row's own index (its V row is read anyway)
                while (j < clen)
                    put((int32_t)p, 0.0, 0.0);
            }
        }
    });
    std::memcpy(perm_out, perm.data(), sizeof(int32_t) * n_pad);

    out->n = n;
    out->n_pad = n_pad;
    out->C = C;
    out->sigma = sigma;
    out->n_chunks = n_chunks;
    out->nnz = nnz;
    out->n_stored = n_stored;
    out->chunk_ptr = chunk_ptr;
    out->chunk_len = chunk_len;
    out->col = scol;
    out->val_ri = sval;
    out->perm = perm_out;
    return KPM_OK;
}

extern "C" {

void kpm_sell_release(kpm_sell *s)
{
    if (!s)
        return;
    std::free(s->chunk_ptr);
    std::free(s->chunk_len);
    std::free(s->col);
    std::free(s->val_ri);
    std::free(s->perm);
    std::memset(s, 0, sizeof(*s));
}

}  // extern "C"

extern "C" {

int kpm_gather_build(const kpm_sell *s, kpm_gather *out)
{
    if (!out)
        return KPM_EINVAL;
    std::memset(out, 0, sizeof(*out));
    if (!s || !s->chunk_ptr || !s->chunk_len || (s->n_stored > 0 && !s->col))
        return KPM_EINVAL;
    if (s->C < 8)
        return KPM_EINVAL;
    const int64_t C = s->C;
    const int64_t n_chunks = s->n_chunks;
    uint16_t *lidx = (uint16_t *)std::malloc(sizeof(uint16_t) * (s->n_stored ? s->n_stored : 1));
    int64_t *run_ptr = (int64_t *)std::malloc(sizeof(int64_t) * (n_chunks + 1));
    if (!lidx || !run_ptr) {
        std::free(lidx);
        std::free(run_ptr);
        return KPM_ENOMEM;
    }
    // chunks are independent: each part of the chunk range builds its runs
    // (pairs) and per-chunk run counts, written to lidx directly; the parts'
    // runs are then concatenated in order
    std::vector<std::vector<int32_t>> part_runs(kMaxHostThreads);
    std::vector<int32_t> part_umax(kMaxHostThreads, 0), part_lmax(kMaxHostThreads, 0);
    std::atomic<bool> too_long(false), no_mem(false);
    std::vector<int64_t> run_cnt(n_chunks, 0);
    const int parts = parallel_parts(n_chunks, 1 << 9, [&](int64_t lo, int64_t hi, int part) {
        try {
            std::vector<int32_t> &runs = part_runs[part];
            std::vector<int32_t> others;
            int32_t u_max = 0, l_max = 0;
            for (int64_t c = lo; c < hi && !too_long; c++) {
                const int64_t r0 = c * C;
                const int64_t e0 = s->chunk_ptr[c];
                const int64_t cnt = (int64_t)s->chunk_len[c] * C;
                l_max = std::max(l_max, s->chunk_len[c]);
                others.clear();
                for (int64_t e = e0; e < e0 + cnt; e++) {
                    const int64_t j = s->col[e];
                    if (j < r0 || j >= r0 + C)
                        others.push_back((int32_t)j);
                }
                std::sort(others.begin(), others.end());
                others.erase(std::unique(others.begin(), others.end()), others.end());
                const int64_t u = C + (int64_t)others.size();
                if (u > 65535) {
                    too_long = true;
                    return;
                }
                u_max = std::max<int32_t>(u_max, (int32_t)u);
                // own rows, then the others; a row that continues the last run joins it
                const size_t first = runs.size();
                runs.push_back((int32_t)r0);
                runs.push_back((int32_t)C);
                for (int32_t j : others) {
                    const size_t last = runs.size() - 2;
                    if ((int64_t)runs[last] + runs[last + 1] == j)
                        runs[last + 1]++;
                    else {
                        runs.push_back(j);
                        runs.push_back(1);
                    }
                }
                run_cnt[c] = (int64_t)(runs.size() - first) / 2;
                for (int64_t e = e0; e < e0 + cnt; e++) {
                    const int64_t j = s->col[e];
                    int64_t pos;
                    if (j >= r0 && j < r0 + C)
                        pos = j - r0;
                    else
                        pos = C + (std::lower_bound(others.begin(), others.end(), (int32_t)j) -
                                   others.begin());
                    lidx[e] = (uint16_t)pos;
                }
            }
            part_umax[part] = u_max;
            part_lmax[part] = l_max;
        } catch (const std::bad_alloc &) {
            no_mem = true;
        }
    });
    if (too_long || no_mem) {
        std::free(lidx);
        std::free(run_ptr);
        return too_long ? KPM_EUNSUPPORTED : KPM_ENOMEM;
    }
    int32_t u_max = 0, l_max = 0;
    size_t total = 0;
    for (int p = 0; p < parts; p++) {
        u_max = std::max(u_max, part_umax[p]);
        l_max = std::max(l_max, part_lmax[p]);
        total += part_runs[p].size();
    }
    run_ptr[0] = 0;
    for (int64_t c = 0; c < n_chunks; c++)
        run_ptr[c + 1] = run_ptr[c] + run_cnt[c];
    int32_t *runs_out = (int32_t *)std::malloc(sizeof(int32_t) * (total ? total : 1));
    if (!runs_out) {
        std::free(lidx);
        std::free(run_ptr);
        return KPM_ENOMEM;
    }
    size_t at = 0;
    for (int p = 0; p < parts; p++) {
        if (!part_runs[p].empty())
            std::memcpy(runs_out + at, part_runs[p].data(), sizeof(int32_t) * part_runs[p].size());
        at += part_runs[p].size();
    }
    out->n_chunks = n_chunks;
    out->n_runs = (int64_t)total / 2;
    out->u_max = u_max;
    out->l_max = l_max;
    out->lidx = lidx;
    out->run_ptr = run_ptr;
    out->runs = runs_out;
    return KPM_OK;
}

void kpm_gather_release(kpm_gather *g)
{
    if (!g)
        return;
    std::free(g->lidx);
    std::free(g->run_ptr);
    std::free(g->runs);
    std::memset(g, 0, sizeof(*g));
}

}  // extern "C"

// ------------------------------------------------ staged entry arrays
namespace kpm {
namespace {

// Offset (in entries) of entry j < n of row r in a region of n entries per
// row laid out in groups of 8, then of 4, 2 and 1 entries (the binary digits
// of n mod 8), each group row-major (see kpm_staged in kpm.h).
int64_t group_offset(int64_t C, int n, int j, int64_t r)
{
    const int full = n & ~7;
    if (j < full)
        return C * (j & ~7) + 8 * r + (j & 7);
    int base = full;
    for (int g = 4; g >= 1; g >>= 1) {
        if ((n - full) & g) {
            if (j < base + g)
                return C * base + g * r + (j - base);
            base += g;
        }
    }
    return -1;  // not reached for j < n
}

// Offset of the index of entry j of row r within its chunk (forms 0-2: the
// first len - 1 entries grouped, the own entry last).
int64_t staged_index_offset(int64_t C, int len, int j, int64_t r)
{
    const int nm = len - 1;
    return j == nm ? C * nm + r : group_offset(C, nm, j, r);
}

// Offset (in complex numbers) of the value of entry j of row r: form 1
// pairs entries j, j+1 for even j below (len - 1) rounded down to even.
int64_t staged_value_offset(int64_t C, int len, int j, int64_t r, int form)
{
    if (form == 1) {
        const int np = (len - 1) & ~1;
        if (j < np)
            return C * (j & ~1) + 2 * r + (j & 1);
    }
    return C * j + r;
}

}  // namespace
}  // namespace kpm

extern "C" {

int kpm_staged_build(const kpm_sell *s, const kpm_gather *g, int32_t form, kpm_staged *out)
{
    if (!out)
        return KPM_EINVAL;
    std::memset(out, 0, sizeof(*out));
    if (!s || !g || form < 0 || form > 3 || !s->chunk_ptr || !s->chunk_len || s->C < 8 ||
        g->n_chunks != s->n_chunks || (s->n_stored > 0 && (!s->col || !s->val_ri || !g->lidx)))
        return KPM_EINVAL;
    if (form == 2 && g->u_max > 32768)
        return KPM_EINVAL;
    const int64_t C = s->C, n_chunks = s->n_chunks;
    // the last SELL entry of row r of chunk c that reads the row's own V row
    auto own_entry = [&](int64_t c, int64_t r) {
        int own = -1;
        for (int j = 0; j < s->chunk_len[c]; j++)
            if (s->col[s->chunk_ptr[c] + (int64_t)j * C + r] == c * C + r)
                own = j;
        return own;
    };
    if (form >= 2) {
        // every entry purely real or purely imaginary; form 3: own entries real
        std::atomic<bool> bad(false);
        parallel_parts(n_chunks, 1 << 10, [&](int64_t lo, int64_t hi, int) {
            for (int64_t c = lo; c < hi && !bad; c++)
                for (int64_t r = 0; r < C; r++) {
                    for (int j = 0; j < s->chunk_len[c]; j++) {
                        const int64_t e = s->chunk_ptr[c] + (int64_t)j * C + r;
                        if (s->val_ri[2 * e] != 0.0 && s->val_ri[2 * e + 1] != 0.0)
                            bad = true;
                    }
                    const int own = own_entry(c, r);
                    if (form == 3 && own >= 0 &&
                        s->val_ri[2 * (s->chunk_ptr[c] + (int64_t)own * C + r) + 1] != 0.0)
                        bad = true;
                }
        });
        if (bad)
            return KPM_EINVAL;
    }
    int64_t *chunk_ptr = (int64_t *)std::malloc(sizeof(int64_t) * (n_chunks + 1));
    int32_t *chunk_len = (int32_t *)std::malloc(sizeof(int32_t) * (n_chunks ? n_chunks : 1));
    int32_t *chunk_nre = form == 3 ? (int32_t *)std::malloc(sizeof(int32_t) * (n_chunks ? n_chunks : 1))
                                   : nullptr;
    if (!chunk_ptr || !chunk_len || (form == 3 && !chunk_nre)) {
        std::free(chunk_ptr);
        std::free(chunk_len);
        std::free(chunk_nre);
        return KPM_ENOMEM;
    }
    auto is_imag = [&](int64_t e) { return s->val_ri[2 * e] == 0.0 && s->val_ri[2 * e + 1] != 0.0; };
    parallel_parts(n_chunks, 1 << 10, [&](int64_t lo, int64_t hi, int) {
        for (int64_t c = lo; c < hi; c++) {
            const int len = s->chunk_len[c];
            if (form == 3) {
                // real region: the largest count of real entries besides the
                // own one; imaginary region: the largest count of imaginary
                int n_re = 0, n_im = 0;
                for (int64_t r = 0; r < C; r++) {
                    const int own = own_entry(c, r);
                    int re = 0, im = 0;
                    for (int j = 0; j < len; j++) {
                        if (j == own)
                            continue;
                        if (is_imag(s->chunk_ptr[c] + (int64_t)j * C + r))
                            im++;
                        else
                            re++;
                    }
                    n_re = std::max(n_re, re);
                    n_im = std::max(n_im, im);
                }
                chunk_nre[c] = n_re;
                chunk_len[c] = n_re + n_im + 1;
                continue;
            }
            bool all_own = len > 0;
            for (int64_t r = 0; r < C && all_own; r++)
                all_own = own_entry(c, r) >= 0;
            chunk_len[c] = len + (all_own ? 0 : 1);
        }
    });
    chunk_ptr[0] = 0;
    int32_t l_max = 0;
    for (int64_t c = 0; c < n_chunks; c++) {
        chunk_ptr[c + 1] = chunk_ptr[c] + C * chunk_len[c];
        l_max = std::max(l_max, chunk_len[c]);
    }
    const int64_t n_stored = chunk_ptr[n_chunks];
    const int64_t nv = form == 3 ? n_stored : 2 * n_stored;  // value words
    uint16_t *lidx = (uint16_t *)std::malloc(sizeof(uint16_t) * (n_stored ? n_stored : 1));
    double *val = (form == 0 || form == 2) ? (double *)std::malloc(sizeof(double) * (nv ? nv : 1))
                                           : nullptr;
    float *valf = (form == 1 || form == 3) ? (float *)std::malloc(sizeof(float) * (nv ? nv : 1))
                                           : nullptr;
    if (!lidx || (!val && !valf)) {
        std::free(chunk_ptr);
        std::free(chunk_len);
        std::free(chunk_nre);
        std::free(lidx);
        std::free(val);
        std::free(valf);
        return KPM_ENOMEM;
    }
    parallel_parts(n_chunks, 1 << 9, [&](int64_t lo, int64_t hi, int) {
        std::vector<int> order;
        for (int64_t c = lo; c < hi; c++) {
            const int len = s->chunk_len[c], len_s = chunk_len[c];
            const int64_t e0 = s->chunk_ptr[c], s0 = chunk_ptr[c];
            for (int64_t r = 0; r < C; r++) {
                const int own = own_entry(c, r);
                // staged entry k of this row: SELL entry j (or -1: value 0,
                // own row), written at index offset io and value offset vo
                auto put = [&](int j, int64_t io, int64_t vo) {
                    double re = 0.0, im = 0.0;
                    uint16_t li = (uint16_t)r;
                    if (j >= 0) {
                        const int64_t e = e0 + (int64_t)j * C + r;
                        re = s->val_ri[2 * e];
                        im = s->val_ri[2 * e + 1];
                        li = g->lidx[e];
                    }
                    if (form == 1) {
                        valf[2 * (s0 + vo)] = (float)re;
                        valf[2 * (s0 + vo) + 1] = (float)im;
                    } else if (form == 3) {
                        valf[s0 + vo] = (float)(im != 0.0 ? im : re);
                    } else if (form == 0) {
                        val[2 * (s0 + vo)] = re;
                        val[2 * (s0 + vo) + 1] = im;
                    } else {
                        const bool imag = re == 0.0 && im != 0.0;
                        val[2 * (s0 + vo)] = imag ? -im : re;
                        val[2 * (s0 + vo) + 1] = imag ? im : re;
                        if (imag)
                            li = (uint16_t)(li | 0x8000u);
                    }
                    lidx[s0 + io] = li;
                };
                if (form == 3) {
                    const int n_re = chunk_nre[c], n_im = len_s - 1 - n_re;
                    int kr = 0, ki = 0;
                    for (int j = 0; j < len; j++) {
                        if (j == own)
                            continue;
                        if (is_imag(e0 + (int64_t)j * C + r)) {
                            const int64_t o = C * n_re + group_offset(C, n_im, ki++, r);
                            put(j, o, o);
                        } else {
                            const int64_t o = group_offset(C, n_re, kr++, r);
                            put(j, o, o);
                        }
                    }
                    while (kr < n_re) {
                        const int64_t o = group_offset(C, n_re, kr++, r);
                        put(-1, o, o);
                    }
                    while (ki < n_im) {
                        const int64_t o = C * n_re + group_offset(C, n_im, ki++, r);
                        put(-1, o, o);
                    }
                    put(own, C * (len_s - 1) + r, C * (len_s - 1) + r);
                    continue;
                }
                const int vf = form == 1 ? 1 : 0;
                int k = 0;
                auto put_k = [&](int j) {
                    put(j, staged_index_offset(C, len_s, k, r),
                        staged_value_offset(C, len_s, k, r, vf));
                    k++;
                };
                for (int j = 0; j < len; j++)
                    if (j != own)
                        put_k(j);
                while (k < len_s - 1)
                    put_k(-1);
                put_k(own);
            }
        }
    });
    out->n_chunks = n_chunks;
    out->n_stored = n_stored;
    out->l_max = l_max;
    out->form = form;
    out->chunk_ptr = chunk_ptr;
    out->chunk_len = chunk_len;
    out->chunk_nre = chunk_nre;
    out->lidx = lidx;
    out->val = val;
    out->valf = valf;
    return KPM_OK;
}

void kpm_staged_release(kpm_staged *st)
{
    if (!st)
        return;
    std::free(st->chunk_ptr);
    std::free(st->chunk_len);
    std::free(st->chunk_nre);
    std::free(st->lidx);
    std::free(st->val);
    std::free(st->valf);
    std::memset(st, 0, sizeof(*st));
}

}  // extern "C"
