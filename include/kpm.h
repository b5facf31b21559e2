/*
 * kpm.h -- C interface of libkpm, a GB300 (sm_103a) implementation of the
 * hot path of the Kernel Polynomial Method for the density of states
 * (KPM-DOS), after Kreutzer, Hager, Wellein, Pieper, Alvermann, Fehske,
 * "Performance Engineering of the Kernel Polynomial Method on Large-Scale
 * CPU-GPU Systems", IPDPS 2015.
 *
 * The method (Sec. "Problem Description", Eq. 3): rescale H~ = a (H - b 1),
 * iterate the Chebyshev recurrence nu_1 = H~ nu_0, nu_{m+1} = 2 H~ nu_m -
 * nu_{m-1} on R start vectors at once, and collect in every step the scalar
 * products eta_{2m} = <nu_m|nu_m> and eta_{2m+1} = <nu_{m+1}|nu_m>.  The
 * library fuses one step into the "augmented sparse matrix multiple-vector
 * product" of Fig. 5 (aug_spmmv):
 *     W <- 2a (H - b 1) V - W,  eta_{2m}[:] = <V|V>,  eta_{2m+1}[:] = <W|V>
 * over an N x R block of vectors stored row-major (interleaved, Sec.
 * "General Notes on the Implementation"), with H held in a SELL-C-sigma
 * layout.
 *
 * General rules
 *   - Every function returns KPM_OK (0) or a negative KPM_E* status; no C++
 *     exception crosses this interface.  kpm_status_string() names a status.
 *   - Complex numbers are passed as interleaved (re, im) doubles ("_ri").
 *   - The caller owns every buffer it passes; functions copy what they keep.
 *   - A context (kpm_ctx) is used by one host thread at a time.
 *   - "host" pointers must be host memory, "device" pointers memory of the
 *     context's CUDA device; "stream" is a cudaStream_t passed as void*
 *     (NULL = the legacy default stream).
 */
#ifndef KPM_H
#define KPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define KPM_OK 0
#define KPM_EINVAL (-1)          /* bad argument: malformed CSR, odd or <2 M, R < 1, ... */
#define KPM_ENOTHERMITIAN (-2)   /* check_hermitian set and H != H^dagger */
#define KPM_ENOMEM (-3)          /* host or device allocation failed */
#define KPM_ECUDA (-4)           /* a CUDA runtime call failed */
#define KPM_ETIMEOUT (-5)        /* a bounded device-side wait gave up */
#define KPM_EUNSUPPORTED (-6)    /* valid request this build cannot serve */

/* ------------------------------------------------------------- precision */
/* KPM_PREC_FP64: H' and the vector blocks stored as complex double, all
 *   arithmetic in IEEE double.
 * KPM_PREC_FP32: H' and the vector blocks stored as complex float (half the
 *   bytes of the bandwidth-bound sweep), the sparse product in single
 *   precision.  The eta scalar products: each thread's products of at most
 *   8 rows per column are summed in single precision, the partial sums of
 *   the rows of one warp are added in single precision (at most 32 rows in
 *   all), and every such partial is accumulated in double, as are the sums
 *   across warps and blocks.  a, b, the fold H' = 2a(H - b 1) and the
 *   moment-to-DOS steps stay double in both forms. */
#define KPM_PREC_FP64 0
#define KPM_PREC_FP32 1

typedef struct kpm_ctx kpm_ctx;

/* Optional device allocator used for every device buffer of a context.
 * alloc returns NULL on failure; free accepts what alloc returned. */
typedef void *(*kpm_alloc_fn)(size_t bytes, void *user);
typedef void (*kpm_free_fn)(void *ptr, void *user);

typedef struct kpm_options {
    int32_t precision;        /* KPM_PREC_FP64 (default) or KPM_PREC_FP32 */
    int32_t chunk_height;     /* SELL chunk height C (rows per chunk); 0 = 32 */
    int32_t sigma;            /* SELL sorting window sigma (rows); 0 = 256, 1 = no sort */
    int32_t check_hermitian;  /* nonzero: kpm_create verifies H == H^dagger (1e-12 rel) */
    int32_t autotune;         /* nonzero: the first moment call for a block width R times the
                                 launch variants (kpm_autotune) and keeps the fastest */
    int32_t device;           /* CUDA device ordinal */
    kpm_alloc_fn alloc_fn;    /* NULL = cudaMalloc */
    kpm_free_fn free_fn;      /* NULL = cudaFree */
    void *alloc_user;
    const int32_t *row_order; /* NULL, or int32[n]: a permutation of the rows (new position ->
                                 original row) applied before the sigma sort, e.g. to place
                                 rows that share neighbours together for cache reuse; moments
                                 do not depend on it beyond rounding.  Read during kpm_create. */
    /* One part of a row-partitioned problem (kpm_partition_build): */
    int64_t n_halo;           /* 0, or the part's halo rows: the CSR's columns run to
                                 n + n_halo, column n + h reading halo slot h of the vector
                                 blocks (kpm_halo_unpack); such a context serves the
                                 device-resident sweep calls only */
    int64_t global_n;         /* 0 = n; else the rows of the whole problem: start vectors
                                 draw their phases by global row (stream 1 at index
                                 r * global_n + global row) */
    int64_t row0;             /* global row of local row 0 (with global_n) */
} kpm_options;

/* Fills *opt with the defaults listed above. */
void kpm_default_options(kpm_options *opt);

/* Name of a status code (static string). */
const char *kpm_status_string(int status);

/* ======================================================= host-only calls
 * These run on the CPU and need no GPU.  Large inputs are split among host
 * threads (CSR validation, Gershgorin bounds, the SELL-C-sigma build, the
 * gather lists; kpm_create uses the same code): at most the environment
 * variable KPM_HOST_THREADS if set, else the hardware concurrency (<= 64).
 * The results do not depend on the thread count. */

/* Spectral bounds of a Hermitian CSR matrix by Gershgorin's circle theorem
 * (Sec. "Problem Description": a, b are found "with Gershgorin's circle
 * theorem or a few Lanczos sweeps").  emin = min_i (Re h_ii - r_i),
 * emax = max_i (Re h_ii + r_i), r_i = sum_{j != i} |h_ij|, in double.
 *   n        rows (>= 1); row_ptr int64[n+1] (row_ptr[0] = 0, nondecreasing);
 *   col      int32[nnz] in [0, n), strictly increasing within a row;
 *   val_ri   double[2*nnz] interleaved (re, im).
 * KPM_EINVAL on a malformed CSR or a non-finite value. */
int kpm_gershgorin(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val_ri,
                   double *emin, double *emax);

/* Spectral bounds from a few Lanczos steps (Sec. "Problem Description": the
 * alternative to Gershgorin).  steps Lanczos iterations in double from a
 * random-phase start vector (SplitMix64 stream 3 of seed), no
 * reorthogonalisation; the smallest and largest Ritz values of the
 * tridiagonal matrix, each within r = |beta_k s_k| of an eigenvalue of H
 * (s_k the last component of its eigenvector), give
 * [theta_min - r_min, theta_max + r_max], intersected with the Gershgorin
 * interval.  The interval is tighter than Gershgorin's but, like
 * any Krylov estimate, covers the spectrum only to the accuracy the
 * residuals state: widen it (kpm_scale_from_bounds' eps) before use.
 * Host only.  KPM_EINVAL for steps < 2 or a malformed CSR. */
int kpm_lanczos_bounds(int64_t n, const int64_t *row_ptr, const int32_t *col,
                       const double *val_ri, int32_t steps, uint64_t seed, double *emin,
                       double *emax);

/* Rescaling of Sec. "Problem Description": b = (emax + emin)/2 and
 * a = (1 - eps) * 2/(emax - emin), mapping [emin, emax] onto
 * [-(1-eps), 1-eps].  KPM_EINVAL unless emax > emin and 0 <= eps < 1. */
int kpm_scale_from_bounds(double emin, double emax, double eps, double *a, double *b);

/* Chebyshev moments mu_0..mu_{M-1} from the eta of R vectors (the
 * reconstruction step the paper leaves to the application, Sec. "Problem
 * Description").  Per vector: c_0 = eta_0, c_1 = eta_1,
 * c_{2k} = 2 eta_{2k} - eta_0, c_{2k+1} = 2 eta_{2k+1} - eta_1 (from
 * T_{2k} = 2 T_k^2 - 1, T_{2k+1} = 2 T_{k+1} T_k - T_1); then the stochastic
 * trace mu_n = sum_r c_n^(r) / sum_r eta_0^(r), so mu_0 = 1.
 *   eta  host double[R][M] (row r = vector r);  mu  host double[M].
 * KPM_EINVAL for odd or < 2 M, R < 1, or sum_r eta_0^(r) <= 0. */
int kpm_eta_to_mu(const double *eta, int32_t M, int32_t R, double *mu);

/* Jackson-damped density of states on K Chebyshev nodes.
 *   x_k = cos(pi (k + 1/2)/K), k = 0..K-1 (descending x),
 *   g_n = [(M-n+1) cos(pi n/(M+1)) + sin(pi n/(M+1)) cot(pi/(M+1))]/(M+1),
 *   rho~(x) = [g_0 mu_0 + 2 sum_{n=1}^{M-1} g_n mu_n T_n(x)] / (pi sqrt(1-x^2)),
 *   energy[k] = x_k/a + b,  rho[k] = a rho~(x_k).
 * rho integrates to mu_0 over energy (Eq. 2 divided by N).  Host, double.
 * KPM_EINVAL for M < 1, K < 1 or a <= 0. */
int kpm_dos(const double *mu, int32_t M, int32_t K, double a, double b,
            double *energy, double *rho);

/* Host-side view of the sparse layout built by kpm_create (for inspection
 * and tests).  Rows are permuted: new row p holds original row perm[p].
 * Chunk c covers new rows [c*C, (c+1)*C); its entries start at chunk_ptr[c]
 * and are stored column-major, entry j of row r in the chunk at
 * chunk_ptr[c] + j*C + r, for j < chunk_len[c].  Padding entries have value
 * 0 and a valid column index.  val_ri holds the folded matrix
 * H' = 2a(H - b 1) (diagonal entries are added where H lacks them), in
 * double, with column indices already mapped to new row numbers. */
typedef struct kpm_sell {
    int64_t n;           /* rows of H */
    int64_t n_pad;       /* n rounded up to a multiple of C */
    int32_t C, sigma;
    int64_t n_chunks;
    int64_t nnz;         /* stored entries of H' without padding */
    int64_t n_stored;    /* stored entries including padding = chunk_ptr[n_chunks] */
    int64_t *chunk_ptr;  /* [n_chunks + 1] */
    int32_t *chunk_len;  /* [n_chunks] */
    int32_t *col;        /* [n_stored] */
    double *val_ri;      /* [2 * n_stored] */
    int32_t *perm;       /* [n_pad]: new row -> original row (rows >= n map to themselves) */
} kpm_sell;

/* Builds the SELL-C-sigma form of H' = 2a(H - b 1) from CSR (host only).
 * Rows are taken in the order row_order (NULL = 0..n-1; otherwise a
 * permutation of 0..n-1, new position -> original row, else KPM_EINVAL),
 * sorted by descending length inside windows of sigma rows (stable),
 * grouped into chunks of C rows, and the permutation is applied
 * symmetrically (rows and columns).  C in [1, 1024], sigma >= 1.
 * Free with kpm_sell_release.  KPM_EINVAL on a malformed CSR. */
int kpm_sell_build(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val_ri,
                   double a, double b, int32_t C, int32_t sigma, const int32_t *row_order,
                   kpm_sell *out);
void kpm_sell_release(kpm_sell *s);

/* Gather lists of the staged sweep (host view, for inspection and tests).
 * The staged aug_spmmv kernel copies, for each chunk, every V row the
 * chunk's entries read into shared memory once, however many entries read
 * it.  For chunk c of a kpm_sell (rows r0 = c*C .. r0+C-1) that list holds
 * the chunk's own C rows first (local positions 0..C-1), then every other
 * row its stored entries reference, in increasing order.  It is stored as
 * runs of consecutive rows: runs[2q] = first row, runs[2q+1] = row count,
 * for q in [run_ptr[c], run_ptr[c+1]); local positions count through the
 * runs in order (adjacent runs are merged).  lidx[e] is the local position
 * of the row that stored entry e reads (indexed like kpm_sell.col), so
 * col[e] is the row at position lidx[e] of its chunk's list.  u_max is the
 * longest list in rows, l_max the largest chunk_len.
 * KPM_EINVAL for C < 8 (16-byte multiples of 16-bit indices per chunk
 * column); KPM_EUNSUPPORTED if a list exceeds 65535 rows.  Host only; free
 * with kpm_gather_release. */
typedef struct kpm_gather {
    int64_t n_chunks, n_runs;
    int32_t u_max, l_max;
    uint16_t *lidx;    /* [n_stored] */
    int64_t *run_ptr;  /* [n_chunks + 1] */
    int32_t *runs;     /* [2 * n_runs] */
} kpm_gather;
int kpm_gather_build(const kpm_sell *s, kpm_gather *out);
void kpm_gather_release(kpm_gather *g);

/* Entry arrays of the staged sweep (host view, for inspection and tests;
 * kpm_create builds the same arrays for the device).  The staged kernel
 * reads a chunk's entries from arrays of its own, derived from a kpm_sell
 * and its kpm_gather.  Fig. 5's sweep needs <V|V> per row, and the kernel
 * takes the row's own V operand from the row's last entry, so:
 *   - The "own" entry of a row is its last SELL entry that reads the row's
 *     own V row (its diagonal, or a padding entry); it is stored last.
 *     Where a row has none, a zero entry on the row's own index stands in.
 *   - Forms 0-2: a row's entries are its SELL entries except the own one,
 *     in SELL order, then the own entry.  In a chunk where some row has no
 *     own entry, every row gets one more entry (value 0, own index: the own
 *     entry of the rows without one, a filler before the own entry of the
 *     others).  chunk_len[c] = len >= 1 is the resulting length.
 *   - Form 3: a row's real entries except the own one first (region A,
 *     chunk_nre[c] entries), then its imaginary entries (region B), in SELL
 *     order, each region filled up to the chunk's largest count with zero
 *     entries on the row's own index, then the own entry (which must be
 *     real); len = chunk_nre[c] + (imaginary count) + 1.
 *   - Local indices (lidx, 16-bit positions in the chunk's gather list, the
 *     row's own position being r) and, for form 3, values: a region of n
 *     entries per row is stored in groups of 8 entries, then one group each
 *     of 4, 2 and 1 entries for the binary digits of n mod 8, high to low;
 *     a group of g entries starting at entry j of the region holds row r's
 *     entries at (region start) + C*j + g*r, so one 16-, 8- or 4-byte load
 *     per row reads a whole group.  Forms 0-2 have one region, the first
 *     nm = len - 1 entries; form 3 has region A at the chunk's start and
 *     region B at C*chunk_nre[c].  The own entry sits at C*(len - 1) + r.
 *   - Values of forms 0-2: form 1 (complex float) stores entries j, j+1 of
 *     row r together at complex offset chunk_ptr[c] + C*j + 2r for even
 *     j < (nm & ~1), the others at chunk_ptr[c] + C*j + r; forms 0 and 2
 *     (complex double) store entry j at chunk_ptr[c] + C*j + r.  Form 2 is
 *     the half-complex form of complex double matrices whose every stored
 *     entry is purely real or purely imaginary: a real entry h stores the
 *     operand pair (h, h), an imaginary entry i*m stores (-m, m) and has bit
 *     15 of its local index set (the kernel reads the V row's two halves in
 *     swapped order for it).  Form 3, the half-complex form of complex float
 *     matrices of that kind, stores one float per entry: h of a real entry,
 *     m of an imaginary one (the region says which).  A zero entry counts as
 *     real.
 * form: 0 complex double, 1 complex float (values rounded to float), 2
 * half-complex double, 3 half-complex float.  KPM_EINVAL for another form;
 * for forms 2 and 3 if an entry has both parts nonzero; for form 2 if a
 * gather list is longer than 32768 rows (bit 15 is taken); for form 3 if an
 * own entry is imaginary.  Host only; free with kpm_staged_release. */
typedef struct kpm_staged {
    int64_t n_chunks;
    int64_t n_stored;    /* C * sum of chunk_len */
    int32_t l_max;       /* largest chunk_len */
    int32_t form;
    int64_t *chunk_ptr;  /* [n_chunks + 1] first entry of each chunk */
    int32_t *chunk_len;  /* [n_chunks] */
    int32_t *chunk_nre;  /* form 3: [n_chunks] real-region length; otherwise NULL */
    uint16_t *lidx;      /* [n_stored] */
    double *val;         /* forms 0, 2: double[2 * n_stored]; otherwise NULL */
    float *valf;         /* form 1: float[2 * n_stored]; form 3: float[n_stored];
                            otherwise NULL */
} kpm_staged;
int kpm_staged_build(const kpm_sell *s, const kpm_gather *g, int32_t form, kpm_staged *out);
void kpm_staged_release(kpm_staged *st);

/* Row partition for several processes (Sec. "Symmetric Heterogeneous
 * Execution": each process holds a contiguous, weighted share of the rows,
 * receives before every sweep the rows of the vector block its rows read
 * from other processes -- the halo -- and the scalar products are summed
 * over processes once, at the end, as in the single global reduction of
 * Table III).  Host only.
 *
 * kpm_partition_rows: boundaries row_start[0..parts] (row_start[0] = 0,
 * row_start[parts] = n) of parts contiguous shares of n rows, part k about
 * weights[k]/sum(weights) of them (weights NULL = equal), every boundary a
 * multiple of align rows (a lattice plane: z-slabs for the numbering of Eq.
 * 1) and every part at least align rows.  KPM_EINVAL unless n is a multiple
 * of align, there are at least parts planes and the weights are positive.
 *
 * kpm_partition_build: part `part` of the CSR matrix under row_start: its
 * rows [row0, row0 + n_local) as a local CSR whose columns are the local
 * row (columns in the part) or n_local + h for halo slot h (the other
 * parts' rows the part's rows read, halo_rows[h] increasing); within a row
 * local columns come first, each group increasing.  The peers are the
 * parts it receives from or sends to (increasing): halo slots
 * [recv_ptr[q], recv_ptr[q+1]) come from peer[q], and peer[q] needs this
 * part's local rows send_rows[send_ptr[q] .. send_ptr[q+1]), in the order
 * of its own halo slots.  The whole CSR is read (every part sees the whole
 * matrix here).  Free with kpm_partition_release. */
typedef struct kpm_part {
    int64_t n;            /* rows of the whole matrix */
    int64_t row0;         /* global row of local row 0 */
    int64_t n_local;      /* rows of this part */
    int64_t n_halo;       /* halo slots */
    int64_t nnz;          /* entries of the local CSR */
    int32_t n_peers;
    int32_t reserved;
    int64_t *row_ptr;     /* [n_local + 1] */
    int32_t *col;         /* [nnz] */
    double *val_ri;       /* [2 * nnz] */
    int64_t *halo_rows;   /* [n_halo] global rows */
    int32_t *peer;        /* [n_peers] */
    int64_t *recv_ptr;    /* [n_peers + 1] */
    int64_t *send_ptr;    /* [n_peers + 1] */
    int32_t *send_rows;   /* [send_ptr[n_peers]] local rows */
} kpm_part;
int kpm_partition_rows(int64_t n, int32_t parts, const double *weights, int64_t align,
                       int64_t *row_start);
int kpm_partition_build(int64_t n, const int64_t *row_ptr, const int32_t *col,
                        const double *val_ri, int32_t parts, const int64_t *row_start,
                        int32_t part, kpm_part *out);
void kpm_partition_release(kpm_part *p);

/* ============================================================ GPU calls */

/* Creates a context on opt->device: validates the CSR (and, if asked,
 * Hermiticity), folds H' = 2a(H - b 1) in double, converts to SELL-C-sigma,
 * rounds to complex float for KPM_PREC_FP32, and uploads.  The CSR may be
 * freed on return.  a > 0 and b are the rescaling of Sec. "Problem
 * Description" (see kpm_gershgorin / kpm_scale_from_bounds); the caller is
 * responsible for the spectrum of a(H - b) lying in [-1, 1].
 * opt may be NULL (defaults).  Errors: KPM_EINVAL, KPM_ENOTHERMITIAN,
 * KPM_ENOMEM, KPM_ECUDA. */
int kpm_create(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val_ri,
               double a, double b, const kpm_options *opt, kpm_ctx **out);

/* Releases the context and its device memory (waits for its work). */
void kpm_destroy(kpm_ctx *ctx);

/* eta moments for R random-phase start vectors drawn from seed (Fig. 5):
 * entry i of vector r is exp(2 pi i u), u = SplitMix64 stream 1 at index
 * r*n + i (key = mix(seed + 2*0x9E3779B97F4A7C15), u = top 53 bits of
 * mix(key + (index+1)*0x9E3779B97F4A7C15) times 2^-53), so vector r does not
 * depend on R.  One initial sweep (eta_0, eta_1) and M/2 - 1 aug_spmmv
 * sweeps give eta_0..eta_{M-1}.
 *   eta       host double[R][M]: Re eta_k of vector r at eta[r*M + k]
 *   eta_imag  host double[R][M] or NULL: Im eta_k (zero in exact arithmetic)
 * Synchronous: returns after eta is on the host.  M even and >= 2, R >= 1,
 * otherwise KPM_EINVAL. */
int kpm_moments(kpm_ctx *ctx, int32_t M, int32_t R, uint64_t seed, double *eta,
                double *eta_imag, void *stream);

/* As kpm_moments with caller-given start vectors (Fig. 5 with nu_0 given,
 * Eq. 3 unchanged): v0_ri is host double[2 * n * R], row-major complex
 * n x R (entry (i, r) at 2*(i*R + r)), in the original row numbering.  The
 * n basis vectors give the exact trace tr T_m(H~) in place of the
 * stochastic estimate of Sec. "Problem Description" (the sum over r of
 * <r|T_m|r> with random phases). */
int kpm_moments_v0(kpm_ctx *ctx, int32_t M, int32_t R, const double *v0_ri, double *eta,
                   double *eta_imag, void *stream);

/* Local and momentum-resolved quantities (Sec. "Application Scenario": the
 * local DOS and the spectral function A(k, E) of Fig. 2): the same moments
 * as kpm_moments from start vectors built on the device, so no n x R block
 * crosses the bus.  Output, synchronisation and M as in kpm_moments.
 *
 * kpm_moments_local: vector r is the unit vector of original row rows[r]
 * (host int64[R]); its moments are those of the local DOS of that row,
 * <e_i|T_n(H~)|e_i> after kpm_eta_to_mu (summing a site's orbitals with
 * kpm_eta_to_mu over their R rows gives the site's LDOS).  KPM_EINVAL for a
 * row outside [0, n).
 *
 * kpm_moments_plane_wave: for a lattice of nx*ny*nz sites with norb
 * orbitals per site, original row i = norb*(x + nx*(y + ny*z)) + alpha (the
 * numbering of the Hamiltonian of Eq. 1), vector r is the Bloch wave
 * exp(2 pi i q_r . (x, y, z)) / sqrt(nx*ny*nz) on orbital orb[r] of every
 * site (q host double[R][3], the wave vector k = 2 pi q per lattice
 * spacing; orb host int32[R]).  Its moments after kpm_eta_to_mu are those of
 * A(k, E) restricted to that orbital; kpm_eta_to_mu over the norb vectors of
 * one q gives A(k, E) / norb.  KPM_EINVAL unless nx*ny*nz*norb = n,
 * 0 <= orb[r] < norb and q is finite. */
int kpm_moments_local(kpm_ctx *ctx, int32_t M, int32_t R, const int64_t *rows, double *eta,
                      double *eta_imag, void *stream);
int kpm_moments_plane_wave(kpm_ctx *ctx, int32_t M, int32_t R, int32_t nx, int32_t ny, int32_t nz,
                           int32_t norb, const double *q, const int32_t *orb, double *eta,
                           double *eta_imag, void *stream);

/* Ensemble (not in the paper, which scales one problem over many nodes; each
 * problem is the KPM-DOS of Sec. "Problem Description" and Fig. 5, run as
 * in kpm_moments): count independent problems (each its own context, all on the
 * same device and of the same precision), problem p with M[p] moments
 * (even, >= 2), R[p] >= 1 random-phase vectors from seed[p]; eta[p] is host
 * double[R[p]][M[p]].  All problems advance together.  Each problem's R[p]
 * columns are split into column blocks of power-of-two widths up to 64,
 * widest first (one block where R[p] is such a power), as kpm_moments splits
 * them; the blocks of one width, across all problems, form a class.  Every
 * sweep step is, per class, one batched launch covering the class's blocks
 * still running plus one batched eta reduction, and the whole schedule is
 * captured into a CUDA graph and run as one graph launch.  Complex float
 * classes of width 8..64 whose contexts all have gather lists with one chunk
 * height run the staged kernel (kpm_launch.stages) over the class's chunks,
 * the others the register-path kernel.  A class takes the launch shape and
 * stage count that the context of its first block (the one with the largest
 * M) uses for the width -- the default, or what kpm_autotune /
 * kpm_set_launch chose -- with fewer stages where the class's widest gather
 * list needs it.  Synchronous.  Equivalent to kpm_batch_create + kpm_batch_launch
 * + kpm_batch_eta for every problem + kpm_batch_destroy. */
int kpm_moments_batch(kpm_ctx *const *ctx, int32_t count, const int32_t *M, const int32_t *R,
                      const uint64_t *seed, double *const *eta, void *stream);

/* A captured ensemble schedule that can be launched repeatedly.  It uses the
 * contexts' own work buffers: while it exists, run no other moment call on
 * those contexts, and destroy it before them.  Each context may appear
 * once. */
typedef struct kpm_batch kpm_batch;

typedef struct kpm_batch_info {
    int32_t count;             /* problems */
    int32_t steps;             /* sweep steps = max M/2 */
    int32_t grid;              /* blocks of each batched sweep launch (register path) */
    int16_t classes;           /* block-width classes */
    int16_t staged_classes;    /* of which run the staged kernel */
    int64_t kernel_launches;   /* kernel nodes in the graph */
    int64_t sweeps;            /* sum over problems of M/2 */
    double algorithmic_bytes;  /* Eq. 4 bytes of one run, summed over problems */
} kpm_batch_info;

int kpm_batch_create(kpm_ctx *const *ctx, int32_t count, const int32_t *M, const int32_t *R,
                     const uint64_t *seed, kpm_batch **out);
/* One run of the whole ensemble: a single graph launch, asynchronous on
 * stream.  Each run redraws the start vectors from the seeds. */
int kpm_batch_launch(kpm_batch *batch, void *stream);
/* Copies problem p's eta (host double[R[p]][M[p]]) after the launch on
 * stream; synchronises the stream.  KPM_ETIMEOUT if a bounded device-side
 * wait of the last launch gave up (the moments are then invalid). */
int kpm_batch_eta(kpm_batch *batch, int32_t p, double *eta, void *stream);
int kpm_batch_get_info(const kpm_batch *batch, kpm_batch_info *out);
void kpm_batch_destroy(kpm_batch *batch);

/* ------------------------------------------------- device-resident calls
 * For benchmarks and sweep-level tests: inputs and outputs stay on the GPU
 * and nothing is synchronised. */

typedef struct kpm_info {
    int64_t n, n_pad, nnz, n_stored, n_chunks;
    int32_t C, sigma, precision, device;
    double a, b;
    int64_t matrix_bytes;   /* device bytes of values + column indices */
    int64_t kernel_launches; /* kernels this context has launched so far */
    int32_t gather_lists;    /* 1: the staged kernel's gather lists were built */
    int32_t half_complex;    /* 1: every stored entry purely real or purely imaginary (and,
                                for complex float, every row's own entry real): the staged
                                kernel's half-complex form, two real FMAs per entry and
                                column instead of four */
    int64_t upload_bytes;    /* host -> device bytes kpm_create copied (matrix, indices,
                                gather lists and records, half-complex operands) */
} kpm_info;

int kpm_get_info(const kpm_ctx *ctx, kpm_info *out);

/* Reads and clears the context's device error word: KPM_OK; KPM_ETIMEOUT
 * if a bounded device-side wait of the staged kernel gave up since the last
 * check (its results are then invalid); KPM_EINVAL if a kernel met an index
 * outside its array and skipped it (kpm_halo_pack's rows).  The moment calls
 * check it themselves before returning; the device-resident calls leave it
 * to the caller.  Synchronous. */
int kpm_check_device_error(kpm_ctx *ctx);

/* Test hook for the bounded waits (not for production use): from now on the
 * staged kernel's producer stops after chunks_per_block chunks in every
 * block, so the consumers' waits for the next stage expire (after about two
 * seconds of SM clock), the launch records a timeout in the device error word
 * (kpm_check_device_error then returns KPM_ETIMEOUT) and its results are
 * invalid; the context stays usable.  A batch (kpm_batch_create) built while
 * the hook is set on its first context stalls the same way in each of its
 * staged launches; kpm_batch_eta then returns KPM_ETIMEOUT.  -1 switches the
 * hook off.  KPM_EINVAL for values below -1. */
int kpm_test_stall_staged(kpm_ctx *ctx, int64_t chunks_per_block);

/* Bytes of one device vector block of width R in the context's layout:
 * n_pad (+ n_halo for a part) rows of ld(R) complex numbers (complex double
 * for FP64, complex float for FP32), ld(R) = R, rounded up to even for
 * FP32 when R > 1, rows in the permuted order of the sparse layout, halo
 * slots after them. */
int64_t kpm_block_bytes(const kpm_ctx *ctx, int32_t R);

/* Host (original row order, double complex n x R row-major) <-> device block
 * (context layout).  Padding rows and columns are written as zero. */
int kpm_block_upload(kpm_ctx *ctx, int32_t R, const double *host_ri, void *dev_block, void *stream);
int kpm_block_download(kpm_ctx *ctx, int32_t R, const void *dev_block, double *host_ri, void *stream);

/* One fused sweep on device blocks V, W of width R (Fig. 5, one iteration):
 *   init = 0:  W <- H' V - W        (H' = 2a(H - b 1))
 *   init = 1:  W <- (1/2) H' V      (= a(H - b 1) V, the initial step; W is not read)
 * and eta_dev (device double[3][R]) receives, per column r, <V|V>,
 * Re <W|V> and Im <W|V> of the updated W.  with_imag = 0 skips Im (written
 * as 0).  eta_dev = NULL leaves the per-block partial sums in the context's
 * scratch and launches no reduction (for timing the sweep kernel alone).
 * V and W must not overlap. */
int kpm_aug_spmmv(kpm_ctx *ctx, int32_t R, const void *V, void *W, double *eta_dev,
                  int32_t init, int32_t with_imag, void *stream);

/* Allocation-free variant of kpm_aug_spmmv (the paper has no counterpart;
 * it serves callers that may not allocate device memory at the time of the
 * call: code whose device memory is owned by another allocator or pool,
 * and latency-critical loops in which cudaMalloc/cudaFree would implicitly
 * synchronise the device).  Same arguments, same kernels and the same
 * results as kpm_aug_spmmv; the caller still passes V, W and eta_dev.  The
 * per-block partial sums go to a fixed scratch array of 1,048,576 doubles
 * (8 MiB) that every GPU loading this library holds until the process
 * exits; the call makes no cudaMalloc, cudaFree or other allocating call.
 *   - The first call on a device looks up the scratch's device address
 *     (cudaGetSymbolAddress) and caches it for the life of the process;
 *     make that first call before any stream capture on that device.  A
 *     device reset (cudaDeviceReset) reloads the library's module and is
 *     not supported between calls.
 *   - R needing more partials than the scratch holds is rejected with
 *     KPM_EINVAL before anything is launched.  The need is the sum over
 *     column blocks of grid * 3 * width doubles, grid depending on the
 *     launch shape and the device's SM count; with the default staged
 *     shapes of both forms on a 152-SM GB300 every R <= 256 fits (tested).
 *     The register-path shapes (contexts without gather lists) and shapes
 *     from kpm_autotune or kpm_set_launch can need more and then get
 *     KPM_EINVAL.
 *   - Nothing in the scratch has to start at zero: every call writes each
 *     partial it later reads.  Calls share the one array and it keeps the
 *     last call's contents, so calls that overlap on the GPU (other streams,
 *     other host threads, other contexts on the same device) race; order
 *     them on one stream. */
int kpm_aug_spmmv_static(kpm_ctx *ctx, int32_t R, const void *V, void *W, double *eta_dev,
                         int32_t init, int32_t with_imag, void *stream);

/* Halo exchange of a part's context (kpm_options.n_halo > 0): the vector
 * blocks hold the part's rows and then n_halo halo slots.
 * kpm_halo_pack copies local rows rows_dev[0..count) (device int32, local
 * row numbers) of block V to buf (device, count rows of the block's row
 * length: kpm_block_bytes / rows); kpm_halo_unpack copies count rows of buf
 * into halo slots first .. first + count - 1 of V.  Asynchronous on stream.
 * KPM_EINVAL for a range outside the block; a row of rows_dev outside
 * [0, n) is skipped and reported by kpm_check_device_error (KPM_EINVAL). */
int kpm_halo_pack(kpm_ctx *ctx, int32_t R, const void *V, const int32_t *rows_dev, int32_t count,
                  void *buf, void *stream);
int kpm_halo_unpack(kpm_ctx *ctx, int32_t R, void *V, const void *buf, int64_t first,
                    int32_t count, void *stream);
/* Start block of random phases for a part (or any context): entry (p, r)
 * of V for the context's rows exp(2 pi i u), u from stream 1 at index
 * r * global_n + global row (kpm_moments' start vectors of the whole
 * problem); halo slots and padding rows zero.  Asynchronous on stream. */
int kpm_block_phases(kpm_ctx *ctx, int32_t R, uint64_t seed, void *V, void *stream);

/* kpm_moments with everything on the device: random-phase start vectors
 * from seed are generated on the GPU and eta_dev / eta_imag_dev (device
 * double[R][M], eta_imag_dev may be NULL) are written without a host copy.
 * Work buffers are kept in the context between calls with the same R. */
int kpm_moments_device(kpm_ctx *ctx, int32_t M, int32_t R, uint64_t seed, double *eta_dev,
                       double *eta_imag_dev, void *stream);

/* ------------------------------------------------------- ablation calls
 * The optimisation stages of the paper on this GPU (Secs. "Algorithm
 * Analysis and Optimization" and "GPU Performance Model"). */

/* One sweep of a reduced kernel (Fig. 10's three kernels), on device blocks
 * as in kpm_aug_spmmv:
 *   variant 0: fully augmented sweep (kpm_aug_spmmv with eta_dev = NULL),
 *   variant 1: augmented SpMMV without the scalar products, W <- H'V - W,
 *   variant 2: plain SpMMV, W <- (1/2) H'V (W not read).
 * Variants 1 and 2 run the kernel the context uses for the full sweep
 * (register path or staged kernel) without the scalar products.  KPM_EINVAL for another variant. */
int kpm_sweep_variant(kpm_ctx *ctx, int32_t R, const void *V, void *W, int32_t variant,
                      void *stream);

/* Sweeps whose per-block eta partials one reduction launch sums in the
 * moment calls: 0 (default) = as many as fit 64 MB; 1 = a reduction after
 * every sweep, the single-GPU form of the paper's aug_spmmv* (a global
 * reduction in every iteration, Table III). */
int kpm_set_reduce_interval(kpm_ctx *ctx, int32_t sweeps);

/* How consecutive staged sweeps overlap.  A sweep launch carries a fixed
 * cost (~20 us against ~0.18 ms for the 64^3 lattice at R = 32): the
 * launch, its blocks' set-up and the filling of their first stages, and
 * the blocks that finish last.
 *   KPM_OVERLAP_NONE  one plain launch per sweep;
 *   KPM_OVERLAP_PDL   (default) each staged sweep is a programmatic
 *                     dependent launch: its blocks are scheduled as the
 *                     previous kernel's blocks retire, set up and fetch
 *                     their first chunk records, and wait (griddepcontrol)
 *                     for that kernel's completion and writes before they
 *                     touch the vector blocks or the eta partials.  Results
 *                     are those of plain launches, bit for bit.
 * KPM_EINVAL for a NULL context or another mode. */
/* Checked build.  Compiling the library with -DKPM_CHECK (build.py
 * build(check=True): _build_check/libkpm_check.so, which the Python binding
 * loads when the environment has KPM_CHECK=1) adds bounds checks to every
 * access of the staged sweep that depends on the context's device arrays:
 * each chunk record's entry range, run rows, overflow runs, gathered-row
 * count and W rows against the arrays' extents and the stage's areas
 * (checked by the producer warp before it copies anything), and every local
 * index against the chunk's gathered rows (checked by the consumer warps).
 * A failed check records KPM_DEVERR_RANGE in the device error word, stops
 * the launch's blocks, and kpm_check_device_error returns KPM_EINVAL.
 * kpm_checked_build returns 1 in a checked build, 0 otherwise.
 * kpm_test_corrupt_record (test hook, checked builds only, else
 * KPM_EUNSUPPORTED) overwrites word `word` (0..31) of chunk `chunk`'s device
 * record with (x, y): word 0 = first staged entry (low, high 32 bits), word
 * 1 = (staged length | real-region length << 16, run count), word 2 =
 * overflow offset, words 3..31 = inline runs (first row, row count). */
int kpm_checked_build(void);
int kpm_test_corrupt_record(kpm_ctx *ctx, int64_t chunk, int32_t word, int32_t x, int32_t y);

#define KPM_OVERLAP_NONE 0
#define KPM_OVERLAP_PDL 1
int kpm_set_sweep_overlap(kpm_ctx *ctx, int32_t mode);

/* The naive KPM-DOS of Fig. 3 from library calls: for each start vector in
 * turn, per step one cuSPARSE CSR SpMV (u = H v) and the cuBLAS level-1 calls
 * axpy (u -= b v), scal (w = -w), axpy (w += 2a u), nrm2 (eta_2m) and dotc
 * (eta_2m+1), in complex double on the original CSR matrix.  A baseline for
 * the ablation, not the production path. */
typedef struct kpm_naive kpm_naive;
int kpm_naive_create(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val_ri,
                     double a, double b, int32_t device, kpm_naive **out);
/* eta_dev: device double[R][M]; random-phase start vectors as kpm_moments. */
int kpm_naive_moments(kpm_naive *nv, int32_t M, int32_t R, uint64_t seed, double *eta_dev,
                      void *stream);
void kpm_naive_destroy(kpm_naive *nv);

/* Launch variant the context uses for block width R: lanes per row (T),
 * complex columns per lane (E, T*E = R), threads per block, blocks per SM
 * (0 = occupancy maximum), row groups per warp in one block tile (a
 * tile is threads/32 * (32/T) * tile_groups consecutive rows; 0 = 4) and
 * the kernel (stages), as chosen by the defaults or the autotuner.  The
 * default is the staged kernel with two stages wherever the context has
 * gather lists (C >= 8), the width is 2..64 (complex float: 4 columns per
 * lane, at widths 2 and 4 the whole row in one lane) or 1..32 (complex
 * double: 2 columns per lane, 1 at width 1) and two stages fit in shared
 * memory; everything else (complex float width 1) runs the register-path
 * kernel.  Complex
 * double contexts with gather lists split R into blocks of at most 32
 * columns (kpm_get_max_block_width).  For a matrix whose every stored
 * entry is purely real or purely imaginary (the topological insulator,
 * Sec. "Application Scenario"), the staged kernel multiplies with two real
 * FMAs per entry and column instead of four in both forms (the skipped
 * products are exact zeros, so W is the same); complex float then stores
 * one float per entry.  Complex float stages also carry the chunk's old W
 * rows where the larger stages keep the number of blocks per SM (else each
 * lane loads its old W a chunk ahead). */
typedef struct kpm_launch {
    int32_t lanes_per_row, cols_per_lane, block_threads, blocks_per_sm, tile_groups;
    int32_t stages;  /* 0: register-path kernel (block_threads per block, tile_groups);
                        1..8: the staged kernel -- per SELL chunk
                        one producer warp copies the matrix entries and each V row the
                        chunk reads (once, kpm_gather_build) into one of
                        `stages` shared-memory stages with bulk copies, and C*T/32
                        consumer warps compute from there; block_threads = 32 + C*T;
                        complex float: cols_per_lane 4 (width 4..64) or 2 (width
                        2..32); complex double: cols_per_lane 2 (width 2..32) or 1
                        (width 1) */
} kpm_launch;
int kpm_get_launch(const kpm_ctx *ctx, int32_t R, kpm_launch *out);
/* Forces a launch variant for width R (KPM_EUNSUPPORTED if not built). */
int kpm_set_launch(kpm_ctx *ctx, int32_t R, const kpm_launch *launch);

/* Autotuner for block width R: times `sweeps` aug_spmmv sweeps (after two
 * untimed ones) on the context's work blocks for every built launch shape
 * -- lanes per row T and columns per lane E with T*E = width, 128..512
 * threads per block, 1 or 4 row groups per tile, and the staged kernel
 * with 1..3 stages where they fit -- and for the widest
 * column block (64, 32 or 16 columns, R split into powers of two up to
 * it), and keeps the fastest for later calls.  best (may be NULL) receives
 * the shape chosen for the widest block.  Synchronises stream. */
int kpm_autotune(kpm_ctx *ctx, int32_t R, int32_t sweeps, void *stream, kpm_launch *best);

/* Widest column block the context uses (64, or 32 for complex double
 * contexts with gather lists, unless the autotuner chose otherwise). */
int kpm_get_max_block_width(const kpm_ctx *ctx);

/* Layout autotuner: builds trial contexts with SELL chunk heights C in
 * {8, 16, 32, 64, 128} and, for matrices with rows of different lengths, sorting
 * windows sigma in {1, 256, 4096}, tunes the launch shape of each for width
 * R (as kpm_autotune) and returns in *best the options of the fastest
 * (base's other fields kept, autotune set) and its time per sweep in
 * *best_ms (may be NULL).  Costs one kpm_create per trial. */
int kpm_autotune_layout(int64_t n, const int64_t *row_ptr, const int32_t *col,
                        const double *val_ri, double a, double b, const kpm_options *base,
                        int32_t R, int32_t sweeps, kpm_options *best, double *best_ms);

#ifdef __cplusplus
}
#endif
#endif /* KPM_H */
