// Context management and the KPM-DOS driver of libkpm: device layout,
// start vectors, the sweep schedule of Fig. 5 (one initial step, then
// swap + aug_spmmv), the deterministic eta reduction, and the ensemble.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "aug_spmmv.cuh"
#include "kpm_internal.h"

using namespace kpm;

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ULL;

// SplitMix64 output function (Steele, Lea, Flood 2014).
__host__ __device__ inline uint64_t splitmix_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// ------------------------------------------------------------- kernels
// Random-phase start block: V[p][r] = exp(2 pi i u), u from stream 1 at
// index r*gn + row0 + perm[p] (gn = the whole problem's rows, row0 = the
// global row of local row 0; n and 0 for an unpartitioned problem); rows
// p >= n (padding, halo slots) and columns r >= R are zero.  rows = the
// block's rows.
template <typename Real>
__global__ void phases_kernel(Real *V, const int32_t *perm, int64_t n, int64_t rows, int R,
                              int ld, uint64_t key, int64_t gn, int64_t row0)
{
    const int64_t total = rows * ld;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = idx / ld;
        const int r = (int)(idx - p * ld);
        Real re = 0, im = 0;
        if (p < n && r < R) {
            const uint64_t i = (uint64_t)row0 + (perm ? (uint64_t)perm[p] : (uint64_t)p);
            const uint64_t x = splitmix_mix(key + ((uint64_t)r * (uint64_t)gn + i + 1) * kGolden);
            const double u = (double)(x >> 11) * 0x1.0p-53;
            if constexpr (sizeof(Real) == 8) {
                double s, c;
                sincospi(2.0 * u, &s, &c);
                re = c;
                im = s;
            } else {
                // 2u or 2u - 2 in [-1, 1): the float argument keeps 25 bits
                const float x2 = (float)(u < 0.5 ? 2.0 * u : 2.0 * u - 2.0);
                float s, c;
                sincospif(x2, &s, &c);
                re = c;
                im = s;
            }
        }
        V[2 * idx] = re;
        V[2 * idx + 1] = im;
    }
}

// Start block of basis vectors (local quantities, Sec. "Application
// Scenario"): column r is the unit vector of original row rows[r].
template <typename Real>
__global__ void basis_kernel(Real *V, const int32_t *perm, int64_t n, int64_t n_pad, int R,
                             int ld, const int64_t *rows)
{
    const int64_t total = n_pad * ld;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = idx / ld;
        const int r = (int)(idx - p * ld);
        const bool one = p < n && r < R && (int64_t)perm[p] == rows[r];
        V[2 * idx] = one ? Real(1) : Real(0);
        V[2 * idx + 1] = Real(0);
    }
}

// Halo exchange of a part: out row k = V row iperm[rows[k]]; rows of ld
// complex numbers.  A row outside [0, n) is skipped (its output stays as
// it was) and recorded in the error word.
template <typename Real>
__global__ void halo_pack_kernel(const Real *V, const int32_t *iperm, const int32_t *rows,
                                 int64_t count, int ld, int64_t n, Real *out, int *err)
{
    const int64_t total = count * ld;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx / ld, r = idx - k * ld;
        const int32_t row = rows[k];
        if (row < 0 || row >= n) {
            atomicExch(err, KPM_DEVERR_RANGE);
            continue;
        }
        const int64_t src = ((int64_t)iperm[row] * ld + r) * 2;
        out[2 * idx] = V[src];
        out[2 * idx + 1] = V[src + 1];
    }
}

// Start block of Bloch plane waves (momentum-resolved quantities, A(k, E)):
// on a lattice of nx*ny*nz sites with norb orbitals per site, original row
// i = norb*(x + nx*(y + ny*z)) + alpha; column r is
// exp(2 pi i q_r . (x, y, z)) / sqrt(sites) on orbital orb[r] of every site
// and zero on the others (k = 2 pi q in units of the inverse lattice
// spacing).  The phase's fraction of a turn is reduced to [0, 1) before
// sincospi.
template <typename Real>
__global__ void plane_wave_kernel(Real *V, const int32_t *perm, int64_t n, int64_t n_pad, int R,
                                  int ld, const double *q, const int32_t *orb, int nx, int ny,
                                  int norb, double scale)
{
    const int64_t total = n_pad * ld;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = idx / ld;
        const int r = (int)(idx - p * ld);
        double re = 0.0, im = 0.0;
        if (p < n && r < R) {
            const int64_t i = perm[p];
            const int64_t site = i / norb;
            if ((int)(i - site * norb) == orb[r]) {
                const int64_t x = site % nx, y = (site / nx) % ny, z = site / ((int64_t)nx * ny);
                double f = q[3 * r] * (double)x + q[3 * r + 1] * (double)y + q[3 * r + 2] * (double)z;
                f -= floor(f);
                double sn, cs;
                sincospi(2.0 * f, &sn, &cs);
                re = scale * cs;
                im = scale * sn;
            }
        }
        V[2 * idx] = (Real)re;
        V[2 * idx + 1] = (Real)im;
    }
}

// Sum the per-block partials of `slots` consecutive sweeps in block order.
// partial: [slots][G][3][RB] (slot stride `slot_stride` doubles).  Sweep
// m = m0 + s writes eta[(col0 + r) * M + 2m] = <V|V>,
// eta[... + 2m + 1] = Re<W|V>, and, if eta_im, the imaginary parts.
__global__ void reduce_moments_kernel(const double *partial, int64_t slot_stride, int slots, int G,
                                      int RB, int col0, int M, int m0, double *eta, double *eta_im)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= slots * 3 * RB)
        return;
    const int s = t / (3 * RB);
    const int q = (t / RB) % 3;
    const int r = t % RB;
    const double *src = partial + s * slot_stride + q * RB + r;
    double sum = 0.0;
    for (int g = 0; g < G; g++)
        sum += src[(int64_t)g * 3 * RB];
    const int m = m0 + s;
    const int64_t row = (int64_t)(col0 + r) * M;
    if (q == 0) {
        eta[row + 2 * m] = sum;
        if (eta_im)
            eta_im[row + 2 * m] = 0.0;
    } else if (q == 1) {
        eta[row + 2 * m + 1] = sum;
    } else if (eta_im) {
        eta_im[row + 2 * m + 1] = sum;
    }
}

// Single sweep: out[q * R + col0 + r] = sum_g partial[g][q][r].
__global__ void reduce_single_kernel(const double *partial, int G, int RB, int col0, int R,
                                     double *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * RB)
        return;
    const int q = t / RB, r = t % RB;
    double sum = 0.0;
    for (int g = 0; g < G; g++)
        sum += partial[(int64_t)g * 3 * RB + q * RB + r];
    out[q * R + col0 + r] = sum;
}

}  // namespace

namespace kpm {

static std::mutex g_attr_lock;
// (kernel, device, attribute) -> the value set last
static std::map<std::tuple<const void *, int, int>, size_t> g_attr_set;

int ensure_max_dynamic_smem(const void *func, size_t smem)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return KPM_ECUDA;
    std::lock_guard<std::mutex> lock(g_attr_lock);
    size_t &have = g_attr_set[std::make_tuple(func, dev, 0)];
    if (have >= smem)
        return KPM_OK;
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return KPM_ECUDA;
    }
    have = smem;
    return KPM_OK;
}

int ensure_carveout_max_l1(const void *func)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return KPM_ECUDA;
    std::lock_guard<std::mutex> lock(g_attr_lock);
    size_t &have = g_attr_set[std::make_tuple(func, dev, 1)];
    if (have)
        return KPM_OK;
    if (cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxL1) != cudaSuccess) {
        cudaGetLastError();
        return KPM_ECUDA;
    }
    have = 1;
    return KPM_OK;
}

void *dev_alloc(kpm_ctx *c, size_t bytes)
{
    if (bytes == 0)
        bytes = 16;
    if (c->alloc_fn)
        return c->alloc_fn(bytes, c->alloc_user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(kpm_ctx *c, void *p)
{
    if (!p)
        return;
    if (c->free_fn)
        c->free_fn(p, c->alloc_user);
    else
        cudaFree(p);
}

int64_t block_ld(const kpm_ctx *c, int R)
{
    if (c->precision == KPM_PREC_FP32 && R > 1 && (R & 1))
        return R + 1;
    return R;
}

// Column blocks: R split into powers of two <= cap (64 by default), widest
// first, so each block starts on a column that keeps its vector accesses
// aligned.
std::vector<int> column_widths(int R, int cap)
{
    std::vector<int> w;
    int rest = R;
    for (int b = cap; b >= 1; b >>= 1)
        while (rest >= b) {
            w.push_back(b);
            rest -= b;
        }
    return w;
}

// Complex float staged shapes: the old W rows travel with each stage (the
// producer copies them, the consumers read them from shared memory) where
// the larger stages keep the same number of blocks per SM; otherwise each
// consumer lane loads its row's old W into registers a chunk ahead.
// (Complex double keeps its lanes' cp.async of the old W: staging it, with
// the sums started from -W, measured slower on the FP64-bound sweep.)
int choose_wstage(const kpm_ctx *c, const LaunchShape &s)
{
    if (c->precision != KPM_PREC_FP32 || s.stages < 1 || !c->gather_ok)
        return 0;
    const int vs = staged_value_bytes(false, c->half_ok);
    StagedLayout L0, L1;
    if (!staged_layout(c->C, s.T, s.T * s.E, 8, vs, c->u_max, c->l_max, s.stages, 1, false,
                       c->max_smem, L0) ||
        !staged_layout(c->C, s.T, s.T * s.E, 8, vs, c->u_max, c->l_max, s.stages, 1, true,
                       c->max_smem, L1))
        return 0;
    const int o0 = staged_max_blocks_per_sm(s.T, s.E, c->C, L0.smem, false, c->half_ok);
    const int o1 = staged_max_blocks_per_sm(s.T, s.E, c->C, L1.smem, false, c->half_ok);
    return o1 >= o0 && o1 > 0 ? 1 : 0;
}

LaunchShape default_shape(const kpm_ctx *c, int RB)
{
    LaunchShape s;
    const bool fp64 = c->precision == KPM_PREC_FP64;
    s.threads = fp64 ? 256 : 128;
    if (fp64) {
        s.E = RB >= 64 ? 2 : 1;
        s.T = RB / s.E;
    } else {
        s.E = RB >= 4 ? 4 : RB;
        s.T = RB / s.E;
    }
    s.blocks_per_sm = 0;  // 0 = occupancy maximum
    s.tile_groups = fp64 ? 8 : 1;
    s.stages = 0;
    // The staged kernel where it is built and two stages fit: the copies of
    // one chunk fly while the consumers work on the other.  Complex float
    // takes 4 columns per lane (two blocks per SM at width 32; measured best
    // at widths 16..64 on the 64^3 lattice, a third stage costs the second
    // block), at widths 2 and 4 the whole row in one lane (93 % of HBM at
    // width 4 on the 64^3 lattice against 50 % on the register path);
    // complex double 2 columns per lane at widths 2..32 and 1 at width 1
    // (one block per SM at width 32; measured faster than the register path
    // at every width on the 64^3 lattice, 2.2x at widths 1..4, with and
    // without the half-complex form).
    const int E = fp64 ? std::min(RB, 2) : std::min(RB, 4);
    if (c->gather_ok && RB >= (fp64 ? 1 : 2) && RB % E == 0 &&
        staged_shape_supported(RB / E, E, fp64)) {
        StagedLayout L;
        if (staged_layout(c->C, RB / E, RB, fp64 ? 16 : 8, staged_value_bytes(fp64, c->half_ok),
                          c->u_max, c->l_max, 2, 1, false, c->max_smem, L)) {
            s.E = E;
            s.T = RB / E;
            s.stages = 2;
            s.wstage = choose_wstage(c, s);
        }
    }
    return s;
}

// Shared-memory layout of a staged shape on this context (false if it does
// not fit or the context has no gather lists).
bool shape_layout(const kpm_ctx *c, const LaunchShape &s, StagedLayout &L)
{
    const bool fp64 = c->precision == KPM_PREC_FP64;
    if (s.stages < 1 || !c->gather_ok || !staged_shape_supported(s.T, s.E, fp64))
        return false;
    return staged_layout(c->C, s.T, s.T * s.E, fp64 ? 16 : 8, staged_value_bytes(fp64, c->half_ok),
                         c->u_max, c->l_max, s.stages, 1, s.wstage != 0,
                         c->max_smem, L);
}

// Blocks per SM of a staged shape with layout L.
int staged_occupancy(const kpm_ctx *c, const LaunchShape &s, const StagedLayout &L)
{
    return staged_max_blocks_per_sm(s.T, s.E, c->C, L.smem, c->precision == KPM_PREC_FP64,
                                    c->half_ok);
}

int resolve_grid(kpm_ctx *c, LaunchShape &s)
{
    int occ = 0;
    if (s.stages > 0) {
        StagedLayout L;
        if (!shape_layout(c, s, L))
            return -1;
        occ = staged_occupancy(c, s, L);
    } else {
        occ = sweep_max_blocks_per_sm(c->precision, s, false);
    }
    if (occ < 1)
        return -1;
    if (s.blocks_per_sm < 1 || s.blocks_per_sm > occ)
        s.blocks_per_sm = occ;
    return s.blocks_per_sm * c->n_sm;
}

int plan_blocks(kpm_ctx *c, int R, std::vector<ColumnBlock> &blocks, int64_t &slot_doubles)
{
    blocks.clear();
    slot_doubles = 0;
    int col0 = 0;
    for (int RB : column_widths(R, c->max_rb)) {
        ColumnBlock cb;
        cb.col0 = col0;
        cb.RB = RB;
        auto it = c->shapes.find(RB);
        cb.shape = it != c->shapes.end() ? it->second : default_shape(c, RB);
        cb.grid = resolve_grid(c, cb.shape);
        if (cb.grid < 1)
            return KPM_EUNSUPPORTED;
        cb.partial_offset = slot_doubles;
        slot_doubles += (int64_t)cb.grid * 3 * RB;
        blocks.push_back(cb);
        col0 += RB;
    }
    return KPM_OK;
}

int ensure_vectors(kpm_ctx *c, int R)
{
    const int64_t bytes = (c->n_pad + c->n_halo) * block_ld(c, R) * (int64_t)c->sdc;
    if (bytes <= c->vw_bytes)
        return KPM_OK;
    dev_free(c, c->d_V);
    dev_free(c, c->d_W);
    c->d_V = c->d_W = nullptr;
    c->vw_bytes = 0;
    c->d_V = dev_alloc(c, bytes);
    c->d_W = dev_alloc(c, bytes);
    if (!c->d_V || !c->d_W)
        return KPM_ENOMEM;
    c->vw_bytes = bytes;
    return KPM_OK;
}

int ensure_partial(kpm_ctx *c, int64_t doubles)
{
    if (doubles <= c->partial_doubles)
        return KPM_OK;
    dev_free(c, c->d_partial);
    c->d_partial = (double *)dev_alloc(c, doubles * sizeof(double));
    c->partial_doubles = c->d_partial ? doubles : 0;
    return c->d_partial ? KPM_OK : KPM_ENOMEM;
}

int ensure_eta(kpm_ctx *c, int64_t doubles)
{
    if (doubles <= c->eta_doubles)
        return KPM_OK;
    dev_free(c, c->d_eta);
    dev_free(c, c->d_eta_im);
    c->d_eta = (double *)dev_alloc(c, doubles * sizeof(double));
    c->d_eta_im = (double *)dev_alloc(c, doubles * sizeof(double));
    c->eta_doubles = (c->d_eta && c->d_eta_im) ? doubles : 0;
    return c->eta_doubles ? KPM_OK : KPM_ENOMEM;
}

int ensure_aux(kpm_ctx *c, int64_t bytes)
{
    if (bytes <= c->aux_bytes)
        return KPM_OK;
    dev_free(c, c->d_aux);
    c->d_aux = dev_alloc(c, bytes);
    c->aux_bytes = c->d_aux ? bytes : 0;
    return c->d_aux ? KPM_OK : KPM_ENOMEM;
}

}  // namespace kpm

namespace {

SweepParams sweep_params(const kpm_ctx *c, const ColumnBlock &cb, int R, const void *V, void *W,
                         double *partial, bool imag)
{
    SweepParams p;
    p.chunk_ptr = c->d_chunk_ptr;
    p.chunk_len = c->d_chunk_len;
    p.col = c->d_col;
    p.val = c->d_val;
    p.V = V;
    p.W = W;
    p.partial = partial;
    p.n_pad = c->n_pad;
    p.log2C = c->log2C;
    p.ld = (int32_t)block_ld(c, R);
    p.col0 = cb.col0;
    p.tile_groups = cb.shape.tile_groups > 0 ? cb.shape.tile_groups : 4;
    p.with_imag = imag ? 1 : 0;
    return p;
}

// The staged kernel's arguments for one sweep of column block cb.
int staged_params(const kpm_ctx *c, const ColumnBlock &cb, const SweepParams &p, bool init,
                  bool dots, StagedParams &q, StagedLayout &L)
{
    if (!shape_layout(c, cb.shape, L))
        return KPM_EUNSUPPORTED;
    q.one.rec = c->d_rec;
    q.one.ovf = c->d_ovf;
    q.one.lidx = c->d_lidx;
    q.one.val = c->d_val_staged;
    q.one.buf[0] = const_cast<void *>(p.V);
    q.one.buf[1] = p.W;
    q.one.partial = p.partial;
    q.one.tile0 = 0;
    q.one.n_tiles = c->n_chunks;
    q.one.ps = 3 * cb.RB;  // [grid][3][RB]
    q.one.qs = 1;
    q.one.ld = p.ld;
    q.one.col0 = p.col0;
    q.one.rows = c->n_pad + c->n_halo;
    q.one.entries = c->n_staged;
    q.one.n_ovf = c->n_ovf;
    q.probs = nullptr;
    q.n_probs = 1;
    q.parity = 0;
    q.C = c->C;
    q.stages = L.stages;
    q.with_imag = p.with_imag;
    q.init = init ? 1 : 0;
    q.dots = dots ? 1 : 0;
    q.fp64 = c->precision == KPM_PREC_FP64 ? 1 : 0;
    q.half = c->half_ok ? 1 : 0;
    q.stall_after = c->stall_after;
    q.err = c->d_err;
    q.bar_bytes = L.bar_bytes;
    q.stage_bytes = L.stage_bytes;
    q.off_val = L.off_val;
    q.off_lidx = L.off_lidx;
    q.off_aux = L.off_aux;
    q.off_w = L.off_w;
    return KPM_OK;
}

int launch_one(kpm_ctx *c, const ColumnBlock &cb, const SweepParams &p, bool init,
               cudaStream_t st, bool dots = true)
{
    c->launches++;
    if (cb.shape.stages > 0) {
        StagedLayout L;
        StagedParams q;
        KPM_TRY(staged_params(c, cb, p, init, dots, q, L));
        return launch_sweep_staged(q, cb.shape.T, cb.shape.E, cb.grid, L.smem, st,
                                   c->overlap != KPM_OVERLAP_NONE);
    }
    if (c->precision == KPM_PREC_FP64)
        return launch_sweep_fp64(p, cb.shape, cb.grid, init, st);
    return launch_sweep_fp32(p, cb.shape, cb.grid, init, st);
}

}  // namespace

int kpm::launch_phases_raw(void *V, bool fp64, const int32_t *perm, int64_t n, int64_t n_pad,
                           int R, int ld, uint64_t seed, int n_sm, cudaStream_t st)
{
    const uint64_t key = splitmix_mix(seed + 2 * kGolden);  // stream 1
    const int grid = n_sm * 8;
    if (fp64)
        phases_kernel<double><<<grid, 256, 0, st>>>((double *)V, perm, n, n_pad, R, ld, key, n, 0);
    else
        phases_kernel<float><<<grid, 256, 0, st>>>((float *)V, perm, n, n_pad, R, ld, key, n, 0);
    return cuda_status(cudaGetLastError());
}

int kpm::launch_phases(kpm_ctx *c, void *V, int R, uint64_t seed, cudaStream_t st)
{
    const uint64_t key = splitmix_mix(seed + 2 * kGolden);  // stream 1
    const int ld = (int)block_ld(c, R);
    const int grid = c->n_sm * 8;
    const int64_t rows = c->n_pad + c->n_halo;
    const int64_t gn = c->global_n > 0 ? c->global_n : c->n;
    c->launches++;
    if (c->precision == KPM_PREC_FP64)
        phases_kernel<double><<<grid, 256, 0, st>>>((double *)V, c->d_perm, c->n, rows, R, ld,
                                                    key, gn, c->row0);
    else
        phases_kernel<float><<<grid, 256, 0, st>>>((float *)V, c->d_perm, c->n, rows, R, ld,
                                                   key, gn, c->row0);
    return cuda_status(cudaGetLastError());
}

namespace {

int autotune_shapes(kpm_ctx *c, int R, int sweeps, cudaStream_t st, float *ms_per_sweep = nullptr);

// The sweep schedule of Fig. 5 on device buffers already holding V = nu_0:
// sweep m reads V = d_V (m even) or d_W (m odd) and overwrites the other.
// Sweeps run in batches of `slots` between eta reductions, column block by
// column block.
int run_schedule(kpm_ctx *c, int M, int R, double *eta, double *eta_im, cudaStream_t st)
{
    NvtxRange range("sweeps and eta reductions (enqueue)");
    std::vector<ColumnBlock> blocks;
    int64_t slot_doubles = 0;
    KPM_TRY(plan_blocks(c, R, blocks, slot_doubles));
    const int sweeps = M / 2;
    // as many sweeps of partials as fit in ~64 MB (at least one)
    int slots = (int)std::max<int64_t>(1, std::min<int64_t>(sweeps, (64LL << 20) / 8 / slot_doubles));
    if (c->reduce_interval > 0)
        slots = std::min(slots, c->reduce_interval);
    KPM_TRY(ensure_partial(c, slots * slot_doubles));
    const bool imag = eta_im != nullptr;
    for (int m0 = 0; m0 < sweeps; m0 += slots) {
        const int pending = std::min(slots, sweeps - m0);
        for (const ColumnBlock &cb : blocks) {
            for (int j = 0; j < pending; j++) {
                const int m = m0 + j;
                void *V = (m & 1) ? c->d_W : c->d_V, *W = (m & 1) ? c->d_V : c->d_W;
                double *slot = c->d_partial + (int64_t)j * slot_doubles;
                SweepParams p = sweep_params(c, cb, R, V, W, slot + cb.partial_offset, imag);
                KPM_TRY(launch_one(c, cb, p, m == 0, st));
            }
        }
        for (const ColumnBlock &cb : blocks) {
            const int threads = pending * 3 * cb.RB;
            c->launches++;
            reduce_moments_kernel<<<(threads + 255) / 256, 256, 0, st>>>(
                c->d_partial + cb.partial_offset, slot_doubles, pending, cb.grid, cb.RB, cb.col0, M,
                m0, eta, eta_im);
            KPM_CUDA(cudaGetLastError());
        }
    }
    return KPM_OK;
}

int upload_block(kpm_ctx *c, int R, const double *host_ri, void *dev, cudaStream_t st)
{
    const int64_t ld = block_ld(c, R);
    const int64_t count = c->n_pad * ld * 2;
    std::vector<double> staging;
    try {
        staging.assign(count, 0.0);
    } catch (const std::bad_alloc &) {
        return KPM_ENOMEM;
    }
    for (int64_t p = 0; p < c->n; p++) {
        const int64_t i = c->perm[p];
        std::memcpy(&staging[p * ld * 2], host_ri + i * R * 2, sizeof(double) * 2 * R);
    }
    if (c->precision == KPM_PREC_FP64) {
        KPM_CUDA(cudaMemcpyAsync(dev, staging.data(), count * sizeof(double),
                                 cudaMemcpyHostToDevice, st));
    } else {
        std::vector<float> f(count);
        for (int64_t k = 0; k < count; k++)
            f[k] = (float)staging[k];
        KPM_CUDA(cudaMemcpyAsync(dev, f.data(), count * sizeof(float), cudaMemcpyHostToDevice, st));
        KPM_CUDA(cudaStreamSynchronize(st));
    }
    KPM_CUDA(cudaStreamSynchronize(st));
    return KPM_OK;
}

}  // namespace

namespace kpm {
int sweep_max_blocks_per_sm_fp64(const LaunchShape &s);
int sweep_max_blocks_per_sm_fp32(const LaunchShape &s);
int sweep_max_blocks_per_sm(int precision, const LaunchShape &s, bool)
{
    return precision == KPM_PREC_FP64 ? sweep_max_blocks_per_sm_fp64(s)
                                      : sweep_max_blocks_per_sm_fp32(s);
}
}  // namespace kpm

// ================================================================= C ABI
extern "C" {

int kpm_create(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val_ri,
               double a, double b, const kpm_options *opt_in, kpm_ctx **out)
{
    NvtxRange range("kpm_create");
    if (!out)
        return KPM_EINVAL;
    *out = nullptr;
    kpm_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        kpm_default_options(&opt);
    if (opt.chunk_height == 0)
        opt.chunk_height = 32;
    if (opt.sigma == 0)
        opt.sigma = 256;
    if (opt.precision != KPM_PREC_FP64 && opt.precision != KPM_PREC_FP32)
        return KPM_EINVAL;
    if (!(a > 0.0) || !std::isfinite(a) || !std::isfinite(b))
        return KPM_EINVAL;
    if ((opt.alloc_fn == nullptr) != (opt.free_fn == nullptr))
        return KPM_EINVAL;
    // a part of a row-partitioned problem: halo columns, global row numbers
    if (opt.n_halo < 0 || opt.global_n < 0 || opt.row0 < 0 ||
        (opt.global_n > 0 && opt.row0 + n > opt.global_n) ||
        (opt.n_halo > 0 && opt.check_hermitian))
        return KPM_EINVAL;
    int rc = validate_csr_rect(n, n + opt.n_halo, row_ptr, col, val_ri);
    if (rc)
        return rc;
    if (opt.check_hermitian) {
        rc = check_hermitian(n, row_ptr, col, val_ri, 1e-12);
        if (rc)
            return rc;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || opt.device < 0 || opt.device >= ndev) {
        cudaGetLastError();
        return ndev == 0 ? KPM_ECUDA : KPM_EINVAL;
    }
    kpm_sell sell;
    {
        NvtxRange r("kpm_create: SELL-C-sigma build (host)");
        rc = sell_build_rect(n, opt.n_halo, row_ptr, col, val_ri, a, b, opt.chunk_height,
                             opt.sigma, opt.row_order, &sell);
    }
    if (rc)
        return rc;

    kpm_ctx *c = new (std::nothrow) kpm_ctx;
    if (!c) {
        kpm_sell_release(&sell);
        return KPM_ENOMEM;
    }
    c->device = opt.device;
    c->precision = opt.precision;
    c->n = n;
    c->n_pad = sell.n_pad;
    c->nnz = sell.nnz;
    c->n_stored = sell.n_stored;
    c->n_chunks = sell.n_chunks;
    c->C = sell.C;
    c->log2C = 0;
    while ((1 << c->log2C) < c->C)
        c->log2C++;
    c->sigma = sell.sigma;
    c->a = a;
    c->b = b;
    c->sdc = opt.precision == KPM_PREC_FP64 ? 16 : 8;
    c->autotune = opt.autotune;
    c->alloc_fn = opt.alloc_fn;
    c->free_fn = opt.free_fn;
    c->alloc_user = opt.alloc_user;
    c->perm.assign(sell.perm, sell.perm + sell.n_pad);
    c->n_halo = opt.n_halo;
    c->global_n = opt.global_n;
    c->row0 = opt.row0;

    DeviceGuard guard(c->device);
    auto fail = [&](int code) {
        kpm_sell_release(&sell);
        kpm_destroy(c);
        return code;
    };
    if (!guard.ok)
        return fail(KPM_ECUDA);
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        return fail(KPM_ECUDA);
    {
        int optin = 0;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device) !=
            cudaSuccess)
            return fail(KPM_ECUDA);
        c->max_smem = (size_t)optin;
    }
    c->d_err = (int *)dev_alloc(c, sizeof(int));
    if (!c->d_err)
        return fail(KPM_ENOMEM);
    if (cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess)
        return fail(KPM_ECUDA);

    c->d_chunk_ptr = (int64_t *)dev_alloc(c, sizeof(int64_t) * (sell.n_chunks + 1));
    c->d_chunk_len = (int32_t *)dev_alloc(c, sizeof(int32_t) * sell.n_chunks);
    c->d_col = (int32_t *)dev_alloc(c, sizeof(int32_t) * sell.n_stored);
    c->d_val = dev_alloc(c, c->sdc * sell.n_stored);
    c->d_perm = (int32_t *)dev_alloc(c, sizeof(int32_t) * sell.n_pad);
    if (!c->d_chunk_ptr || !c->d_chunk_len || !c->d_col || !c->d_val || !c->d_perm)
        return fail(KPM_ENOMEM);
    if (cudaMemcpy(c->d_chunk_ptr, sell.chunk_ptr, sizeof(int64_t) * (sell.n_chunks + 1),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_chunk_len, sell.chunk_len, sizeof(int32_t) * sell.n_chunks,
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_col, sell.col, sizeof(int32_t) * sell.n_stored, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(c->d_perm, sell.perm, sizeof(int32_t) * sell.n_pad, cudaMemcpyHostToDevice) !=
            cudaSuccess)
        return fail(KPM_ECUDA);
    if (c->n_halo > 0) {
        // local row -> position in the vector blocks, for the halo exchange
        std::vector<int32_t> iperm(n);
        for (int64_t p = 0; p < n; p++)
            iperm[sell.perm[p]] = (int32_t)p;
        c->d_iperm = (int32_t *)dev_alloc(c, sizeof(int32_t) * n);
        if (!c->d_iperm)
            return fail(KPM_ENOMEM);
        if (cudaMemcpy(c->d_iperm, iperm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return fail(KPM_ECUDA);
    }
    if (c->precision == KPM_PREC_FP64) {
        if (cudaMemcpy(c->d_val, sell.val_ri, 16 * sell.n_stored, cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return fail(KPM_ECUDA);
    } else {
        std::vector<float> f;
        try {
            f.resize(2 * sell.n_stored);
        } catch (const std::bad_alloc &) {
            return fail(KPM_ENOMEM);
        }
        for (int64_t k = 0; k < 2 * sell.n_stored; k++)
            f[k] = (float)sell.val_ri[k];
        if (cudaMemcpy(c->d_val, f.data(), 8 * sell.n_stored, cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return fail(KPM_ECUDA);
    }
    c->upload_bytes = (int64_t)sizeof(int64_t) * (sell.n_chunks + 1) +
                      (int64_t)sizeof(int32_t) * (sell.n_chunks + sell.n_stored + sell.n_pad) +
                      (int64_t)c->sdc * sell.n_stored;
    // every stored entry purely real or purely imaginary: the staged
    // kernel's two-FMA (half-complex) form
    bool half = true;
    for (int64_t k = 0; k < sell.n_stored && half; k++)
        half = sell.val_ri[2 * k] == 0.0 || sell.val_ri[2 * k + 1] == 0.0;
    if (sell.C >= 8) {
        // gather lists and staged entry arrays for the staged kernel; a
        // matrix whose lists do not fit the 16-bit local indices keeps the
        // register-path kernel only
        NvtxRange r("kpm_create: gather lists, staged arrays, upload");
        kpm_gather g;
        const int grc = kpm_gather_build(&sell, &g);
        if (grc == KPM_ENOMEM)
            return fail(KPM_ENOMEM);
        if (grc == KPM_OK) {
            // complex double: the two-FMA form's operands need bit 15 of the
            // local indices; complex float: every row's own entry real (else
            // kpm_staged_build refuses form 3 and the general form is built)
            const bool fp32 = c->precision == KPM_PREC_FP32;
            half = half && (fp32 || g.u_max <= 32768);
            int form = fp32 ? (half ? 3 : 1) : (half ? 2 : 0);
            kpm_staged sg;
            int src = kpm_staged_build(&sell, &g, form, &sg);
            if (src == KPM_EINVAL && form == 3) {
                half = false;
                form = 1;
                src = kpm_staged_build(&sell, &g, form, &sg);
            }
            if (src != KPM_OK) {
                kpm_gather_release(&g);
                return fail(src);
            }
            // producer records: fixed 256-byte entries, runs past the inline
            // ones in the overflow array
            std::vector<int2> rec, ovf;
            try {
                rec.assign((size_t)g.n_chunks * KPM_REC_WORDS, make_int2(0, 0));
                for (int64_t ch = 0; ch < g.n_chunks; ch++) {
                    int2 *r = &rec[(size_t)ch * KPM_REC_WORDS];
                    const int64_t e0 = sg.chunk_ptr[ch];
                    const int64_t q0 = g.run_ptr[ch], nr = g.run_ptr[ch + 1] - q0;
                    const int64_t of = (int64_t)ovf.size();
                    r[0] = make_int2((int)(uint32_t)e0, (int)(e0 >> 32));
                    // staged length, and (half-complex float) the real
                    // region's length in the upper 16 bits
                    const int nre = sg.chunk_nre ? sg.chunk_nre[ch] : 0;
                    r[1] = make_int2(sg.chunk_len[ch] | (nre << 16), (int)nr);
                    r[2] = make_int2((int)(uint32_t)of, (int)(of >> 32));
                    for (int64_t q = 0; q < nr; q++) {
                        const int2 run = make_int2(g.runs[2 * (q0 + q)], g.runs[2 * (q0 + q) + 1]);
                        if (q < KPM_REC_INLINE_RUNS)
                            r[3 + q] = run;
                        else
                            ovf.push_back(run);
                    }
                }
            } catch (const std::bad_alloc &) {
                kpm_staged_release(&sg);
                kpm_gather_release(&g);
                return fail(KPM_ENOMEM);
            }
            const size_t vbytes = (size_t)staged_value_bytes(!fp32, half) * sg.n_stored;
            c->d_val_staged = dev_alloc(c, vbytes);
            c->d_lidx = (uint16_t *)dev_alloc(c, sizeof(uint16_t) * sg.n_stored);
            c->d_rec = (int2 *)dev_alloc(c, sizeof(int2) * rec.size());
            c->d_ovf = (int2 *)dev_alloc(c, sizeof(int2) * (ovf.empty() ? 1 : ovf.size()));
            const bool alloc_ok = c->d_val_staged && c->d_lidx && c->d_rec && c->d_ovf;
            const void *vsrc = sg.valf ? (const void *)sg.valf : (const void *)sg.val;
            const bool ok =
                alloc_ok &&
                cudaMemcpy(c->d_val_staged, vsrc, vbytes, cudaMemcpyHostToDevice) == cudaSuccess &&
                cudaMemcpy(c->d_lidx, sg.lidx, sizeof(uint16_t) * sg.n_stored,
                           cudaMemcpyHostToDevice) == cudaSuccess &&
                cudaMemcpy(c->d_rec, rec.data(), sizeof(int2) * rec.size(),
                           cudaMemcpyHostToDevice) == cudaSuccess &&
                (ovf.empty() || cudaMemcpy(c->d_ovf, ovf.data(), sizeof(int2) * ovf.size(),
                                           cudaMemcpyHostToDevice) == cudaSuccess);
            c->u_max = g.u_max;
            c->l_max = sg.l_max;
            c->n_staged = sg.n_stored;
            c->n_ovf = (int64_t)ovf.size();
            const int64_t n_staged = sg.n_stored;
            kpm_staged_release(&sg);
            kpm_gather_release(&g);
            if (!ok)
                return fail(alloc_ok ? KPM_ECUDA : KPM_ENOMEM);
            c->gather_ok = true;
            c->half_ok = half;
            c->upload_bytes += (int64_t)vbytes + (int64_t)sizeof(uint16_t) * n_staged +
                               (int64_t)sizeof(int2) * (int64_t)(rec.size() + ovf.size());
            // complex double: the staged kernel's widest block is 32 columns
            // (wider rows would leave room for one stage only), and two
            // 32-wide staged sweeps beat one 64-wide register-path sweep
            if (c->precision == KPM_PREC_FP64)
                c->max_rb = 32;
        }
    }
    kpm_sell_release(&sell);
    *out = c;
    return KPM_OK;
}

void kpm_destroy(kpm_ctx *c)
{
    if (!c)
        return;
    DeviceGuard guard(c->device);
    cudaDeviceSynchronize();
    dev_free(c, c->d_chunk_ptr);
    dev_free(c, c->d_chunk_len);
    dev_free(c, c->d_col);
    dev_free(c, c->d_val);
    dev_free(c, c->d_perm);
    dev_free(c, c->d_iperm);
    dev_free(c, c->d_V);
    dev_free(c, c->d_W);
    dev_free(c, c->d_partial);
    dev_free(c, c->d_eta);
    dev_free(c, c->d_eta_im);
    dev_free(c, c->d_lidx);
    dev_free(c, c->d_val_staged);
    dev_free(c, c->d_aux);
    dev_free(c, c->d_rec);
    dev_free(c, c->d_ovf);
    dev_free(c, c->d_err);
    delete c;
}

int kpm_test_stall_staged(kpm_ctx *c, int64_t chunks_per_block)
{
    if (!c || chunks_per_block < -1)
        return KPM_EINVAL;
    c->stall_after = chunks_per_block;
    return KPM_OK;
}

int kpm_check_device_error(kpm_ctx *c)
{
    if (!c)
        return KPM_EINVAL;
    DeviceGuard guard(c->device);
    int word = 0;
    KPM_CUDA(cudaMemcpy(&word, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (word == 0)
        return KPM_OK;
    KPM_CUDA(cudaMemset(c->d_err, 0, sizeof(int)));
    return word == KPM_DEVERR_RANGE ? KPM_EINVAL : KPM_ETIMEOUT;
}

int kpm_get_info(const kpm_ctx *c, kpm_info *out)
{
    if (!c || !out)
        return KPM_EINVAL;
    out->n = c->n;
    out->n_pad = c->n_pad;
    out->nnz = c->nnz;
    out->n_stored = c->n_stored;
    out->n_chunks = c->n_chunks;
    out->C = c->C;
    out->sigma = c->sigma;
    out->precision = c->precision;
    out->device = c->device;
    out->a = c->a;
    out->b = c->b;
    out->matrix_bytes = c->n_stored * ((int64_t)c->sdc + 4);
    out->gather_lists = c->gather_ok ? 1 : 0;
    out->half_complex = c->half_ok ? 1 : 0;
    out->upload_bytes = c->upload_bytes;
    out->kernel_launches = c->launches;
    return KPM_OK;
}

int64_t kpm_block_bytes(const kpm_ctx *c, int32_t R)
{
    if (!c || R < 1)
        return -1;
    return (c->n_pad + c->n_halo) * block_ld(c, R) * (int64_t)c->sdc;
}

int kpm_block_upload(kpm_ctx *c, int32_t R, const double *host_ri, void *dev, void *stream)
{
    if (!c || R < 1 || !host_ri || !dev)
        return KPM_EINVAL;
    DeviceGuard guard(c->device);
    return upload_block(c, R, host_ri, dev, (cudaStream_t)stream);
}

int kpm_block_download(kpm_ctx *c, int32_t R, const void *dev, double *host_ri, void *stream)
{
    if (!c || R < 1 || !host_ri || !dev)
        return KPM_EINVAL;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t ld = block_ld(c, R);
    const int64_t count = c->n_pad * ld * 2;
    std::vector<double> staging;
    try {
        staging.resize(count);
    } catch (const std::bad_alloc &) {
        return KPM_ENOMEM;
    }
    if (c->precision == KPM_PREC_FP64) {
        KPM_CUDA(cudaMemcpyAsync(staging.data(), dev, count * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
        KPM_CUDA(cudaStreamSynchronize(st));
    } else {
        std::vector<float> f(count);
        KPM_CUDA(cudaMemcpyAsync(f.data(), dev, count * sizeof(float), cudaMemcpyDeviceToHost, st));
        KPM_CUDA(cudaStreamSynchronize(st));
        for (int64_t k = 0; k < count; k++)
            staging[k] = f[k];
    }
    for (int64_t p = 0; p < c->n; p++) {
        const int64_t i = c->perm[p];
        std::memcpy(host_ri + i * R * 2, &staging[p * ld * 2], sizeof(double) * 2 * R);
    }
    return KPM_OK;
}

int kpm_halo_pack(kpm_ctx *c, int32_t R, const void *V, const int32_t *rows_dev, int32_t count,
                  void *buf, void *stream)
{
    if (!c || R < 1 || !V || !buf || count < 0 || (count > 0 && !rows_dev) || c->n_halo < 1)
        return KPM_EINVAL;
    if (count == 0)
        return KPM_OK;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int ld = (int)block_ld(c, R);
    const int grid = c->n_sm * 4;
    c->launches++;
    if (c->precision == KPM_PREC_FP64)
        halo_pack_kernel<double><<<grid, 256, 0, st>>>((const double *)V, c->d_iperm, rows_dev,
                                                       count, ld, c->n, (double *)buf, c->d_err);
    else
        halo_pack_kernel<float><<<grid, 256, 0, st>>>((const float *)V, c->d_iperm, rows_dev,
                                                      count, ld, c->n, (float *)buf, c->d_err);
    return cuda_status(cudaGetLastError());
}

int kpm_halo_unpack(kpm_ctx *c, int32_t R, void *V, const void *buf, int64_t first, int32_t count,
                    void *stream)
{
    if (!c || R < 1 || !V || !buf || count < 0 || first < 0 || first + count > c->n_halo)
        return KPM_EINVAL;
    if (count == 0)
        return KPM_OK;
    DeviceGuard guard(c->device);
    const int64_t row_bytes = block_ld(c, R) * (int64_t)c->sdc;
    char *dst = static_cast<char *>(V) + (c->n_pad + first) * row_bytes;
    return cuda_status(cudaMemcpyAsync(dst, buf, (size_t)count * row_bytes,
                                       cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
}

int kpm_block_phases(kpm_ctx *c, int32_t R, uint64_t seed, void *V, void *stream)
{
    if (!c || R < 1 || !V)
        return KPM_EINVAL;
    DeviceGuard guard(c->device);
    return launch_phases(c, V, R, seed, (cudaStream_t)stream);
}

int kpm_aug_spmmv(kpm_ctx *c, int32_t R, const void *V, void *W, double *eta_dev, int32_t init,
                  int32_t with_imag, void *stream)
{
    if (!c || R < 1 || !V || !W || V == W)
        return KPM_EINVAL;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<ColumnBlock> blocks;
    int64_t slot_doubles = 0;
    KPM_TRY(plan_blocks(c, R, blocks, slot_doubles));
    KPM_TRY(ensure_partial(c, slot_doubles));
    for (const ColumnBlock &cb : blocks) {
        SweepParams p = sweep_params(c, cb, R, V, W, c->d_partial + cb.partial_offset, with_imag);
        KPM_TRY(launch_one(c, cb, p, init != 0, st));
        if (!eta_dev)
            continue;
        c->launches++;
        reduce_single_kernel<<<(3 * cb.RB + 127) / 128, 128, 0, st>>>(
            c->d_partial + cb.partial_offset, cb.grid, cb.RB, cb.col0, R, eta_dev);
        KPM_CUDA(cudaGetLastError());
    }
    return KPM_OK;
}

int kpm_sweep_variant(kpm_ctx *c, int32_t R, const void *V, void *W, int32_t variant,
                      void *stream)
{
    if (!c || R < 1 || !V || !W || V == W || variant < 0 || variant > 2)
        return KPM_EINVAL;
    if (variant == 0)
        return kpm_aug_spmmv(c, R, V, W, nullptr, 0, 0, stream);
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<ColumnBlock> blocks;
    int64_t slot_doubles = 0;
    KPM_TRY(plan_blocks(c, R, blocks, slot_doubles));
    for (const ColumnBlock &cb : blocks) {
        SweepParams p = sweep_params(c, cb, R, V, W, nullptr, false);
        if (cb.shape.stages > 0) {
            // the staged kernel without its scalar products
            KPM_TRY(launch_one(c, cb, p, variant == 2, st, false));
            continue;
        }
        c->launches++;
        KPM_TRY(c->precision == KPM_PREC_FP64
                    ? launch_nodot_fp64(p, cb.shape, cb.grid, variant == 2, st)
                    : launch_nodot_fp32(p, cb.shape, cb.grid, variant == 2, st));
    }
    return KPM_OK;
}

int kpm_set_reduce_interval(kpm_ctx *c, int32_t sweeps)
{
    if (!c || sweeps < 0)
        return KPM_EINVAL;
    c->reduce_interval = sweeps;
    return KPM_OK;
}

int kpm_checked_build(void)
{
#ifdef KPM_CHECK
    return 1;
#else
    return 0;
#endif
}

int kpm_test_corrupt_record(kpm_ctx *c, int64_t chunk, int32_t word, int32_t x, int32_t y)
{
#ifdef KPM_CHECK
    if (!c || !c->d_rec || chunk < 0 || chunk >= c->n_chunks || word < 0 || word >= KPM_REC_WORDS)
        return KPM_EINVAL;
    DeviceGuard guard(c->device);
    const int2 v = make_int2(x, y);
    return cuda_status(cudaMemcpy(c->d_rec + chunk * KPM_REC_WORDS + word, &v, sizeof(v),
                                  cudaMemcpyHostToDevice));
#else
    (void)c;
    (void)chunk;
    (void)word;
    (void)x;
    (void)y;
    return KPM_EUNSUPPORTED;
#endif
}

int kpm_set_sweep_overlap(kpm_ctx *c, int32_t mode)
{
    if (!c || mode < KPM_OVERLAP_NONE || mode > KPM_OVERLAP_PDL)
        return KPM_EINVAL;
    c->overlap = mode;
    return KPM_OK;
}

int kpm_moments_device(kpm_ctx *c, int32_t M, int32_t R, uint64_t seed, double *eta_dev,
                       double *eta_imag_dev, void *stream)
{
    if (c && c->n_halo > 0)
        return KPM_EUNSUPPORTED;  // a part runs its sweeps with halo exchanges
    if (!c || M < 2 || (M & 1) || R < 1 || !eta_dev)
        return KPM_EINVAL;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (c->autotune && !c->tuned.count(R))
        KPM_TRY(autotune_shapes(c, R, 5, st));
    KPM_TRY(ensure_vectors(c, R));
    KPM_TRY(launch_phases(c, c->d_V, R, seed, st));
    return run_schedule(c, M, R, eta_dev, eta_imag_dev, st);
}

static int moments_to_host(kpm_ctx *c, int32_t M, int32_t R, double *eta, double *eta_imag,
                           cudaStream_t st)
{
    NvtxRange range("eta to host (waits for the sweeps)");
    const int64_t count = (int64_t)M * R;
    KPM_CUDA(cudaMemcpyAsync(eta, c->d_eta, count * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (eta_imag)
        KPM_CUDA(cudaMemcpyAsync(eta_imag, c->d_eta_im, count * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
    KPM_CUDA(cudaStreamSynchronize(st));
    return kpm_check_device_error(c);
}

int kpm_moments(kpm_ctx *c, int32_t M, int32_t R, uint64_t seed, double *eta, double *eta_imag,
                void *stream)
{
    NvtxRange range("kpm_moments");
    if (c && c->n_halo > 0)
        return KPM_EUNSUPPORTED;  // a part runs its sweeps with halo exchanges
    if (!c || M < 2 || (M & 1) || R < 1 || !eta)
        return KPM_EINVAL;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    KPM_TRY(ensure_eta(c, (int64_t)M * R));
    if (c->autotune && !c->tuned.count(R))
        KPM_TRY(autotune_shapes(c, R, 5, st));
    KPM_TRY(ensure_vectors(c, R));
    KPM_TRY(launch_phases(c, c->d_V, R, seed, st));
    KPM_TRY(run_schedule(c, M, R, c->d_eta, eta_imag ? c->d_eta_im : nullptr, st));
    return moments_to_host(c, M, R, eta, eta_imag, st);
}

int kpm_moments_v0(kpm_ctx *c, int32_t M, int32_t R, const double *v0_ri, double *eta,
                   double *eta_imag, void *stream)
{
    if (c && c->n_halo > 0)
        return KPM_EUNSUPPORTED;  // a part runs its sweeps with halo exchanges
    if (!c || M < 2 || (M & 1) || R < 1 || !eta || !v0_ri)
        return KPM_EINVAL;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    KPM_TRY(ensure_eta(c, (int64_t)M * R));
    if (c->autotune && !c->tuned.count(R))
        KPM_TRY(autotune_shapes(c, R, 5, st));
    KPM_TRY(ensure_vectors(c, R));
    KPM_TRY(upload_block(c, R, v0_ri, c->d_V, st));
    KPM_TRY(run_schedule(c, M, R, c->d_eta, eta_imag ? c->d_eta_im : nullptr, st));
    return moments_to_host(c, M, R, eta, eta_imag, st);
}

int kpm_moments_local(kpm_ctx *c, int32_t M, int32_t R, const int64_t *rows, double *eta,
                      double *eta_imag, void *stream)
{
    if (c && c->n_halo > 0)
        return KPM_EUNSUPPORTED;  // a part runs its sweeps with halo exchanges
    if (!c || M < 2 || (M & 1) || R < 1 || !eta || !rows)
        return KPM_EINVAL;
    for (int32_t r = 0; r < R; r++)
        if (rows[r] < 0 || rows[r] >= c->n)
            return KPM_EINVAL;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    KPM_TRY(ensure_eta(c, (int64_t)M * R));
    KPM_TRY(ensure_aux(c, (int64_t)R * sizeof(int64_t)));
    if (c->autotune && !c->tuned.count(R))
        KPM_TRY(autotune_shapes(c, R, 5, st));
    KPM_TRY(ensure_vectors(c, R));
    KPM_CUDA(cudaMemcpyAsync(c->d_aux, rows, R * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    const int ld = (int)block_ld(c, R);
    c->launches++;
    if (c->precision == KPM_PREC_FP64)
        basis_kernel<double><<<c->n_sm * 8, 256, 0, st>>>((double *)c->d_V, c->d_perm, c->n,
                                                          c->n_pad, R, ld, (const int64_t *)c->d_aux);
    else
        basis_kernel<float><<<c->n_sm * 8, 256, 0, st>>>((float *)c->d_V, c->d_perm, c->n,
                                                         c->n_pad, R, ld, (const int64_t *)c->d_aux);
    KPM_CUDA(cudaGetLastError());
    KPM_TRY(run_schedule(c, M, R, c->d_eta, eta_imag ? c->d_eta_im : nullptr, st));
    return moments_to_host(c, M, R, eta, eta_imag, st);
}

int kpm_moments_plane_wave(kpm_ctx *c, int32_t M, int32_t R, int32_t nx, int32_t ny, int32_t nz,
                           int32_t norb, const double *q, const int32_t *orb, double *eta,
                           double *eta_imag, void *stream)
{
    if (c && c->n_halo > 0)
        return KPM_EUNSUPPORTED;  // a part runs its sweeps with halo exchanges
    if (!c || M < 2 || (M & 1) || R < 1 || !eta || !q || !orb || nx < 1 || ny < 1 || nz < 1 ||
        norb < 1 || (int64_t)nx * ny * nz * norb != c->n)
        return KPM_EINVAL;
    for (int32_t r = 0; r < R; r++) {
        if (orb[r] < 0 || orb[r] >= norb)
            return KPM_EINVAL;
        for (int j = 0; j < 3; j++)
            if (!std::isfinite(q[3 * r + j]))
                return KPM_EINVAL;
    }
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    KPM_TRY(ensure_eta(c, (int64_t)M * R));
    const int64_t qbytes = ((int64_t)R * 3 * sizeof(double) + 15) / 16 * 16;
    KPM_TRY(ensure_aux(c, qbytes + (int64_t)R * sizeof(int32_t)));
    if (c->autotune && !c->tuned.count(R))
        KPM_TRY(autotune_shapes(c, R, 5, st));
    KPM_TRY(ensure_vectors(c, R));
    char *aux = (char *)c->d_aux;
    KPM_CUDA(cudaMemcpyAsync(aux, q, R * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
    KPM_CUDA(cudaMemcpyAsync(aux + qbytes, orb, R * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    const int ld = (int)block_ld(c, R);
    const double scale = 1.0 / std::sqrt((double)nx * ny * nz);
    c->launches++;
    if (c->precision == KPM_PREC_FP64)
        plane_wave_kernel<double><<<c->n_sm * 8, 256, 0, st>>>(
            (double *)c->d_V, c->d_perm, c->n, c->n_pad, R, ld, (const double *)aux,
            (const int32_t *)(aux + qbytes), nx, ny, norb, scale);
    else
        plane_wave_kernel<float><<<c->n_sm * 8, 256, 0, st>>>(
            (float *)c->d_V, c->d_perm, c->n, c->n_pad, R, ld, (const double *)aux,
            (const int32_t *)(aux + qbytes), nx, ny, norb, scale);
    KPM_CUDA(cudaGetLastError());
    KPM_TRY(run_schedule(c, M, R, c->d_eta, eta_imag ? c->d_eta_im : nullptr, st));
    return moments_to_host(c, M, R, eta, eta_imag, st);
}

}  // extern "C"

// ------------------------------------------------------------ autotuner
namespace {

// Candidate launch shapes for a column block of width RB.
std::vector<LaunchShape> shape_candidates(const kpm_ctx *c, int RB)
{
    std::vector<LaunchShape> out;
    const int max_threads = c->precision == KPM_PREC_FP64 ? 256 : 512;
    for (int E = 1; E <= 4; E <<= 1) {
        if (RB % E)
            continue;
        const int T = RB / E;
        if (T < 1 || T > 32)
            continue;
        for (int threads = 128; threads <= max_threads; threads <<= 1)
            for (int tg : {1, 4}) {
                LaunchShape s{T, E, threads, 0, tg};
                if (sweep_max_blocks_per_sm(c->precision, s, false) > 0)
                    out.push_back(s);
            }
        // the staged kernel with 1..3 stages where they fit
        for (int ns = 1; ns <= 3; ns++) {
            LaunchShape s{T, E, 128, 0, 1};
            s.stages = ns;
            s.wstage = choose_wstage(c, s);
            StagedLayout L;
            if (shape_layout(c, s, L) &&
                staged_occupancy(c, s, L) > 0)
                out.push_back(s);
        }
    }
    return out;
}

// Average time of `sweeps` non-initial sweeps of one column block with
// shape s (V, W are the context's work blocks holding a recurrence).
int time_block(kpm_ctx *c, int R, int col0, int RB, LaunchShape s, int sweeps, cudaStream_t st,
               cudaEvent_t e0, cudaEvent_t e1, float *ms)
{
    ColumnBlock cb;
    cb.col0 = col0;
    cb.RB = RB;
    cb.shape = s;
    cb.grid = resolve_grid(c, cb.shape);
    if (cb.grid < 1)
        return KPM_EUNSUPPORTED;
    cb.partial_offset = 0;
    KPM_TRY(ensure_partial(c, (int64_t)cb.grid * 3 * RB));
    void *V = c->d_V, *W = c->d_W;
    for (int k = 0; k < 2 + sweeps; k++) {
        if (k == 2)
            KPM_CUDA(cudaEventRecord(e0, st));
        SweepParams p = sweep_params(c, cb, R, V, W, c->d_partial, false);
        KPM_TRY(launch_one(c, cb, p, false, st));
        std::swap(V, W);
    }
    KPM_CUDA(cudaEventRecord(e1, st));
    KPM_CUDA(cudaEventSynchronize(e1));
    KPM_CUDA(cudaEventElapsedTime(ms, e0, e1));
    *ms /= sweeps;
    return KPM_OK;
}

int autotune_shapes(kpm_ctx *c, int R, int sweeps, cudaStream_t st, float *ms_per_sweep)
{
    KPM_TRY(ensure_vectors(c, R));
    // a bounded recurrence to time on: random phases in V, W = (1/2) H' V
    KPM_TRY(launch_phases(c, c->d_V, R, 0x5EED, st));
    {
        std::vector<ColumnBlock> blocks;
        int64_t slot = 0;
        KPM_TRY(plan_blocks(c, R, blocks, slot));
        KPM_TRY(ensure_partial(c, slot));
        for (const ColumnBlock &cb : blocks) {
            SweepParams p = sweep_params(c, cb, R, c->d_V, c->d_W, c->d_partial + cb.partial_offset,
                                         false);
            KPM_TRY(launch_one(c, cb, p, true, st));
        }
    }
    cudaEvent_t e0, e1;
    KPM_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return KPM_ECUDA;
    }
    int rc = KPM_OK;
    std::map<int, std::pair<float, LaunchShape>> best;  // per width
    int best_cap = 64;
    float best_total = 1e30f;
    for (int cap = 64; cap >= 16 && rc == KPM_OK; cap >>= 1) {
        if (cap > 64 || (cap < 64 && R < 2 * cap))
            continue;
        float total = 0.f;
        int col0 = 0;
        for (int RB : column_widths(R, cap)) {
            if (!best.count(RB)) {
                float bt = 1e30f;
                LaunchShape bs = default_shape(c, RB);
                for (const LaunchShape &s : shape_candidates(c, RB)) {
                    float ms = 0.f;
                    rc = time_block(c, R, col0, RB, s, sweeps, st, e0, e1, &ms);
                    if (rc != KPM_OK)
                        break;
                    if (ms < bt)
                        bt = ms, bs = s;
                }
                if (rc != KPM_OK)
                    break;
                best[RB] = {bt, bs};
            }
            total += best[RB].first;
            col0 += RB;
        }
        if (rc == KPM_OK && total < best_total)
            best_total = total, best_cap = cap;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != KPM_OK)
        return rc;
    c->max_rb = best_cap;
    for (auto &kv : best)
        c->shapes[kv.first] = kv.second.second;
    c->tuned[R] = 1;
    if (ms_per_sweep)
        *ms_per_sweep = best_total;
    return KPM_OK;
}

}  // namespace

extern "C" {

int kpm_autotune(kpm_ctx *c, int32_t R, int32_t sweeps, void *stream,
                            kpm_launch *best)
{
    if (!c || R < 1 || sweeps < 1)
        return KPM_EINVAL;
    DeviceGuard guard(c->device);
    KPM_TRY(autotune_shapes(c, R, sweeps, (cudaStream_t)stream));
    if (best) {
        const int RB = column_widths(R, c->max_rb).front();
        const LaunchShape &s = c->shapes[RB];
        best->lanes_per_row = s.T;
        best->cols_per_lane = s.E;
        best->block_threads = s.threads;
        best->blocks_per_sm = s.blocks_per_sm;
        best->tile_groups = s.tile_groups;
        best->stages = s.stages;
    }
    return KPM_OK;
}

int kpm_autotune_layout(int64_t n, const int64_t *row_ptr, const int32_t *col,
                                   const double *val_ri, double a, double b,
                                   const kpm_options *base, int32_t R, int32_t sweeps,
                                   kpm_options *best, double *best_ms)
{
    if (!best || R < 1 || sweeps < 1)
        return KPM_EINVAL;
    kpm_options opt;
    if (base)
        opt = *base;
    else
        kpm_default_options(&opt);
    KPM_TRY(validate_csr(n, row_ptr, col, val_ri));
    // sigma only matters when row lengths differ
    bool uniform = true;
    for (int64_t i = 1; i < n && uniform; i++)
        uniform = (row_ptr[i + 1] - row_ptr[i]) == (row_ptr[1] - row_ptr[0]);
    const int Cs[] = {8, 16, 32, 64, 128};
    const int sigmas_ragged[] = {1, 256, 4096};
    double best_t = 1e300;
    int rc = KPM_EUNSUPPORTED;
    for (int C : Cs) {
        for (int si = 0; si < (uniform ? 1 : 3); si++) {
            kpm_options o = opt;
            o.chunk_height = C;
            o.sigma = uniform ? 1 : sigmas_ragged[si];
            if (o.sigma > 1 && o.sigma < C)
                continue;
            o.autotune = 0;
            kpm_ctx *t = nullptr;
            int r = kpm_create(n, row_ptr, col, val_ri, a, b, &o, &t);
            if (r != KPM_OK)
                return r;
            float ms = 0.f;
            {
                DeviceGuard guard(t->device);
                r = autotune_shapes(t, R, sweeps, nullptr, &ms);
            }
            kpm_destroy(t);
            if (r != KPM_OK)
                return r;
            rc = KPM_OK;
            if (ms < best_t) {
                best_t = ms;
                *best = o;
            }
        }
    }
    best->autotune = 1;
    if (best_ms)
        *best_ms = best_t;
    return rc;
}

int kpm_get_max_block_width(const kpm_ctx *c)
{
    return c ? c->max_rb : -1;
}

int kpm_get_launch(const kpm_ctx *c, int32_t R, kpm_launch *out)
{
    if (!c || !out || R < 1 || R > 64 || (R & (R - 1)))
        return KPM_EINVAL;
    auto it = c->shapes.find(R);
    LaunchShape s = it != c->shapes.end() ? it->second : default_shape(c, R);
    if (s.blocks_per_sm < 1) {
        DeviceGuard guard(c->device);
        StagedLayout L;
        if (s.stages > 0)
            s.blocks_per_sm = shape_layout(c, s, L)
                                  ? staged_occupancy(c, s, L)
                                  : 0;
        else
            s.blocks_per_sm = sweep_max_blocks_per_sm(c->precision, s, false);
    }
    out->lanes_per_row = s.T;
    out->cols_per_lane = s.E;
    out->block_threads = s.stages > 0 ? 32 + c->C * s.T : s.threads;
    out->blocks_per_sm = s.blocks_per_sm;
    out->tile_groups = s.tile_groups;
    out->stages = s.stages;
    return KPM_OK;
}

int kpm_set_launch(kpm_ctx *c, int32_t R, const kpm_launch *l)
{
    if (!c || !l || R < 1 || R > 64 || (R & (R - 1)))
        return KPM_EINVAL;
    if (l->lanes_per_row * l->cols_per_lane != R || l->block_threads < 32 ||
        l->block_threads > 1024 || (l->block_threads % 32) ||
        l->blocks_per_sm < 0 || l->tile_groups < 0 || l->tile_groups > 1024)
        return KPM_EINVAL;
    if (l->stages < 0 || l->stages > 8)
        return KPM_EINVAL;
    LaunchShape s{l->lanes_per_row, l->cols_per_lane, l->block_threads, l->blocks_per_sm,
                  l->tile_groups > 0 ? l->tile_groups : 4};
    s.stages = l->stages;
    DeviceGuard guard(c->device);
    s.wstage = choose_wstage(c, s);
    if (s.stages > 0) {
        StagedLayout L;
        if (!shape_layout(c, s, L) || staged_occupancy(c, s, L) < 1)
            return KPM_EUNSUPPORTED;
        // the register-path fields stay valid for the ablation variants
        if (sweep_max_blocks_per_sm(c->precision, s, false) < 1)
            s.threads = 128;
    } else if (sweep_max_blocks_per_sm(c->precision, s, false) < 1)
        return KPM_EUNSUPPORTED;
    c->shapes[R] = s;
    return KPM_OK;
}

}  // extern "C"

// =====================================================================
// Allocation-free sweep (kpm_aug_spmmv_static).
//
// kpm_aug_spmmv keeps the per-block partial sums of eta in a device buffer
// that it allocates on first use.  This variant runs the same kernels but
// takes that scratch from the fixed array below.  The CUDA runtime places
// the array in device memory when this library's module is loaded on a
// device and keeps it there until the process exits, so a call never
// allocates.  Host code cannot use the symbol as a pointer; its device
// address is looked up once per device with cudaGetSymbolAddress.
// =====================================================================
#include <mutex>

#define KPM_STATIC_SCRATCH_DOUBLES (1024 * 1024)  // 8 MiB per device

static __device__ __align__(256) double g_static_scratch[KPM_STATIC_SCRATCH_DOUBLES];

namespace {

constexpr int kMaxStaticDevices = 64;
std::mutex g_static_scratch_lock;
double *g_static_scratch_addr[kMaxStaticDevices] = {};

// Device address of g_static_scratch on `device`, which must be current.
int static_scratch_address(int device, double **out)
{
    if (device < 0 || device >= kMaxStaticDevices)
        return KPM_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_static_scratch_lock);
    if (!g_static_scratch_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return KPM_ECUDA;
        }
        g_static_scratch_addr[device] = static_cast<double *>(p);
    }
    *out = g_static_scratch_addr[device];
    return KPM_OK;
}

}  // namespace

extern "C" int kpm_aug_spmmv_static(kpm_ctx *c, int32_t R, const void *V, void *W,
                                    double *eta_dev, int32_t init, int32_t with_imag,
                                    void *stream)
{
    if (!c || R < 1 || !V || !W || V == W)
        return KPM_EINVAL;
    DeviceGuard guard(c->device);
    if (!guard.ok)
        return KPM_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    double *scratch = nullptr;
    KPM_TRY(static_scratch_address(c->device, &scratch));

    // Column blocks as in kpm_aug_spmmv (powers of two <= max_rb, widest first),
    // visited twice without any container: first to size the scratch, then
    // to launch.
    auto block_shape = [&](int RB, LaunchShape &s, int &grid) {
        auto it = c->shapes.find(RB);
        s = it != c->shapes.end() ? it->second : default_shape(c, RB);
        grid = resolve_grid(c, s);
        return grid >= 1;
    };
    int64_t need = 0;
    for (int rest = R, RB = c->max_rb; RB >= 1; RB >>= 1) {
        for (; rest >= RB; rest -= RB) {
            LaunchShape s;
            int grid = 0;
            if (!block_shape(RB, s, grid))
                return KPM_EUNSUPPORTED;
            need += (int64_t)grid * 3 * RB;
        }
    }
    if (need > KPM_STATIC_SCRATCH_DOUBLES)
        return KPM_EINVAL;

    int64_t offset = 0;
    int col0 = 0;
    for (int rest = R, RB = c->max_rb; RB >= 1; RB >>= 1) {
        for (; rest >= RB; rest -= RB) {
            ColumnBlock cb;
            cb.col0 = col0;
            cb.RB = RB;
            block_shape(RB, cb.shape, cb.grid);
            cb.partial_offset = offset;
            SweepParams p = sweep_params(c, cb, R, V, W, scratch + offset, with_imag != 0);
            KPM_TRY(launch_one(c, cb, p, init != 0, st));
            if (eta_dev) {
                c->launches++;
                reduce_single_kernel<<<(3 * RB + 127) / 128, 128, 0, st>>>(scratch + offset,
                                                                           cb.grid, RB, col0, R,
                                                                           eta_dev);
                KPM_CUDA(cudaGetLastError());
            }
            offset += (int64_t)cb.grid * 3 * RB;
            col0 += RB;
        }
    }
    return KPM_OK;
}
