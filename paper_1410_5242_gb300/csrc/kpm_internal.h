// Internal declarations shared by the translation units of libkpm.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstddef>
#include <map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kpm.h"

namespace kpm {

// Validates a CSR matrix (see kpm_gershgorin in kpm.h for the rules).
int validate_csr(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val_ri);
// The same for n rows with columns in [0, n_cols) (a part's local matrix).
int validate_csr_rect(int64_t n, int64_t n_cols, const int64_t *row_ptr, const int32_t *col,
                      const double *val_ri);
// kpm_sell_build for a part's local matrix: columns n .. n + n_halo - 1 are
// halo slots, stored as vector rows n_pad + (column - n).
int sell_build_rect(int64_t n, int64_t n_halo, const int64_t *row_ptr, const int32_t *col,
                    const double *val_ri, double a, double b, int32_t C, int32_t sigma,
                    const int32_t *row_order, kpm_sell *out);
// KPM_OK if H == H^dagger within rel_tol * max|h_ij|, else KPM_ENOTHERMITIAN.
int check_hermitian(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val_ri,
                    double rel_tol);

// Arguments of one aug_spmmv sweep over a column block of width RB = T*E
// starting at column col0 of blocks whose rows hold ld complex numbers.
struct SweepParams {
    const int64_t *chunk_ptr;  // [n_chunks + 1]
    const int32_t *chunk_len;  // [n_chunks]
    const int32_t *col;        // [n_stored]
    const void *val;           // [n_stored] complex (double2 or float2)
    const void *V;             // [n_pad][ld] complex, read only
    void *W;                   // [n_pad][ld] complex, updated in place
    double *partial;           // [grid][3][RB]: per-block <V|V>, Re<W|V>, Im<W|V>
    int64_t n_pad;
    int32_t log2C;
    int32_t ld;
    int32_t col0;
    int32_t tile_groups;       // row groups (of P rows) per warp per block tile
    int32_t with_imag;
};

// Device-side error codes a kernel records in the context's error word.
#define KPM_DEVERR_TIMEOUT 1  // a bounded wait gave up (KPM_ETIMEOUT)
#define KPM_DEVERR_RANGE 2    // an index outside its array was skipped (KPM_EINVAL)

// Per-chunk producer record of the staged kernel: 32 int2 (256 bytes),
// [0] = first entry of the chunk in the staged entry arrays (int64 as lo,
// hi), [1] = (staged chunk length, run count), [2] = index of run
// KPM_REC_INLINE_RUNS in the overflow array (int64), [3 + q] = run q (first
// row, row count) for q < KPM_REC_INLINE_RUNS.
#define KPM_REC_WORDS 32
#define KPM_REC_INLINE_RUNS 29

// One problem of a staged launch: its arrays, where its chunks sit in the
// launch's global tile sequence, and where its eta partials go (slot s,
// entry t = q*RB + r at partial[s*ps + t*qs]; slot = the first chunk of the
// problem a block handled, so slots < min(grid, n_tiles)).  The entry
// arrays are the staged ones (kpm_staged in kpm.h: per row the own entry
// last, indices in groups of 8/4/2/1, complex float values in pairs).
struct StagedProblem {
    const int2 *rec;       // [n_tiles][KPM_REC_WORDS]
    const int2 *ovf;       // runs beyond the inline ones
    const uint16_t *lidx;  // staged local indices
    const void *val;       // staged values: complex float, complex double, or
                           // the half-complex form's operand pairs
    void *buf[2];          // vector blocks: V = buf[parity], W = buf[parity ^ 1]
    double *partial;
    int64_t tile0, n_tiles;
    int64_t ps, qs;
    int32_t ld, col0;
    // extents for the bounds checks of a KPM_CHECK build: rows of each
    // vector block, staged entries, overflow runs
    int64_t rows, entries, n_ovf;
};

static_assert(sizeof(StagedProblem) % 8 == 0, "copied to shared memory in 8-byte words");

// Arguments of one staged sweep (aug_spmmv_staged.cu) over a table of
// problems (probs, n_probs entries, in device memory) or the single problem
// `one` (probs = NULL, n_probs = 1), and the shared-memory layout of one
// stage: V rows [u_max][RB] at 0, the chunk's staged values at off_val and
// staged local indices at off_lidx (l_max * C entries each).  Stages start
// at bar_bytes; the barriers, each stage's chunk length, the record ring,
// the eta sum and the problem table sit before them; after them, at
// off_aux, the block's W buffer (complex double: C rows of RB columns).
// off_w != 0 (complex float): each stage also holds the chunk's old W rows
// at off_w, copied by the producer.
struct StagedParams {
    StagedProblem one;
    const StagedProblem *probs;
    int32_t n_probs, parity;
    int32_t C, stages, with_imag, init;
    int32_t dots;  // 0: no scalar products (the ablation's reduced sweeps)
    int64_t stall_after;  // >= 0: the producer stops after this many chunks per
                          // block (test of the bounded waits); -1: never
    int *err;  // device error word (KPM_DEVERR_*)
    uint32_t bar_bytes, stage_bytes, off_val, off_lidx, off_aux, off_w;
    int32_t fp64;  // complex double (else complex float)
    int32_t half;  // every stored entry purely real or imaginary (the half-complex form)
};

// The shared-memory layout of a staged launch; false if fewer than
// min_stages stages fit in max_smem bytes.
struct StagedLayout {
    uint32_t bar_bytes, stage_bytes, off_val, off_lidx, off_aux, off_w;
    int stages;
    size_t smem;
};
// csize: bytes of one complex number of the vector blocks (8 or 16);
// vsize: bytes of one staged value (staged_value_bytes); wstage: the old W
// rows travel with each stage (complex float only).
bool staged_layout(int C, int T, int RB, int csize, int vsize, int u_max, int l_max, int stages,
                   int n_probs, bool wstage, size_t max_smem, StagedLayout &out);
bool staged_shape_supported(int T, int E, bool fp64);
// pdl: launched as a programmatic dependent of the previous kernel in the
// stream (its blocks set up while that kernel finishes).
int launch_sweep_staged(const StagedParams &p, int T, int E, int grid, size_t smem, void *stream,
                        bool pdl = false);
int staged_max_blocks_per_sm(int T, int E, int C, size_t smem, bool fp64, bool half);
// Bytes of one staged value: complex double or its operand pair (16),
// complex float (8), one float of the complex float half form (4).
inline int staged_value_bytes(bool fp64, bool half)
{
    return fp64 ? 16 : (half ? 4 : 8);
}

// stages = 0: the register-path kernel of aug_spmmv.cuh with `threads` per
// block; stages >= 1: the staged kernel of aug_spmmv_staged.cu with that
// many shared-memory stages and 32 + C*T threads per block.
struct LaunchShape {
    int T, E, threads, blocks_per_sm, tile_groups;
    int stages = 0;
    int wstage = 0;  // staged complex float: the old W rows travel with each stage
};

// Launch one sweep of the given shape; grid = blocks_per_sm * n_sm.
// Returns KPM_EUNSUPPORTED for a (T, E) pair that is not instantiated.
int launch_sweep_fp64(const SweepParams &p, const LaunchShape &s, int grid, bool init,
                      void *stream);
int launch_sweep_fp32(const SweepParams &p, const LaunchShape &s, int grid, bool init,
                      void *stream);
// The same sweep without scalar products (ablation variants).
int launch_nodot_fp64(const SweepParams &p, const LaunchShape &s, int grid, bool init, void *stream);
int launch_nodot_fp32(const SweepParams &p, const LaunchShape &s, int grid, bool init, void *stream);
// Occupancy query for the same kernels (blocks per SM, 0 if unsupported).
int sweep_max_blocks_per_sm(int precision, const LaunchShape &s, bool init);

// Makes a device current for the lifetime of the object and restores the
// previous one afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

// Kernel attributes are per function and per device (context).  These set
// one on the current device, once per kernel, device and value, and are
// safe to call from several host threads.
// The dynamic shared-memory limit of func raised to at least smem bytes.
int ensure_max_dynamic_smem(const void *func, size_t smem);
// The shared-memory carve-out preference of func set to the maximum L1.
int ensure_carveout_max_l1(const void *func);

// A named NVTX range for the lifetime of the object (the phases of a call
// in profiler timelines; no cost without a profiler attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

inline int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess)
        return KPM_OK;
    if (e == cudaErrorMemoryAllocation)
        return KPM_ENOMEM;
    return KPM_ECUDA;
}

#define KPM_TRY(expr)                 \
    do {                              \
        int rc_ = (expr);             \
        if (rc_ != KPM_OK)            \
            return rc_;               \
    } while (0)
#define KPM_CUDA(expr) KPM_TRY(cuda_status(expr))


}  // namespace kpm

// ------------------------------------------------------------ context
struct ColumnBlock {
    int col0, RB;
    kpm::LaunchShape shape;
    int grid;
    int64_t partial_offset;  // doubles from the start of a slot
};

struct kpm_ctx {
    int device = 0;
    int precision = KPM_PREC_FP64;
    int64_t n = 0, n_pad = 0, nnz = 0, n_stored = 0, n_chunks = 0;
    int32_t C = 32, log2C = 5, sigma = 1;
    double a = 0, b = 0;
    int n_sm = 1;
    size_t sdc = 16;  // bytes per complex entry of matrix and vectors

    kpm_alloc_fn alloc_fn = nullptr;
    kpm_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;

    // a part of a row-partitioned problem: halo slots after the n_pad rows
    // of each vector block; start vectors by global row
    int64_t n_halo = 0, global_n = 0, row0 = 0;
    int32_t *d_iperm = nullptr;  // [n] local row -> position (parts only)

    int64_t *d_chunk_ptr = nullptr;
    int32_t *d_chunk_len = nullptr;
    int32_t *d_col = nullptr;
    void *d_val = nullptr;
    int32_t *d_perm = nullptr;
    std::vector<int32_t> perm;  // host copy: new row -> original row

    // gather lists of the staged kernel (contexts with C >= 8)
    bool gather_ok = false;
    // every stored entry purely real or purely imaginary (complex double
    // contexts: the staged kernel's two-FMA form, with its own operand
    // array and bit 15 of d_lidx marking the imaginary entries)
    bool half_ok = false;
    void *d_val_staged = nullptr;  // staged values (kpm_staged; form by precision and half_ok)
    int64_t upload_bytes = 0;    // host -> device bytes kpm_create copied
    uint16_t *d_lidx = nullptr;  // staged local indices (kpm_staged)
    int2 *d_rec = nullptr;       // [n_chunks][KPM_REC_WORDS]
    int2 *d_ovf = nullptr;
    int64_t n_staged = 0, n_ovf = 0;  // entries of the staged arrays, overflow runs
    int32_t u_max = 0, l_max = 0;
    int overlap = KPM_OVERLAP_PDL;  // kpm_set_sweep_overlap
    int *d_err = nullptr;  // device error word, KPM_DEVERR_*
    int64_t stall_after = -1;  // kpm_test_stall_staged
    size_t max_smem = 0;   // opt-in shared memory per block

    // work buffers (grown on demand)
    void *d_V = nullptr, *d_W = nullptr;
    int64_t vw_bytes = 0;
    double *d_partial = nullptr;
    int64_t partial_doubles = 0;
    double *d_eta = nullptr, *d_eta_im = nullptr;
    void *d_aux = nullptr;  // small per-call inputs of the start-block kernels
    int64_t aux_bytes = 0;
    int64_t eta_doubles = 0;

    std::map<int, kpm::LaunchShape> shapes;  // per column-block width
    int max_rb = 64;        // widest column block (a power of two <= 64)
    int autotune = 0;       // tune the launch shape on first use of each R
    int reduce_interval = 0;  // sweeps per eta reduction launch (0 = as many as fit 64 MB)
    std::map<int, int> tuned;  // R -> already tuned
    int64_t launches = 0;  // kernels launched by this context
};


namespace kpm {
void *dev_alloc(kpm_ctx *c, size_t bytes);
void dev_free(kpm_ctx *c, void *p);
int64_t block_ld(const kpm_ctx *c, int R);
// R split into power-of-two column blocks <= cap, widest first.
std::vector<int> column_widths(int R, int cap);
int ensure_vectors(kpm_ctx *c, int R);
int ensure_partial(kpm_ctx *c, int64_t doubles);
int ensure_eta(kpm_ctx *c, int64_t doubles);
int ensure_aux(kpm_ctx *c, int64_t bytes);
int launch_phases(kpm_ctx *c, void *V, int R, uint64_t seed, cudaStream_t st);
// Random-phase block without a context: perm may be NULL (identity).
int launch_phases_raw(void *V, bool fp64, const int32_t *perm, int64_t n, int64_t n_pad, int R,
                      int ld, uint64_t seed, int n_sm, cudaStream_t st);
LaunchShape default_shape(const kpm_ctx *c, int RB);
int choose_wstage(const kpm_ctx *c, const LaunchShape &s);
}  // namespace kpm
