// Ensembles of independent KPM-DOS problems (disorder realisations of
// different sizes, moment counts M and block widths R) advanced together.
//
// Each problem's R columns are split into column blocks of power-of-two
// widths up to 64 (one block where R is such a power), and the blocks --
// the units below -- are grouped into classes of equal width.  Every sweep
// step is, per class, one launch of batch_sweep_kernel over the tiles of
// the class's units still running at that step (sorted by M, so the
// running set is always a prefix; blocks stride over the concatenated tile
// list and keep their eta terms in registers for as long as they stay in
// one unit), followed by one launch of batch_reduce_kernel that turns
// the per-block eta partials of the step into eta_{2m}, eta_{2m+1} of every
// running unit's columns.  The whole schedule (start
// vectors, the initial sweep, the M/2 - 1 sweeps of the longest problem)
// is captured once into a CUDA graph and replayed with one graph launch.
#define KPM_SWEEP_MAX_THREADS 512
#define KPM_SWEEP_MIN_BLOCKS 2
#define KPM_SWEEP_INDEX_RUN 2
#define KPM_SWEEP_PREFETCH 1
#include "aug_spmmv.cuh"

#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "kpm_internal.h"

using namespace kpm;

namespace {

constexpr int kBatchThreads = 128;  // 4 warps per block
// block tile: one row group per warp (complex float), four (complex double),
// as measured best for the single-problem sweep
constexpr int kBatchTileGroups[2] = {4, 1};  // [precision]
constexpr int kReduceThreads = 128;

// One unit: columns col0 .. col0 + RB - 1 of a problem's vector block.
struct BatchProblem {
    const int64_t *chunk_ptr;
    const int32_t *chunk_len;
    const int32_t *col;
    const void *val;
    void *buf0, *buf1;  // nu_0 lives in buf0; sweep s reads buf[s & 1], writes the other
    double *partial;    // [3 * RB][slots], the unit's own
    double *eta;        // [RB][M]: rows col0 .. of the problem's eta
    int64_t n_pad, n_tiles, tile_rows;
    int64_t slots;  // min(grid, n_tiles): blocks that touch the unit in a step
    int32_t log2C, ld, RB, shape, tile_groups, M, col0;  // ld: the problem's row stride
};

// L2 prefetch of a run's first tile (the later ones are prefetched one tile
// ahead inside the run).
template <typename Real>
__device__ __forceinline__ void prefetch_first(const BatchProblem &bp, int64_t t0, int step)
{
    SweepParams p;
    p.chunk_ptr = bp.chunk_ptr;
    p.val = bp.val;
    p.col = bp.col;
    p.V = (step & 1) ? bp.buf1 : bp.buf0;
    p.W = (step & 1) ? bp.buf0 : bp.buf1;
    p.n_pad = bp.n_pad;
    p.log2C = bp.log2C;
    p.ld = bp.ld;
    prefetch_tile<Real>(p, t0, bp.tile_rows, step != 0);
}

// Lane shape of a problem with block width RB = 2^shape: complex float
// uses 4 columns (two 16-byte accesses) per lane, complex double one.
template <typename Real, int S>
struct BatchShape {
    static constexpr int RB = 1 << S;
    static constexpr int E = sizeof(Real) == 4 ? (RB < 4 ? RB : 4) : (RB < 64 ? 1 : 2);
    static constexpr int T = RB / E;
};

template <typename Real>
int batch_team(int shape)
{
    switch (shape) {
    case 0: return BatchShape<Real, 0>::T;
    case 1: return BatchShape<Real, 1>::T;
    case 2: return BatchShape<Real, 2>::T;
    case 3: return BatchShape<Real, 3>::T;
    case 4: return BatchShape<Real, 4>::T;
    case 5: return BatchShape<Real, 5>::T;
    default: return BatchShape<Real, 6>::T;
    }
}

// One block's run of tiles within one problem: local tiles t0, t0 + G, ...
// (G = gridDim.x), accumulated in registers and written once, as the
// block's partial in slot t0 of the problem's [3*RB][slots] array.
template <typename Real, int S>
__device__ __forceinline__ void batch_run(const BatchProblem &bp, int64_t t0, int step,
                                          double *red)
{
    using Sh = BatchShape<Real, S>;
    constexpr int T = Sh::T, E = Sh::E, P = 32 / T;
    SweepParams p;
    p.chunk_ptr = bp.chunk_ptr;
    p.chunk_len = bp.chunk_len;
    p.col = bp.col;
    p.val = bp.val;
    p.V = (step & 1) ? bp.buf1 : bp.buf0;
    p.W = (step & 1) ? bp.buf0 : bp.buf1;
    p.partial = bp.partial;
    p.n_pad = bp.n_pad;
    p.log2C = bp.log2C;
    p.ld = bp.ld;
    p.col0 = bp.col0;
    p.tile_groups = bp.tile_groups;
    p.with_imag = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int tl = lane % T, team = lane / T;
    const int64_t cbase = (int64_t)p.col0 + tl * Pieces<Real, E>::EV;
    const Real *__restrict__ val = static_cast<const Real *>(p.val);
    const Real *__restrict__ V = static_cast<const Real *>(p.V);
    Real *W = static_cast<Real *>(p.W);
    EtaAcc<Real, false> acc[E];
    const int64_t rows_per_tile = (int64_t)nwarps * P * bp.tile_groups;
    for (int64_t tile = t0; tile < bp.n_tiles; tile += gridDim.x) {
        if (threadIdx.x == 0)
            prefetch_tile<Real>(p, tile + gridDim.x, rows_per_tile, step != 0);
        for (int g = 0; g < bp.tile_groups; g++) {
            const int64_t row = tile * rows_per_tile + ((int64_t)g * nwarps + warp) * P + team;
            if (row < p.n_pad)
                sweep_row<Real, T, E, false>(p, val, V, W, row, step == 0, cbase, acc);
        }
    }
    block_eta_sum<Real, T, E, false>(acc, red, bp.partial + t0, bp.slots);
}

template <typename Real>
__global__ void __launch_bounds__(KPM_SWEEP_MAX_THREADS, KPM_SWEEP_MIN_BLOCKS)
    batch_sweep_kernel(const BatchProblem *__restrict__ probs,
                       const int64_t *__restrict__ tile_prefix, int n_active, int step)
{
    extern __shared__ double red_smem[];
    const int64_t total = tile_prefix[n_active];
    int64_t gt = blockIdx.x;
    while (gt < total) {
        // the running problem owning global tile gt
        int lo = 0, hi = n_active - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile_prefix[mid] <= gt)
                lo = mid;
            else
                hi = mid - 1;
        }
        const BatchProblem bp = probs[lo];
        const int64_t t0 = gt - tile_prefix[lo];  // < gridDim.x: first tile of this block's run
        if (threadIdx.x == 0)
            prefetch_first<Real>(bp, t0, step);
        switch (bp.shape) {
        case 0: batch_run<Real, 0>(bp, t0, step, red_smem); break;
        case 1: batch_run<Real, 1>(bp, t0, step, red_smem); break;
        case 2: batch_run<Real, 2>(bp, t0, step, red_smem); break;
        case 3: batch_run<Real, 3>(bp, t0, step, red_smem); break;
        case 4: batch_run<Real, 4>(bp, t0, step, red_smem); break;
        case 5: batch_run<Real, 5>(bp, t0, step, red_smem); break;
        default: batch_run<Real, 6>(bp, t0, step, red_smem); break;
        }
        __syncthreads();  // red_smem is reused by the next run
        // next tile of this block after the run
        const int64_t run = (bp.n_tiles - t0 + gridDim.x - 1) / gridDim.x;
        gt += run * (int64_t)gridDim.x;
    }
}

// One block per (running unit, quantity q in {<V|V>, Re<W|V>}, column r):
// sums the unit's per-block partials of this step in slot order.
__global__ void batch_reduce_kernel(const BatchProblem *__restrict__ probs, int n_active, int step)
{
    __shared__ double red[kReduceThreads];
    const int k = blockIdx.x / 128;
    const int qr = blockIdx.x % 128;
    const int q = qr / 64, r = qr % 64;
    if (k >= n_active)
        return;
    const int RB = probs[k].RB;
    if (r >= RB)
        return;
    const int64_t slots = probs[k].slots;
    const double *src = probs[k].partial + (int64_t)(q * RB + r) * slots;
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < slots; t += blockDim.x)
        s += src[t];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        probs[k].eta[(int64_t)r * probs[k].M + 2 * step + q] = red[0];
}

template <typename Real>
int batch_grid(int n_sm)
{
    int nb = 0;
    const size_t smem = (size_t)(kBatchThreads / 32) * 3 * 64 * sizeof(double);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_sweep_kernel<Real>, kBatchThreads,
                                                      smem) != cudaSuccess)
        return 0;
    return nb * n_sm;
}

}  // namespace

// A class whose problems run the staged kernel (complex float with gather
// lists): its launch shape and shared-memory layout.
struct StagedClass {
    bool on = false, half = false;  // half: the half-complex float form
    int T = 0, E = 4, grid = 0;
    StagedLayout L{};
};

struct kpm_batch {
    int device = 0, precision = 0, count = 0, n_units = 0, steps = 0, grid = 0;
    std::vector<StagedClass> staged;       // per class
    StagedProblem *d_sprobs = nullptr;     // per sorted unit (staged classes)
    std::vector<kpm_ctx *> ctx;      // original order
    std::vector<int> M, R;           // original order
    std::vector<int> n_active;       // [step][class]: running units of each class
    std::vector<int> class_first;    // first sorted unit of each class (+ n_units)
    std::vector<int> class_prefix;   // offset of each class's tile prefix array
    BatchProblem *d_probs = nullptr;
    int64_t *d_prefix = nullptr;
    cudaStream_t capture = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    kpm_batch_info info{};
};

namespace {

void batch_release(kpm_batch *b)
{
    if (!b)
        return;
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    if (b->capture)
        cudaStreamDestroy(b->capture);
    if (!b->ctx.empty()) {
        dev_free(b->ctx[0], b->d_probs);
        dev_free(b->ctx[0], b->d_prefix);
        dev_free(b->ctx[0], b->d_sprobs);
    }
    delete b;
}

}  // namespace

extern "C" {

int kpm_batch_create(kpm_ctx *const *ctx, int32_t count, const int32_t *M, const int32_t *R,
                     const uint64_t *seed, kpm_batch **out)
{
    if (!out)
        return KPM_EINVAL;
    *out = nullptr;
    if (!ctx || count < 1 || !M || !R || !seed)
        return KPM_EINVAL;
    for (int32_t p = 0; p < count; p++) {
        if (!ctx[p] || M[p] < 2 || (M[p] & 1) || R[p] < 1)
            return KPM_EINVAL;
        if (ctx[p]->n_halo > 0)
            return KPM_EUNSUPPORTED;  // a part runs its sweeps with halo exchanges
        if (ctx[p]->device != ctx[0]->device || ctx[p]->precision != ctx[0]->precision)
            return KPM_EINVAL;
        for (int32_t q = 0; q < p; q++)
            if (ctx[q] == ctx[p])
                return KPM_EINVAL;  // each problem needs its own work buffers
    }
    kpm_batch *b = new (std::nothrow) kpm_batch;
    if (!b)
        return KPM_ENOMEM;
    b->device = ctx[0]->device;
    b->precision = ctx[0]->precision;
    b->count = count;
    b->ctx.assign(ctx, ctx + count);
    b->M.assign(M, M + count);
    b->R.assign(R, R + count);
    DeviceGuard guard(b->device);
    auto fail = [&](int rc) {
        batch_release(b);
        return rc;
    };
    if (!guard.ok)
        return fail(KPM_ECUDA);

    // Units: each problem's columns in power-of-two blocks of at most 64,
    // widest first, as the single-problem sweeps split them (a block's first
    // column is a multiple of its width, which keeps its accesses aligned).
    struct Unit {
        int p, col0, RB, shape;  // shape = log2(RB)
    };
    std::vector<Unit> units;
    for (int p = 0; p < count; p++) {
        int col0 = 0;
        for (int RB : column_widths(R[p], 64)) {
            int shape = 0;
            while ((1 << shape) < RB)
                shape++;
            units.push_back({p, col0, RB, shape});
            col0 += RB;
        }
    }
    const int n_units = (int)units.size();
    b->n_units = n_units;
    // Units grouped by width (one batched launch per width class and step:
    // a launch whose blocks all run the same (T, E) loop keeps the SMs
    // evenly loaded; mixing widths in one launch ran 12% slower on the
    // 64-lattice ensemble), each class by decreasing M, so that the running
    // set of a class is a prefix of it.
    std::vector<int> order(n_units);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        if (units[x].shape != units[y].shape)
            return units[x].shape < units[y].shape;
        return M[units[x].p] > M[units[y].p];
    });
    auto unit_ctx = [&](int i) { return ctx[units[order[i]].p]; };  // i: sorted unit
    const bool fp64 = b->precision == KPM_PREC_FP64;
    const int sd = fp64 ? 16 : 8;
    b->grid = fp64 ? batch_grid<double>(ctx[0]->n_sm) : batch_grid<float>(ctx[0]->n_sm);
    if (b->grid < 1)
        return fail(KPM_ECUDA);
    std::vector<BatchProblem> probs(n_units);
    std::vector<StagedProblem> sprobs(n_units);
    std::vector<int64_t> prefix;  // per class: tile prefix over its units (count_c + 1)
    double bytes = 0.0;
    for (int i = 0; i < n_units; i++)
        if (i == 0 || units[order[i]].shape != units[order[i - 1]].shape)
            b->class_first.push_back(i);
    b->class_first.push_back(n_units);
    // Complex float classes run the staged kernel when every unit's context
    // has gather lists with one chunk height and the stages fit.  The class
    // takes the lane shape and stage count its first unit's context uses for
    // the width (as tuned by kpm_autotune or kpm_set_launch, else the
    // default); a register-path choice there keeps the class on the register
    // path.
    b->staged.assign(b->class_first.size() - 1, StagedClass());
    for (size_t cl = 0; cl + 1 < b->class_first.size() && !fp64; cl++) {
        const int first = b->class_first[cl], last = b->class_first[cl + 1];
        const int RB = units[order[first]].RB;
        const kpm_ctx *c0 = unit_ctx(first);
        auto it = c0->shapes.find(RB);
        const LaunchShape sh = it != c0->shapes.end() ? it->second : default_shape(c0, RB);
        StagedClass &sc = b->staged[cl];
        sc.T = sh.T;
        sc.E = sh.E;
        bool ok = sh.stages > 0 && RB >= 8 && sh.T * sh.E == RB &&
                  staged_shape_supported(sc.T, sc.E, false);
        int u_max = 0, l_max = 0;
        for (int i = first; i < last && ok; i++) {
            const kpm_ctx *c = unit_ctx(i);
            ok = c->gather_ok && c->C == c0->C && c->half_ok == c0->half_ok;
            u_max = std::max(u_max, c->u_max);
            l_max = std::max(l_max, c->l_max);
        }
        // the class's stage count, or fewer where the wider gather lists of
        // other units (or the unit table) do not leave room; the old
        // W rows travel with the stages where that keeps the blocks per SM
        bool fits = false;
        const int vs = staged_value_bytes(false, c0->half_ok);
        for (int ns = ok ? sh.stages : 0; ns >= 1 && !fits; ns--)
            fits = staged_layout(c0->C, sc.T, RB, 8, vs, u_max, l_max, ns, last - first, false,
                                 ctx[0]->max_smem, sc.L);
        ok = ok && fits;
        if (ok) {
            int bps = staged_max_blocks_per_sm(sc.T, sc.E, c0->C, sc.L.smem, false, c0->half_ok);
            StagedLayout Lw;
            if (staged_layout(c0->C, sc.T, RB, 8, vs, u_max, l_max, sc.L.stages, last - first, true,
                              ctx[0]->max_smem, Lw)) {
                const int bw = staged_max_blocks_per_sm(sc.T, sc.E, c0->C, Lw.smem, false,
                                                        c0->half_ok);
                if (bw >= bps && bw > 0) {
                    sc.L = Lw;
                    bps = bw;
                }
            }
            sc.grid = bps * ctx[0]->n_sm;
            ok = bps > 0;
        }
        sc.on = ok;
        sc.half = ok && c0->half_ok;
    }
    // Pass 1: every unit's tiles and partial slots, and its partials'
    // offset within its context's partial buffer (the units of a problem
    // share its context's buffers: V and W at their own columns, eta at
    // their own rows, partials one after the other).
    auto class_of = [&](int i) {
        int cl = 0;
        while (b->class_first[cl + 1] <= i)
            cl++;
        return cl;
    };
    std::vector<int64_t> u_tiles(n_units), u_rows(n_units), u_slots(n_units), u_poff(n_units);
    std::vector<int64_t> p_partial(count, 0);
    for (int i = 0; i < n_units; i++) {
        const Unit &u = units[order[i]];
        const StagedClass &sc = b->staged[class_of(i)];
        const kpm_ctx *c = ctx[u.p];
        const int T = fp64 ? batch_team<double>(u.shape) : batch_team<float>(u.shape);
        const int rows_per_group = (kBatchThreads / 32) * (32 / T);
        const int tg = kBatchTileGroups[fp64 ? 0 : 1];
        u_rows[i] = sc.on ? c->C : (int64_t)rows_per_group * tg;
        u_tiles[i] = (c->n_pad + u_rows[i] - 1) / u_rows[i];
        u_slots[i] = std::min<int64_t>(sc.on ? sc.grid : b->grid, u_tiles[i]);
        u_poff[i] = p_partial[u.p];
        p_partial[u.p] += 3 * (int64_t)u.RB * u_slots[i];
    }
    for (int p = 0; p < count; p++) {
        kpm_ctx *c = ctx[p];
        int rc = ensure_vectors(c, R[p]);
        if (!rc)
            rc = ensure_partial(c, p_partial[p]);
        if (!rc)
            rc = ensure_eta(c, (int64_t)M[p] * R[p]);
        if (rc)
            return fail(rc);
        const double mat = (double)c->nnz * (sd + 4);
        bytes += mat + 2.0 * R[p] * sd * c->n + (M[p] / 2 - 1) * (mat + 3.0 * R[p] * sd * c->n);
        b->info.sweeps += M[p] / 2;
    }
    // Pass 2: the unit tables, with the buffers in place.
    for (int i = 0; i < n_units; i++) {
        const int cl = class_of(i);
        if (i == b->class_first[cl]) {
            b->class_prefix.push_back((int)prefix.size());
            prefix.push_back(0);
        }
        const StagedClass &sc = b->staged[cl];
        const Unit &u = units[order[i]];
        const int p = u.p;
        kpm_ctx *c = ctx[p];
        BatchProblem &bp = probs[i];
        bp.chunk_ptr = c->d_chunk_ptr;
        bp.chunk_len = c->d_chunk_len;
        bp.col = c->d_col;
        bp.val = c->d_val;
        bp.buf0 = c->d_V;
        bp.buf1 = c->d_W;
        bp.partial = c->d_partial + u_poff[i];
        bp.eta = c->d_eta + (int64_t)u.col0 * M[p];
        bp.n_pad = c->n_pad;
        bp.n_tiles = u_tiles[i];
        bp.tile_rows = u_rows[i];
        bp.slots = u_slots[i];
        bp.log2C = c->log2C;
        bp.ld = (int32_t)block_ld(c, R[p]);
        bp.RB = u.RB;
        bp.shape = u.shape;
        bp.tile_groups = kBatchTileGroups[fp64 ? 0 : 1];
        bp.M = M[p];
        bp.col0 = u.col0;
        if (sc.on) {
            StagedProblem &sp = sprobs[i];
            sp.rec = c->d_rec;
            sp.ovf = c->d_ovf;
            sp.lidx = c->d_lidx;
            sp.val = c->d_val_staged;
            sp.buf[0] = c->d_V;
            sp.buf[1] = c->d_W;
            sp.partial = bp.partial;  // [3*RB][slots]
            sp.tile0 = prefix.back();
            sp.n_tiles = u_tiles[i];
            sp.ps = 1;
            sp.qs = u_slots[i];
            sp.ld = bp.ld;
            sp.col0 = u.col0;
            sp.rows = c->n_pad + c->n_halo;
            sp.entries = c->n_staged;
            sp.n_ovf = c->n_ovf;
        }
        prefix.push_back(prefix.back() + u_tiles[i]);
    }
    b->steps = 0;
    for (int p = 0; p < count; p++)
        b->steps = std::max(b->steps, M[p] / 2);
    const int n_classes = (int)b->class_first.size() - 1;
    b->n_active.assign((size_t)b->steps * n_classes, 0);
    for (int cl = 0; cl < n_classes; cl++)
        for (int s = 0; s < b->steps; s++) {
            int k = b->class_first[cl];
            while (k < b->class_first[cl + 1] && M[units[order[k]].p] / 2 > s)
                k++;
            b->n_active[(size_t)s * n_classes + cl] = k - b->class_first[cl];
        }

    b->d_probs = (BatchProblem *)dev_alloc(ctx[0], sizeof(BatchProblem) * n_units);
    b->d_prefix = (int64_t *)dev_alloc(ctx[0], sizeof(int64_t) * prefix.size());
    if (!b->d_probs || !b->d_prefix)
        return fail(KPM_ENOMEM);
    if (cudaMemcpy(b->d_probs, probs.data(), sizeof(BatchProblem) * n_units,
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_prefix, prefix.data(), sizeof(int64_t) * prefix.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(KPM_ECUDA);
    bool any_staged = false;
    for (const StagedClass &sc : b->staged)
        any_staged = any_staged || sc.on;
    if (any_staged) {
        b->d_sprobs = (StagedProblem *)dev_alloc(ctx[0], sizeof(StagedProblem) * n_units);
        if (!b->d_sprobs)
            return fail(KPM_ENOMEM);
        if (cudaMemcpy(b->d_sprobs, sprobs.data(), sizeof(StagedProblem) * n_units,
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(KPM_ECUDA);
    }

    // ---- capture the schedule
    NvtxRange range("kpm_batch_create: capture");
    if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess)
        return fail(KPM_ECUDA);
    if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(KPM_ECUDA);
    int rc = KPM_OK;
    int64_t launches = 0;
    for (int p = 0; p < count && rc == KPM_OK; p++) {
        rc = launch_phases(ctx[p], ctx[p]->d_V, R[p], seed[p], b->capture);
        launches++;
    }
    const size_t smem = (size_t)(kBatchThreads / 32) * 3 * 64 * sizeof(double);
    // The classes of a step run one after the other (as concurrent graph
    // branches they ran 3% slower on the 64-lattice ensemble).
    for (int s = 0; s < b->steps && rc == KPM_OK; s++) {
        for (int cl = 0; cl < n_classes && rc == KPM_OK; cl++) {
            const int na = b->n_active[(size_t)s * n_classes + cl];
            if (na == 0)
                continue;
            const BatchProblem *cp = b->d_probs + b->class_first[cl];
            const int64_t *cpre = b->d_prefix + b->class_prefix[cl];
            const StagedClass &sc = b->staged[cl];
            if (sc.on) {
                // the running units are a prefix of the class: a table of na
                StagedParams q{};
                q.probs = b->d_sprobs + b->class_first[cl];
                q.n_probs = na;
                q.parity = s & 1;
                q.C = unit_ctx(b->class_first[cl])->C;
                q.stages = sc.L.stages;
                q.with_imag = 0;
                q.init = s == 0 ? 1 : 0;
                q.half = sc.half ? 1 : 0;
                q.dots = 1;
                q.stall_after = ctx[0]->stall_after;
                q.err = ctx[0]->d_err;
                q.bar_bytes = sc.L.bar_bytes;
                q.stage_bytes = sc.L.stage_bytes;
                q.off_val = sc.L.off_val;
                q.off_lidx = sc.L.off_lidx;
                q.off_aux = sc.L.off_aux;
                q.off_w = sc.L.off_w;
                // a programmatic dependent of the step's previous kernel:
                // its blocks set up while that kernel finishes
                rc = launch_sweep_staged(q, sc.T, sc.E, sc.grid, sc.L.smem, b->capture, true);
                if (rc != KPM_OK)
                    break;
            } else if (fp64)
                batch_sweep_kernel<double><<<b->grid, kBatchThreads, smem, b->capture>>>(
                    cp, cpre, na, s);
            else
                batch_sweep_kernel<float><<<b->grid, kBatchThreads, smem, b->capture>>>(
                    cp, cpre, na, s);
            batch_reduce_kernel<<<na * 128, kReduceThreads, 0, b->capture>>>(cp, na, s);
            launches += 2;
            rc = cuda_status(cudaGetLastError());
        }
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->capture, &graph);
    b->graph = graph;
    if (rc != KPM_OK)
        return fail(rc);
    if (ec != cudaSuccess || !graph)
        return fail(KPM_ECUDA);
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
        return fail(KPM_ECUDA);
    b->info.count = count;
    b->info.steps = b->steps;
    b->info.kernel_launches = launches;
    b->info.algorithmic_bytes = bytes;
    b->info.grid = b->grid;
    b->info.classes = (int16_t)b->staged.size();
    b->info.staged_classes = 0;
    for (const StagedClass &sc : b->staged)
        b->info.staged_classes += sc.on ? 1 : 0;
    *out = b;
    return KPM_OK;
}

int kpm_batch_launch(kpm_batch *b, void *stream)
{
    NvtxRange range("kpm_batch_launch");
    if (!b || !b->exec)
        return KPM_EINVAL;
    DeviceGuard guard(b->device);
    // the staged launches record bounded-wait expiries in the first
    // context's error word; kpm_batch_eta reports them
    KPM_CUDA(cudaMemsetAsync(b->ctx[0]->d_err, 0, sizeof(int), (cudaStream_t)stream));
    return cuda_status(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
}

int kpm_batch_eta(kpm_batch *b, int32_t p, double *eta, void *stream)
{
    if (!b || p < 0 || p >= b->count || !eta)
        return KPM_EINVAL;
    DeviceGuard guard(b->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = (int64_t)b->M[p] * b->R[p];
    KPM_CUDA(cudaMemcpyAsync(eta, b->ctx[p]->d_eta, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    int word = 0;
    KPM_CUDA(cudaMemcpyAsync(&word, b->ctx[0]->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    KPM_CUDA(cudaStreamSynchronize(st));
    return word ? KPM_ETIMEOUT : KPM_OK;
}

int kpm_batch_get_info(const kpm_batch *b, kpm_batch_info *out)
{
    if (!b || !out)
        return KPM_EINVAL;
    *out = b->info;
    return KPM_OK;
}

void kpm_batch_destroy(kpm_batch *b)
{
    if (!b)
        return;
    DeviceGuard guard(b->device);
    cudaDeviceSynchronize();
    batch_release(b);
}

int kpm_moments_batch(kpm_ctx *const *ctx, int32_t count, const int32_t *M, const int32_t *R,
                      const uint64_t *seed, double *const *eta, void *stream)
{
    if (!eta)
        return KPM_EINVAL;
    for (int32_t p = 0; p < count; p++)
        if (!eta[p])
            return KPM_EINVAL;
    kpm_batch *b = nullptr;
    int rc = kpm_batch_create(ctx, count, M, R, seed, &b);
    if (rc)
        return rc;
    rc = kpm_batch_launch(b, stream);
    for (int32_t p = 0; p < count && rc == KPM_OK; p++)
        rc = kpm_batch_eta(b, p, eta[p], stream);
    kpm_batch_destroy(b);
    return rc;
}

}  // extern "C"
