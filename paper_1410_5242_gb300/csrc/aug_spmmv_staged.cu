// The aug_spmmv sweep of Fig. 5 with the gathered V rows staged in shared
// memory by the bulk-copy (TMA) engine, for complex float and complex double
// storage.
//
// Why: in the register-path kernel every entry's gather of R complex values
// is a load into registers, so the bytes a streaming multiprocessor can
// have in flight are capped by its register file, and each V row is read
// from L2 once per entry that uses it (13 times at 13 entries per row).
// Here one producer warp per block copies, per SELL chunk, the matrix
// values, the 16-bit local column indices and every V row the chunk reads
// -- once, however many of its entries read it (the chunk's gather list,
// kpm_gather_build) -- into a ring of shared-memory stages with
// cp.async.bulk, which completes on an mbarrier and occupies no registers.
// The consumer warps compute the chunk's rows from shared memory; each
// reads its row's old W from global memory (requested in L2 by the
// producer) while the entry loop runs.
//
// Per stage s: full[s] (the producer's arrive + the copies' byte count)
// and empty[s] (one arrive per consumer warp once it has read the stage).
// A chunk is one tile; blocks stride over chunks, so all blocks sweep the
// matrix together and the V rows one chunk gathers are recent in L2.
//
// One launch may cover several independent problems (an ensemble: one
// batched launch per step, kpm_batch.cu): their chunks form one global tile
// sequence, a table in shared memory gives each problem's arrays, and the
// consumer warps flush their eta sums to a problem's partial slot when the
// tile sequence moves on to the next problem.  A single problem is a table
// of one.
//
// Lane/column ownership is that of aug_spmmv.cuh.  Complex float: the
// products are accumulated with paired FMAs (real and imaginary parts of h
// times a column in two packed sums), so W agrees with the register path to
// single-precision rounding, and eta (packed 8-row partials folded into
// TwoSum pairs, StagedEta) is reproducible run to run.  Complex double: four
// FMAs per entry and column, or two in the half-complex form (every stored
// entry purely real or purely imaginary: the host stores operand pairs and
// marks imaginary entries in bit 15 of the local index), the FP64 pipe
// being this form's bound on GB300; eta in plain FMA chains (StagedEta64).
//
// Every wait is bounded (about two seconds of SM clock): on expiry the
// thread records KPM_DEVERR_TIMEOUT in *err, raises the block's abort flag
// (which every other wait polls), and the block stops; before exiting the
// producer waits (bounded again) for the copies it issued.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "aug_spmmv.cuh"
#include "kpm_internal.h"

namespace kpm {
namespace {

constexpr long long kWaitLimitCycles = 4LL << 30;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Global -> shared bulk copy completing on mbarrier bar.  dst, src and
// bytes are multiples of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Wait for the phase of parity `parity` of bar to complete.  Gives up when
// the block's abort flag is raised (returns false) or after
// kWaitLimitCycles (records the timeout, raises the flag, returns false).
// honour_abort = false waits for the copies themselves even after an abort.
__device__ __forceinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity,
                                            volatile int *abort_flag, int *err, bool honour_abort)
{
    const long long t0 = clock64();
    for (uint32_t it = 1;; it++) {
        if (mbar_try_wait(bar, parity))
            return true;
        if ((it & 31) == 0) {
            if (honour_abort && *abort_flag)
                return false;
            if (clock64() - t0 > kWaitLimitCycles) {
                *abort_flag = 1;
                if (err)
                    atomicExch(err, KPM_DEVERR_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  volatile int *abort_flag, int *err,
                                                  bool honour_abort)
{
    if (mbar_try_wait(bar, parity))
        return true;
    return mbar_wait_slow(bar, parity, abort_flag, err, honour_abort);
}

// The producer's record ring: the 256-byte records of the next kMetaDepth
// tiles are fetched with cp.async (8 bytes per lane) into shared memory, so
// the per-tile metadata never waits on a memory round trip.
constexpr int kMetaDepth = 8;
constexpr uint32_t kMetaOffset = 256;  // per stage: chunk length, problem, chunk number
constexpr uint32_t kRingOffset = kMetaOffset + 8 * 16;
constexpr uint32_t kRedOffset = kRingOffset + kMetaDepth * KPM_REC_WORDS * 8;
constexpr uint32_t kTableOffset = kRedOffset + 3 * 64 * 8;  // eta sum of up to 64 columns

__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copies rows [row0, row0 + nrows) of a vector block (rows of ld complex
// numbers of csize bytes; columns col0 .. col0 + RB - 1) to consecutive
// RB-wide rows at dst: one copy when the block's rows are exactly RB wide,
// else one per row.
__device__ __forceinline__ void copy_rows(uint32_t dst, const char *block, int64_t row0, int nrows,
                                          int ld, int col0, uint32_t row_bytes, uint32_t bar,
                                          int csize)
{
    const int64_t ld_bytes = (int64_t)ld * csize;
    const char *src = block + row0 * ld_bytes + (int64_t)col0 * csize;
    if (ld_bytes == (int64_t)row_bytes) {
        bulk_g2s(dst, src, (uint32_t)nrows * row_bytes, bar);
    } else {
        for (int i = 0; i < nrows; i++)
            bulk_g2s(dst + (uint32_t)i * row_bytes, src + i * ld_bytes, row_bytes, bar);
    }
}

// Two floats in one 64-bit register pair, and the paired FMA of sm_100+
// (d.lo = a.lo * b.lo + c.lo, d.hi = a.hi * b.hi + c.hi, each rounded once).
__device__ __forceinline__ uint64_t pack2(float lo, float hi)
{
    uint64_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}

__device__ __forceinline__ void unpack2(uint64_t v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// One 16-byte piece (one complex double) from shared memory.
__device__ __forceinline__ void lds_piece(const double *src, double (&out)[2])
{
    const double2 t = *reinterpret_cast<const double2 *>(src);
    out[0] = t.x;
    out[1] = t.y;
}

// ------------------------------------------------------------------ eta
// Complex float eta.  Each row adds, per column, |v|^2 and Re(conj(w) v)
// (IMAG: also Im(conj(w) v)) to single-precision pending sums, one FMA
// chain per value.  Every kEtaFold rows (one row per chunk) fold() sums the
// pending values of the warp's P = 32/T rows (teams of equal lane-in-team)
// by an xor butterfly and adds each sum, error-free, to a float-float
// (TwoSum, Knuth) running pair held by one team: value i = q*E + k goes to
// team i % P, slot i / P.  A single-precision partial thus never holds more
// than kEtaFold rows of one lane plus the additions across the warp's rows,
// and nothing here uses the FP64 pipe, which on this GPU runs at 1/64 of
// the FP32 rate.
constexpr int kEtaFold = 8;

__device__ __forceinline__ void two_sum_pair(float &hi, float &lo, float p)
{
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float ap = __fsub_rn(s, bp);
    const float e = __fadd_rn(__fsub_rn(hi, ap), __fsub_rn(p, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

template <bool IMAG, int T, int E>
struct WarpEta {
    static constexpr int NQ = IMAG ? 3 : 2, P = 32 / T, NV = NQ * E, KH = (NV + P - 1) / P;
    float pend[NV];
    float hi[KH], lo[KH];
    __device__ __forceinline__ void clear()
    {
#pragma unroll
        for (int i = 0; i < NV; i++)
            pend[i] = 0.f;
#pragma unroll
        for (int i = 0; i < KH; i++)
            hi[i] = lo[i] = 0.f;
    }
    __device__ __forceinline__ void add(int k, float wr, float wi, float vr, float vi)
    {
        pend[k] = __fmaf_rn(vr, vr, pend[k]);
        pend[k] = __fmaf_rn(vi, vi, pend[k]);
        pend[E + k] = __fmaf_rn(wr, vr, pend[E + k]);
        pend[E + k] = __fmaf_rn(wi, vi, pend[E + k]);
        if constexpr (IMAG) {
            pend[2 * E + k] = __fmaf_rn(wr, vi, pend[2 * E + k]);
            pend[2 * E + k] = __fmaf_rn(-wi, vr, pend[2 * E + k]);
        }
    }
    // E = 4: the pending terms of columns k and k ^ 2 (the lane's two
    // pieces) exchanged where sw is set
    __device__ __forceinline__ void swap_pieces(int sw)
    {
#pragma unroll
        for (int q = 0; q < NQ; q++)
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const float a = pend[q * E + k], b = pend[q * E + k + 2];
                pend[q * E + k] = sw ? b : a;
                pend[q * E + k + 2] = sw ? a : b;
            }
    }
    // all lanes of the warp take part
    __device__ __forceinline__ void fold(int team)
    {
#pragma unroll
        for (int off = T; off < 32; off <<= 1)
#pragma unroll
            for (int i = 0; i < NV; i++)
                pend[i] = __fadd_rn(pend[i], __shfl_xor_sync(0xffffffffu, pend[i], off));
#pragma unroll
        for (int i = 0; i < NV; i++) {
            if (team == i % P)
                two_sum_pair(hi[i / P], lo[i / P], pend[i]);
            pend[i] = 0.f;
        }
    }
    // after fold(): this lane's running sums added to red (double [3][RB],
    // column c of quantity q at q*RB + c), or written if first; then cleared
    __device__ __forceinline__ void add_to(double *red, int tl, int team, bool first)
    {
#pragma unroll
        for (int i = 0; i < NV; i++) {
            if (team == i % P) {
                double &d = red[(i / E) * (T * E) + owned_column<float, T, E>(tl, i % E)];
                const double v = (double)hi[i / P] + (double)lo[i / P];
                d = first ? v : d + v;
            }
        }
#pragma unroll
        for (int i = 0; i < KH; i++)
            hi[i] = lo[i] = 0.f;
    }
};

// A lane's eta terms for one column in complex double: plain FMA chains
// (aug_spmmv.cuh's EtaAcc).
template <bool IMAG>
struct StagedEta64 {
    EtaAcc<double, IMAG> a;
    __device__ __forceinline__ void add(double wr, double wi, double vr, double vi)
    {
        a.add(wr, wi, vr, vi);
    }
    __device__ __forceinline__ double get(int k) const { return a.get(k); }
};

// Inclusive prefix sum over the warp's lanes.
__device__ __forceinline__ int warp_incl_scan(int v, int lane)
{
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off)
            v += t;
    }
    return v;
}

// The problem table in shared memory and the problem owning a global tile
// (cursor moves forward only: a block's tiles increase).
__device__ __forceinline__ int advance_problem(const StagedProblem *tab, int n_probs, int pi,
                                               int64_t gt)
{
    while (pi + 1 < n_probs && gt >= tab[pi].tile0 + tab[pi].n_tiles)
        pi++;
    return pi;
}

// Programmatic dependent launch: a launch that may start while the kernel
// before it in the stream still runs lets its blocks set up (barriers,
// problem table, the first records: data no kernel writes) and then waits
// here, before its first access to the vector blocks or the eta partials,
// until that kernel has completed and its writes are visible.  Without
// such a predecessor the wait returns at once.
__device__ __forceinline__ void grid_dependency_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Lets the next launch in the stream (if it was launched as a programmatic
// dependent) schedule its blocks as this grid's blocks retire.
__device__ __forceinline__ void allow_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The producer warp: for each tile of this block, wait until its stage is
// free, announce the bytes on full[s], and issue the copies.  Lane l holds
// word l of the tile's record, i.e. inline run l - 3; runs past the inline
// ones are read from the overflow array 32 at a time.  Returns the number
// of tiles armed.
template <int RB, int CSIZE, int VSIZE>
__device__ __forceinline__ int64_t produce(const StagedParams &p, unsigned char *smem,
                                           const StagedProblem *tab, int64_t total,
                                           volatile int *abort_flag)
{
    constexpr uint32_t row_bytes = RB * CSIZE;
    const int lane = threadIdx.x & 31;
    const int NS = p.stages;
    const uint32_t full0 = smem_u32(smem), empty0 = full0 + 8 * NS;
    const uint32_t ring0 = smem_u32(smem + kRingOffset);
    const int2 *ring = reinterpret_cast<const int2 *>(smem + kRingOffset);
    const uint32_t stage0 = smem_u32(smem + p.bar_bytes);
    const int64_t G = gridDim.x;
    const int par = p.parity;

    // the record stream runs kMetaDepth tiles ahead of the issue stream; the
    // fields of the problem each stream is in are kept in registers
    int pj = -1;
    int64_t j_end = -1, j_tile0 = 0;
    const int2 *j_rec = nullptr;
    auto fetch_record = [&](int64_t t, uint32_t slot) {
        if (t < total) {
            if (t >= j_end) {
                pj = advance_problem(tab, p.n_probs, pj < 0 ? 0 : pj, t);
                j_rec = tab[pj].rec;
                j_tile0 = tab[pj].tile0;
                j_end = j_tile0 + tab[pj].n_tiles;
            }
            cp_async8(ring0 + (slot * KPM_REC_WORDS + lane) * 8,
                      j_rec + (t - j_tile0) * KPM_REC_WORDS + lane);
        }
        cp_async_commit();
    };
    for (int i = 0; i < kMetaDepth; i++)
        fetch_record(blockIdx.x + i * G, (uint32_t)i);
    grid_dependency_wait();
    int pi = -1;
    int64_t i_end = -1, i_tile0 = 0;
    const char *Vb = nullptr, *Wb = nullptr, *valb = nullptr, *lidxb = nullptr;
    const int2 *ovfp = nullptr;
    int ld = 0, col0 = 0;
    int64_t k = 0;
    int s = 0;          // stage of tile k
    uint32_t ph = 0;    // parity of that stage's current use
    for (int64_t gt = blockIdx.x; gt < total; gt += G, k++) {
        if (p.stall_after >= 0 && k >= p.stall_after)
            break;  // test hook: leave the remaining stages unarmed
        const int slot = (int)(k % kMetaDepth);
        cp_async_wait<kMetaDepth - 1>();
        __syncwarp();
        const int2 word = ring[slot * KPM_REC_WORDS + lane];
        __syncwarp();
        fetch_record(gt + kMetaDepth * G, (uint32_t)slot);
        if (gt >= i_end) {
            pi = advance_problem(tab, p.n_probs, pi < 0 ? 0 : pi, gt);
            const StagedProblem &P = tab[pi];
            i_tile0 = P.tile0;
            i_end = i_tile0 + P.n_tiles;
            Vb = static_cast<const char *>(P.buf[par]);
            Wb = static_cast<const char *>(P.buf[par ^ 1]);
            valb = static_cast<const char *>(P.val);
            lidxb = reinterpret_cast<const char *>(P.lidx);
            ovfp = P.ovf;
            ld = P.ld;
            col0 = P.col0;
        }
        const int64_t lt = gt - i_tile0;  // chunk within the problem

        auto word64 = [&](int w) {
            return (int64_t)(uint32_t)__shfl_sync(0xffffffffu, word.x, w) |
                   ((int64_t)__shfl_sync(0xffffffffu, word.y, w) << 32);
        };
        const int64_t e0 = word64(0), ovf0 = word64(2);
        const int lenw = __shfl_sync(0xffffffffu, word.x, 1);
        const int len = lenw & 0xffff, nre = lenw >> 16;
        const int nruns = __shfl_sync(0xffffffffu, word.y, 1);
        const int n_inline = min(nruns, KPM_REC_INLINE_RUNS);
        const bool has_run = lane >= 3 && lane - 3 < n_inline;
#ifdef KPM_CHECK
        // checked build: the chunk's record must keep every copy inside the
        // arrays it reads and the stage areas it fills; else the launch stops
        // with KPM_DEVERR_RANGE before any copy
        const StagedProblem &PC = tab[pi];
        bool bad = len < 1 || nre < 0 || nre > len || nruns < 1 ||
                   (uint64_t)p.C * len * VSIZE > p.off_lidx - p.off_val ||
                   (uint64_t)p.C * len * 2 > (p.off_w ? p.off_w : p.stage_bytes) - p.off_lidx ||
                   e0 < 0 || e0 + (int64_t)p.C * len > PC.entries ||
                   (nruns > KPM_REC_INLINE_RUNS &&
                    (ovf0 < 0 || ovf0 + (nruns - KPM_REC_INLINE_RUNS) > PC.n_ovf)) ||
                   (lt + 1) * p.C > PC.rows;
        if (has_run && (word.x < 0 || word.y < 0 || (int64_t)word.x + word.y > PC.rows))
            bad = true;
        if (__any_sync(0xffffffffu, bad)) {
            if (lane == 0 && p.err) {
                atomicExch(p.err, KPM_DEVERR_RANGE);
                *abort_flag = 1;
            }
            break;
        }
#endif
        const int count = has_run ? word.y : 0;
        const int incl = warp_incl_scan(count, lane);
        uint32_t total_rows = (uint32_t)__shfl_sync(0xffffffffu, incl, 31);
        for (int g = KPM_REC_INLINE_RUNS; g < nruns; g += 32) {
            const int2 r = g + lane < nruns
                               ? __ldg(ovfp + ovf0 + (g - KPM_REC_INLINE_RUNS) + lane)
                               : make_int2(0, 0);
#ifdef KPM_CHECK
            if (r.x < 0 || r.y < 0 || (int64_t)r.x + r.y > PC.rows)
                bad = true;
#endif
            total_rows += (uint32_t)__shfl_sync(0xffffffffu, warp_incl_scan(r.y, lane), 31);
        }
#ifdef KPM_CHECK
        if (__any_sync(0xffffffffu, bad || total_rows < (uint32_t)p.C ||
                                        total_rows > p.off_val / row_bytes)) {
            if (lane == 0 && p.err) {
                atomicExch(p.err, KPM_DEVERR_RANGE);
                *abort_flag = 1;
            }
            break;
        }
#endif

        const uint32_t full = full0 + 8 * s, empty = empty0 + 8 * s;
        if (k >= NS) {
            // every lane waits (and acquires); the warp leaves together
            const bool ok = mbar_wait_bounded(empty, ph ^ 1u, abort_flag, p.err, true);
            if (!__all_sync(0xffffffffu, ok))
                break;
        }
        const uint32_t st = stage0 + (uint32_t)s * p.stage_bytes;
        const uint32_t val_bytes = (uint32_t)p.C * (uint32_t)len * (uint32_t)VSIZE;
        const uint32_t lidx_bytes = (uint32_t)p.C * (uint32_t)len * 2u;
        // the chunk's old W rows with the stage (complex float, off_w set)
        const bool w_in_stage = p.off_w != 0 && !p.init;
        const uint32_t bytes = total_rows * row_bytes + val_bytes + lidx_bytes +
                               (w_in_stage ? (uint32_t)p.C * row_bytes : 0u);
        if (lane == 0) {
            volatile int *meta = reinterpret_cast<volatile int *>(smem + kMetaOffset + 16 * s);
            meta[0] = len;
            meta[1] = nre;
#ifdef KPM_CHECK
            meta[2] = (int)total_rows;
#endif
            mbar_arrive_expect_tx(full, bytes);
        }
        __syncwarp();
        if (len > 0) {
            if (lane == 0)
                bulk_g2s(st + p.off_val, valb + e0 * VSIZE, val_bytes, full);
            if (lane == 1)
                bulk_g2s(st + p.off_lidx, lidxb + e0 * 2, lidx_bytes, full);
        }
        if (w_in_stage) {
            if (lane == 2)
                copy_rows(st + p.off_w, Wb, lt * (int64_t)p.C, p.C, ld, col0, row_bytes, full, CSIZE);
        } else if (!p.init && lane == 2 && ((int64_t)ld * CSIZE & 15) == 0) {
            // the consumers read the chunk's old W rows themselves; ask L2
            // for them now (whole rows: contiguous, 16-byte multiples)
            prefetch_l2(Wb + lt * (int64_t)p.C * ld * CSIZE, (uint64_t)p.C * ld * CSIZE);
        }
        if (has_run && count > 0)
            copy_rows(st + (uint32_t)(incl - count) * row_bytes, Vb, word.x, count, ld, col0,
                      row_bytes, full, CSIZE);
        uint32_t base = (uint32_t)__shfl_sync(0xffffffffu, incl, 31);
        for (int g = KPM_REC_INLINE_RUNS; g < nruns; g += 32) {
            const int2 r = g + lane < nruns
                               ? __ldg(ovfp + ovf0 + (g - KPM_REC_INLINE_RUNS) + lane)
                               : make_int2(0, 0);
            const int ri = warp_incl_scan(r.y, lane);
            if (r.y > 0)
                copy_rows(st + (base + (uint32_t)(ri - r.y)) * row_bytes, Vb, r.x, r.y, ld, col0,
                          row_bytes, full, CSIZE);
            base += (uint32_t)__shfl_sync(0xffffffffu, ri, 31);
        }
        if (++s == NS) {
            s = 0;
            ph ^= 1u;
        }
    }
    cp_async_wait<0>();
    return k;
}

__device__ __forceinline__ void consumer_bar(int n_cw)
{
    asm volatile("bar.sync 1, %0;" ::"r"(n_cw * 32) : "memory");
}

// Complex float: one problem's eta sums, warp after warp into red (3*RB
// doubles) from each warp's running pairs, then red to the problem's
// partial slot.  The caller has folded its pending terms.
template <int T, int E, bool IMAG>
__device__ __forceinline__ void flush_eta32(WarpEta<IMAG, T, E> &pe, double *red,
                                            const StagedProblem &P, int64_t slot, int cw, int n_cw)
{
    constexpr int RB = T * E;
    const int lane = threadIdx.x & 31;
    const int tl = lane % T, team = lane / T;
    for (int w = 0; w < n_cw; w++) {
        if (cw == w)
            pe.add_to(red, tl, team, w == 0);
        consumer_bar(n_cw);
    }
    for (int t = cw * 32 + lane; t < 3 * RB; t += n_cw * 32)
        P.partial[slot * P.ps + t * P.qs] = (!IMAG && t >= 2 * RB) ? 0.0 : red[t];
    consumer_bar(n_cw);
}

// Complex double: the consumer warps' eta sums for one problem, in a fixed
// order: lanes of equal columns by an xor butterfly, then warp after warp
// into red (3*RB doubles), then red to the problem's partial slot.  Resets
// acc.
template <int T, int E, typename Acc>
__device__ __forceinline__ void flush_eta64(Acc (&acc)[E], double *red, const StagedProblem &P,
                                            int64_t slot, int cw, int n_cw)
{
    constexpr int RB = T * E;
    const int lane = threadIdx.x & 31;
    const int tl = lane % T, team = lane / T;
    double out[3 * E];
#pragma unroll
    for (int k = 0; k < E; k++)
#pragma unroll
        for (int q = 0; q < 3; q++)
            out[q * E + k] = acc[k].get(q);
#pragma unroll
    for (int off = T; off < 32; off <<= 1)
#pragma unroll
        for (int i = 0; i < 3 * E; i++)
            out[i] += __shfl_xor_sync(0xffffffffu, out[i], off);
    for (int w = 0; w < n_cw; w++) {
        if (cw == w && team == 0) {
#pragma unroll
            for (int q = 0; q < 3; q++)
#pragma unroll
                for (int k = 0; k < E; k++) {
                    double &d = red[q * RB + owned_column<double, T, E>(tl, k)];
                    d = w == 0 ? out[q * E + k] : d + out[q * E + k];
                }
        }
        consumer_bar(n_cw);
    }
    for (int t = cw * 32 + lane; t < 3 * RB; t += n_cw * 32)
        P.partial[slot * P.ps + t * P.qs] = red[t];
    consumer_bar(n_cw);
#pragma unroll
    for (int k = 0; k < E; k++)
        acc[k] = Acc();
}

// Up to 32 + C*T = 544 threads (C = 32, T = 16).  A launch bound of 576
// threads caps four columns per lane (E = 4) at 96 registers: 18 warps of
// that size fit the register file of an SM's four sub-partitions (two
// 288-thread blocks at width 32, or one 544-thread block at width 64); two
// columns per lane get 56 (two 544-thread blocks).  Complex double keeps
// one block per SM: its stages are twice as large.
#define KPM_STAGED_MAX_THREADS 576

template <typename Real, int E>
struct StagedMinBlocks {
    static constexpr int value = (E >= 4 || sizeof(Real) == 8) ? 1 : 2;
};

// Visits the index groups of a row's first nm entries in a stage (layout of
// kpm_staged in kpm.h: groups of 8, then of 4, 2 and 1 entries; one load per
// group): pair(j, u_j, u_{j+1}) for the entries of the groups of two or
// more, in pairs starting at even j, and single(j, u_j) for a group of one.
template <typename F2, typename F1>
__device__ __forceinline__ void walk_index_groups(const uint16_t *lid, int C, int rit, int nm,
                                                  F2 &&pair, F1 &&single)
{
    int j = 0;
    for (; j + 8 <= nm; j += 8) {
        const uint4 g = *reinterpret_cast<const uint4 *>(lid + C * j + 8 * rit);
        pair(j, g.x & 0xffffu, g.x >> 16);
        pair(j + 2, g.y & 0xffffu, g.y >> 16);
        pair(j + 4, g.z & 0xffffu, g.z >> 16);
        pair(j + 6, g.w & 0xffffu, g.w >> 16);
    }
    if (nm - j >= 4) {
        const uint2 g = *reinterpret_cast<const uint2 *>(lid + C * j + 4 * rit);
        pair(j, g.x & 0xffffu, g.x >> 16);
        pair(j + 2, g.y & 0xffffu, g.y >> 16);
        j += 4;
    }
    if (nm - j >= 2) {
        const uint32_t g = *reinterpret_cast<const uint32_t *>(lid + C * j + 2 * rit);
        pair(j, g & 0xffffu, g >> 16);
        j += 2;
    }
    if (nm - j >= 1)
        single(j, (uint32_t)lid[C * j + rit]);
}

// Visits entries [j0, j0 + n) of a row whose indices and one-float values
// share the grouped layout of a region (groups of 8, 4, 2, 1 entries; one
// load per group for the indices and one or two for the values):
// f(u_j, s_j) for each entry in order.
template <typename F>
__device__ __forceinline__ void walk_region(const uint16_t *lid, const float *hv, int C, int rit,
                                            int j0, int n, F &&f)
{
    const uint16_t *L = lid + C * j0;
    const float *H = hv + C * j0;
    int j = 0;
    for (; j + 8 <= n; j += 8) {
        const uint4 g = *reinterpret_cast<const uint4 *>(L + C * j + 8 * rit);
        const float4 h0 = *reinterpret_cast<const float4 *>(H + C * j + 8 * rit);
        const float4 h1 = *reinterpret_cast<const float4 *>(H + C * j + 8 * rit + 4);
        f(g.x & 0xffffu, h0.x);
        f(g.x >> 16, h0.y);
        f(g.y & 0xffffu, h0.z);
        f(g.y >> 16, h0.w);
        f(g.z & 0xffffu, h1.x);
        f(g.z >> 16, h1.y);
        f(g.w & 0xffffu, h1.z);
        f(g.w >> 16, h1.w);
    }
    if (n - j >= 4) {
        const uint2 g = *reinterpret_cast<const uint2 *>(L + C * j + 4 * rit);
        const float4 h = *reinterpret_cast<const float4 *>(H + C * j + 4 * rit);
        f(g.x & 0xffffu, h.x);
        f(g.x >> 16, h.y);
        f(g.y & 0xffffu, h.z);
        f(g.y >> 16, h.w);
        j += 4;
    }
    if (n - j >= 2) {
        const uint32_t g = *reinterpret_cast<const uint32_t *>(L + C * j + 2 * rit);
        const float2 h = *reinterpret_cast<const float2 *>(H + C * j + 2 * rit);
        f(g & 0xffffu, h.x);
        f(g >> 16, h.y);
        j += 2;
    }
    if (n - j >= 1)
        f((uint32_t)L[C * j + rit], H[C * j + rit]);
}

// The problem a consumer warp's tile belongs to, with the fields the
// consumers use.  Every consumer warp derives it from the tile number and
// the problem table alone (never from what the producer wrote), so all of
// them see the same sequence of problems.
struct ConsumerProblem {
    int pi = 0, cur = -1;
    int64_t slot = 0;
    void *W = nullptr;
    int ld = 0, col0 = 0;
};

// Complex float consumer warp.  Per chunk: the row's old W is loaded into
// registers one chunk ahead, when the previous chunk is done, so its latency
// passes while the entries are summed; the entries are read from the stage
// group by group (one 16-byte load per 8 indices, one per 2 values); each
// entry adds its products with Re h and Im h to two packed (re, im) sums
// per column with paired FMAs, and H'V - W = (a.re - b.im - w.re,
// a.im + b.re - w.im); the last entry reads the row's own V row, whose
// operand stays in registers for the scalar products.  HALF (every entry
// purely real or purely imaginary, one float per entry, real entries before
// imaginary ones): a real entry r adds (r, r) * (v.re, v.im) to a, an
// imaginary one i*m adds (m, m) * (v.re, v.im) to b -- the nonzero products
// of the general form, so W is the same -- with one paired FMA per column.
//
// Abort safety: the only barriers among consumer warps are in flush_eta32.
// Every consumer warp walks the same tiles (blockIdx.x, + gridDim.x, ...)
// and derives each tile's problem from the table, so every consumer warp
// calls flush_eta32 at the same tiles whatever happens to its waits.  A
// warp whose wait fails (timeout, or the block's abort flag) sets `failed`
// and skips the work and the waits of its remaining tiles, but not the
// flushes: the barrier counts always match.
template <int T, int E, bool IMAG, bool HALF>
__device__ __forceinline__ void consume32(const StagedParams &p, unsigned char *smem,
                                          const StagedProblem *tab, int64_t total,
                                          volatile int *abort_flag)
{
    constexpr int P = 32 / T, RB = T * E;
    constexpr int EV = Pieces<float, E>::EV, NP = Pieces<float, E>::NP;
    static_assert(EV == 2, "two complex floats per 16-byte piece");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cw = warp - 1, n_cw = (blockDim.x >> 5) - 1;
    const int tl = lane % T, team = lane / T;
    // The order of a lane's two 16-byte pieces (E = 4).  A 16-byte shared
    // load serves eight lanes per pass; with four lanes per row (T = 4) the
    // two teams of a pass would read the same 64-byte half of their V rows,
    // i.e. the same 16 banks, so odd teams take their pieces in the other
    // order.  With two lanes per row (rows 64 bytes apart), the third and
    // fourth team of a pass do.  The old W, the stored W and the eta terms
    // follow the same order (swapped back before eta is summed across
    // teams).
    constexpr bool kSwap = NP == 2 && (T == 4 || T == 2);
    const int sw = kSwap ? (T == 4 ? (team & 1) : ((team >> 1) & 1)) : 0;
    // this lane's pieces within a row, in floats
    const int pofs0 = 2 * tl * EV + 2 * sw * T * EV, pofs1 = 2 * tl * EV + 2 * (sw ^ 1) * T * EV;
    auto po = [&](int q) { return q == 0 ? pofs0 : pofs1; };
    WarpEta<IMAG, T, E> pe;
    pe.clear();
    auto fold = [&]() {
        if constexpr (kSwap)
            pe.swap_pieces(sw);
        pe.fold(team);
    };
    grid_dependency_wait();
    const int rit = cw * P + team;  // row within the chunk
    const int C = p.C, NS = p.stages;
    const int64_t G = gridDim.x;
    const uint32_t full0 = smem_u32(smem), empty0 = full0 + 8 * NS;
    double *red = reinterpret_cast<double *>(smem + kRedOffset);
    int nfold = 0;
    uint64_t pa[E], pb[E];
    float4 wo[NP];  // the row's old W pieces
    // the old W of the row of tile gt (problem q) into wo
    auto load_w = [&](int64_t gt, int q) {
        const StagedProblem &Q = tab[q];
        const float *Wq = static_cast<const float *>(Q.buf[p.parity ^ 1]);
        const int64_t row = (gt - Q.tile0) * (int64_t)C + rit;
        const float *wr = Wq + 2 * (row * Q.ld + Q.col0);
#pragma unroll
        for (int q2 = 0; q2 < NP; q2++)
            wo[q2] = __ldcg(reinterpret_cast<const float4 *>(wr + po(q2)));
    };
    ConsumerProblem cp;
    bool failed = false, have_w = false;
    int64_t k = 0;
    int s_next = 0;          // stage of the next tile
    uint32_t ph_next = 0;    // parity of that stage's current use
    for (int64_t gt = blockIdx.x; gt < total; gt += G, k++) {
        const int s = s_next;
        const uint32_t ph = ph_next;
        if (++s_next == NS) {
            s_next = 0;
            ph_next ^= 1u;
        }
        cp.pi = advance_problem(tab, p.n_probs, cp.pi, gt);
        const int64_t lt = gt - tab[cp.pi].tile0;
        if (cp.pi != cp.cur) {
            if (cp.cur >= 0 && p.dots) {
                fold();
                nfold = 0;
                flush_eta32<T, E, IMAG>(pe, red, tab[cp.cur], cp.slot, cw, n_cw);
            }
            cp.cur = cp.pi;
            cp.slot = lt;
            cp.W = tab[cp.pi].buf[p.parity ^ 1];
            cp.ld = tab[cp.pi].ld;
            cp.col0 = tab[cp.pi].col0;
        }
        if (failed)
            continue;
        if (!p.init && !p.off_w && !have_w)
            load_w(gt, cp.pi);
        const bool ok = mbar_wait_bounded(full0 + 8 * s, ph, abort_flag, p.err, true);
        if (!__all_sync(0xffffffffu, ok)) {
            failed = true;
            continue;
        }
        const unsigned char *st = smem + p.bar_bytes + (size_t)s * p.stage_bytes;
        const volatile int *meta = reinterpret_cast<const volatile int *>(smem + kMetaOffset + 16 * s);
        const int len = meta[0];
        const float *vb = reinterpret_cast<const float *>(st);
        const uint16_t *lid = reinterpret_cast<const uint16_t *>(st + p.off_lidx);
#ifdef KPM_CHECK
        // checked build: a local index past the chunk's gathered rows reads
        // row 0 instead and stops the launch with KPM_DEVERR_RANGE
        const uint32_t ntot = (uint32_t)meta[2];
        auto check_u = [&](uint32_t &u) {
            if (u >= ntot) {
                if (p.err)
                    atomicExch(p.err, KPM_DEVERR_RANGE);
                *abort_flag = 1;
                u = 0;
            }
        };
#endif
#pragma unroll
        for (int c = 0; c < E; c++)
            pa[c] = pb[c] = 0ull;
        auto entry = [&](uint32_t u, float hx, float hy) {
#ifdef KPM_CHECK
            check_u(u);
#endif
            const uint64_t hx2 = pack2(hx, hx), hy2 = pack2(hy, hy);
            const float *vr = vb + (size_t)u * 2 * RB;
#pragma unroll
            for (int q = 0; q < NP; q++) {
                const float4 v4 = *reinterpret_cast<const float4 *>(vr + po(q));
                const uint64_t v0 = pack2(v4.x, v4.y), v1 = pack2(v4.z, v4.w);
                pa[2 * q] = ffma2(hx2, v0, pa[2 * q]);
                pb[2 * q] = ffma2(hy2, v0, pb[2 * q]);
                pa[2 * q + 1] = ffma2(hx2, v1, pa[2 * q + 1]);
                pb[2 * q + 1] = ffma2(hy2, v1, pb[2 * q + 1]);
            }
        };
        const int nm = len - 1;
        float hox, hoy;  // the own entry's value
        if constexpr (HALF) {
            const float *hv = reinterpret_cast<const float *>(st + p.off_val);
            const int nre = meta[1];
            auto half_entry = [&](uint64_t (&acc)[E], uint32_t u, float h) {
#ifdef KPM_CHECK
                check_u(u);
#endif
                const uint64_t h2 = pack2(h, h);
                const float *vr = vb + (size_t)u * 2 * RB;
#pragma unroll
                for (int q = 0; q < NP; q++) {
                    const float4 v4 = *reinterpret_cast<const float4 *>(vr + po(q));
                    acc[2 * q] = ffma2(h2, pack2(v4.x, v4.y), acc[2 * q]);
                    acc[2 * q + 1] = ffma2(h2, pack2(v4.z, v4.w), acc[2 * q + 1]);
                }
            };
            walk_region(lid, hv, C, rit, 0, nre, [&](uint32_t u, float h) { half_entry(pa, u, h); });
            walk_region(lid, hv, C, rit, nre, nm - nre,
                        [&](uint32_t u, float h) { half_entry(pb, u, h); });
            hox = hv[C * nm + rit];
            hoy = 0.f;
        } else {
            const float2 *vals = reinterpret_cast<const float2 *>(st + p.off_val);
            walk_index_groups(
                lid, C, rit, nm,
                [&](int j, uint32_t u0, uint32_t u1) {
                    const float4 h = *reinterpret_cast<const float4 *>(vals + C * j + 2 * rit);
                    entry(u0, h.x, h.y);
                    entry(u1, h.z, h.w);
                },
                [&](int j, uint32_t u) {
                    const float2 h = vals[C * j + rit];
                    entry(u, h.x, h.y);
                });
            const float2 h = vals[C * nm + rit];
            hox = h.x;
            hoy = h.y;
        }
        // the own entry: local position rit; its V operand stays for eta
        float4 vo[NP];
        {
            const uint64_t hx2 = pack2(hox, hox), hy2 = pack2(hoy, hoy);
            const float *vr = vb + (size_t)rit * 2 * RB;
#pragma unroll
            for (int q = 0; q < NP; q++) {
                vo[q] = *reinterpret_cast<const float4 *>(vr + po(q));
                const uint64_t v0 = pack2(vo[q].x, vo[q].y), v1 = pack2(vo[q].z, vo[q].w);
                pa[2 * q] = ffma2(hx2, v0, pa[2 * q]);
                pa[2 * q + 1] = ffma2(hx2, v1, pa[2 * q + 1]);
                if constexpr (!HALF) {
                    pb[2 * q] = ffma2(hy2, v0, pb[2 * q]);
                    pb[2 * q + 1] = ffma2(hy2, v1, pb[2 * q + 1]);
                }
            }
        }
        float w[2 * E];
#pragma unroll
        for (int c = 0; c < E; c++) {
            float ar, ai, br, bi;
            unpack2(pa[c], ar, ai);
            unpack2(pb[c], br, bi);
            w[2 * c] = ar - bi;
            w[2 * c + 1] = ai + br;
        }
        if (p.init) {
#pragma unroll
            for (int i = 0; i < 2 * E; i++)
                w[i] *= 0.5f;
        } else {
            if (p.off_w) {
                // the old W rows came with the stage
                const float *ws = reinterpret_cast<const float *>(st + p.off_w) + (size_t)rit * 2 * RB;
#pragma unroll
                for (int q = 0; q < NP; q++)
                    wo[q] = *reinterpret_cast<const float4 *>(ws + po(q));
            }
#pragma unroll
            for (int q = 0; q < NP; q++) {
                w[4 * q] -= wo[q].x;
                w[4 * q + 1] -= wo[q].y;
                w[4 * q + 2] -= wo[q].z;
                w[4 * q + 3] -= wo[q].w;
            }
        }
        const int64_t wbase = (lt * (int64_t)C + rit) * cp.ld + cp.col0 + tl * EV;
        if constexpr (kSwap) {
            // the pieces back in column order for the store
            float wc[2 * E];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                wc[i] = sw ? w[i + 4] : w[i];
                wc[i + 4] = sw ? w[i] : w[i + 4];
            }
            store_owned<float, T, E>(static_cast<float *>(cp.W), wbase, wc);
        } else {
            store_owned<float, T, E>(static_cast<float *>(cp.W), wbase, w);
        }
        // the next tile's old W, while this one's scalar products are added
        have_w = false;
        if (!p.init && !p.off_w && gt + G < total) {
            load_w(gt + G, advance_problem(tab, p.n_probs, cp.pi, gt + G));
            have_w = true;
        }
        if (p.dots) {
#pragma unroll
            for (int q = 0; q < NP; q++) {
                pe.add(2 * q, w[4 * q], w[4 * q + 1], vo[q].x, vo[q].y);
                pe.add(2 * q + 1, w[4 * q + 2], w[4 * q + 3], vo[q].z, vo[q].w);
            }
            if (++nfold == kEtaFold) {
                fold();
                nfold = 0;
            }
        }
        __syncwarp();
        if (lane == 0)
            mbar_arrive(empty0 + 8 * s);
    }
    if (!p.dots)
        return;
    if (cp.cur >= 0) {
        fold();
        flush_eta32<T, E, IMAG>(pe, red, tab[cp.cur], cp.slot, cw, n_cw);
    } else if (p.probs == nullptr) {
        // a single problem's partials are read for every block: a block
        // without chunks contributes zeros
        for (int t = cw * 32 + lane; t < 3 * RB; t += n_cw * 32)
            tab[0].partial[(int64_t)blockIdx.x * tab[0].ps + t * tab[0].qs] = 0.0;
    }
}

// Complex double consumer warp (the FP64 pipe is this form's bound): the
// old W row is fetched with cp.async into the block's W buffer while the
// entry loop runs; per entry and column four FMAs on one 16-byte V piece,
// or, HALF (every stored entry purely real or purely imaginary), two on its
// 8-byte halves: the value array holds operand pairs (a, b) and bit 15 of
// the local index marks an imaginary entry -- a real one, (r, r), adds
// (r x, r y) to (re, im); an imaginary one, (-m, m), adds (-m y, m x), so
// the halves are read in swapped order.  The two FMAs are the general
// form's nonzero products in the same order (the skipped ones add exact
// zeros), so both forms give the same W.  Eta in plain FMA chains.  Abort
// safety as in consume32.
template <int T, int E, bool IMAG, bool HALF>
__device__ __forceinline__ void consume64(const StagedParams &p, unsigned char *smem,
                                          const StagedProblem *tab, int64_t total,
                                          volatile int *abort_flag)
{
    constexpr int P = 32 / T, RB = T * E;
    grid_dependency_wait();
    constexpr int EV = Pieces<double, E>::EV, NP = Pieces<double, E>::NP;
    static_assert(EV == 1, "one complex double per 16-byte piece");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cw = warp - 1, n_cw = (blockDim.x >> 5) - 1;
    const int tl = lane % T, team = lane / T;
    const int rit = cw * P + team;
    const int C = p.C, NS = p.stages;
    const int64_t G = gridDim.x;
    const uint32_t full0 = smem_u32(smem), empty0 = full0 + 8 * NS;
    double *red = reinterpret_cast<double *>(smem + kRedOffset);
    StagedEta64<IMAG> acc[E];
    ConsumerProblem cp;
    bool failed = false;
    int64_t k = 0;
    int s_next = 0;          // stage of the next tile
    uint32_t ph_next = 0;    // parity of that stage's current use
    for (int64_t gt = blockIdx.x; gt < total; gt += G, k++) {
        const int s = s_next;
        const uint32_t ph = ph_next;
        if (++s_next == NS) {
            s_next = 0;
            ph_next ^= 1u;
        }
        cp.pi = advance_problem(tab, p.n_probs, cp.pi, gt);
        const int64_t lt = gt - tab[cp.pi].tile0;
        if (cp.pi != cp.cur) {
            if (cp.cur >= 0 && p.dots)
                flush_eta64<T, E>(acc, red, tab[cp.cur], cp.slot, cw, n_cw);
            cp.cur = cp.pi;
            cp.slot = lt;
            cp.W = tab[cp.pi].buf[p.parity ^ 1];
            cp.ld = tab[cp.pi].ld;
            cp.col0 = tab[cp.pi].col0;
        }
        if (failed)
            continue;
        const bool ok = mbar_wait_bounded(full0 + 8 * s, ph, abort_flag, p.err, true);
        if (!__all_sync(0xffffffffu, ok)) {
            failed = true;
            continue;
        }
        const unsigned char *st = smem + p.bar_bytes + (size_t)s * p.stage_bytes;
        const int len = *reinterpret_cast<const volatile int *>(smem + kMetaOffset + 16 * s);
        const double *vb = reinterpret_cast<const double *>(st);
#ifdef KPM_CHECK
        // checked build: as in consume32
        const uint32_t ntot = (uint32_t)(reinterpret_cast<const volatile int *>(
            smem + kMetaOffset + 16 * s))[2];
#endif
        const double2 *vals = reinterpret_cast<const double2 *>(st + p.off_val);
        const uint16_t *lid = reinterpret_cast<const uint16_t *>(st + p.off_lidx);
        double *Wp = static_cast<double *>(cp.W);

        // the old W row is requested first (the producer asked L2 for it):
        // this lane's 16-byte pieces go to the row's slot of the W buffer
        // (written and read by this lane only) with cp.async
        const int64_t wbase = (lt * (int64_t)C + rit) * cp.ld + cp.col0 + tl * EV;
        double *wsm = reinterpret_cast<double *>(smem + p.off_aux) + rit * 2 * RB;
        if (!p.init) {
#pragma unroll
            for (int q = 0; q < NP; q++)
                cp_async16(smem_u32(wsm + 2 * (q * T * EV + tl * EV)),
                           Wp + 2 * (wbase + (int64_t)q * T * EV));
            cp_async_commit();
        }
        double a[2 * E];
#pragma unroll
        for (int q = 0; q < 2 * E; q++)
            a[q] = 0.0;
        auto entry = [&](uint32_t l, const double2 h) {
#ifdef KPM_CHECK
            if ((HALF ? (l & 0x7fffu) : l) >= ntot) {
                if (p.err)
                    atomicExch(p.err, KPM_DEVERR_RANGE);
                *abort_flag = 1;
                l = HALF ? (l & 0x8000u) : 0u;
            }
#endif
            if constexpr (HALF) {
                const int sw = (int)(l >> 15);
                const double *vr = vb + (size_t)(l & 0x7fffu) * 2 * RB + 2 * tl;
                const double *v0 = vr + sw, *v1 = vr + (sw ^ 1);
#pragma unroll
                for (int c = 0; c < E; c++) {
                    a[2 * c] = fma(h.x, v0[2 * c * T], a[2 * c]);
                    a[2 * c + 1] = fma(h.y, v1[2 * c * T], a[2 * c + 1]);
                }
            } else {
                const double *vr = vb + (size_t)l * 2 * RB;
#pragma unroll
                for (int c = 0; c < E; c++) {
                    const double2 v = *reinterpret_cast<const double2 *>(vr + 2 * (c * T + tl));
                    a[2 * c] = fma(h.x, v.x, a[2 * c]);
                    a[2 * c] = fma(-h.y, v.y, a[2 * c]);
                    a[2 * c + 1] = fma(h.x, v.y, a[2 * c + 1]);
                    a[2 * c + 1] = fma(h.y, v.x, a[2 * c + 1]);
                }
            }
        };
        const int nm = len - 1;
        walk_index_groups(
            lid, C, rit, nm,
            [&](int j, uint32_t u0, uint32_t u1) {
                entry(u0, vals[C * j + rit]);
                entry(u1, vals[C * (j + 1) + rit]);
            },
            [&](int j, uint32_t u) { entry(u, vals[C * j + rit]); });
        entry((uint32_t)lid[C * nm + rit], vals[C * nm + rit]);
        if (p.init) {
#pragma unroll
            for (int q = 0; q < 2 * E; q++)
                a[q] *= 0.5;
        } else {
            cp_async_wait<0>();
#pragma unroll
            for (int q = 0; q < NP; q++) {
                double wo[2];
                lds_piece(wsm + 2 * (q * T * EV + tl * EV), wo);
                a[2 * q] -= wo[0];
                a[2 * q + 1] -= wo[1];
            }
        }
        store_owned<double, T, E>(Wp, wbase, a);
        if (p.dots) {
            // the row's own V entries: local position rit of the list
            const double *ov = vb + (size_t)rit * 2 * RB;
#pragma unroll
            for (int q = 0; q < NP; q++) {
                double v[2];
                lds_piece(ov + 2 * (q * T * EV + tl * EV), v);
                acc[q].add(a[2 * q], a[2 * q + 1], v[0], v[1]);
            }
        }
        __syncwarp();
        if (lane == 0)
            mbar_arrive(empty0 + 8 * s);
    }
    if (!p.dots)
        return;
    if (cp.cur >= 0) {
        flush_eta64<T, E>(acc, red, tab[cp.cur], cp.slot, cw, n_cw);
    } else if (p.probs == nullptr) {
        for (int t = cw * 32 + lane; t < 3 * RB; t += n_cw * 32)
            tab[0].partial[(int64_t)blockIdx.x * tab[0].ps + t * tab[0].qs] = 0.0;
    }
}

template <typename Real, int T, int E, bool IMAG, bool HALF>
__global__ void __launch_bounds__(KPM_STAGED_MAX_THREADS, StagedMinBlocks<Real, E>::value)
    aug_spmmv_staged_kernel(const StagedParams p)
{
    static_assert(T >= 1 && T <= 32 && (32 % T) == 0, "team size divides the warp");
    constexpr int RB = T * E;
    constexpr int CSIZE = 2 * (int)sizeof(Real);
    // bytes of one staged value: a complex number, an operand pair (complex
    // double half form) or one float (complex float half form)
    constexpr int VSIZE = (sizeof(Real) == 4 && HALF) ? 4 : CSIZE;
    // [full[NS], empty[NS] | abort flag at 128 | stage chunk lengths at
    //  kMetaOffset | record ring at kRingOffset | eta sum at kRedOffset |
    //  problem table at kTableOffset | stages from bar_bytes on | at
    //  off_aux: the W buffer (complex double) or the consumer warps' eta
    //  accumulators (complex float)]
    extern __shared__ __align__(128) unsigned char smem[];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NS = p.stages;
    const uint32_t full0 = smem_u32(smem), empty0 = full0 + 8 * NS;
    const int n_cw = (blockDim.x >> 5) - 1;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 128);
    StagedProblem *tab = reinterpret_cast<StagedProblem *>(smem + kTableOffset);
    if (threadIdx.x == 0) {
        allow_dependents();
        *abort_flag = 0;
        for (int s = 0; s < NS; s++) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, (uint32_t)n_cw);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    {
        const StagedProblem *src = p.probs ? p.probs : &p.one;
        const int words = p.n_probs * (int)(sizeof(StagedProblem) / 8);
        for (int i = threadIdx.x; i < words; i += blockDim.x)
            reinterpret_cast<uint64_t *>(tab)[i] = reinterpret_cast<const uint64_t *>(src)[i];
    }
    __syncthreads();
    const int64_t total = tab[p.n_probs - 1].tile0 + tab[p.n_probs - 1].n_tiles;

    if (warp == 0) {
        const int64_t armed = produce<RB, CSIZE, VSIZE>(p, smem, tab, total, abort_flag);
        // the copies of the last armed stages must land before the block's
        // shared memory is released
        if (lane == 0)
            for (int64_t k = armed > NS ? armed - NS : 0; k < armed; k++)
                mbar_wait_bounded(full0 + 8 * (uint32_t)(k % NS), (uint32_t)((k / NS) & 1),
                                  abort_flag, p.err, false);
        __syncwarp();
    } else if constexpr (sizeof(Real) == 4) {
        consume32<T, E, IMAG, HALF>(p, smem, tab, total, abort_flag);
    } else {
        consume64<T, E, IMAG, HALF>(p, smem, tab, total, abort_flag);
    }
}

}  // namespace

// (T, E) shapes of the staged kernel.  Complex float: 4 columns per lane
// as two 16-byte pieces (widths 4..64), or 2 as one piece (widths 2..32:
// twice the lanes per row, for more warps per SM); at widths 2 and 4 one
// lane holds a whole row.  Complex double: 2 columns per lane as two
// pieces (widths 2..32; a 64-wide stage would not fit twice), or 1 (width
// 1), each with and without the half-complex shortcut.
#define KPM_STAGED_SHAPES(X) X(1, 4) X(2, 4) X(4, 4) X(8, 4) X(16, 4) X(1, 2) X(4, 2) X(8, 2) X(16, 2)
#define KPM_STAGED_SHAPES64(X) X(1, 1) X(1, 2) X(2, 2) X(4, 2) X(8, 2) X(16, 2)

bool staged_shape_supported(int T, int E, bool fp64)
{
#define KPM_CASE(T_, E_) \
    if (T == T_ && E == E_) \
        return true;
    if (fp64) {
        KPM_STAGED_SHAPES64(KPM_CASE)
    } else {
        KPM_STAGED_SHAPES(KPM_CASE)
    }
#undef KPM_CASE
    return false;
}

bool staged_layout(int C, int T, int RB, int csize, int vsize, int u_max, int l_max, int stages,
                   int n_probs, bool wstage, size_t max_smem, StagedLayout &o)
{
    auto up = [](uint64_t x, uint64_t a) { return (x + a - 1) / a * a; };
    if (C < 8 || T < 1 || RB < 1 || RB > 64 || (csize != 8 && csize != 16) ||
        (vsize != 4 && vsize != 8 && vsize != 16) || (wstage && csize != 8) || u_max < C ||
        l_max < 0 || stages < 1 || stages > 8 || n_probs < 1 || (C * T) % 32 != 0 ||
        32 + C * T > KPM_STAGED_MAX_THREADS)
        return false;
    const uint64_t row_bytes = (uint64_t)RB * csize;
    uint64_t off = up((uint64_t)u_max * row_bytes, 128);
    o.off_val = (uint32_t)off;
    off = up(off + (uint64_t)C * l_max * vsize, 128);
    o.off_lidx = (uint32_t)off;
    off = up(off + (uint64_t)C * l_max * 2, 128);
    o.off_w = 0;
    if (wstage) {
        // the chunk's old W rows (complex float)
        o.off_w = (uint32_t)off;
        off = up(off + (uint64_t)C * row_bytes, 128);
    }
    o.stage_bytes = (uint32_t)off;
    o.bar_bytes = (uint32_t)up(kTableOffset + (uint64_t)n_probs * sizeof(StagedProblem), 128);
    o.stages = stages;
    // after the stages: complex double, the block's W buffer (one slot per
    // row of a chunk); complex float nothing
    o.off_aux = (uint32_t)(o.bar_bytes + (uint64_t)stages * o.stage_bytes);
    o.smem = o.off_aux + (csize == 16 ? (uint64_t)C * row_bytes : 0);
    return o.smem <= max_smem && o.stage_bytes < (1u << 20);
}

// Host launch helpers: occupancy queries and launches, no device code.

namespace {

// Blocks per SM at smem bytes of dynamic shared memory.  The query needs the
// kernel's dynamic shared-memory limit at least smem; it only ever raises
// the limit, through the same per-device record the launches use, so that a
// query for a small layout never lowers it under a larger layout that an
// earlier launch or a captured graph of the same instantiation relies on.
template <typename Real, int T, int E, bool IMAG, bool HALF>
int occupancy_of(int threads, size_t smem)
{
    int nb = 0;
    if (ensure_max_dynamic_smem((const void *)aug_spmmv_staged_kernel<Real, T, E, IMAG, HALF>,
                                smem) != KPM_OK ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, aug_spmmv_staged_kernel<Real, T, E, IMAG, HALF>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

// Launches one instantiation, raising its dynamic shared-memory limit on
// the current device the first time a launch there needs more.
template <typename Real, int T, int E, bool IMAG, bool HALF>
int launch_one_staged(const StagedParams &p, int grid, int threads, size_t smem, cudaStream_t st,
                      bool pdl)
{
    KPM_TRY(ensure_max_dynamic_smem((const void *)aug_spmmv_staged_kernel<Real, T, E, IMAG, HALF>,
                                    smem));
    if (pdl) {
        // may start while the previous kernel in the stream finishes
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, aug_spmmv_staged_kernel<Real, T, E, IMAG, HALF>, p) ==
                       cudaSuccess
                   ? KPM_OK
                   : KPM_ECUDA;
    }
    aug_spmmv_staged_kernel<Real, T, E, IMAG, HALF><<<grid, threads, smem, st>>>(p);
    return cudaGetLastError() == cudaSuccess ? KPM_OK : KPM_ECUDA;
}

}  // namespace

int staged_max_blocks_per_sm(int T, int E, int C, size_t smem, bool fp64, bool half)
{
    const int threads = 32 + C * T;
#define KPM_CASE(T_, E_) \
    if (T == T_ && E == E_) \
        return half ? occupancy_of<float, T_, E_, false, true>(threads, smem) \
                    : occupancy_of<float, T_, E_, false, false>(threads, smem);
#define KPM_CASE64(T_, E_) \
    if (T == T_ && E == E_) \
        return occupancy_of<double, T_, E_, false, false>(threads, smem);
    if (fp64) {
        KPM_STAGED_SHAPES64(KPM_CASE64)
    } else {
        KPM_STAGED_SHAPES(KPM_CASE)
    }
#undef KPM_CASE
#undef KPM_CASE64
    return 0;
}

int launch_sweep_staged(const StagedParams &p, int T, int E, int grid, size_t smem, void *stream,
                        bool pdl)
{
    const int threads = 32 + p.C * T;
    if (grid < 1 || threads > KPM_STAGED_MAX_THREADS || p.stages < 1 || p.stages > 8 ||
        p.n_probs < 1 || (p.probs == nullptr && p.n_probs != 1))
        return KPM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
#define KPM_CASE(T_, E_)                                                                       \
    if (T == T_ && E == E_) {                                                                  \
        if (p.half)                                                                            \
            return p.with_imag                                                                 \
                       ? launch_one_staged<float, T_, E_, true, true>(p, grid, threads, smem, st, pdl) \
                       : launch_one_staged<float, T_, E_, false, true>(p, grid, threads, smem, st, pdl); \
        return p.with_imag ? launch_one_staged<float, T_, E_, true, false>(p, grid, threads, smem, st, pdl) \
                           : launch_one_staged<float, T_, E_, false, false>(p, grid, threads, smem, st, pdl); \
    }
#define KPM_CASE64(T_, E_)                                                                     \
    if (T == T_ && E == E_) {                                                                  \
        if (p.half)                                                                            \
            return p.with_imag                                                                 \
                       ? launch_one_staged<double, T_, E_, true, true>(p, grid, threads, smem, st, pdl) \
                       : launch_one_staged<double, T_, E_, false, true>(p, grid, threads, smem, st, pdl); \
        return p.with_imag                                                                     \
                   ? launch_one_staged<double, T_, E_, true, false>(p, grid, threads, smem, st, pdl) \
                   : launch_one_staged<double, T_, E_, false, false>(p, grid, threads, smem, st, pdl); \
    }
    if (p.fp64) {
        KPM_STAGED_SHAPES64(KPM_CASE64)
    } else {
        KPM_STAGED_SHAPES(KPM_CASE)
    }
#undef KPM_CASE
#undef KPM_CASE64
    return KPM_EUNSUPPORTED;
}

}  // namespace kpm
