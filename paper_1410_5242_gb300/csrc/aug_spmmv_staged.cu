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

// A lane's eta terms for one column.  Each row adds |v|^2 and Re(conj(w) v)
// as paired FMAs into packed single-precision pending sums ((v_re^2, v_im^2)
// and (w_re v_re, w_im v_im)); every kEtaFold chunks fold() adds the pending
// sums to (hi, lo) pairs with Knuth's TwoSum, so the running sum is carried
// without rounding loss and only an 8-row partial is ever rounded in single
// precision.  IMAG adds Im(conj(w) v) the same way in scalar form.
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

template <bool IMAG>
struct StagedEta {
    uint64_t pvv = 0ull, pwv = 0ull;
    float pwvi = 0.f;
    float vv_h = 0.f, vv_l = 0.f, wv_h = 0.f, wv_l = 0.f, wvi_h = 0.f, wvi_l = 0.f;
    __device__ __forceinline__ void add(float wr, float wi, float vr, float vi)
    {
        const uint64_t v2 = pack2(vr, vi), w2 = pack2(wr, wi);
        pvv = ffma2(v2, v2, pvv);
        pwv = ffma2(w2, v2, pwv);
        if constexpr (IMAG) {
            pwvi = __fmaf_rn(wr, vi, pwvi);
            pwvi = __fmaf_rn(-wi, vr, pwvi);
        }
    }
    __device__ __forceinline__ void fold()
    {
        float a, b;
        unpack2(pvv, a, b);
        two_sum_pair(vv_h, vv_l, __fadd_rn(a, b));
        unpack2(pwv, a, b);
        two_sum_pair(wv_h, wv_l, __fadd_rn(a, b));
        pvv = pwv = 0ull;
        if constexpr (IMAG) {
            two_sum_pair(wvi_h, wvi_l, pwvi);
            pwvi = 0.f;
        }
    }
    // after fold()
    __device__ __forceinline__ double get(int k) const
    {
        if (k == 0)
            return (double)vv_h + (double)vv_l;
        if (k == 1)
            return (double)wv_h + (double)wv_l;
        return IMAG ? (double)wvi_h + (double)wvi_l : 0.0;
    }
};

// A lane's eta terms for one column in complex double: plain FMA chains
// (aug_spmmv.cuh's EtaAcc); fold() has nothing to do.
template <bool IMAG>
struct StagedEta64 {
    EtaAcc<double, IMAG> a;
    __device__ __forceinline__ void add(double wr, double wi, double vr, double vi)
    {
        a.add(wr, wi, vr, vi);
    }
    __device__ __forceinline__ void fold() {}
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

// The producer warp: for each tile of this block, wait until its stage is
// free, announce the bytes on full[s], and issue the copies.  Lane l holds
// word l of the tile's record, i.e. inline run l - 3; runs past the inline
// ones are read from the overflow array 32 at a time.  Returns the number
// of tiles armed.
template <int RB, int CSIZE>
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
    int pi = -1;
    int64_t i_end = -1, i_tile0 = 0;
    const char *Vb = nullptr, *Wb = nullptr, *valb = nullptr, *lidxb = nullptr;
    const int2 *ovfp = nullptr;
    int ld = 0, col0 = 0;
    int64_t k = 0;
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
        const int len = __shfl_sync(0xffffffffu, word.x, 1);
        const int nruns = __shfl_sync(0xffffffffu, word.y, 1);
        const int n_inline = min(nruns, KPM_REC_INLINE_RUNS);
        const bool has_run = lane >= 3 && lane - 3 < n_inline;
        const int count = has_run ? word.y : 0;
        const int incl = warp_incl_scan(count, lane);
        uint32_t total_rows = (uint32_t)__shfl_sync(0xffffffffu, incl, 31);
        for (int g = KPM_REC_INLINE_RUNS; g < nruns; g += 32) {
            const int2 r = g + lane < nruns
                               ? __ldg(ovfp + ovf0 + (g - KPM_REC_INLINE_RUNS) + lane)
                               : make_int2(0, 0);
            total_rows += (uint32_t)__shfl_sync(0xffffffffu, warp_incl_scan(r.y, lane), 31);
        }

        const int s = (int)(k % NS);
        const uint32_t ph = (uint32_t)((k / NS) & 1);
        const uint32_t full = full0 + 8 * s, empty = empty0 + 8 * s;
        if (k >= NS) {
            // every lane waits (and acquires); the warp leaves together
            const bool ok = mbar_wait_bounded(empty, ph ^ 1u, abort_flag, p.err, true);
            if (!__all_sync(0xffffffffu, ok))
                break;
        }
        const uint32_t st = stage0 + (uint32_t)s * p.stage_bytes;
        const uint32_t val_bytes = (uint32_t)p.C * (uint32_t)len * (uint32_t)CSIZE;
        const uint32_t lidx_bytes = (uint32_t)p.C * (uint32_t)len * 2u;
        const uint32_t bytes = total_rows * row_bytes + val_bytes + lidx_bytes;
        if (lane == 0) {
            volatile int *meta = reinterpret_cast<volatile int *>(smem + kMetaOffset + 16 * s);
            meta[0] = len;
            meta[1] = pi;
            meta[2] = (int)lt;
            mbar_arrive_expect_tx(full, bytes);
        }
        __syncwarp();
        if (len > 0) {
            if (lane == 0)
                bulk_g2s(st + p.off_val, valb + e0 * CSIZE, val_bytes, full);
            if (lane == 1)
                bulk_g2s(st + p.off_lidx, lidxb + e0 * 2, lidx_bytes, full);
        }
        // the consumers read the chunk's old W rows themselves; ask L2 for
        // them now (whole rows: contiguous, 16-byte multiples)
        if (!p.init && lane == 2 && ((int64_t)ld * CSIZE & 15) == 0)
            prefetch_l2(Wb + lt * (int64_t)p.C * ld * CSIZE, (uint64_t)p.C * ld * CSIZE);
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
    }
    cp_async_wait<0>();
    return k;
}

__device__ __forceinline__ void consumer_bar(int n_cw)
{
    asm volatile("bar.sync 1, %0;" ::"r"(n_cw * 32) : "memory");
}

// The consumer warps' eta sums for one problem, in a fixed order: lanes of
// equal columns by an xor butterfly, then warp after warp into red (3*RB
// doubles), then red to the problem's partial slot.  Resets acc.
template <typename Real, int T, int E, typename Acc>
__device__ __forceinline__ void flush_eta(Acc (&acc)[E], double *red,
                                          const StagedProblem &P, int64_t slot, int cw, int n_cw)
{
    constexpr int RB = T * E;
    const int lane = threadIdx.x & 31;
    const int tl = lane % T, team = lane / T;
    double out[3 * E];
#pragma unroll
    for (int k = 0; k < E; k++) {
        acc[k].fold();
#pragma unroll
        for (int q = 0; q < 3; q++)
            out[q * E + k] = acc[k].get(q);
    }
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
                    double &d = red[q * RB + owned_column<Real, T, E>(tl, k)];
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

// One row's H' V for this lane's E columns from a stage, complex double:
// one 16-byte piece per column and lane and four FMAs per entry and column;
// or, with HALF (every stored entry purely real or purely imaginary), two.
// There the value array holds operand pairs (a, b) and bit 15 of the local
// index marks an imaginary entry: a real one, (r, r), adds (r x, r y) to
// (re, im); an imaginary one, (-m, m), adds (-m y, m x), so the halves of v
// are read in swapped order.  The two FMAs are the general form's nonzero
// products in the same order (the skipped ones add exact zeros), so both
// forms give the same W.
template <int T, int E, bool HALF>
__device__ __forceinline__ void row_product(const double *vb, const double2 *vals,
                                            const uint16_t *lid, int C, int len, int rit, int tl,
                                            double (&acc_s)[2 * E])
{
    constexpr int RB = T * E;
#pragma unroll
    for (int q = 0; q < 2 * E; q++)
        acc_s[q] = 0.0;
#pragma unroll 4
    for (int j = 0; j < len; j++) {
        const int l = lid[j * C + rit];
        const double2 h = vals[j * C + rit];
        if constexpr (HALF) {
            const int sw = l >> 15;
            const double *vr = vb + (size_t)(l & 0x7fff) * 2 * RB + 2 * tl;
            const double *v0 = vr + sw, *v1 = vr + (sw ^ 1);
#pragma unroll
            for (int k = 0; k < E; k++) {
                acc_s[2 * k] = fma(h.x, v0[2 * k * T], acc_s[2 * k]);
                acc_s[2 * k + 1] = fma(h.y, v1[2 * k * T], acc_s[2 * k + 1]);
            }
        } else {
            const double *vr = vb + (size_t)l * 2 * RB;
#pragma unroll
            for (int k = 0; k < E; k++) {
                const double2 v = *reinterpret_cast<const double2 *>(vr + 2 * (k * T + tl));
                acc_s[2 * k] = fma(h.x, v.x, acc_s[2 * k]);
                acc_s[2 * k] = fma(-h.y, v.y, acc_s[2 * k]);
                acc_s[2 * k + 1] = fma(h.x, v.y, acc_s[2 * k + 1]);
                acc_s[2 * k + 1] = fma(h.y, v.x, acc_s[2 * k + 1]);
            }
        }
    }
}

// One 16-byte piece (two complex floats or one complex double) from
// shared memory.
__device__ __forceinline__ void lds_piece(const float *src, float (&out)[4])
{
    const float4 t = *reinterpret_cast<const float4 *>(src);
    out[0] = t.x;
    out[1] = t.y;
    out[2] = t.z;
    out[3] = t.w;
}

__device__ __forceinline__ void lds_piece(const double *src, double (&out)[2])
{
    const double2 t = *reinterpret_cast<const double2 *>(src);
    out[0] = t.x;
    out[1] = t.y;
}

template <typename Real, int T, int E, bool IMAG, bool HALF>
__global__ void __launch_bounds__(KPM_STAGED_MAX_THREADS, StagedMinBlocks<Real, E>::value)
    aug_spmmv_staged_kernel(const StagedParams p)
{
    static_assert(T >= 1 && T <= 32 && (32 % T) == 0, "team size divides the warp");
    static_assert(!HALF || sizeof(Real) == 8, "the half-complex form is complex double only");
    constexpr int P = 32 / T;
    constexpr int RB = T * E;
    constexpr int CSIZE = 2 * (int)sizeof(Real);
    constexpr int EV = Pieces<Real, E>::EV, NP = Pieces<Real, E>::NP;
    static_assert(2 * EV * sizeof(Real) == 16, "16-byte pieces");
    using Acc = typename std::conditional<sizeof(Real) == 4, StagedEta<IMAG>,
                                          StagedEta64<IMAG>>::type;
    // [full[NS], empty[NS] | abort flag at 128 | stage metadata at
    //  kMetaOffset | record ring at kRingOffset | eta sum at kRedOffset |
    //  problem table at kTableOffset | stages from bar_bytes on | W buffer
    //  at off_wbuf]
    extern __shared__ __align__(128) unsigned char smem[];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NS = p.stages;
    const uint32_t full0 = smem_u32(smem), empty0 = full0 + 8 * NS;
    const int n_cw = (blockDim.x >> 5) - 1;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 128);
    StagedProblem *tab = reinterpret_cast<StagedProblem *>(smem + kTableOffset);
    double *red = reinterpret_cast<double *>(smem + kRedOffset);
    if (threadIdx.x == 0) {
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
        const int64_t armed = produce<RB, CSIZE>(p, smem, tab, total, abort_flag);
        // the copies of the last armed stages must land before the block's
        // shared memory is released
        if (lane == 0)
            for (int64_t k = armed > NS ? armed - NS : 0; k < armed; k++)
                mbar_wait_bounded(full0 + 8 * (uint32_t)(k % NS), (uint32_t)((k / NS) & 1),
                                  abort_flag, p.err, false);
        __syncwarp();
    } else {
        const int cw = warp - 1;
        const int tl = lane % T, team = lane / T;
        const int rit = cw * P + team;  // row within the chunk
        const int C = p.C;
        Acc acc[E];
        int cur = -1;        // problem whose eta terms acc holds
        int64_t slot = 0;    // its partial slot: this block's first chunk of it
        Real *Wp = nullptr;  // its W block, row length and first column
        int ldw = 0, col0 = 0;
        int64_t k = 0;
        for (int64_t gt = blockIdx.x; gt < total; gt += gridDim.x, k++) {
            const int s = (int)(k % NS);
            const uint32_t ph = (uint32_t)((k / NS) & 1);
            const bool ok = mbar_wait_bounded(full0 + 8 * s, ph, abort_flag, p.err, true);
            if (!__all_sync(0xffffffffu, ok))
                break;
            const unsigned char *st = smem + p.bar_bytes + (size_t)s * p.stage_bytes;
            const volatile int *meta =
                reinterpret_cast<const volatile int *>(smem + kMetaOffset + 16 * s);
            const int len = meta[0], pi = meta[1];
            const int64_t lt = meta[2];
            if (pi != cur) {
                if (cur >= 0 && p.dots)
                    flush_eta<Real, T, E>(acc, red, tab[cur], slot, cw, n_cw);
                cur = pi;
                slot = lt;
                Wp = static_cast<Real *>(tab[pi].buf[p.parity ^ 1]);
                ldw = tab[pi].ld;
                col0 = tab[pi].col0;
            }
            using Real2 = typename std::conditional<sizeof(Real) == 4, float2, double2>::type;
            const Real *vb = reinterpret_cast<const Real *>(st);
            const Real2 *vals = reinterpret_cast<const Real2 *>(st + p.off_val);
            const uint16_t *lid = reinterpret_cast<const uint16_t *>(st + p.off_lidx);

            // The old W row is requested from global memory first (the
            // producer asked L2 for it when it armed the stage): this lane's
            // 16-byte pieces go to the block's W buffer (the row's slot,
            // written and read by this lane only) with cp.async, and the
            // entry loop hides their latency.
            const int64_t row = lt * (int64_t)C + rit;
            const int64_t wbase = row * ldw + col0 + tl * EV;
            Real *wsm = reinterpret_cast<Real *>(smem + p.off_wbuf) + rit * 2 * RB;
            if (!p.init) {
#pragma unroll
                for (int q = 0; q < NP; q++)
                    cp_async16(smem_u32(wsm + 2 * (q * T * EV + tl * EV)),
                               Wp + 2 * (wbase + (int64_t)q * T * EV));
                cp_async_commit();
            }
            Real acc_s[2 * E];
            if constexpr (sizeof(Real) == 4) {
                // complex float: two packed (re, im) accumulators per
                // column, a = sum_j Re(h_j) v_j and b = sum_j Im(h_j) v_j, so
                // each entry costs two paired FMAs per column; then
                // H' V = (a.re - b.im, a.im + b.re)
                uint64_t pa[E], pb[E];
#pragma unroll
                for (int c = 0; c < E; c++)
                    pa[c] = pb[c] = 0ull;
#pragma unroll 4
                for (int j = 0; j < len; j++) {
                    const int u = lid[j * C + rit];
                    const float2 h = vals[j * C + rit];
                    const uint64_t hx2 = pack2(h.x, h.x), hy2 = pack2(h.y, h.y);
                    const float *vr = vb + (size_t)u * 2 * RB;
#pragma unroll
                    for (int q = 0; q < NP; q++) {
                        const float4 v4 =
                            *reinterpret_cast<const float4 *>(vr + 2 * (q * T * EV + tl * EV));
                        const uint64_t v0 = pack2(v4.x, v4.y);
                        pa[q * EV] = ffma2(hx2, v0, pa[q * EV]);
                        pb[q * EV] = ffma2(hy2, v0, pb[q * EV]);
                        if constexpr (EV == 2) {
                            const uint64_t v1 = pack2(v4.z, v4.w);
                            pa[q * EV + 1] = ffma2(hx2, v1, pa[q * EV + 1]);
                            pb[q * EV + 1] = ffma2(hy2, v1, pb[q * EV + 1]);
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < E; c++) {
                    float ar, ai, br, bi;
                    unpack2(pa[c], ar, ai);
                    unpack2(pb[c], br, bi);
                    acc_s[2 * c] = ar - bi;
                    acc_s[2 * c + 1] = ai + br;
                }
            } else {
                row_product<T, E, HALF>(vb, vals, lid, C, len, rit, tl, acc_s);
            }
            if (p.init) {
#pragma unroll
                for (int q = 0; q < 2 * E; q++)
                    acc_s[q] *= Real(0.5);
            } else {
                cp_async_wait<0>();
#pragma unroll
                for (int q = 0; q < NP; q++) {
                    Real w[2 * EV];
                    lds_piece(wsm + 2 * (q * T * EV + tl * EV), w);
#pragma unroll
                    for (int i = 0; i < 2 * EV; i++)
                        acc_s[q * 2 * EV + i] -= w[i];
                }
            }
            store_owned<Real, T, E>(Wp, wbase, acc_s);
            // the row's own V entries: local position rit of the list
            if (p.dots) {
                const Real *ov = vb + (size_t)rit * 2 * RB;
#pragma unroll
                for (int q = 0; q < NP; q++) {
                    Real v[2 * EV];
                    lds_piece(ov + 2 * (q * T * EV + tl * EV), v);
#pragma unroll
                    for (int e = 0; e < EV; e++)
                        acc[q * EV + e].add(acc_s[q * 2 * EV + 2 * e],
                                            acc_s[q * 2 * EV + 2 * e + 1], v[2 * e],
                                            v[2 * e + 1]);
                }
                if ((k % kEtaFold) == kEtaFold - 1) {
#pragma unroll
                    for (int c = 0; c < E; c++)
                        acc[c].fold();
                }
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(empty0 + 8 * s);
        }
        if (!p.dots) {
            // no scalar products: nothing to write
        } else if (cur >= 0) {
            flush_eta<Real, T, E>(acc, red, tab[cur], slot, cw, n_cw);
        } else if (p.probs == nullptr) {
            // a single problem's partials are read for every block: a block
            // without chunks contributes zeros
            for (int t = cw * 32 + lane; t < 3 * RB; t += n_cw * 32)
                tab[0].partial[(int64_t)blockIdx.x * tab[0].ps + t * tab[0].qs] = 0.0;
        }
    }
}

}  // namespace

// (T, E) shapes of the staged kernel.  Complex float: 4 columns per lane
// as two 16-byte pieces (widths 8..64), or 2 as one piece (widths 8..32:
// twice the lanes per row, for more warps per SM).  Complex double: 2
// columns per lane as two pieces (widths 8..32; a 64-wide stage would not
// fit twice), each with and without the half-complex shortcut.
#define KPM_STAGED_SHAPES(X) X(2, 4) X(4, 4) X(8, 4) X(16, 4) X(4, 2) X(8, 2) X(16, 2)
#define KPM_STAGED_SHAPES64(X) X(4, 2) X(8, 2) X(16, 2)

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

bool staged_layout(int C, int T, int RB, int csize, int u_max, int l_max, int stages,
                   int n_probs, size_t max_smem, StagedLayout &o)
{
    auto up = [](uint64_t x, uint64_t a) { return (x + a - 1) / a * a; };
    if (C < 8 || T < 1 || RB < 1 || RB > 64 || (csize != 8 && csize != 16) || u_max < C ||
        l_max < 0 || stages < 1 || stages > 8 || n_probs < 1 || (C * T) % 32 != 0 ||
        32 + C * T > KPM_STAGED_MAX_THREADS)
        return false;
    const uint64_t row_bytes = (uint64_t)RB * csize;
    uint64_t off = up((uint64_t)u_max * row_bytes, 128);
    o.off_val = (uint32_t)off;
    off = up(off + (uint64_t)C * l_max * csize, 128);
    o.off_lidx = (uint32_t)off;
    off = up(off + (uint64_t)C * l_max * 2, 128);
    o.stage_bytes = (uint32_t)off;
    o.bar_bytes = (uint32_t)up(kTableOffset + (uint64_t)n_probs * sizeof(StagedProblem), 128);
    o.stages = stages;
    // after the stages: the block's W buffer, one slot per row of a chunk
    o.off_wbuf = (uint32_t)(o.bar_bytes + (uint64_t)stages * o.stage_bytes);
    o.smem = o.off_wbuf + (uint64_t)C * row_bytes;
    return o.smem <= max_smem && o.stage_bytes < (1u << 20);
}

namespace {

template <typename Real, int T, int E, bool IMAG, bool HALF>
int occupancy_of(int threads, size_t smem)
{
    int nb = 0;
    if (cudaFuncSetAttribute(aug_spmmv_staged_kernel<Real, T, E, IMAG, HALF>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, aug_spmmv_staged_kernel<Real, T, E, IMAG, HALF>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

// Launches one instantiation, raising its dynamic shared-memory limit the
// first time a launch needs more.
template <typename Real, int T, int E, bool IMAG, bool HALF>
int launch_one_staged(const StagedParams &p, int grid, int threads, size_t smem, cudaStream_t st)
{
    static size_t set = 0;
    if (set < smem) {
        if (cudaFuncSetAttribute(aug_spmmv_staged_kernel<Real, T, E, IMAG, HALF>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return KPM_ECUDA;
        set = smem;
    }
    aug_spmmv_staged_kernel<Real, T, E, IMAG, HALF><<<grid, threads, smem, st>>>(p);
    return cudaGetLastError() == cudaSuccess ? KPM_OK : KPM_ECUDA;
}

}  // namespace

int staged_max_blocks_per_sm(int T, int E, int C, size_t smem, bool fp64)
{
    const int threads = 32 + C * T;
#define KPM_CASE(T_, E_) \
    if (T == T_ && E == E_) \
        return occupancy_of<float, T_, E_, false, false>(threads, smem);
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

int launch_sweep_staged(const StagedParams &p, int T, int E, int grid, size_t smem, void *stream)
{
    const int threads = 32 + p.C * T;
    if (grid < 1 || threads > KPM_STAGED_MAX_THREADS || p.stages < 1 || p.stages > 8 ||
        p.n_probs < 1 || (p.probs == nullptr && p.n_probs != 1) || (p.half && !p.fp64))
        return KPM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
#define KPM_CASE(T_, E_)                                                                       \
    if (T == T_ && E == E_)                                                                    \
        return p.with_imag ? launch_one_staged<float, T_, E_, true, false>(p, grid, threads, smem, st) \
                           : launch_one_staged<float, T_, E_, false, false>(p, grid, threads, smem, st);
#define KPM_CASE64(T_, E_)                                                                     \
    if (T == T_ && E == E_) {                                                                  \
        if (p.half)                                                                            \
            return p.with_imag                                                                 \
                       ? launch_one_staged<double, T_, E_, true, true>(p, grid, threads, smem, st) \
                       : launch_one_staged<double, T_, E_, false, true>(p, grid, threads, smem, st); \
        return p.with_imag                                                                     \
                   ? launch_one_staged<double, T_, E_, true, false>(p, grid, threads, smem, st) \
                   : launch_one_staged<double, T_, E_, false, false>(p, grid, threads, smem, st); \
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
