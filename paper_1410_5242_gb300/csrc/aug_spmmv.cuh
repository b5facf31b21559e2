// The fused augmented sparse-matrix multiple-vector product (aug_spmmv) of
// Fig. 5 for sm_103a.  One sweep computes, for every row i and every column
// r of a row-major block of width RB = T*E,
//     W_ir <- sum_j H'_ij V_jr - W_ir          (H' = 2a(H - b 1), folded)
//     (init: W_ir <- (1/2) sum_j H'_ij V_jr,   W not read)
// and accumulates <V|V>, Re<W|V>, Im<W|V> per column with the updated W.
//
// Thread mapping (Sec. "GPU Implementation": warps along block-vector rows so
// that the R columns load coalesced; the dot products are reduced with warp
// shuffles): a row is handled by a team of T lanes, lane t owning the E
// consecutive complex columns t*E .. t*E+E-1, so each lane moves 16 bytes
// (or 8 for one complex float) per access; a warp holds P = 32/T rows.
// Matrix values and column indices are read once per team (identical
// addresses within the team are one broadcast access) from SELL-C-sigma
// chunks stored column-major, so the P rows of a warp read adjacent entries.
//
// Work split: a block tile is nwarps * P * tile_groups consecutive rows;
// blocks stride over tiles, so all blocks sweep the matrix as one moving
// window and the neighbour rows of V each gather needs are recent in L2.
//
// eta: every lane accumulates over all rows it handles (double: plain FMA
// chains; float: each row's product pair is added error-free with Knuth's
// TwoSum into a (hi, lo) float pair).  At the end lanes of equal columns are
// combined by an xor butterfly (identical result on every lane, fixed
// order), warps through shared memory in warp order, and each block writes
// its [3][RB] partial in double.  Nothing depends on timing, so eta is
// bitwise reproducible for a fixed launch shape.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>

#include "kpm_internal.h"

namespace kpm {

#ifndef KPM_SWEEP_MAX_THREADS
#define KPM_SWEEP_MAX_THREADS 256
#endif
#ifndef KPM_SWEEP_INDEX_RUN
#define KPM_SWEEP_INDEX_RUN 4
#endif
#ifndef KPM_SWEEP_MIN_BLOCKS
#define KPM_SWEEP_MIN_BLOCKS 2
#endif
#ifndef KPM_SWEEP_PREFETCH
#define KPM_SWEEP_PREFETCH 1
#endif
#ifndef KPM_SWEEP_PIPELINE_INDEX
#define KPM_SWEEP_PIPELINE_INDEX 1
#endif


// ---------------------------------------------------------------- loads
// N reals from read-only memory as 16-byte (or one 8-byte) accesses.
template <typename Real, int N>
__device__ __forceinline__ void load_nc(const Real *__restrict__ p, Real (&out)[N])
{
    constexpr int bytes = N * (int)sizeof(Real);
    static_assert(bytes % 8 == 0, "vector access of 8 or 16k bytes");
    if constexpr (bytes % 16 == 0) {
        const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
        for (int i = 0; i < bytes / 16; i++) {
            uint4 u = __ldg(q + i);
            memcpy(reinterpret_cast<char *>(out) + 16 * i, &u, 16);
        }
    } else {
        uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
        memcpy(out, &u, 8);
    }
}

template <typename Real, int N>
__device__ __forceinline__ void load_rw(const Real *p, Real (&out)[N])
{
    constexpr int bytes = N * (int)sizeof(Real);
    if constexpr (bytes % 16 == 0) {
        const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
        for (int i = 0; i < bytes / 16; i++) {
            uint4 u = q[i];
            memcpy(reinterpret_cast<char *>(out) + 16 * i, &u, 16);
        }
    } else {
        uint2 u = *reinterpret_cast<const uint2 *>(p);
        memcpy(out, &u, 8);
    }
}

template <typename Real, int N>
__device__ __forceinline__ void store(Real *p, const Real (&in)[N])
{
    constexpr int bytes = N * (int)sizeof(Real);
    if constexpr (bytes % 16 == 0) {
        uint4 *q = reinterpret_cast<uint4 *>(p);
#pragma unroll
        for (int i = 0; i < bytes / 16; i++) {
            uint4 u;
            memcpy(&u, reinterpret_cast<const char *>(in) + 16 * i, 16);
            q[i] = u;
        }
    } else {
        uint2 u;
        memcpy(&u, in, 8);
        *reinterpret_cast<uint2 *>(p) = u;
    }
}

// Bulk prefetch of a contiguous range into L2 (a hint: no completion to
// wait for).  Start and size must be multiples of 16 bytes.
__device__ __forceinline__ void prefetch_l2(const void *ptr, uint64_t bytes)
{
    const char *p = static_cast<const char *>(ptr);
    while (bytes > 0) {
        const uint32_t n = bytes > (1u << 20) ? (1u << 20) : (uint32_t)bytes;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(n) : "memory");
        p += n;
        bytes -= n;
    }
}

// The streamed inputs of one block tile (rows [r0, r1)): the SELL entries
// of the chunks covering it, the old W rows and the tile's own V rows.
// Every range starts and ends on a multiple of 16 bytes: chunk offsets are
// multiples of C entries, and a block row holds ld complex numbers with ld
// even in the float form.
template <typename Real>
__device__ __forceinline__ void prefetch_tile(const SweepParams &p, int64_t tile,
                                              int64_t rows_per_tile, bool read_w)
{
    const int64_t r0 = tile * rows_per_tile;
    const int64_t r1 = min(p.n_pad, r0 + rows_per_tile);
    if (r0 >= r1)
        return;
    const int64_t e0 = __ldg(p.chunk_ptr + (r0 >> p.log2C));
    const int64_t e1 = __ldg(p.chunk_ptr + ((r1 - 1) >> p.log2C) + 1);
    constexpr int64_t cplx = 2 * (int64_t)sizeof(Real);
    if (e1 > e0) {
        prefetch_l2(static_cast<const char *>(p.val) + e0 * cplx, (e1 - e0) * cplx);
        if (((e0 | e1) & 3) == 0)
            prefetch_l2(p.col + e0, (e1 - e0) * 4);
    }
    const int64_t row_bytes = (int64_t)p.ld * cplx;
    if ((row_bytes & 15) == 0) {
        prefetch_l2(static_cast<const char *>(p.V) + r0 * row_bytes, (r1 - r0) * row_bytes);
        if (read_w)
            prefetch_l2(static_cast<const char *>(p.W) + r0 * row_bytes, (r1 - r0) * row_bytes);
    }
}

// ------------------------------------------------------ column ownership
// A lane owns E complex columns of its row as NP pieces of EV consecutive
// complex numbers (EV = 2 for complex float, so a piece is one 16-byte
// access; EV = 1 for complex double).  Piece k of team lane tl starts at
// column k*T*EV + tl*EV, so the T lanes of a team read one contiguous
// T*EV-column span per access: a row's 16-byte pieces are interleaved
// across the team instead of each lane owning a contiguous E-column run,
// which halves the cache lines one warp access touches.
template <typename Real, int E>
struct Pieces {
    static constexpr int EV = (sizeof(Real) == 4 && E % 2 == 0) ? 2 : 1;
    static constexpr int NP = E / EV;
};

// Column (within the block) of accumulator k of team lane tl.
template <typename Real, int T, int E>
__device__ __forceinline__ int owned_column(int tl, int k)
{
    constexpr int EV = Pieces<Real, E>::EV;
    return (k / EV) * T * EV + tl * EV + (k % EV);
}

// E complex numbers of a row whose pieces start at base (complex units),
// base + T*EV, ...; read-only and read-write variants, and the store.
template <typename Real, int T, int E>
__device__ __forceinline__ void load_owned_nc(const Real *__restrict__ p, int64_t base,
                                              Real (&out)[2 * E])
{
    constexpr int EV = Pieces<Real, E>::EV, NP = Pieces<Real, E>::NP;
#pragma unroll
    for (int k = 0; k < NP; k++) {
        Real piece[2 * EV];
        load_nc<Real, 2 * EV>(p + (base + (int64_t)k * T * EV) * 2, piece);
#pragma unroll
        for (int i = 0; i < 2 * EV; i++)
            out[k * 2 * EV + i] = piece[i];
    }
}

template <typename Real, int T, int E>
__device__ __forceinline__ void load_owned_rw(const Real *p, int64_t base, Real (&out)[2 * E])
{
    constexpr int EV = Pieces<Real, E>::EV, NP = Pieces<Real, E>::NP;
#pragma unroll
    for (int k = 0; k < NP; k++) {
        Real piece[2 * EV];
        load_rw<Real, 2 * EV>(p + (base + (int64_t)k * T * EV) * 2, piece);
#pragma unroll
        for (int i = 0; i < 2 * EV; i++)
            out[k * 2 * EV + i] = piece[i];
    }
}

template <typename Real, int T, int E>
__device__ __forceinline__ void store_owned(Real *p, int64_t base, const Real (&in)[2 * E])
{
    constexpr int EV = Pieces<Real, E>::EV, NP = Pieces<Real, E>::NP;
#pragma unroll
    for (int k = 0; k < NP; k++) {
        Real piece[2 * EV];
#pragma unroll
        for (int i = 0; i < 2 * EV; i++)
            piece[i] = in[k * 2 * EV + i];
        store<Real, 2 * EV>(p + (base + (int64_t)k * T * EV) * 2, piece);
    }
}

// ------------------------------------------------------- eta accumulation
// IMAG: also accumulate Im<W|V> (only needed for the Hermiticity check).
template <typename Real, bool IMAG>
struct EtaAcc;

template <bool IMAG>
struct EtaAcc<double, IMAG> {
    double vv = 0.0, wv = 0.0, wvi = 0.0;
    __device__ __forceinline__ void add(double wr, double wi, double vr, double vi)
    {
        vv = fma(vr, vr, vv);
        vv = fma(vi, vi, vv);
        wv = fma(wr, vr, wv);
        wv = fma(wi, vi, wv);
        if constexpr (IMAG) {
            wvi = fma(wr, vi, wvi);
            wvi = fma(-wi, vr, wvi);
        }
    }
    __device__ __forceinline__ double get(int k) const
    {
        return k == 0 ? vv : (k == 1 ? wv : (IMAG ? wvi : 0.0));
    }
};

// (hi, lo) += p without rounding loss in the running sum: Knuth's TwoSum
// gives hi + p = s + e exactly; e goes to the low word.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float p)
{
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float ap = __fsub_rn(s, bp);
    const float e = __fadd_rn(__fsub_rn(hi, ap), __fsub_rn(p, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

template <bool IMAG>
struct EtaAcc<float, IMAG> {
    float vv_h = 0.f, vv_l = 0.f, wv_h = 0.f, wv_l = 0.f, wvi_h = 0.f, wvi_l = 0.f;
    __device__ __forceinline__ void add(float wr, float wi, float vr, float vi)
    {
        two_sum_acc(vv_h, vv_l, __fmaf_rn(vr, vr, __fmul_rn(vi, vi)));
        two_sum_acc(wv_h, wv_l, __fmaf_rn(wr, vr, __fmul_rn(wi, vi)));
        if constexpr (IMAG)
            two_sum_acc(wvi_h, wvi_l, __fmaf_rn(wr, vi, -__fmul_rn(wi, vr)));
    }
    __device__ __forceinline__ double get(int k) const
    {
        if (k == 0)
            return (double)vv_h + (double)vv_l;
        if (k == 1)
            return (double)wv_h + (double)wv_l;
        return IMAG ? (double)wvi_h + (double)wvi_l : 0.0;
    }
};

// ------------------------------------------------------------------ one row
// W row <- H' V - W (or (1/2) H' V when init) for this lane's E owned
// columns (pieces from column cbase on, see owned_column), and this row's
// terms of the scalar products (DOTS = false leaves them out: the ablation
// variants of the paper's GPU model, augmented SpMMV without dot products
// and plain SpMMV).
template <typename Real, int T, int E, bool IMAG, bool DOTS = true>
__device__ __forceinline__ void sweep_row(const SweepParams &p, const Real *__restrict__ val,
                                          const Real *__restrict__ V, Real *W, int64_t row,
                                          int init, int64_t cbase, EtaAcc<Real, IMAG> (&acc)[E])
{
    constexpr int NC = KPM_SWEEP_INDEX_RUN;  // entries whose indices are fetched together
    const int Cmask = (1 << p.log2C) - 1;
    const int64_t ch = row >> p.log2C;
    const int64_t e0 = __ldg(p.chunk_ptr + ch) + (row & Cmask);
    const int len = __ldg(p.chunk_len + ch);
    const int64_t wbase = row * p.ld + cbase;

    // the old W first (not read by the initial sweep): it is independent of
    // the gathers and its latency overlaps theirs
    Real s[2 * E];
    if (init) {
#pragma unroll
        for (int k = 0; k < 2 * E; k++)
            s[k] = Real(0);
    } else {
        load_owned_rw<Real, T, E>(W, wbase, s);
#pragma unroll
        for (int k = 0; k < 2 * E; k++)
            s[k] = -s[k];
    }
    // Entries in runs of NC: all column indices of a run are fetched first
    // (one memory latency), then the run's gathers, whose loads are in
    // flight together.  The indices of the next run are requested before
    // the gathers of the current one, so that their latencies overlap.
    const int64_t C = (int64_t)Cmask + 1;
    int cj[NC];
#pragma unroll
    for (int q = 0; q < NC; q++)
        cj[q] = q < len ? __ldg(p.col + e0 + (int64_t)q * C) : 0;
    for (int j0 = 0; j0 < len; j0 += NC) {
        const int nb = min(NC, len - j0);
        const int64_t eb = e0 + (int64_t)j0 * C;
        int cn[NC];
        if constexpr (KPM_SWEEP_PIPELINE_INDEX) {
#pragma unroll
            for (int q = 0; q < NC; q++)
                cn[q] = j0 + NC + q < len ? __ldg(p.col + eb + (int64_t)(NC + q) * C) : 0;
        }
#pragma unroll
        for (int q = 0; q < NC; q++) {
            if (q < nb) {
                Real h[2];
                load_nc<Real, 2>(val + 2 * (eb + (int64_t)q * C), h);
                Real v[2 * E];
                load_owned_nc<Real, T, E>(V, (int64_t)cj[q] * p.ld + cbase, v);
#pragma unroll
                for (int k = 0; k < E; k++) {
                    s[2 * k] = fma(h[0], v[2 * k], s[2 * k]);
                    s[2 * k] = fma(-h[1], v[2 * k + 1], s[2 * k]);
                    s[2 * k + 1] = fma(h[0], v[2 * k + 1], s[2 * k + 1]);
                    s[2 * k + 1] = fma(h[1], v[2 * k], s[2 * k + 1]);
                }
            }
        }
        if constexpr (KPM_SWEEP_PIPELINE_INDEX) {
#pragma unroll
            for (int q = 0; q < NC; q++)
                cj[q] = cn[q];
        } else if (j0 + NC < len) {
#pragma unroll
            for (int q = 0; q < NC; q++)
                cj[q] = j0 + NC + q < len ? __ldg(p.col + eb + (int64_t)(NC + q) * C) : 0;
        }
    }
    if (init) {
#pragma unroll
        for (int k = 0; k < 2 * E; k++)
            s[k] *= Real(0.5);
    }
    store_owned<Real, T, E>(W, wbase, s);
    if constexpr (DOTS) {
        // the row's own V entries (recently touched by the diagonal gather)
        Real vs[2 * E];
        load_owned_nc<Real, T, E>(V, wbase, vs);
#pragma unroll
        for (int k = 0; k < E; k++)
            acc[k].add(s[2 * k], s[2 * k + 1], vs[2 * k], vs[2 * k + 1]);
    }
}

// Block-wide sum of every lane's eta terms per column in a fixed order:
// lanes of equal columns by an xor butterfly (the same result on every
// lane), then warps in warp order through shared memory.  The sum for
// (quantity q, column r) is stored to dst[(q * RB + r) * stride].  red
// holds nwarps * 3 * RB doubles; the caller synchronises before reusing it.
template <typename Real, int T, int E, bool IMAG>
__device__ __forceinline__ void block_eta_sum(const EtaAcc<Real, IMAG> (&acc)[E], double *red,
                                              double *dst, int64_t stride)
{
    constexpr int RB = T * E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
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
    if (team == 0) {
#pragma unroll
        for (int q = 0; q < 3; q++)
#pragma unroll
            for (int k = 0; k < E; k++)
                red[(warp * 3 + q) * RB + owned_column<Real, T, E>(tl, k)] = out[q * E + k];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * RB; t += blockDim.x) {
        double sum = 0.0;
        for (int w = 0; w < nwarps; w++)
            sum += red[w * 3 * RB + t];
        dst[t * stride] = sum;
    }
}

// ------------------------------------------------------------------ kernel
template <typename Real, int T, int E, bool IMAG>
__global__ void __launch_bounds__(KPM_SWEEP_MAX_THREADS, KPM_SWEEP_MIN_BLOCKS)
    aug_spmmv_kernel(const SweepParams p, const int init)
{
    static_assert(T >= 1 && T <= 32 && (32 % T) == 0, "team size divides the warp");
    constexpr int P = 32 / T;   // rows per warp
    constexpr int RB = T * E;   // columns of this block
    extern __shared__ double red_smem[];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int tl = lane % T;
    const int team = lane / T;
    const int64_t cbase = (int64_t)p.col0 + tl * Pieces<Real, E>::EV;
    const Real *__restrict__ val = static_cast<const Real *>(p.val);
    const Real *__restrict__ V = static_cast<const Real *>(p.V);
    Real *W = static_cast<Real *>(p.W);
    EtaAcc<Real, IMAG> acc[E];

    const int64_t rows_per_tile = (int64_t)nwarps * P * p.tile_groups;
    const int64_t n_tiles = (p.n_pad + rows_per_tile - 1) / rows_per_tile;
    // One thread keeps the next KPM_SWEEP_PREFETCH tiles of this block
    // requested in L2, so that the threads' own loads of the streamed data
    // (matrix, old W, own V rows) are L2 hits rather than DRAM round trips.
    constexpr int D = KPM_SWEEP_PREFETCH;
    if (D > 0 && threadIdx.x == 0)
        for (int k = 0; k < D; k++)
            prefetch_tile<Real>(p, blockIdx.x + (int64_t)k * gridDim.x, rows_per_tile, !init);
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        if (D > 0 && threadIdx.x == 0)
            prefetch_tile<Real>(p, tile + (int64_t)D * gridDim.x, rows_per_tile, !init);
        for (int g = 0; g < p.tile_groups; g++) {
            const int64_t row = tile * rows_per_tile + ((int64_t)g * nwarps + warp) * P + team;
            if (row >= p.n_pad)
                continue;
            sweep_row<Real, T, E, IMAG>(p, val, V, W, row, init, cbase, acc);
        }
    }

    block_eta_sum<Real, T, E, IMAG>(acc, red_smem, p.partial + (int64_t)blockIdx.x * 3 * RB, 1);
}

// The sweep without the scalar products (ablation variants): the same
// loop and prefetching as aug_spmmv_kernel, no eta accumulation or
// reduction.  init = 1 gives plain SpMMV (W <- (1/2) H' V, W not read),
// init = 0 the augmented SpMMV without dots (W <- H' V - W).
template <typename Real, int T, int E>
__global__ void __launch_bounds__(KPM_SWEEP_MAX_THREADS, KPM_SWEEP_MIN_BLOCKS)
    spmmv_nodot_kernel(const SweepParams p, const int init)
{
    constexpr int P = 32 / T;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int tl = lane % T;
    const int team = lane / T;
    const int64_t cbase = (int64_t)p.col0 + tl * Pieces<Real, E>::EV;
    const Real *__restrict__ val = static_cast<const Real *>(p.val);
    const Real *__restrict__ V = static_cast<const Real *>(p.V);
    Real *W = static_cast<Real *>(p.W);
    EtaAcc<Real, false> acc[E];
    const int64_t rows_per_tile = (int64_t)nwarps * P * p.tile_groups;
    const int64_t n_tiles = (p.n_pad + rows_per_tile - 1) / rows_per_tile;
    constexpr int D = KPM_SWEEP_PREFETCH;
    if (D > 0 && threadIdx.x == 0)
        for (int k = 0; k < D; k++)
            prefetch_tile<Real>(p, blockIdx.x + (int64_t)k * gridDim.x, rows_per_tile, !init);
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        if (D > 0 && threadIdx.x == 0)
            prefetch_tile<Real>(p, tile + (int64_t)D * gridDim.x, rows_per_tile, !init);
        for (int g = 0; g < p.tile_groups; g++) {
            const int64_t row = tile * rows_per_tile + ((int64_t)g * nwarps + warp) * P + team;
            if (row >= p.n_pad)
                continue;
            sweep_row<Real, T, E, false, false>(p, val, V, W, row, init, cbase, acc);
        }
    }
}

// Instantiated (T, E) shapes; X(T, E) is expanded for each.
#define KPM_SHAPES_FP64(X) \
    X(1, 1) X(2, 1) X(4, 1) X(8, 1) X(16, 1) X(32, 1) X(1, 2) X(2, 2) X(4, 2) X(8, 2) X(16, 2) X(32, 2)
#define KPM_SHAPES_FP32(X)                                                                     \
    X(1, 1) X(2, 1) X(1, 2) X(2, 2) X(4, 2) X(8, 2) X(16, 2) X(32, 2) X(1, 4) X(2, 4) X(4, 4) \
        X(8, 4) X(16, 4)

template <typename Real>
inline size_t sweep_smem_bytes(int threads, int RB)
{
    return (size_t)(threads / 32) * 3 * RB * sizeof(double);
}

}  // namespace kpm
