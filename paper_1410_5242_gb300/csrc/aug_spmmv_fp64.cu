// Instantiations and launcher of the aug_spmmv sweep for complex double
// storage (one translation unit per precision so they compile in parallel).
// The double form is bound by the FP64 pipe: more warps per SM and index
// runs of 4 measured best (3.7-3.9 ms per sweep at 64^3, R = 32).  The L2
// prefetch runs one tile ahead: two tiles were 0.3 % faster but evicted V
// rows before their last use (3.33 GB of DRAM traffic per sweep against
// 2.84 GB at one tile and 1.88 GB algorithmic).
#ifndef KPM_SWEEP_MAX_THREADS
#define KPM_SWEEP_MAX_THREADS 256
#endif
#ifndef KPM_SWEEP_MIN_BLOCKS
#define KPM_SWEEP_MIN_BLOCKS 3
#endif
#ifndef KPM_SWEEP_INDEX_RUN
#define KPM_SWEEP_INDEX_RUN 4
#endif
#ifndef KPM_SWEEP_PREFETCH
#define KPM_SWEEP_PREFETCH 1
#endif
#ifndef KPM_SWEEP_MAX_L1
#define KPM_SWEEP_MAX_L1 0
#endif
#include "aug_spmmv.cuh"

namespace kpm {

int launch_sweep_fp64(const SweepParams &p, const LaunchShape &s, int grid, bool init,
                      void *stream)
{
    if (s.threads < 32 || s.threads > KPM_SWEEP_MAX_THREADS || (s.threads % 32) || grid < 1)
        return KPM_EINVAL;
    const size_t smem = sweep_smem_bytes<double>(s.threads, s.T * s.E);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
#define KPM_CASE(T_, E_)                                                                       \
    if (s.T == T_ && s.E == E_) {                                                              \
        if (KPM_SWEEP_MAX_L1) {                                                                \
            if (ensure_carveout_max_l1((const void *)aug_spmmv_kernel<double, T_, E_, false>) != \
                KPM_OK)                                                                        \
                return KPM_ECUDA;                                                              \
        }                                                                                      \
        if (p.with_imag)                                                                       \
            aug_spmmv_kernel<double, T_, E_, true><<<grid, s.threads, smem, st>>>(p, init ? 1 : 0);  \
        else                                                                                   \
            aug_spmmv_kernel<double, T_, E_, false><<<grid, s.threads, smem, st>>>(p, init ? 1 : 0); \
        return cudaGetLastError() == cudaSuccess ? KPM_OK : KPM_ECUDA;                         \
    }
    KPM_SHAPES_FP64(KPM_CASE)
#undef KPM_CASE
    return KPM_EUNSUPPORTED;
}

int launch_nodot_fp64(const SweepParams &p, const LaunchShape &s, int grid, bool init, void *stream)
{
    if (s.threads < 32 || s.threads > KPM_SWEEP_MAX_THREADS || (s.threads % 32) || grid < 1)
        return KPM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
#define KPM_CASE(T_, E_)                                                                       \
    if (s.T == T_ && s.E == E_) {                                                              \
        spmmv_nodot_kernel<double, T_, E_><<<grid, s.threads, 0, st>>>(p, init ? 1 : 0);           \
        return cudaGetLastError() == cudaSuccess ? KPM_OK : KPM_ECUDA;                         \
    }
    KPM_SHAPES_FP64(KPM_CASE)
#undef KPM_CASE
    return KPM_EUNSUPPORTED;
}

int sweep_max_blocks_per_sm_fp64(const LaunchShape &s)
{
    int nb = 0;
    if (s.threads < 32 || s.threads > KPM_SWEEP_MAX_THREADS || (s.threads % 32))
        return 0;
    const size_t smem = sweep_smem_bytes<double>(s.threads, s.T * s.E);
#define KPM_CASE(T_, E_)                                                                       \
    if (s.T == T_ && s.E == E_) {                                                              \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, aug_spmmv_kernel<double, T_, E_, false>, \
                                                          s.threads, smem) != cudaSuccess)    \
            return 0;                                                                          \
        return nb;                                                                             \
    }
    KPM_SHAPES_FP64(KPM_CASE)
#undef KPM_CASE
    return 0;
}

}  // namespace kpm
