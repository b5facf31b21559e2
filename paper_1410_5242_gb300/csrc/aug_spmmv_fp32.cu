// Instantiations and launcher of the aug_spmmv sweep for complex float
// storage (one translation unit per precision so they compile in parallel).
// The float form is bound by memory-level parallelism: 64 registers per
// thread (launched as 8 blocks of 4 warps per SM; blocks of up to 1024
// threads are allowed for the autotuner), pipelined index runs of 2
// entries and an L2 bulk prefetch one tile ahead measured best (0.32 ms
// per sweep at 64^3, R = 32).
#ifndef KPM_SWEEP_MAX_THREADS
#define KPM_SWEEP_MAX_THREADS 1024
#endif
#ifndef KPM_SWEEP_MIN_BLOCKS
#define KPM_SWEEP_MIN_BLOCKS 1
#endif
#ifndef KPM_SWEEP_INDEX_RUN
#define KPM_SWEEP_INDEX_RUN 2
#endif
#ifndef KPM_SWEEP_PREFETCH
#define KPM_SWEEP_PREFETCH 1
#endif
#ifndef KPM_SWEEP_MAX_L1
#define KPM_SWEEP_MAX_L1 0
#endif
#include "aug_spmmv.cuh"

namespace kpm {

int launch_sweep_fp32(const SweepParams &p, const LaunchShape &s, int grid, bool init,
                      void *stream)
{
    if (s.threads < 32 || s.threads > KPM_SWEEP_MAX_THREADS || (s.threads % 32) || grid < 1)
        return KPM_EINVAL;
    const size_t smem = sweep_smem_bytes<float>(s.threads, s.T * s.E);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
#define KPM_CASE(T_, E_)                                                                       \
    if (s.T == T_ && s.E == E_) {                                                              \
        if (KPM_SWEEP_MAX_L1) {                                                                \
            if (ensure_carveout_max_l1((const void *)aug_spmmv_kernel<float, T_, E_, false>) != \
                KPM_OK)                                                                        \
                return KPM_ECUDA;                                                              \
        }                                                                                      \
        if (p.with_imag)                                                                       \
            aug_spmmv_kernel<float, T_, E_, true><<<grid, s.threads, smem, st>>>(p, init ? 1 : 0);  \
        else                                                                                   \
            aug_spmmv_kernel<float, T_, E_, false><<<grid, s.threads, smem, st>>>(p, init ? 1 : 0); \
        return cudaGetLastError() == cudaSuccess ? KPM_OK : KPM_ECUDA;                         \
    }
    KPM_SHAPES_FP32(KPM_CASE)
#undef KPM_CASE
    return KPM_EUNSUPPORTED;
}

int launch_nodot_fp32(const SweepParams &p, const LaunchShape &s, int grid, bool init, void *stream)
{
    if (s.threads < 32 || s.threads > KPM_SWEEP_MAX_THREADS || (s.threads % 32) || grid < 1)
        return KPM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
#define KPM_CASE(T_, E_)                                                                       \
    if (s.T == T_ && s.E == E_) {                                                              \
        spmmv_nodot_kernel<float, T_, E_><<<grid, s.threads, 0, st>>>(p, init ? 1 : 0);           \
        return cudaGetLastError() == cudaSuccess ? KPM_OK : KPM_ECUDA;                         \
    }
    KPM_SHAPES_FP32(KPM_CASE)
#undef KPM_CASE
    return KPM_EUNSUPPORTED;
}

int sweep_max_blocks_per_sm_fp32(const LaunchShape &s)
{
    int nb = 0;
    if (s.threads < 32 || s.threads > KPM_SWEEP_MAX_THREADS || (s.threads % 32))
        return 0;
    const size_t smem = sweep_smem_bytes<float>(s.threads, s.T * s.E);
#define KPM_CASE(T_, E_)                                                                       \
    if (s.T == T_ && s.E == E_) {                                                              \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, aug_spmmv_kernel<float, T_, E_, false>, \
                                                          s.threads, smem) != cudaSuccess)    \
            return 0;                                                                          \
        return nb;                                                                             \
    }
    KPM_SHAPES_FP32(KPM_CASE)
#undef KPM_CASE
    return 0;
}

}  // namespace kpm
