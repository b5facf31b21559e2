// Instantiations and launcher of the aug_spmmv sweep for complex double
// storage (one translation unit per precision so they compile in parallel).
#include "aug_spmmv.cuh"

namespace kpm {

int launch_sweep_fp64(const SweepParams &p, const LaunchShape &s, int grid, bool init,
                      void *stream)
{
    if (s.threads < 32 || s.threads > 512 || (s.threads % 32) || grid < 1)
        return KPM_EINVAL;
    const size_t smem = sweep_smem_bytes<double>(s.threads, s.T * s.E);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
#define KPM_CASE(T_, E_)                                                                       \
    if (s.T == T_ && s.E == E_) {                                                              \
        aug_spmmv_kernel<double, T_, E_><<<grid, s.threads, smem, st>>>(p, init ? 1 : 0);       \
        return cudaGetLastError() == cudaSuccess ? KPM_OK : KPM_ECUDA;                         \
    }
    KPM_SHAPES_FP64(KPM_CASE)
#undef KPM_CASE
    return KPM_EUNSUPPORTED;
}

int sweep_max_blocks_per_sm_fp64(const LaunchShape &s)
{
    int nb = 0;
    const size_t smem = sweep_smem_bytes<double>(s.threads, s.T * s.E);
#define KPM_CASE(T_, E_)                                                                       \
    if (s.T == T_ && s.E == E_) {                                                              \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, aug_spmmv_kernel<double, T_, E_>, \
                                                          s.threads, smem) != cudaSuccess)    \
            return 0;                                                                          \
        return nb;                                                                             \
    }
    KPM_SHAPES_FP64(KPM_CASE)
#undef KPM_CASE
    return 0;
}

}  // namespace kpm
