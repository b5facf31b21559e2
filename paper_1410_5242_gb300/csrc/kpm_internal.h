// Internal declarations shared by the translation units of libkpm.
#pragma once

#include <cstdint>
#include <cstddef>

#include "kpm.h"

namespace kpm {

// Validates a CSR matrix (see kpm_gershgorin in kpm.h for the rules).
int validate_csr(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val_ri);
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

struct LaunchShape {
    int T, E, threads, blocks_per_sm, tile_groups;
};

// Launch one sweep of the given shape; grid = blocks_per_sm * n_sm.
// Returns KPM_EUNSUPPORTED for a (T, E) pair that is not instantiated.
int launch_sweep_fp64(const SweepParams &p, const LaunchShape &s, int grid, bool init,
                      void *stream);
int launch_sweep_fp32(const SweepParams &p, const LaunchShape &s, int grid, bool init,
                      void *stream);
// Occupancy query for the same kernels (blocks per SM, 0 if unsupported).
int sweep_max_blocks_per_sm(int precision, const LaunchShape &s, bool init);

}  // namespace kpm
