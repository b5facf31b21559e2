// The naive KPM-DOS algorithm of Fig. 3 built from library calls (cuSPARSE
// SpMV, cuBLAS level-1), the starting point of the paper's optimisation
// stages.  It runs one start vector after the other, each step as six
// separate calls over complex-double vectors, with the scalar products
// written to device memory (device pointer mode) so that nothing
// synchronises inside the loop.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusparse.h>

#include <cstring>
#include <new>

#include "kpm_internal.h"

using namespace kpm;

struct kpm_naive {
    int device = 0, n_sm = 1;
    int64_t n = 0, nnz = 0;
    double a = 0, b = 0;
    cusparseHandle_t sp = nullptr;
    cublasHandle_t bl = nullptr;
    int32_t *d_rowptr = nullptr, *d_col = nullptr;
    cuDoubleComplex *d_val = nullptr;
    cusparseSpMatDescr_t A = nullptr;
    cuDoubleComplex *d_v = nullptr, *d_w = nullptr, *d_u = nullptr;
    cusparseDnVecDescr_t dv = nullptr, dw = nullptr, du = nullptr;
    void *spmv_buf = nullptr;
    size_t spmv_bytes = 0;
    cuDoubleComplex *d_block = nullptr;  // start vectors [n][R]
    int block_R = 0;
    double *d_nrm = nullptr;             // [R][M/2]
    cuDoubleComplex *d_dot = nullptr;    // [R][M/2]
    int64_t scalars = 0;
};

namespace {

void naive_release(kpm_naive *nv)
{
    if (!nv)
        return;
    if (nv->A)
        cusparseDestroySpMat(nv->A);
    if (nv->dv)
        cusparseDestroyDnVec(nv->dv);
    if (nv->dw)
        cusparseDestroyDnVec(nv->dw);
    if (nv->du)
        cusparseDestroyDnVec(nv->du);
    if (nv->sp)
        cusparseDestroy(nv->sp);
    if (nv->bl)
        cublasDestroy(nv->bl);
    cudaFree(nv->d_rowptr);
    cudaFree(nv->d_col);
    cudaFree(nv->d_val);
    cudaFree(nv->d_v);
    cudaFree(nv->d_w);
    cudaFree(nv->d_u);
    cudaFree(nv->spmv_buf);
    cudaFree(nv->d_block);
    cudaFree(nv->d_nrm);
    cudaFree(nv->d_dot);
    delete nv;
}

// eta[r][2m] = nrm[r][m]^2, eta[r][2m+1] = Re dot[r][m]
__global__ void naive_eta_kernel(const double *nrm, const cuDoubleComplex *dot, int R, int half,
                                 double *eta)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= R * half)
        return;
    const int r = t / half, m = t % half;
    eta[(int64_t)r * 2 * half + 2 * m] = nrm[t] * nrm[t];
    eta[(int64_t)r * 2 * half + 2 * m + 1] = dot[t].x;
}

}  // namespace

extern "C" {

int kpm_naive_create(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val_ri,
                     double a, double b, int32_t device, kpm_naive **out)
{
    if (!out)
        return KPM_EINVAL;
    *out = nullptr;
    KPM_TRY(validate_csr(n, row_ptr, col, val_ri));
    if (!(a > 0.0) || row_ptr[n] > INT32_MAX)
        return KPM_EINVAL;
    kpm_naive *nv = new (std::nothrow) kpm_naive;
    if (!nv)
        return KPM_ENOMEM;
    nv->device = device;
    nv->n = n;
    nv->nnz = row_ptr[n];
    nv->a = a;
    nv->b = b;
    DeviceGuard guard(device);
    auto fail = [&](int rc) {
        naive_release(nv);
        return rc;
    };
    if (!guard.ok)
        return fail(KPM_ECUDA);
    cudaDeviceGetAttribute(&nv->n_sm, cudaDevAttrMultiProcessorCount, device);
    int32_t *rp32 = new (std::nothrow) int32_t[n + 1];
    if (!rp32)
        return fail(KPM_ENOMEM);
    for (int64_t i = 0; i <= n; i++)
        rp32[i] = (int32_t)row_ptr[i];
    const size_t vbytes = sizeof(cuDoubleComplex) * (size_t)n;
    bool ok = cudaMalloc(&nv->d_rowptr, sizeof(int32_t) * (n + 1)) == cudaSuccess &&
              cudaMalloc(&nv->d_col, sizeof(int32_t) * (nv->nnz ? nv->nnz : 1)) == cudaSuccess &&
              cudaMalloc(&nv->d_val, 16 * (nv->nnz ? nv->nnz : 1)) == cudaSuccess &&
              cudaMalloc(&nv->d_v, vbytes) == cudaSuccess &&
              cudaMalloc(&nv->d_w, vbytes) == cudaSuccess &&
              cudaMalloc(&nv->d_u, vbytes) == cudaSuccess;
    if (!ok) {
        delete[] rp32;
        cudaGetLastError();
        return fail(KPM_ENOMEM);
    }
    ok = cudaMemcpy(nv->d_rowptr, rp32, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemcpy(nv->d_col, col, sizeof(int32_t) * nv->nnz, cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemcpy(nv->d_val, val_ri, 16 * nv->nnz, cudaMemcpyHostToDevice) == cudaSuccess;
    delete[] rp32;
    if (!ok)
        return fail(KPM_ECUDA);
    if (cusparseCreate(&nv->sp) != CUSPARSE_STATUS_SUCCESS ||
        cublasCreate(&nv->bl) != CUBLAS_STATUS_SUCCESS)
        return fail(KPM_ECUDA);
    cublasSetPointerMode(nv->bl, CUBLAS_POINTER_MODE_DEVICE);
    if (cusparseCreateCsr(&nv->A, n, n, nv->nnz, nv->d_rowptr, nv->d_col, nv->d_val,
                          CUSPARSE_INDEX_32I, CUSPARSE_INDEX_32I, CUSPARSE_INDEX_BASE_ZERO,
                          CUDA_C_64F) != CUSPARSE_STATUS_SUCCESS ||
        cusparseCreateDnVec(&nv->dv, n, nv->d_v, CUDA_C_64F) != CUSPARSE_STATUS_SUCCESS ||
        cusparseCreateDnVec(&nv->dw, n, nv->d_w, CUDA_C_64F) != CUSPARSE_STATUS_SUCCESS ||
        cusparseCreateDnVec(&nv->du, n, nv->d_u, CUDA_C_64F) != CUSPARSE_STATUS_SUCCESS)
        return fail(KPM_ECUDA);
    const cuDoubleComplex one = {1.0, 0.0}, zero = {0.0, 0.0};
    if (cusparseSpMV_bufferSize(nv->sp, CUSPARSE_OPERATION_NON_TRANSPOSE, &one, nv->A, nv->dv,
                                &zero, nv->du, CUDA_C_64F, CUSPARSE_SPMV_ALG_DEFAULT,
                                &nv->spmv_bytes) != CUSPARSE_STATUS_SUCCESS)
        return fail(KPM_ECUDA);
    if (cudaMalloc(&nv->spmv_buf, nv->spmv_bytes ? nv->spmv_bytes : 16) != cudaSuccess)
        return fail(KPM_ENOMEM);
    *out = nv;
    return KPM_OK;
}

int kpm_naive_moments(kpm_naive *nv, int32_t M, int32_t R, uint64_t seed, double *eta_dev,
                      void *stream)
{
    if (!nv || M < 2 || (M & 1) || R < 1 || !eta_dev)
        return KPM_EINVAL;
    DeviceGuard guard(nv->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int half = M / 2;
    const int64_t n = nv->n;
    if (R > nv->block_R) {
        cudaFree(nv->d_block);
        nv->d_block = nullptr;
        nv->block_R = 0;
        if (cudaMalloc(&nv->d_block, sizeof(cuDoubleComplex) * n * R) != cudaSuccess)
            return KPM_ENOMEM;
        nv->block_R = R;
    }
    if ((int64_t)R * half > nv->scalars) {
        cudaFree(nv->d_nrm);
        cudaFree(nv->d_dot);
        nv->d_nrm = nullptr;
        nv->d_dot = nullptr;
        nv->scalars = 0;
        if (cudaMalloc(&nv->d_nrm, sizeof(double) * R * half) != cudaSuccess ||
            cudaMalloc(&nv->d_dot, sizeof(cuDoubleComplex) * R * half) != cudaSuccess)
            return KPM_ENOMEM;
        nv->scalars = (int64_t)R * half;
    }
    if (cusparseSetStream(nv->sp, st) != CUSPARSE_STATUS_SUCCESS ||
        cublasSetStream(nv->bl, st) != CUBLAS_STATUS_SUCCESS)
        return KPM_ECUDA;
    KPM_TRY(launch_phases_raw(nv->d_block, true, nullptr, n, n, R, R, seed, nv->n_sm, st));

    // constants the level-1 calls read through device pointers
    double *d_c = nullptr;
    if (cudaMallocAsync((void **)&d_c, sizeof(double) * 8, st) != cudaSuccess)
        return KPM_ENOMEM;
    const double host_c[8] = {-nv->b, 0.0, 2.0 * nv->a, 0.0, -1.0, nv->a, 0.0, 0.0};
    if (cudaMemcpyAsync(d_c, host_c, sizeof(host_c), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return KPM_ECUDA;
    const cuDoubleComplex *minus_b = (const cuDoubleComplex *)(d_c + 0);
    const cuDoubleComplex *two_a = (const cuDoubleComplex *)(d_c + 2);
    const double *minus_one = d_c + 4;
    const double *a_real = d_c + 5;
    const cuDoubleComplex one = {1.0, 0.0}, zero = {0.0, 0.0};
    int rc = KPM_OK;
    auto spmv = [&](cuDoubleComplex *x) {
        cusparseDnVecSetValues(nv->dv, x);
        return cusparseSpMV(nv->sp, CUSPARSE_OPERATION_NON_TRANSPOSE, &one, nv->A, nv->dv, &zero,
                            nv->du, CUDA_C_64F, CUSPARSE_SPMV_ALG_DEFAULT, nv->spmv_buf) ==
               CUSPARSE_STATUS_SUCCESS;
    };
    for (int r = 0; r < R && rc == KPM_OK; r++) {
        cuDoubleComplex *v = nv->d_v, *w = nv->d_w, *u = nv->d_u;
        bool ok = cublasZcopy(nv->bl, n, nv->d_block + r, R, v, 1) == CUBLAS_STATUS_SUCCESS;
        // initial step: w = a (H v - b v); eta_0 = <v|v>, eta_1 = <w|v>
        ok = ok && spmv(v);
        ok = ok && cublasZaxpy(nv->bl, n, minus_b, v, 1, u, 1) == CUBLAS_STATUS_SUCCESS;
        ok = ok && cublasZcopy(nv->bl, n, u, 1, w, 1) == CUBLAS_STATUS_SUCCESS;
        ok = ok && cublasZdscal(nv->bl, n, a_real, w, 1) == CUBLAS_STATUS_SUCCESS;
        ok = ok && cublasDznrm2(nv->bl, n, v, 1, nv->d_nrm + (int64_t)r * half) ==
                       CUBLAS_STATUS_SUCCESS;
        ok = ok && cublasZdotc(nv->bl, n, w, 1, v, 1, nv->d_dot + (int64_t)r * half) ==
                       CUBLAS_STATUS_SUCCESS;
        for (int m = 1; m < half && ok; m++) {
            cuDoubleComplex *t = v;  // swap(w, v)
            v = w;
            w = t;
            ok = spmv(v);                                                            // u = H v
            ok = ok && cublasZaxpy(nv->bl, n, minus_b, v, 1, u, 1) == CUBLAS_STATUS_SUCCESS;  // u -= b v
            ok = ok && cublasZdscal(nv->bl, n, minus_one, w, 1) == CUBLAS_STATUS_SUCCESS;     // w = -w
            ok = ok && cublasZaxpy(nv->bl, n, two_a, u, 1, w, 1) == CUBLAS_STATUS_SUCCESS;    // w += 2a u
            ok = ok && cublasDznrm2(nv->bl, n, v, 1, nv->d_nrm + (int64_t)r * half + m) ==
                           CUBLAS_STATUS_SUCCESS;                                            // |v|
            ok = ok && cublasZdotc(nv->bl, n, w, 1, v, 1, nv->d_dot + (int64_t)r * half + m) ==
                           CUBLAS_STATUS_SUCCESS;                                            // <w|v>
        }
        if (!ok)
            rc = KPM_ECUDA;
    }
    if (rc == KPM_OK) {
        const int threads = R * half;
        naive_eta_kernel<<<(threads + 255) / 256, 256, 0, st>>>(nv->d_nrm, nv->d_dot, R, half,
                                                                 eta_dev);
        rc = cuda_status(cudaGetLastError());
    }
    cudaFreeAsync(d_c, st);
    return rc;
}

void kpm_naive_destroy(kpm_naive *nv)
{
    if (!nv)
        return;
    DeviceGuard guard(nv->device);
    cudaDeviceSynchronize();
    naive_release(nv);
}

}  // extern "C"
