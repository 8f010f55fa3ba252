// chem_selftest.cu -- diagnostics: the step kernel's own exp, logarithm and
// reciprocal evaluated next to CUDA's, and its split exponential and
// power-of-two scaling, so tests can bound their error and check their range
// handling.
#include <cuda_runtime.h>

#include <vector>

#include "../../include/chem.h"
#include "chem_handle.h"
#include "chem_kernel.cuh"

namespace chem {

__global__ void selftest_kernel(long long n, const double *x, const double *tab_g, double *y_exp,
                                double *y_exp_ref, double *y_rcp, double *y_rcp_ref) {
    const double *tab = tab_g;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    y_exp[i] = fexp(v, tab);
    y_exp_ref[i] = exp(v);
    y_rcp[i] = frcp(v);
    y_rcp_ref[i] = 1.0 / v;
}

__global__ void selftest_scaled_exp_kernel(long long n, const double *x, const double *tab, double *y_mant,
                                           int *y_pow, const double *v, const int *k, double *y_scaled) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double y;
    int p;
    split_exp(x[i], tab, y, p);
    y_mant[i] = y;
    y_pow[i] = p;
    y_scaled[i] = scale_pow2(v[i], k[i]);
}

// (flog's domain is x >= 2: see its comment)
__global__ void selftest_log_kernel(long long n, const double *x, const double2 *tab, double *y_log,
                                    double *y_log_ref) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    y_log[i] = flog(x[i], tab);
    y_log_ref[i] = log(x[i]);
}

}  // namespace chem

using namespace chem;

extern "C" int chem_selftest_log(int64_t n, const double *x, double *y_log, double *y_log_ref, void *stream) {
    if (n < 0 || !x || !y_log || !y_log_ref) return fail(CHEM_E_INVALID_ARG, "NULL argument");
    if (n == 0) return CHEM_OK;
    std::vector<double> tab;
    fill_log_table(tab);
    double *d_tab = nullptr;
    cudaError_t ce = cudaMalloc(&d_tab, sizeof(double) * tab.size());
    if (ce != cudaSuccess) return fail(CHEM_E_OOM, "self-test table");
    ce = cudaMemcpy(d_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) {
        selftest_log_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
            n, x, reinterpret_cast<const double2 *>(d_tab), y_log, y_log_ref);
        ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = cudaStreamSynchronize((cudaStream_t)stream);
    }
    cudaFree(d_tab);
    if (ce != cudaSuccess) return cuda_fail(ce, "self-test");
    return CHEM_OK;
}

static int upload_exp_table(double **d_tab) {
    std::vector<double> tab(kExpTab);
    for (int j = 0; j < kExpTab; ++j) tab[j] = (double)std::exp2l((long double)j / kExpTab);
    cudaError_t ce = cudaMalloc(d_tab, sizeof(double) * kExpTab);
    if (ce != cudaSuccess) return fail(CHEM_E_OOM, "self-test table");
    ce = cudaMemcpy(*d_tab, tab.data(), sizeof(double) * kExpTab, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        cudaFree(*d_tab);
        return cuda_fail(ce, "self-test table");
    }
    return CHEM_OK;
}

extern "C" int chem_selftest_scaled_exp(int64_t n, const double *x, double *y_mant, int32_t *y_pow, const double *v,
                                        const int32_t *k, double *y_scaled, void *stream) {
    if (n < 0 || !x || !y_mant || !y_pow || !v || !k || !y_scaled) return fail(CHEM_E_INVALID_ARG, "NULL argument");
    if (n == 0) return CHEM_OK;
    double *d_tab = nullptr;
    int rc = upload_exp_table(&d_tab);
    if (rc) return rc;
    selftest_scaled_exp_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        n, x, d_tab, y_mant, y_pow, v, k, y_scaled);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(d_tab);
    if (ce != cudaSuccess) return cuda_fail(ce, "self-test");
    return CHEM_OK;
}

extern "C" int chem_selftest_math(int64_t n, const double *x, double *y_exp, double *y_exp_ref, double *y_rcp,
                                  double *y_rcp_ref, void *stream) {
    if (n < 0 || !x || !y_exp || !y_exp_ref || !y_rcp || !y_rcp_ref)
        return fail(CHEM_E_INVALID_ARG, "NULL argument");
    if (n == 0) return CHEM_OK;
    std::vector<double> tab(kExpTab);
    for (int j = 0; j < kExpTab; ++j) tab[j] = (double)std::exp2l((long double)j / kExpTab);
    double *d_tab = nullptr;
    cudaError_t ce = cudaMalloc(&d_tab, sizeof(double) * kExpTab);
    if (ce != cudaSuccess) return fail(CHEM_E_OOM, "self-test table");
    ce = cudaMemcpy(d_tab, tab.data(), sizeof(double) * kExpTab, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) {
        selftest_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, x, d_tab, y_exp, y_exp_ref,
                                                                                      y_rcp, y_rcp_ref);
        ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = cudaStreamSynchronize((cudaStream_t)stream);
    }
    cudaFree(d_tab);
    if (ce != cudaSuccess) return cuda_fail(ce, "self-test");
    return CHEM_OK;
}
