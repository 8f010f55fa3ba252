// chem_lu.cu -- batched dense solves A x = b, the kinetics-only experiment of
// Sec. 5.2 (Gaussian elimination over many independent systems of size N_s).
//
// Two kernels, both Gaussian elimination with row partial pivoting (ties to
// the lowest row) in FP64, with every arithmetic step of the factorisation
// explicitly rounded and performed in the order of the plain definition
// (multiplier a_ij / a_jj, update a_ik - l a_jk without contraction), so
// factors and pivots are bit-identical to a scalar elimination:
//   * global   one thread per system, the matrices in HBM in the
//              system-interleaved layout A[(i n + j) n_sys + k] (the paper's
//              approach 1: coalesced across threads, every elimination step
//              reads and writes the trailing matrix in HBM);
//   * on-chip  one warp per system, the matrix staged in shared memory once
//              from the contiguous layout A[k][i][j]; the trailing updates
//              and the substitutions are spread over the 32 lanes, HBM sees
//              the matrix once each way.  The back substitution runs by
//              columns, so its x equals the scalar solve to rounding.
#include <cuda_runtime.h>

#include "../../include/chem.h"
#include "chem_handle.h"

namespace chem {

__global__ void lu_global_kernel(int n, long long ns, double *A, double *b, int *piv, int *info) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= ns) return;
    auto a = [&](int i, int j) -> double & { return A[((size_t)i * n + j) * ns + k]; };
    int bad = 0;
    for (int j = 0; j < n; ++j) {
        int p = j;
        double amax = fabs(a(j, j));
        for (int i = j + 1; i < n; ++i) {
            const double v = fabs(a(i, j));
            if (v > amax) {
                amax = v;
                p = i;
            }
        }
        if (piv) piv[(size_t)k * n + j] = p;
        if (!(amax > 0.0) || isinf(amax)) {
            if (!bad) bad = j + 1;
        }
        if (p != j) {
            for (int c = 0; c < n; ++c) {
                const double t = a(j, c);
                a(j, c) = a(p, c);
                a(p, c) = t;
            }
            const double t = b[(size_t)j * ns + k];
            b[(size_t)j * ns + k] = b[(size_t)p * ns + k];
            b[(size_t)p * ns + k] = t;
        }
        const double d = a(j, j);
        for (int i = j + 1; i < n; ++i) {
            const double l = __ddiv_rn(a(i, j), d);
            a(i, j) = l;
            for (int c = j + 1; c < n; ++c) a(i, c) = __dsub_rn(a(i, c), __dmul_rn(l, a(j, c)));
        }
    }
    // forward (unit L) and back substitution, row by row
    for (int i = 0; i < n; ++i) {
        double s = b[(size_t)i * ns + k];
        for (int j = 0; j < i; ++j) s = __dsub_rn(s, __dmul_rn(a(i, j), b[(size_t)j * ns + k]));
        b[(size_t)i * ns + k] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[(size_t)i * ns + k];
        for (int j = i + 1; j < n; ++j) s = __dsub_rn(s, __dmul_rn(a(i, j), b[(size_t)j * ns + k]));
        b[(size_t)i * ns + k] = __ddiv_rn(s, a(i, i));
    }
    if (info) info[k] = bad;
}

__global__ void __launch_bounds__(256) lu_onchip_kernel(int n, long long ns, double *A, double *b, int *piv,
                                                         int *info) {
    extern __shared__ __align__(16) double sm_lu[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    double *M = sm_lu + (size_t)warp * ((size_t)n * n + n);
    double *x = M + (size_t)n * n;
    for (long long k = (long long)blockIdx.x * wpb + warp; k < ns; k += (long long)gridDim.x * wpb) {
        const double *Ak = A + (size_t)k * n * n;
        for (int e = lane; e < n * n; e += 32) M[e] = Ak[e];
        for (int e = lane; e < n; e += 32) x[e] = b[(size_t)k * n + e];
        __syncwarp();
        int bad = 0;
        for (int j = 0; j < n; ++j) {
            // pivot: max |a_ij| over i >= j, lowest row on ties (integer keys)
            unsigned long long best = 0;
            int bi = n;
            for (int i = j + lane; i < n; i += 32) {
                unsigned long long key = (unsigned long long)__double_as_longlong(M[i * n + j]) & 0x7fffffffffffffffULL;
                if (key > 0x7ff0000000000000ULL) key = 0;   // NaN is never the pivot
                if (bi == n || key > best) {
                    best = key;
                    bi = i;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, best, o);
                const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
                if (k2 > best || (k2 == best && i2 < bi)) {
                    best = k2;
                    bi = i2;
                }
            }
            if (lane == 0 && piv) piv[(size_t)k * n + j] = bi;
            if ((best == 0 || best >= 0x7ff0000000000000ULL) && !bad) bad = j + 1;
            if (bi != j) {
                for (int c = lane; c < n; c += 32) {
                    const double t = M[j * n + c];
                    M[j * n + c] = M[bi * n + c];
                    M[bi * n + c] = t;
                }
                if (lane == 0) {
                    const double t = x[j];
                    x[j] = x[bi];
                    x[bi] = t;
                }
            }
            __syncwarp();
            const double d = M[j * n + j];
            for (int i = j + 1 + lane; i < n; i += 32) M[i * n + j] = __ddiv_rn(M[i * n + j], d);
            __syncwarp();
            const int cols = n - j - 1;
            const int tot = (n - j - 1) * cols;
            for (int e = lane; e < tot; e += 32) {
                const int i = j + 1 + e / cols, c = j + 1 + e % cols;
                M[i * n + c] = __dsub_rn(M[i * n + c], __dmul_rn(M[i * n + j], M[j * n + c]));
            }
            __syncwarp();
        }
        // forward substitution by columns: every x_i still receives its
        // updates in increasing j, the scalar order
        for (int j = 0; j < n; ++j) {
            const double xj = x[j];
            for (int i = j + 1 + lane; i < n; i += 32) x[i] = __dsub_rn(x[i], __dmul_rn(M[i * n + j], xj));
            __syncwarp();
        }
        // back substitution by columns (updates arrive in decreasing j, so x
        // matches the scalar solve to rounding, not bit for bit)
        for (int j = n - 1; j >= 0; --j) {
            const double xj = __ddiv_rn(x[j], M[j * n + j]);
            __syncwarp();
            if (lane == 0) x[j] = xj;
            for (int i = lane; i < j; i += 32) x[i] = __dsub_rn(x[i], __dmul_rn(M[i * n + j], xj));
            __syncwarp();
        }
        double *Ao = A + (size_t)k * n * n;
        for (int e = lane; e < n * n; e += 32) Ao[e] = M[e];
        for (int e = lane; e < n; e += 32) b[(size_t)k * n + e] = x[e];
        if (lane == 0 && info) info[k] = bad;
        __syncwarp();
    }
}

}  // namespace chem

using namespace chem;

extern "C" int chem_batched_solve(int32_t method, int32_t n, int64_t n_sys, double *A, double *b, int32_t *pivots,
                                  int32_t *info, void *stream) {
    if (n < 1 || n > CHEM_LU_MAX_N || n_sys < 0 || !A || !b)
        return fail(CHEM_E_INVALID_ARG, "batched solve: n %d, n_sys %lld", n, (long long)n_sys);
    if (n_sys == 0) return CHEM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (method == CHEM_LU_GLOBAL) {
        const int bs = 128;
        lu_global_kernel<<<(unsigned)((n_sys + bs - 1) / bs), bs, 0, st>>>(n, n_sys, A, b, pivots, info);
    } else if (method == CHEM_LU_ONCHIP) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const size_t per = ((size_t)n * n + n) * sizeof(double);
        int wpb = 8;
        while (wpb > 1 && per * wpb > (size_t)optin) wpb >>= 1;
        if (per * wpb > (size_t)optin)
            return fail(CHEM_E_UNSUPPORTED, "on-chip solve: an %dx%d system (%zu bytes) exceeds shared memory", n, n,
                        per);
        cudaError_t ce = cudaFuncSetAttribute(lu_onchip_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaFuncSetAttribute");
        int blocks = 0;
        ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, lu_onchip_kernel, wpb * 32, per * wpb);
        if (ce != cudaSuccess || blocks < 1) return cuda_fail(ce, "occupancy of the on-chip solve");
        long long grid = (long long)blocks * sms;
        const long long need = (n_sys + wpb - 1) / wpb;
        if (grid > need) grid = need;
        lu_onchip_kernel<<<(unsigned)grid, wpb * 32, per * wpb, st>>>(n, n_sys, A, b, pivots, info);
    } else {
        return fail(CHEM_E_INVALID_ARG, "batched solve: method %d", method);
    }
    const cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "batched solve launch");
    return CHEM_OK;
}
