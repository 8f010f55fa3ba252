// chem_lu.cu -- batched dense solves A x = b, the kinetics-only experiment of
// Sec. 5.2 (Gaussian elimination over many independent systems of size N_s).
//
// Two kernels, both Gaussian elimination with row partial pivoting (ties to
// the lowest row) in FP64, with every arithmetic step of the factorisation
// explicitly rounded and performed in the order of the plain definition
// (multiplier a_ij / a_jj, update a_ik - l a_jk without contraction), so
// factors and pivots are bit-identical to a scalar elimination:
//   * global   the matrices in HBM in the system-interleaved layout
//              A[(i n + j) n_sys + k] (the paper's approach 1: coalesced
//              across threads, every elimination step reads and writes the
//              trailing matrix in HBM).  With many systems one thread per
//              system; with few (fewer than fill the SMs), a block of R
//              warps per 32 systems, the trailing rows of each step spread
//              over the R warps, so that enough warps are in flight;
//   * on-chip  one warp per system, the matrix staged in shared memory once
//              from the contiguous layout A[k][i][j]; the trailing updates
//              and the substitutions are spread over the 32 lanes, HBM sees
//              the matrix once each way.  The back substitution runs by
//              columns, so its x equals the scalar solve to rounding.
#include <cuda_runtime.h>

#include "../../include/chem.h"
#include "chem_handle.h"

namespace chem {

// |v| as an ordered integer key; a NaN maps to 0 so it is never the pivot
// (max |a_ij| by the keys is the elimination's pivot, lowest row on ties)
__device__ __forceinline__ unsigned long long lu_key(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
    return b > 0x7ff0000000000000ULL ? 0ULL : b;
}
// The diagonal's key: the search starts from |a_jj| and takes a row only if
// its |a_ij| is larger, so a NaN diagonal (which no comparison exceeds) stays
// the pivot, and the column counts as singular, as in a plain elimination
__device__ __forceinline__ unsigned long long lu_key_diag(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
    return b > 0x7ff0000000000000ULL ? ~0ULL : b;
}

// s - l a, either rounded twice in the plain order (bit-identical to a scalar
// elimination) or contracted to one fused multiply-add (FMA = true)
template <bool FMA>
__device__ __forceinline__ double lu_axpy(double s, double l, double a) {
    return FMA ? __fma_rn(-l, a, s) : __dsub_rn(s, __dmul_rn(l, a));
}

// Forward (unit L) and back substitution of system k, row by row.
template <bool FMA>
__device__ __forceinline__ void lu_global_solve(int n, long long ns, long long k, const double *A, double *b) {
    auto a = [&](int i, int j) -> double { return A[((size_t)i * n + j) * ns + k]; };
    for (int i = 0; i < n; ++i) {
        double s = b[(size_t)i * ns + k];
        for (int j = 0; j < i; ++j) s = lu_axpy<FMA>(s, a(i, j), b[(size_t)j * ns + k]);
        b[(size_t)i * ns + k] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[(size_t)i * ns + k];
        for (int j = i + 1; j < n; ++j) s = lu_axpy<FMA>(s, a(i, j), b[(size_t)j * ns + k]);
        b[(size_t)i * ns + k] = __ddiv_rn(s, a(i, i));
    }
}

// Row update r_i[c] -= l r_j[c] for c in [c0, n) of one system (columns
// `ns` doubles apart).  Rows i and j differ, so each chunk's loads are issued
// together before its stores: kLuChunk loads of each row in flight per thread
// instead of one dependent load-store pair per column.
constexpr int kLuChunk = 4;
template <bool FMA>
__device__ __forceinline__ void lu_row_update(double *ri, const double *rj, double l, int c0, int n, long long ns) {
    int c = c0;
    for (; c + kLuChunk <= n; c += kLuChunk) {
        double x[kLuChunk], y[kLuChunk];
#pragma unroll
        for (int u = 0; u < kLuChunk; ++u) {
            x[u] = ri[(size_t)(c + u) * ns];
            y[u] = rj[(size_t)(c + u) * ns];
        }
#pragma unroll
        for (int u = 0; u < kLuChunk; ++u) ri[(size_t)(c + u) * ns] = lu_axpy<FMA>(x[u], l, y[u]);
    }
    for (; c < n; ++c) ri[(size_t)c * ns] = lu_axpy<FMA>(ri[(size_t)c * ns], l, rj[(size_t)c * ns]);
}

// Exchange of rows j and p (distinct) of one system over the columns
// c0, c0 + step, ... below n, a chunk of loads before its stores.
__device__ __forceinline__ void lu_row_swap(double *rj, double *rp, int c0, int step, int n, long long ns) {
    for (int c = c0; c < n; c += kLuChunk * step) {
        double x[kLuChunk], y[kLuChunk];
#pragma unroll
        for (int u = 0; u < kLuChunk; ++u) {
            const int cu = c + u * step;
            if (cu < n) {
                x[u] = rj[(size_t)cu * ns];
                y[u] = rp[(size_t)cu * ns];
            }
        }
#pragma unroll
        for (int u = 0; u < kLuChunk; ++u) {
            const int cu = c + u * step;
            if (cu < n) {
                rj[(size_t)cu * ns] = y[u];
                rp[(size_t)cu * ns] = x[u];
            }
        }
    }
}

// Multipliers of step j: l_ij = a_ij / a_jj, or, contracted, a_ij times one
// reciprocal of the pivot per column (a correctly rounded FP64 division)
template <bool FMA>
struct LuPivot {
    double d;
    __device__ __forceinline__ explicit LuPivot(double djj) : d(FMA ? 1.0 / djj : djj) {}
    __device__ __forceinline__ double mult(double aij) const { return FMA ? __dmul_rn(aij, d) : __ddiv_rn(aij, d); }
};

template <bool FMA>
__global__ void lu_global_kernel(int n, long long ns, double *A, double *b, int *piv, int *info) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= ns) return;
    auto a = [&](int i, int j) -> double & { return A[((size_t)i * n + j) * ns + k]; };
    int bad = 0;
    for (int j = 0; j < n; ++j) {
        int p = j;
        unsigned long long best = lu_key_diag(a(j, j));
        for (int i = j + 1; i < n; ++i) {
            const unsigned long long key = lu_key(a(i, j));
            if (key > best) {
                best = key;
                p = i;
            }
        }
        if (piv) piv[(size_t)k * n + j] = p;
        if (best == 0 || best >= 0x7ff0000000000000ULL) {
            if (!bad) bad = j + 1;
        }
        if (p != j) {
            lu_row_swap(&a(j, 0), &a(p, 0), 0, 1, n, ns);
            const double t = b[(size_t)j * ns + k];
            b[(size_t)j * ns + k] = b[(size_t)p * ns + k];
            b[(size_t)p * ns + k] = t;
        }
        const LuPivot<FMA> d(a(j, j));
        for (int i = j + 1; i < n; ++i) {
            const double l = d.mult(a(i, j));
            a(i, j) = l;
            lu_row_update<FMA>(&a(i, 0), &a(j, 0), l, j + 1, n, ns);
        }
    }
    lu_global_solve<FMA>(n, ns, k, A, b);
    if (info) info[k] = bad;
}

// The same elimination, element by element, with a block of R warps per 32
// consecutive systems (lane = system): in each step every warp scans its
// share of the pivot column, the shares' maxima meet in shared memory, the
// R warps swap the pivot row's columns between them, and each warp updates
// its trailing rows (row j + 1 + w, j + 1 + w + R, ...).  The substitutions
// run in warp 0, row by row.
template <int R, bool FMA>
__global__ void __maxnreg__(80) lu_global_rows_kernel(int n, long long ns, double *A, double *b, int *piv,
                                                                 int *info) {
    __shared__ unsigned long long s_key[R][32];
    __shared__ int s_row[R][32];
    __shared__ int s_piv[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long k = (long long)blockIdx.x * 32 + lane;
    const bool live = k < ns;
    auto a = [&](int i, int j) -> double & { return A[((size_t)i * n + j) * ns + k]; };
    int bad = 0;
    for (int j = 0; j < n; ++j) {
        // pivot: this warp's rows j + w, j + w + R, ... then the R shares
        unsigned long long best = 0;
        int p = n;
        if (live) {
            for (int i = j + w; i < n; i += R) {
                const unsigned long long key = i == j ? lu_key_diag(a(i, j)) : lu_key(a(i, j));
                if (p == n || key > best) {
                    best = key;
                    p = i;
                }
            }
        }
        s_key[w][lane] = best;
        s_row[w][lane] = p;
        __syncthreads();
        if (w == 0) {
            for (int v = 1; v < R; ++v) {
                const unsigned long long k2 = s_key[v][lane];
                const int r2 = s_row[v][lane];
                if (r2 < n && (p == n || k2 > best || (k2 == best && r2 < p))) {
                    best = k2;
                    p = r2;
                }
            }
            s_piv[lane] = p;
            if (live) {
                if (piv) piv[(size_t)k * n + j] = p;
                if ((best == 0 || best >= 0x7ff0000000000000ULL) && !bad) bad = j + 1;
            }
        }
        __syncthreads();
        p = s_piv[lane];
        if (live && p != j) {
            lu_row_swap(&a(j, 0), &a(p, 0), w, R, n, ns);
            if (w == 0) {
                const double t = b[(size_t)j * ns + k];
                b[(size_t)j * ns + k] = b[(size_t)p * ns + k];
                b[(size_t)p * ns + k] = t;
            }
        }
        __syncthreads();
        if (live) {
            const LuPivot<FMA> d(a(j, j));
            for (int i = j + 1 + w; i < n; i += R) {
                const double l = d.mult(a(i, j));
                a(i, j) = l;
                lu_row_update<FMA>(&a(i, 0), &a(j, 0), l, j + 1, n, ns);
            }
        }
        __syncthreads();
    }
    if (w == 0 && live) {
        lu_global_solve<FMA>(n, ns, k, A, b);
        if (info) info[k] = bad;
    }
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
                const unsigned long long key = i == j ? lu_key_diag(M[i * n + j]) : lu_key(M[i * n + j]);
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

template <bool FMA>
static void launch_global(int R, int n, long long n_sys, double *A, double *b, int *piv, int *info,
                          cudaStream_t st) {
    const unsigned gb = (unsigned)((n_sys + 31) / 32);
    switch (R) {
        case 1: {
            const int bs = 128;
            lu_global_kernel<FMA><<<(unsigned)((n_sys + bs - 1) / bs), bs, 0, st>>>(n, n_sys, A, b, piv, info);
            break;
        }
        case 2: lu_global_rows_kernel<2, FMA><<<gb, 64, 0, st>>>(n, n_sys, A, b, piv, info); break;
        case 4: lu_global_rows_kernel<4, FMA><<<gb, 128, 0, st>>>(n, n_sys, A, b, piv, info); break;
        case 8: lu_global_rows_kernel<8, FMA><<<gb, 256, 0, st>>>(n, n_sys, A, b, piv, info); break;
        default: lu_global_rows_kernel<16, FMA><<<gb, 512, 0, st>>>(n, n_sys, A, b, piv, info); break;
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
    if (method == CHEM_LU_GLOBAL || method == CHEM_LU_GLOBAL_FMA) {
        // one thread per system while the systems alone give every SM at
        // least 16 warps; else R warps per 32 systems, R the power of two
        // that brings the warps to that count (at most 16, and no more than
        // the rows of the first step)
        const long long groups = (n_sys + 31) / 32;
        const long long want = 16LL * sms;
        int R = 1;
        while (R < 16 && groups * R < want && R < n - 1) R <<= 1;
        if (method == CHEM_LU_GLOBAL)
            launch_global<false>(R, n, n_sys, A, b, pivots, info, st);
        else
            launch_global<true>(R, n, n_sys, A, b, pivots, info, st);
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
