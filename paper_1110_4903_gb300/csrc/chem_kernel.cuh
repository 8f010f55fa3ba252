// chem_kernel.cuh -- batched backward-Euler chemistry step (sm_103a).
//
// One warp holds 32/G cell slots; the G lanes of a slot cooperate on one
// cell.  All slots of a warp execute the same instruction stream: one Newton
// iteration of Eq. 29 for every slot per trip of the warp loop, so a slot
// whose cell finishes picks up the next cell from a global work counter
// between iterations, without stalling the other slots.  Per-cell state,
// rates, the Jacobian and its LU live in shared memory; HBM only sees the
// cell state (SoA) on load and store.
//
// FP64 is the binding pipe on this part: 2 DFMA/clk/SM against 128 FFMA, and a
// partly masked FP64 instruction or an FP64<->FP32 conversion costs a full
// FP64 slot.  So:
//   - each phase is one loop over a flat, uniform work list (reactions, D
//     entries, Jacobian entries ordered by gather length and interleaved by
//     pass, fixed-size chunks of the species lists);
//   - coefficients are stored in the type they are used in, and the mixed
//     path converts between FP64 and FP32 on the integer pipe;
//   - pivot searches, range choices and finiteness tests compare integer
//     keys; reciprocals refine rcp.approx; exp is a short table-driven
//     evaluation, once per reaction (K_f) and once per species (the split
//     exponentials the equilibrium constants are multiplied from), and the
//     temperature recovery a multiplied-out polynomial.
// Both paths eliminate the energy unknown through the conservation of total
// energy, so the elimination runs on the ns species unknowns.  The mixed
// path (JT = float) keeps the FP64 residual, rates, sources and
// temperature, and moves everything that only feeds the Jacobian to FP32;
// it writes the Jacobian's rank-two part and the identity densely, four
// rows per store, then adds the sparse reaction sums, and its LU is
// organised by columns.  It is bound by latency, so its slot layout is cut
// to what it reads (20 warps per SM at 36 species).
//   Code size: with 20 warps at different phases, the instructions of one
// Newton iteration have to stay in the SM's instruction caches.  The
// compiler's unrolling of the many short runtime-count loops made the mixed
// kernel 114 KB, and instruction fetch its first stall; every loop below is
// therefore kept rolled (#pragma unroll 1) unless it says otherwise, and
// the few unrolled bodies are written out by hand.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include "chem_internal.h"

namespace chem {

constexpr unsigned kFull = 0xffffffffu;

enum SlotState : int {
    kFree = 0,        // needs a cell
    kInitT = 1,       // needs the temperature of its input state
    kNewtonT = 2,     // needs the temperature of the current Newton iterate
    kNewtonReady = 3, // runs a Newton iteration this trip
    kCheckT = 4,      // needs the temperature of a converged iterate
    kDead = 5         // no more cells
};

template <int G>
struct Grp {
    template <typename V>
    __device__ __forceinline__ static V sum(V v) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        return v;
    }
    template <typename V>
    __device__ __forceinline__ static V max(V v) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
        return v;
    }
    __device__ __forceinline__ static int any(int v) {
        if constexpr (G == 32) {
            return __any_sync(kFull, v);
        } else {
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) v |= __shfl_xor_sync(kFull, v, o);
            return v;
        }
    }
    // maximum of non-negative doubles on the integer pipe (their bit
    // patterns order the same way; a NaN, whose bits are larger than any
    // number's, wins): for a whole warp the high words by redux.sync, then
    // the low words of the lanes holding the high maximum
    __device__ __forceinline__ static double max_nonneg(double v) {
        unsigned long long b = (unsigned long long)__double_as_longlong(v);
        if constexpr (G == 32) {
            const unsigned hi = (unsigned)(b >> 32);
            const unsigned mhi = __reduce_max_sync(kFull, hi);
            const unsigned mlo = __reduce_max_sync(kFull, hi == mhi ? (unsigned)b : 0u);
            return __longlong_as_double((long long)(((unsigned long long)mhi << 32) | mlo));
        } else {
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                const unsigned long long b2 = __shfl_xor_sync(kFull, b, o);
                b = b2 > b ? b2 : b;
            }
            return __longlong_as_double((long long)b);
        }
    }
    // largest key, lowest index on ties
    template <typename K>
    __device__ __forceinline__ static void argmax(K &k, int &i) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const K k2 = __shfl_xor_sync(kFull, k, o);
            const int i2 = __shfl_xor_sync(kFull, i, o);
            if (k2 > k || (k2 == k && i2 < i)) {
                k = k2;
                i = i2;
            }
        }
    }
};

// Conversions between FP64 and FP32 on the integer pipe: on this part a
// conversion instruction occupies the FP64 pipe as long as a DFMA does.
// FP64 -> FP32 rounds toward zero; magnitudes below the smallest normal
// float give a signed zero, above the largest an infinity; NaN stays NaN.
__device__ __forceinline__ float d2f_rz(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;
    const unsigned man = ((hi & 0xfffffu) << 3) | (lo >> 29);
    unsigned f = sign | ((unsigned)e << 23) | man;
    if (e <= 0) f = sign;
    if (e >= 255) f = sign | 0x7f800000u | ((e == 1151 && ((hi & 0xfffffu) | lo)) ? 0x400000u : 0u);
    return __uint_as_float(f);
}
// FP32 -> FP64, exact for normal floats and infinities (NaN stays NaN,
// subnormal floats give a signed zero).
__device__ __forceinline__ double f2d_alu(float v) {
    const unsigned u = __float_as_uint(v);
    const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, man = u & 0x7fffffu;
    unsigned hi = sign | ((e + 896u) << 20) | (man >> 3);
    unsigned lo = man << 29;
    if (e == 0) {
        hi = sign;
        lo = 0u;
    }
    if (e == 255u) hi = sign | 0x7ff00000u | (man >> 3);
    return __hiloint2double((int)hi, (int)lo);
}
template <typename JT> __device__ __forceinline__ JT to_jt(double v);
template <> __device__ __forceinline__ double to_jt<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_jt<float>(double v) { return d2f_rz(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return f2d_alu(v); }

// Order of doubles by their bit patterns (integer pipe): exact for a >= 0
// against b > 0; a negative a counts as smaller, a NaN a as larger.
__device__ __forceinline__ bool bits_gt(double a, double b) {
    return __double_as_longlong(a) > __double_as_longlong(b);
}
__device__ __forceinline__ bool bits_lt(double a, double b) {
    return __double_as_longlong(a) < __double_as_longlong(b);
}
__device__ __forceinline__ bool finite_bits(double v) {
    return ((unsigned)((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ffu) != 0x7ffu;
}

// Argmax over a whole warp (one cell per warp) with redux.sync: the largest
// key, the lowest index on ties, as the shuffle tree gives it.  FP64 keys
// take the high word, then the low word among the lanes holding the high
// maximum; FP32 keys fit one word.
__device__ __forceinline__ void warp_argmax(unsigned long long &k, int &i) {
    const unsigned hi = (unsigned)(k >> 32), lo = (unsigned)k;
    const unsigned mhi = __reduce_max_sync(kFull, hi);
    const unsigned mlo = __reduce_max_sync(kFull, hi == mhi ? lo : 0u);
    i = (int)__reduce_min_sync(kFull, (hi == mhi && lo == mlo) ? (unsigned)i : 0xffffffffu);
    k = ((unsigned long long)mhi << 32) | mlo;
}
__device__ __forceinline__ void warp_argmax(unsigned &k, int &i) {
    const unsigned m = __reduce_max_sync(kFull, k);
    i = (int)__reduce_min_sync(kFull, k == m ? (unsigned)i : 0xffffffffu);
    k = m;
}

// |v| as an ordered integer key (NaN maps to 0 so it is never the pivot).
__device__ __forceinline__ unsigned long long abs_key(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
    return b > 0x7ff0000000000000ULL ? 0ULL : b;
}
__device__ __forceinline__ unsigned abs_key(float v) {
    const unsigned b = __float_as_uint(v) & 0x7fffffffu;
    return b > 0x7f800000u ? 0u : b;
}
__device__ __forceinline__ bool key_is_inf(unsigned long long k) { return k >= 0x7ff0000000000000ULL; }
__device__ __forceinline__ bool key_is_inf(unsigned k) { return k >= 0x7f800000u; }
// the pivot key of a matrix type: 64 bits for FP64, 32 for FP32
template <typename JT>
using PivotKey = decltype(abs_key(JT(0)));

// Reciprocal: the hardware approximation r refined with its residual
// e = 1 - a r as r (1 + e + e^2), whose error is e^3 (the approximation is
// good to about 2^-23, so below FP64 rounding): three FP64 operations.
__device__ __forceinline__ double frcp(double a) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(a));
    const double e = fma(-a, r, 1.0);
    return fma(r, fma(e, e, e), r);
}
// One Newton step only (relative error about 1e-14): for reciprocals that
// scale a convergence ratio or the temperature recovery's Newton step, never
// a rate, an energy or the elimination.
__device__ __forceinline__ double frcp1(double a) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(a));
    const double e = fma(-a, r, 1.0);
    return fma(r, e, r);
}
// FP32 reciprocal of the pivot: the hardware approximation (within an ulp or
// two), enough for an elimination whose result Newton refines in FP64.
__device__ __forceinline__ float frcp(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// The library exp for the arguments the table path does not take; kept out
// of line so its code is not repeated at every call site.
static __device__ __noinline__ double exp_outside(double x) { return exp(x); }

// A small signed integer (|v| < 2^22) as a float without a conversion
// instruction: add it to the bit pattern of 1.5 * 2^23, whose ulp is 1.
__device__ __forceinline__ float small_int_to_float(int v) {
    return __int_as_float(0x4B400000 + v) - 12582912.0f;
}
// The coefficient of a packed list word (a signed power of two stored as
// the sign and exponent bits of its double, over the reaction index in bits
// 0..19) as a double and as a float, by integer operations only: the
// float's exponent is the double's less 1023 - 127.
__device__ __forceinline__ double word_nu_double(unsigned wv) {
    return __hiloint2double((int)(wv & 0xfff00000u), 0);
}
__device__ __forceinline__ float word_nu_float(unsigned wv) {
    const unsigned hi = wv & 0xfff00000u;
    return __int_as_float((int)((hi & 0x80000000u) | (((hi & 0x7ff00000u) - 0x38000000u) << 3)));
}

// A positive integer below 2^20 as a double from integer operations only
// (biased exponent of its top bit, the bits below it), exact.
__device__ __forceinline__ double small_pos_int_to_double(int v) {
    const int e = 31 - __clz(v);
    const unsigned hi = ((unsigned)(1023 + e) << 20) | (((unsigned)v << (20 - e)) & 0xfffffu);
    return __hiloint2double((int)hi, 0);
}

// exp by the table-driven reduction of P. T. P. Tang, ACM TOMS 15(2), 1989:
// x = (256 k + j) ln2/256 + r with |r| <= ln2/512, exp(x) = 2^k 2^(j/256) e^r,
// 2^(j/256) from a 256-entry table and e^r - 1 by its degree-4 Taylor
// polynomial (truncation below 4e-17 on that interval): nine FP64
// operations.  |x| >= 512, infinities and NaN (decided on the exponent bits,
// no FP64 compare) fall back to the library exp.
__device__ __forceinline__ double fexp(double x, const double *tab) {
    const unsigned hi = (unsigned)((unsigned long long)__double_as_longlong(x) >> 32);
    if (((hi >> 20) & 0x7ffu) > 0x407u) return exp_outside(x);
    const double kShift = 6755399441055744.0;               // 1.5 * 2^52
    const double t = fma(x, 369.3299304675746, kShift);     // x * 256/ln2, rounded
    const int n = (int)(unsigned)__double_as_longlong(t);
    const double nd = t - kShift;
    double r = fma(nd, -0x1.62e42fefa0000p-9, x);            // ln2/256, high 36 bits
    r = fma(nd, -0x1.cf79abc9e3b3ap-48, r);                  // ln2/256, low part
    double p = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    p = fma(r, p, 0.5);
    p = fma(r, p, 1.0);
    p *= r;                                                  // e^r - 1
    const double s = __ldg(tab + (n & (kExpTab - 1)));
    const double y = fma(s, p, s);
    const long long k = (long long)(n >> 8);
    return __longlong_as_double(__double_as_longlong(y) + (k << 52));
}

// exp(x) = y 2^k with y in [0.99, 2.01]: the reduction of fexp without its
// final scaling, so that products of many exponentials can be formed
// without overflow.  The reduction is exact up to its two roundings for
// any |x| < 2^22 (the products with ln2/256 are fused, and the table index
// fits an int); beyond that (and for infinities) k saturates at +-2^24 with
// y = 1, and a NaN x gives a NaN y.
__device__ __forceinline__ void split_exp(double x, const double *tab, double &y, int &k) {
    const unsigned hi = (unsigned)((unsigned long long)__double_as_longlong(x) >> 32);
    const unsigned ex = (hi >> 20) & 0x7ffu;
    if (ex >= 0x415u) {
        const bool nan = ex == 0x7ffu && ((hi & 0xfffffu) | (unsigned)__double_as_longlong(x));
        y = nan ? x : 1.0;
        k = (hi >> 31) ? -(1 << 24) : (1 << 24);
        return;
    }
    const double kShift = 6755399441055744.0;               // 1.5 * 2^52
    const double t = fma(x, 369.3299304675746, kShift);     // x * 256/ln2, rounded
    const int n = (int)(unsigned)__double_as_longlong(t);
    const double nd = t - kShift;
    double r = fma(nd, -0x1.62e42fefa0000p-9, x);
    r = fma(nd, -0x1.cf79abc9e3b3ap-48, r);
    double p = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    p = fma(r, p, 0.5);
    p = fma(r, p, 1.0);
    p *= r;
    const double s = __ldg(tab + (n & (kExpTab - 1)));
    y = fma(s, p, s);
    k = n >> 8;
}
// v 2^k on the exponent bits for a normal v; zero, subnormal, infinite and
// NaN v come back unchanged, a result below the normal range is a signed
// zero and one above it an infinity.
__device__ __forceinline__ double scale_pow2(double v, int k) {
    const long long b = __double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0 || e == 0x7ff) return v;
    const int ne = e + k;
    const long long sgn = b & (long long)0x8000000000000000ULL;
    if (ne <= 0) return __longlong_as_double(sgn);
    if (ne >= 0x7ff) return __longlong_as_double(sgn | 0x7ff0000000000000LL);
    return __longlong_as_double(b + ((long long)k << 52));
}

// ln x for x >= 2 by the table-driven reduction of P. T. P. Tang, ACM TOMS
// 16(4), 1990: x = 2^k y with y in [1, 2), F = 1 + j/128 the table point
// nearest to y (j = 0..128), f = y - F (exact, |f| <= 2^-8), u = f (1/F),
// and ln x = k ln2 + ln F + ln(1 + u) with ln(1 + u) by its series to u^6
// (truncation below 2^-56 / 7): ten FP64 operations, within 1.5 ulp.  {1/F,
// ln F} come from a table; k becomes a double on the integer pipe.  (Below 2
// the result can be small next to k ln2 + ln F, and the table's rounding
// then leaves an absolute error near 1e-16.  The kernels take it of T in
// [200, 6000] K.)
__device__ __forceinline__ double flog(double x, const double2 *tab) {
    const long long b = __double_as_longlong(x);
    const int k = (int)(b >> 52) - 1023;
    const double y = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    const int j = (int)((b >> 45) & 0x7f) + (int)((b >> 44) & 1);
    const double F = __longlong_as_double(0x3ff0000000000000LL + ((long long)j << 45));
    const double2 t = __ldg(tab + j);
    const double u = (y - F) * t.x;
    double p = fma(u, -1.0 / 6.0, 0.2);
    p = fma(u, p, -0.25);
    p = fma(u, p, 1.0 / 3.0);
    p = fma(u, p, -0.5);
    p = fma(u, p, 1.0);
    // k as a double: added to the bit pattern of 1.5 * 2^52, whose ulp is 1
    const double kd = __longlong_as_double(0x4338000000000000LL + k) - 6755399441055744.0;
    return fma(u, p, fma(kd, 0.6931471805599453, t.y));
}

// NASA-7 entropy from the thermo coefficients of one species and range
// (layout in chem_internal.h)
__device__ __forceinline__ double nasa_s(const CoefRow<double> &th, double T, double lnT) {
    return th[0] * lnT + T * (th[1] + T * (th[10] + T * (th[11] + T * th[12]))) + th[13];
}
// range of species s at T (1: T > T_mid, the high range)
__device__ __forceinline__ int thermo_range(const DeviceMech &m, int s, long long Tbits) {
    return Tbits > __ldg(reinterpret_cast<const long long *>(m.tmid) + s) ? 1 : 0;
}

// Temperature recovery from (rho_s, e) for every slot whose `need` is set:
// Newton on sum_s rho_s e_s^sens(T) = e, safeguarded by bisection on
// [kTlo, kThi], stop at |dT| <= kTtol T (Eq. 3 with the kinetic energy left to
// the flux stage).  Uniform across the warp.
//   The energies come from the multiplied-out polynomials (five DFMA per
//   species, no 1/T); with F32 the derivative sum c_v is formed in FP32, which
//   changes the Newton steps by a relative 1e-7 and not the root.
template <int G, bool F32>
__device__ __forceinline__ void recover_T(const DeviceMech &m, const double *x, int sl, bool need,
                                          double guess, double &T_out, bool &ok) {
    const int ns = m.ns;
    double lo = kTlo, hi = kThi, T = guess;
    if (!(bits_gt(T, lo) && bits_lt(T, hi))) T = 1500.0;
    bool done = !need;
    ok = false;
    const double e = x[ns];
#pragma unroll 1
    for (int it = 1; it <= kTmaxIter; ++it) {
        if (!__any_sync(kFull, !done)) break;
        const long long Tb = __double_as_longlong(T);
        const float Tf = F32 ? d2f_rz(T) : 0.f;
        double f = 0.0, fp = 0.0;
        float fpf = 0.f;
#pragma unroll 1
        for (int s = sl; s < ns; s += G) {
            const int rg = thermo_range(m, s, Tb);
            const auto c = coef_row(m.tpoly, ns, s, rg);
            const double es = fma(fma(fma(fma(fma(c[5], T, c[4]), T, c[3]), T, c[2]), T, c[1]), T, c[0]);
            f = fma(x[s], es, f);
            if (F32) {
                const auto d = coef_row(m.tpoly_f, ns, s, rg);
                const float cv = fmaf(fmaf(fmaf(fmaf(d[4], Tf, d[3]), Tf, d[2]), Tf, d[1]), Tf, d[0]);
                fpf = fmaf(d2f_rz(x[s]), cv, fpf);
            } else {
                const double cv = fma(fma(fma(fma(c[10], T, c[9]), T, c[8]), T, c[7]), T, c[6]);
                fp = fma(x[s], cv, fp);
            }
        }
        f = Grp<G>::sum(f) - e;
        double rfp;
        if (F32) {
            fpf = Grp<G>::sum(fpf);
            rfp = f2d_alu(__frcp_rn(fpf));
        } else {
            fp = Grp<G>::sum(fp);
            rfp = frcp1(fp);
        }
        if (!done) {
            const long long fb = __double_as_longlong(f);
            if ((fb << 1) == 0) {
                done = true;
                ok = true;
            } else {
                if (fb > 0)
                    hi = T;
                else
                    lo = T;
                double Tn = T - f * rfp;
                if (!(bits_gt(Tn, lo) && bits_lt(Tn, hi))) Tn = 0.5 * (lo + hi);
                const double dT = Tn - T;
                T = Tn;
                // (comparisons of non-negative doubles on their bit patterns)
                if (!bits_gt(fabs(dT), kTtol * T)) {
                    done = true;
                    ok = bits_gt(T, kTlo * (1.0 + 1e-9)) && bits_lt(T, kThi * (1.0 - 1e-9));
                }
            }
        }
    }
    if (need) T_out = T;
}

// FP32 trailing update a_ik -= a_ij (a_jk / a_jj) of elimination step j
// (i > j, k > j, the right-hand side column n included) on the column-major
// matrix A[k*ld + i], ld a multiple of 4.  A lane owns a column, keeps
// a_jk / a_jj in a register and walks its rows four at a time with 16-byte
// loads and stores; the a_ij of the pivot column are 16-byte broadcast
// reads.  When fewer columns than lanes remain, the rows of each column are
// split over 2, 4, ... lanes at multiples of four rows.  The multipliers are
// never stored: the right-hand side is eliminated with the matrix, and back
// substitution reads U only.  Each element gets fma(-a_ij, a_jk / a_jj, a_ik)
// whichever lane computes it.
template <int G>
__device__ __forceinline__ void lu_update_colmajor(float *A, int ld, int n, int j, int sl, float inv) {
    const int C = n - j, r0 = j + 1;
    if (r0 >= n) return;
    int kc = sl, i0 = r0, i1 = n;
    if (C < G) {
        const int lg = C > 1 ? 32 - __clz(C - 1) : 0;   // columns rounded up to 2^lg
        const int lgB = (__ffs(G) - 1) - lg;              // lanes per column, log2
        kc = sl & ((1 << lg) - 1);
        if (kc >= C) return;
        const int part = sl >> lg, base = r0 & ~3;
        const int rows = ((((n - base) + (1 << lgB) - 1) >> lgB) + 3) & ~3;
        i0 = max(r0, base + part * rows);
        i1 = min(n, base + (part + 1) * rows);
    }
    const float *cj = A + j * ld;
#pragma unroll 1
    for (int k = j + 1 + kc; k <= n; k += G) {
        float *ck = A + k * ld;
        const float ajk = ck[j] * inv;
        int i = i0;
#pragma unroll 1
        for (; i < i1 && (i & 3); ++i) ck[i] = fmaf(-cj[i], ajk, ck[i]);
#pragma unroll 1
        for (; i + 4 <= i1; i += 4) {
            const float4 l = *reinterpret_cast<const float4 *>(cj + i);
            float4 v = *reinterpret_cast<const float4 *>(ck + i);
            v.x = fmaf(-l.x, ajk, v.x);
            v.y = fmaf(-l.y, ajk, v.y);
            v.z = fmaf(-l.z, ajk, v.z);
            v.w = fmaf(-l.w, ajk, v.w);
            *reinterpret_cast<float4 *>(ck + i) = v;
        }
#pragma unroll 1
        for (; i < i1; ++i) ck[i] = fmaf(-cj[i], ajk, ck[i]);
    }
}

template <typename JT>
struct SlotMem {
    double *x, *x0, *c, *hRT, *es, *em, *emi, *Q, *part;
    int *ek;
    JT *D, *dTdr, *w, *u, *A, *dQdT, *qtb, *A1, *A2, *rhs;
    JT *cJ, *hJ, *esJ;   // FP32 path: c, h/RT and the energies e_s in the Jacobian type
    // layout and sizes in chem_internal.h (slot_bytes_for, slot_stride); the FP64 path has
    // no FP32 copies (cJ = c, hJ = hRT), the FP32 path no FP64 hRT, es or
    // dTdr.  The species values of the rates (c, the split exponentials em,
    // emi, ek, and h/RT) share the union with the matrix: they are written
    // again every iteration, sentinel included.
    __device__ __forceinline__ void carve(char *base, const DeviceMech &m) {
        const int ns = m.ns, n = ns + 1, nr = m.nr;
        constexpr int jt = (int)sizeof(JT);
        double *p = reinterpret_cast<double *>(base);
        x = p;
        x0 = x + n;
        es = jt == 8 ? x0 + n : nullptr;
        char *q = base + slot_dbl_bytes(ns, jt);
        JT *t = reinterpret_cast<JT *>(q);
        const int ss = small_stride(ns, jt);
        w = t;
        u = w + ss;
        rhs = u + ss;
        if (jt == 8) {
            dTdr = rhs + ss;
            esJ = reinterpret_cast<JT *>(es);
        } else {
            dTdr = nullptr;
            esJ = rhs + ss;
        }
        q += slot_small_bytes(ns, jt);
        // D region: Q and the gather partials until the D entries replace them
        Q = reinterpret_cast<double *>(q);
        part = Q + nr;
        D = reinterpret_cast<JT *>(q);
        q += slot_dreg_bytes(nr, m.nD, m.n_items, jt);
        // union: species values and per-reaction values, then (after the D
        // entries) the matrix
        A = reinterpret_cast<JT *>(q);
        c = reinterpret_cast<double *>(q);
        em = c + ns + 1;
        emi = em + ns + 1;
        hRT = jt == 8 ? emi + ns + 1 : nullptr;
        ek = reinterpret_cast<int *>(emi + (jt == 8 ? 2 : 1) * (ns + 1));
        if (jt == 8) {
            cJ = reinterpret_cast<JT *>(c);
            hJ = reinterpret_cast<JT *>(hRT);
        } else {
            cJ = reinterpret_cast<JT *>(ek + ns + 1);
            hJ = cJ + ns + 1;
        }
        dQdT = reinterpret_cast<JT *>(q + slot_union_species_bytes(ns, jt));
        A1 = dQdT + nr;
        A2 = A1 + nr;
        qtb = A2 + nr;
    }
};

// Sources, Jacobian and one Newton update of Eq. 29 for every slot of the
// warp.  Inputs per slot: x, x0, T, h.  Outputs: x <- x + delta, the scaled
// norm, and a flag for a singular pivot or a non-finite update.
template <int G, typename JT>
__device__ void newton_iteration(const DeviceMech &m, const double *tab, SlotMem<JT> &sm, int sl,
                                 double T, double h, double atol_rho, double atol_e, double rtol,
                                 double &norm, bool &bad, double &T_pred) {
    const int ns = m.ns, nr = m.nr;
    constexpr bool f32 = sizeof(JT) == 4;
    // the linear system solved: the species block, with the energy unknown
    // eliminated (phase 5)
    // the matrix: FP64 row-major with rows of N + 1 (the right-hand side
    // last), FP32 column-major with columns of ldc rows (a multiple of 4, for
    // the 16-byte accesses of its elimination; the right-hand side is column N)
    const int N = ns, ldA = N + 1, ldc = (N + 3) & ~3;
    auto ix = [&](int i, int k) -> int { return f32 ? k * ldc + i : i * ldA + k; };
    const double invT = frcp(T);
    const double lnT = flog(T, m.log_tab);   // T in [200, 6000] K: normal
    const double lnPaRT = kLnPaOverR - lnT;

    // 1. concentrations and thermodynamics (species); the heat capacity only
    //    feeds dT/drho, dT/de and the next temperature guess, so the FP32
    //    path forms it in FP32
    const long long Tb = __double_as_longlong(T);
    const float Tf = f32 ? d2f_rz(T) : 0.f;
    double ctot = 0.0, rhocv = 0.0;
    float rhocvf = 0.f;
#pragma unroll 1
    for (int s = sl; s < ns; s += G) {
        const double *spr = m.sp + s * kSpStride;
        const double xs = sm.x[s];
        const double ci = xs * __ldg(spr + 1);
        sm.c[s] = ci;
        ctot += ci;
        const int rg = thermo_range(m, s, Tb);
        const auto th = coef_row(m.thermo, ns, s, rg);
        const double hRT = th[0] + T * (th[5] + T * (th[6] + T * (th[7] + T * th[8]))) + th[9] * invT;
        const double sR = nasa_s(th, T, lnT);
        const double RM = __ldg(spr + 2);
        // exp(g_s/RT - ln(P_a/RT)) split into mantissa and power of two,
        // for the equilibrium constants (phase 2)
        double ey;
        int eK;
        split_exp(hRT - sR - lnPaRT, tab, ey, eK);
        sm.em[s] = ey;
        sm.emi[s] = frcp(ey);
        sm.ek[s] = eK;
        if (f32) {
            // the species energy with its formation part, e_s = (R/M) T (h/RT
            // - 1): the Jacobian's temperature column (-e_s dT/de) and the
            // linearised temperature guess need no more, so FP32
            const JT hJs = to_jt<JT>(hRT);
            sm.esJ[s] = (JT)__ldg(m.spf + s * kSpStride + 2) * Tf * (hJs - (JT)1);
            const auto d = coef_row(m.tpoly_f, ns, s, rg);
            const float cv = fmaf(fmaf(fmaf(fmaf(d[4], Tf, d[3]), Tf, d[2]), Tf, d[1]), Tf, d[0]);
            rhocvf = fmaf(d2f_rz(xs), cv, rhocvf);
            sm.cJ[s] = to_jt<JT>(ci);
            sm.hJ[s] = hJs;
        } else {
            const double es = RM * T * (hRT - 1.0) - __ldg(spr + 3);
            const auto c = coef_row(m.tpoly, ns, s, rg);
            const double cv = fma(fma(fma(fma(c[10], T, c[9]), T, c[8]), T, c[7]), T, c[6]);
            rhocv = fma(xs, cv, rhocv);
            sm.hRT[s] = hRT;
            sm.es[s] = es;
        }
    }
    if (sl == 0) {
        // sentinel species: concentration 1, no Gibbs or enthalpy contribution
        sm.c[ns] = 1.0;
        sm.em[ns] = 1.0;
        sm.emi[ns] = 1.0;
        sm.ek[ns] = 0;
        if (f32) {
            sm.cJ[ns] = (JT)1;
            sm.hJ[ns] = (JT)0;
        } else {
            sm.hRT[ns] = 0.0;
        }
    }
    ctot = Grp<G>::sum(ctot);
    double dTde;
    float dTdef = 0.f;
    if (f32) {
        rhocvf = Grp<G>::sum(rhocvf);
        dTdef = __frcp_rn(rhocvf);
        dTde = f2d_alu(dTdef);
        // dT/drho_k = -e_k^sens dT/de is formed where the Jacobian needs it
    } else {
        rhocv = Grp<G>::sum(rhocv);
        dTde = frcp(rhocv);
#pragma unroll 1
        for (int s = sl; s < ns; s += G) sm.dTdr[s] = (JT)(-(sm.es[s] + __ldg(m.sp + s * kSpStride + 3)) * dTde);
    }
    __syncwarp();

    // 2. rates per reaction: Eq. 23 forward rate, Eq. 24 equilibrium
    //    constant, Eq. 25 progress rate, and their temperature derivatives
    const JT iT = to_jt<JT>(invT);
    // (the next reaction's parameters are loaded while this one is
    // evaluated: the loop is kept rolled, so nothing else would overlap them)
    static_assert(kRxnDStride == 4, "a reaction's FP64 parameters are two double2");
    double2 nAb = make_double2(0.0, 0.0), nEd = make_double2(0.0, 0.0);
    int2 nf = make_int2(0, 0);
    auto load_rxn = [&](int r) {
        if (r < nr) {
            const double2 *rd = reinterpret_cast<const double2 *>(m.rxn_d + (size_t)r * kRxnDStride);
            nAb = __ldg(rd);
            nEd = __ldg(rd + 1);
            nf = __ldg(reinterpret_cast<const int2 *>(m.rxn_f) + r);
        }
    };
    load_rxn(sl);
#pragma unroll 1
    for (int r = sl; r < nr; r += G) {
        const double lnA = nAb.x, beta = nAb.y, EaR = nEd.x, dnu = nEd.y;
        const int fr = nf.x, fpw = nf.y;
        load_rxn(r + G);
        const int a0 = fr & 0xff, a1 = (fr >> 8) & 0xff, a2 = (fr >> 16) & 0xff;
        const int b0 = fpw & 0xff, b1 = (fpw >> 8) & 0xff, b2 = (fpw >> 16) & 0xff;
        // third factor slots: the sentinel's factors are exactly 1 (0 for the
        // enthalpies), so a pass none of whose reactions has a third factor on
        // either side skips them, with bit-identical results (the 36-species
        // mechanism has at most two per side); the vote makes the branch
        // uniform, so the skipped FP64 products cost no pipe slot
        const bool s3 = __any_sync(__activemask(), (a2 != ns) | (b2 != ns));
        double Pf = sm.c[a0] * sm.c[a1];
        double Pb = sm.c[b0] * sm.c[b1];
        const double lnkf = lnA + beta * lnT - EaR * invT;
        const double kf = fexp(lnkf, tab);
        // K_b = K_f / K_c with 1/K_c = (RT/P_a)^dnu exp(dG/RT) (Eq. 24) as
        // the product over the factor slots of the species' exp(g/RT) (RT/P_a)
        // (products) and their inverses (reactants), the sentinel giving 1:
        // mantissas multiplied in FP64, powers of two added as integers, so no
        // exponential per reaction and no overflow in the partial products
        int K2 = (sm.ek[b0] + sm.ek[b1]) - (sm.ek[a0] + sm.ek[a1]);
        double Pm;
        if (s3) {
            Pf *= sm.c[a2];
            Pb *= sm.c[b2];
            K2 = (sm.ek[b0] + sm.ek[b1] + sm.ek[b2]) - (sm.ek[a0] + sm.ek[a1] + sm.ek[a2]);
            Pm = ((sm.em[b0] * sm.em[b1]) * sm.em[b2]) * ((sm.emi[a0] * sm.emi[a1]) * sm.emi[a2]);
        } else {
            Pm = (sm.em[b0] * sm.em[b1]) * (sm.emi[a0] * sm.emi[a1]);
        }
        const double kb = scale_pow2(kf * Pm, K2);
        double CM = 1.0;
        const bool tb = (fr >> 24) & 1;
        if (tb) {
            CM = ctot;
            const int e0 = __ldg(m.eff_ptr + r), e1 = __ldg(m.eff_ptr + r + 1);
#pragma unroll 1
            for (int e = e0; e < e1; ++e) CM += __ldg(m.eff_c + e) * sm.c[__ldg(m.eff_sp + e)];
        }
        const double fwd = kf * Pf, rev = kb * Pb, q = fwd - rev;
        sm.Q[r] = CM * q;   // in the D region until phase 4
        if (f32) {
            // Jacobian-only quantities in FP32 from FP32 copies
            const float *rf = m.rxn_df + (size_t)r * kRxnDStride;
            // (products formed in FP32 from converted factors: the FP64
            // pipe keeps to the rates the residual needs)
            const JT CMf = to_jt<JT>(CM);
            const JT A1v = CMf * to_jt<JT>(kf), A2v = CMf * to_jt<JT>(kb);
            sm.A1[r] = A1v;
            sm.A2[r] = A2v;
            if (r < m.ntb) sm.qtb[r] = to_jt<JT>(q);
            const JT shf = s3 ? (sm.hJ[b0] + sm.hJ[b1] + sm.hJ[b2]) - (sm.hJ[a0] + sm.hJ[a1] + sm.hJ[a2])
                              : (sm.hJ[b0] + sm.hJ[b1]) - (sm.hJ[a0] + sm.hJ[a1]);
            const JT dlnkf = (JT)__ldg(rf + 1) * iT * iT + (JT)__ldg(rf) * iT;
            const JT dlnKc = (shf - (JT)__ldg(rf + 2)) * iT;
            // concentration products again in FP32 (a conversion costs an
            // FP64-pipe slot, three FP32 products do not)
            JT PfJ = sm.cJ[a0] * sm.cJ[a1], PbJ = sm.cJ[b0] * sm.cJ[b1];
            if (s3) {
                PfJ *= sm.cJ[a2];
                PbJ *= sm.cJ[b2];
            }
            sm.dQdT[r] = A1v * PfJ * dlnkf - A2v * PbJ * (dlnkf - dlnKc);
        } else {
            const double sh = s3 ? (sm.hRT[b0] + sm.hRT[b1] + sm.hRT[b2]) - (sm.hRT[a0] + sm.hRT[a1] + sm.hRT[a2])
                                 : (sm.hRT[b0] + sm.hRT[b1]) - (sm.hRT[a0] + sm.hRT[a1]);
            if (r < m.ntb) sm.qtb[r] = (JT)q;
            sm.A1[r] = (JT)(CM * kf);
            sm.A2[r] = (JT)(CM * kb);
            const double dlnkf = fma(EaR * invT, invT, beta * invT);
            const double dlnKc = (sh - dnu) * invT;
            sm.dQdT[r] = (JT)(CM * (fwd * dlnkf - rev * (dlnkf - dlnKc)));
        }
    }
    __syncwarp();

    // 3. species sources (Eq. 26) and the rank-1 vectors of the Jacobian, as
    //    fixed-size chunks of each species' reaction list, then per species
    //    (an item's partial sums: sum nu Q in FP64, then sum nu dQ/dT and
    //    sum nu q_tb in the Jacobian type, packed into the next 16 bytes)
    const GatherLayout &gl = m.gl[layout_index(G)];
#pragma unroll 1
    for (int it = sl; it < m.n_items; it += G) {
        const int2 im = __ldg(gl.it_meta + it);
        double sq = 0.0;
        JT sdq = 0, squ = 0;
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            if (q < im.y) {
                const int e = im.x + q * G;
                const unsigned wv = __ldg(gl.sp_w + e);
                const int r = (int)(wv & 0xfffffu);
                const double nu = word_nu_double(wv);   // nu_rs != 0 in a list
                const JT nuj = f32 ? (JT)word_nu_float(wv) : (JT)nu;
                sq = fma(nu, sm.Q[r], sq);
                sdq += nuj * sm.dQdT[r];
                if (r < m.ntb) squ += nuj * sm.qtb[r];
            }
        }
        constexpr int iw = (int)(item_bytes((int)sizeof(JT)) / 8);   // doubles per item
        sm.part[iw * it] = sq;
        JT *pj = reinterpret_cast<JT *>(sm.part + iw * it + 1);
        pj[0] = sdq;
        pj[1] = squ;
    }
    __syncwarp();
    double dEt = 0.0;
#pragma unroll 1
    for (int s = sl; s < ns; s += G) {
        double sq = 0.0;
        JT sdq = 0, squ = 0;
        const int i0 = __ldg(m.sp_item_ptr + s), i1 = __ldg(m.sp_item_ptr + s + 1);
        constexpr int iw = (int)(item_bytes((int)sizeof(JT)) / 8);
#pragma unroll 1
        for (int it = i0; it < i1; ++it) {
            sq += sm.part[iw * it];
            const JT *pj = reinterpret_cast<const JT *>(sm.part + iw * it + 1);
            sdq += pj[0];
            squ += pj[1];
        }
        const double M = __ldg(m.sp + s * kSpStride);
        const double ef = __ldg(m.sp + s * kSpStride + 3);
        const JT MJ = f32 ? (JT)__ldg(m.spf + s * kSpStride) : (JT)M;
        const double wds = M * sq;
        // right-hand side -F_s = -(x_s - x0_s - h wdot_s), FP64 until stored
        const double dx = sm.x[s] - sm.x0[s];
        sm.rhs[s] = to_jt<JT>(-(dx - h * wds));
        const JT ws = MJ * sdq, us = MJ * squ;
        sm.w[s] = ws;
        sm.u[s] = us;
        dEt = fma(ef, dx, dEt);
    }
    // the total-energy residual R_E = F_e + sum_s e_f,s F_s = (x_e - x0_e) +
    // sum_s e_f,s (x_s - x0_s), in which the sources cancel (Omega_e =
    // -sum_s e_f,s wdot_s); it replaces the energy equation (phase 5)
    const double RE = Grp<G>::sum(dEt) + (sm.x[ns] - sm.x0[ns]);
    __syncwarp();

    // 4. D entries: d Q_r / d rho_k without the all-ones third-body part,
    //    grouped so that each group is one uniform loop body (FP32: one
    //    branch-free body that selects the sides by their orders, two
    //    entries per trip so their loads overlap; its entries are M_k dQ_r /
    //    drho_k, with integer orders, and the gather applies the 1/M_k)
    if (f32) {
        const JT *__restrict__ A1v = sm.A1;
        const JT *__restrict__ A2v = sm.A2;
        const JT *__restrict__ cJv = sm.cJ;
        const JT *__restrict__ qv = sm.qtb;
        JT *__restrict__ Dw = sm.D;
        auto dval = [&](int j) -> JT {
            const int2 pk = __ldg(m.d_pk + j);
            const int r = pk.x & 0xffff, vf = (pk.x >> 16) & 15, vb = (pk.x >> 20) & 15, i1 = pk.y;
            const JT fwd = (JT)small_int_to_float(vf) * A1v[r] * (cJv[i1 & 0xff] * cJv[(i1 >> 8) & 0xff]);
            const JT bwd = (JT)small_int_to_float(vb) * A2v[r] * (cJv[(i1 >> 16) & 0xff] * cJv[(i1 >> 24) & 0xff]);
            JT d = (vf ? fwd : (JT)0) - (vb ? bwd : (JT)0);
            if (r < m.ntb) d = fma((JT)__ldg(m.d_cef + j), qv[r], d);
            return d;
        };
        int j = sl;
#pragma unroll 1
        for (; j + G < m.nD; j += 2 * G) {
            const JT d0 = dval(j), d1 = dval(j + G);
            Dw[j] = d0;
            Dw[j + G] = d1;
        }
        if (j < m.nD) Dw[j] = dval(j);
    } else
#pragma unroll 1
    for (int j = sl; j < m.nD; j += G) {
        // the FP64 D entries are M_k dQ_r/drho_k as well: integer orders from
        // the descriptor (exact doubles by integer operations), alpha - 1
        // from an 8-byte table, and the gather applies the 1/M_k
        const int2 pk = __ldg(m.d_pk + j);
        const int r = pk.x & 0xffff, vf = (pk.x >> 16) & 15, vb = (pk.x >> 20) & 15, i1 = pk.y;
        const int fa = i1 & 0xff, fb = (i1 >> 8) & 0xff, ba = (i1 >> 16) & 0xff, bb = (i1 >> 24) & 0xff;
        double dd;
        if (j < m.nD_F) {
            dd = small_pos_int_to_double(vf) * sm.A1[r] * (sm.c[fa] * sm.c[fb]);
        } else if (j < m.nD_B) {
            dd = -(small_pos_int_to_double(vb) * sm.A2[r] * (sm.c[ba] * sm.c[bb]));
        } else if (j < m.nD_FB) {
            dd = small_pos_int_to_double(vf) * sm.A1[r] * (sm.c[fa] * sm.c[fb]) -
                 small_pos_int_to_double(vb) * sm.A2[r] * (sm.c[ba] * sm.c[bb]);
        } else {
            dd = 0.0;
        }
        sm.D[j] = r < m.ntb ? (JT)fma(__ldg(m.d_ce + j), (double)sm.qtb[r], dd) : (JT)dd;
    }
    __syncwarp();
    // the per-reaction arrays are dead from here on; the matrix takes their place

    // 5. right-hand side into the matrix, with the energy unknown
    //    eliminated.  The energy row of I - hJ is [e_f, 1] - sum_s e_f,s
    //    (row s) (J_ek = -sum_s e_f,s J_sk), so with the species equations
    //    it reduces to the conservation law de = -R_E - e_f . drho;
    //    substituted into the species rows, whose energy-column entry is
    //    a_s = -h w_s dT/de, it leaves
    //      sum_k (A_sk - a_s e_f,k) drho_k = -F_s + a_s R_E,
    //    the same solution as the full system of Eq. 29 in exact
    //    arithmetic, with one unknown fewer and no energy row to form
    const JT mh = to_jt<JT>(-h);
    {
        const JT cRE = f32 ? mh * (JT)dTdef * d2f_rz(RE) : (JT)(-h * dTde * RE);
#pragma unroll 1
        for (int i = sl; i < N; i += G) sm.A[ix(i, N)] = fma(sm.w[i], cRE, sm.rhs[i]);
    }

    // 6. the reduced system's -h J'_sk = -h (J_sk - w_s e_f,k dT/de), plus
    //    the identity.  J_sk = w_s dT/drho_k + (u_s + M_s sum_r nu_rs D_rk) / M_k
    //    (the D entries carry the factor M_k): a rank-two part, in which
    //    the reduced system's column factor dT/drho_k - e_f,k dT/de stands
    //    for dT/drho_k, plus the gathered sums (longest gather lists
    //    first, so the lanes of a pass run lists of nearly equal length;
    //    four terms in flight per trip, two accumulators)
    const JT *__restrict__ Dv = sm.D;
    if constexpr (f32) {
        // 6a. the rank-two part and the identity, dense: a lane writes
        //     rows 4g..4g+3 of column k with one 16-byte store, from
        //     16-byte reads of w and u (the padding rows of a column take
        //     values that nothing reads).  Task t = k ldc/4 + g steps by G,
        //     the carry taken without a division.
        const int NG = ldc >> 2;
        const unsigned rc = __ldg(m.div16 + NG);
        int k = (int)(((unsigned)sl * rc) >> 16), g = sl - k * NG;
        const int dk = (int)(((unsigned)G * rc) >> 16), dg = G - dk * NG;
        const float cTe = -(mh * dTdef);
#pragma unroll 1
        while (k < N) {
            const float cT = cTe * sm.esJ[k], cU = mh * __ldg(m.spf + k * kSpStride + 1);
            const float4 wv = *reinterpret_cast<const float4 *>(sm.w + 4 * g);
            const float4 uv = *reinterpret_cast<const float4 *>(sm.u + 4 * g);
            const int dd = k - 4 * g;   // the diagonal's row within the four
            float4 a;
            a.x = fmaf(wv.x, cT, uv.x * cU) + (dd == 0 ? 1.f : 0.f);
            a.y = fmaf(wv.y, cT, uv.y * cU) + (dd == 1 ? 1.f : 0.f);
            a.z = fmaf(wv.z, cT, uv.z * cU) + (dd == 2 ? 1.f : 0.f);
            a.w = fmaf(wv.w, cT, uv.w * cU) + (dd == 3 ? 1.f : 0.f);
            *reinterpret_cast<float4 *>(sm.A + k * ldc + 4 * g) = a;
            k += dk;
            g += dg;
            if (g >= NG) {
                g -= NG;
                ++k;
            }
        }
        __syncwarp();
        // 6b. the gathered sums of the entries that have reaction terms,
        //     added as -h (M_s / M_k) sum_r nu_rs D_rk
        //     (the word's top nine bits are those of the float coefficient)
        auto coef = [](unsigned wv) -> float { return __int_as_float((int)(wv & 0xff800000u)); };
#pragma unroll 1
        for (int p = sl; p < m.nJ_nz; p += G) {
            const int4 meta = __ldg(gl.j_meta32 + p);
            const int len = meta.y;
            float a0 = 0.f, a1 = 0.f;
            int e = meta.x, q = 0;
#pragma unroll 1
            for (; q + 4 <= len; q += 4, e += 4 * G) {
                const unsigned w0 = __ldg(gl.j_w + e), w1 = __ldg(gl.j_w + e + G), w2 = __ldg(gl.j_w + e + 2 * G),
                               w3 = __ldg(gl.j_w + e + 3 * G);
                const float v0 = Dv[w0 & 0x7fffffu], v1 = Dv[w1 & 0x7fffffu], v2 = Dv[w2 & 0x7fffffu],
                            v3 = Dv[w3 & 0x7fffffu];
                a0 = fmaf(coef(w0), v0, a0);
                a1 = fmaf(coef(w1), v1, a1);
                a0 = fmaf(coef(w2), v2, a0);
                a1 = fmaf(coef(w3), v3, a1);
            }
#pragma unroll 1
            for (; q < len; ++q, e += G) {
                const unsigned wv = __ldg(gl.j_w + e);
                a0 = fmaf(coef(wv), Dv[wv & 0x7fffffu], a0);
            }
            float *ap = reinterpret_cast<float *>(sm.A) + meta.z;
            *ap = fmaf(mh * __int_as_float(meta.w), a0 + a1, *ap);
        }
        __syncwarp();
    } else {
#pragma unroll 1
        for (int p = sl; p < m.nJ; p += G) {
            const int2 meta = __ldg(gl.j_meta + p);
            const int len = meta.y >> 16;
            const int s = (meta.y >> 8) & 0xff, k = meta.y & 0xff;
            const JT invMk = (JT)__ldg(m.sp + k * kSpStride + 1);
            JT J = sm.w[s] * sm.dTdr[k];
            JT a0 = 0, a1 = 0;
            int e = meta.x, q = 0;
#pragma unroll 1
            for (; q + 4 <= len; q += 4, e += 4 * G) {
                const int d0 = __ldg(gl.j_d + e), d1 = __ldg(gl.j_d + e + G), d2 = __ldg(gl.j_d + e + 2 * G),
                          d3 = __ldg(gl.j_d + e + 3 * G);
                const JT v0 = Dv[d0], v1 = Dv[d1], v2 = Dv[d2], v3 = Dv[d3];
                a0 = fma((JT)__ldg(gl.j_c + e), v0, a0);
                a1 = fma((JT)__ldg(gl.j_c + e + G), v1, a1);
                a0 = fma((JT)__ldg(gl.j_c + e + 2 * G), v2, a0);
                a1 = fma((JT)__ldg(gl.j_c + e + 3 * G), v3, a1);
            }
#pragma unroll 1
            for (; q < len; ++q, e += G) a0 = fma((JT)__ldg(gl.j_c + e), Dv[__ldg(gl.j_d + e)], a0);
            // (D entries scaled by M_k; the FP64 lists' coefficients are nu_rs M_s)
            J = fma(invMk, sm.u[s] + (a0 + a1), J);
            sm.A[ix(s, k)] = mh * J;
        }
        __syncwarp();
#pragma unroll 1
        for (int i = sl; i < N; i += G) sm.A[ix(i, i)] += (JT)1;
        __syncwarp();
    }

    // 7. Gaussian elimination with row partial pivoting on [A | -F]
    //    (Sec. 3.2), ties to the lowest row; the pivot's reciprocal replaces
    //    the diagonal
    bool sing = false;
#pragma unroll 1
    for (int j = 0; j < N; ++j) {
        PivotKey<JT> best = 0;
        int bi = N;
#pragma unroll 1
        for (int i = j + sl; i < N; i += G) {
            const PivotKey<JT> kk = abs_key(sm.A[ix(i, j)]);
            if (bi == N || kk > best) {
                best = kk;
                bi = i;
            }
        }
        if constexpr (G == 32)
            warp_argmax(best, bi);
        else
            Grp<G>::argmax(best, bi);
        if (best == 0 || key_is_inf(best)) sing = true;
        if (bi != j && bi < N) {
#pragma unroll 1
            for (int k = j + sl; k <= N; k += G) {
                const JT t = sm.A[ix(j, k)];
                sm.A[ix(j, k)] = sm.A[ix(bi, k)];
                sm.A[ix(bi, k)] = t;
            }
        }
        __syncwarp();
        // (the FP64 pivot takes the full-precision reciprocal: a 1e-14 error
        // in every multiplier reaches the trace species of ill-conditioned
        // cells at 1e-10)
        const JT inv = frcp(sm.A[ix(j, j)]);
        if (!f32) {
#pragma unroll 1
            for (int i = j + 1 + sl; i < N; i += G) sm.A[i * ldA + j] *= inv;
            __syncwarp();
            if (sl == 0) sm.A[j * ldA + j] = inv;
        }
        if (f32) {
            // FP32: bound by issue and latency, not by the pipe; the update
            // reads column j unscaled and never A[j][j]
            lu_update_colmajor<G>(reinterpret_cast<float *>(sm.A), ldc, N, j, sl, (float)inv);
        } else {
            // FP64: a flat walk over the trailing elements keeps every lane of
            // every FP64 instruction busy (a masked lane costs a full slot)
            // (sl / cols and G / cols by a reciprocal multiply: both numerators
            // are below 64, and an integer division would take conversions on
            // the FP64 pipe)
            const int cols = N - j;
            const int tot = (N - j - 1) * cols;
            const unsigned rc = __ldg(m.div16 + cols);
            int e = sl;
            const int q0 = (int)(((unsigned)sl * rc) >> 16), dq = (int)(((unsigned)G * rc) >> 16);
            int i = j + 1 + q0, k = j + 1 + (sl - q0 * cols);
            const int di = dq, dk = G - dq * cols;
#pragma unroll 1
            for (; e < tot; e += G) {
                sm.A[i * ldA + k] -= sm.A[i * ldA + j] * sm.A[j * ldA + k];
                i += di;
                k += dk;
                if (k > N) {
                    k -= cols;
                    ++i;
                }
            }
        }
        __syncwarp();
        // FP32: the reciprocal replaces the pivot once every lane has read it
        if (f32 && sl == 0) sm.A[ix(j, j)] = inv;
    }
    __syncwarp();
    // back substitution, U delta = y
    if constexpr (f32 && G == 32) {
        // one cell per warp (N <= 64): lane l keeps rows l and l + 32 of the
        // right-hand side in registers, and each solved entry reaches the
        // lanes by a shuffle instead of shared memory and two warp barriers
        // (the FP64 path measured 1 % slower this way)
        JT y0 = sl < N ? sm.A[ix(sl, N)] : JT(0), y1 = sl + 32 < N ? sm.A[ix(sl + 32, N)] : JT(0);
#pragma unroll 1
        for (int j = N - 1; j >= 0; --j) {
            const JT yj = __shfl_sync(kFull, j < 32 ? y0 : y1, j & 31);
            const JT dj = yj * sm.A[ix(j, j)];
            if (sl == (j & 31)) {
                if (j < 32)
                    y0 = dj;
                else
                    y1 = dj;
            }
            if (sl < j) y0 = fma(-sm.A[ix(sl, j)], dj, y0);
            if (sl + 32 < j) y1 = fma(-sm.A[ix(sl + 32, j)], dj, y1);
        }
        __syncwarp();
        if (sl < N) sm.A[ix(sl, N)] = y0;
        if (sl + 32 < N) sm.A[ix(sl + 32, N)] = y1;
        __syncwarp();
    } else {
#pragma unroll 1
        for (int j = N - 1; j >= 0; --j) {
            const JT dj = sm.A[ix(j, N)] * sm.A[ix(j, j)];
            __syncwarp();
            if (sl == 0) sm.A[ix(j, N)] = dj;
#pragma unroll 1
            for (int i = sl; i < j; i += G) sm.A[ix(i, N)] -= sm.A[ix(i, j)] * dj;
            __syncwarp();
        }
    }

    // 8. update, convergence norm, and the linearised temperature of the
    //    new iterate (dT = (de - sum_s e_s^sens drho_s) / (rho cv)) as the
    //    next recovery's starting guess.  The norm's ratios are FP64 on both
    //    paths (they decide acceptance and the divergence abort) and their
    //    maximum is taken on the bit patterns; a zero scale counts a nonzero
    //    update as infinitely large.
    auto ratio = [](double d, double den) -> double {
        if (__double_as_longlong(den) > 0) return fabs(d) * frcp1(den);
        return (__double_as_longlong(d) << 1) != 0 ? CUDART_INF : 0.0;
    };
    double nrm = 0.0, des = 0.0, se = 0.0;
    float desf = 0.f, sef = 0.f;
    int nonfinite = 0;
#pragma unroll 1
    for (int i = sl; i < N; i += G) {
        float df = 0.f;
        double d;
        if (f32) {
            df = (float)sm.A[ix(i, N)];
            d = f2d_alu(df);
            desf -= (float)sm.esJ[i] * df;   // e_s with its formation part: see below
            sef = fmaf(__ldg(m.spf + i * kSpStride + 3), df, sef);
        } else {
            d = (double)sm.A[ix(i, N)];
            des -= sm.es[i] * d;
            se = fma(__ldg(m.sp + i * kSpStride + 3), d, se);
        }
        const double xi = sm.x[i] + d;
        sm.x[i] = xi;
        if (!finite_bits(xi)) nonfinite = 1;
        const double ri = ratio(d, fma(rtol, fabs(xi), atol_rho));
        if (bits_gt(ri, nrm)) nrm = ri;
    }
    {
        // the eliminated energy unknown: de = -R_E - e_f . drho
        const double de = -RE - (f32 ? f2d_alu(Grp<G>::sum(sef)) : Grp<G>::sum(se));
        if (sl == 0) {
            const double xe = sm.x[ns] + de;
            sm.x[ns] = xe;
            if (!finite_bits(xe)) nonfinite = 1;
            const double ri = ratio(de, fma(rtol, fabs(xe), atol_e));
            if (bits_gt(ri, nrm)) nrm = ri;
            // dT = (de - sum_s e_s^sens drho_s) / (rho cv), where de = -R_E -
            // e_f . drho: the FP32 path's e_s carry e_f, so it adds -R_E
            if (f32)
                desf += d2f_rz(-RE);
            else
                des += de;
        }
    }
    nrm = Grp<G>::max_nonneg(nrm);
    nonfinite = Grp<G>::any(nonfinite);
    if (f32)
        des = f2d_alu(Grp<G>::sum(desf));
    else
        des = Grp<G>::sum(des);
    __syncwarp();
    norm = nrm;
    bad = sing || nonfinite;
    T_pred = T + des * dTde;
}

// ---- request-server queue (ServeQueue in chem_internal.h) -----------------
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
template <typename T>
__device__ __forceinline__ T ld_vol(const T *p) {
    return *reinterpret_cast<const volatile T *>(p);
}
// A relaxed load from L2 (not L1, which may hold another launch's or an
// earlier chunk's copy): for device values that are either immutable while
// they are read (a live chunk's descriptor copy) or only hints (`next`, the
// budget copy, the poll time).  Unlike volatile loads, several of these can
// be in flight at once.
template <typename T>
__device__ __forceinline__ T ld_cg(const T *p) {
    static_assert(sizeof(T) == 8 || sizeof(T) == 4, "8- or 4-byte values");
    T r;
    if constexpr (sizeof(T) == 8) {
        const long long v = __ldcg(reinterpret_cast<const long long *>(p));
        memcpy(&r, &v, 8);
    } else {
        const int v = __ldcg(reinterpret_cast<const int *>(p));
        memcpy(&r, &v, 4);
    }
    return r;
}
__device__ __forceinline__ long long ld_acquire_gpu(const long long *p) {
    long long v;
    asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
// Refreshes the device copies of the host's `tail` and of this launch's
// budget, and tells the host where the hand-out of cells stands (`front`:
// the first virtual cell of the current chunk; the cursor only grows, and
// every claim attempt and every idle poll comes here, so the host sees the
// claims catch up with what it published): at most one warp per launch
// every kServePollNs.
__device__ __forceinline__ void serve_refresh(const ServeQueue &q) {
    const unsigned long long now = globaltimer_ns();
    const unsigned long long last = ld_cg(q.dpoll);
    if (now - last < (unsigned long long)kServePollNs || atomicCAS(q.dpoll, last, now) != last) return;
    const unsigned long long t = ld_acquire_sys(q.tail);
    const int bud = ld_vol(q.budget);
    __threadfence();   // what the host wrote before `tail`, before the copy of `tail`
    atomicMax(q.dtail, t);
    *reinterpret_cast<volatile int *>(q.dbudget) = bud;
    *reinterpret_cast<volatile unsigned long long *>(q.front) = ld_cg(q.chunk) << kServeChunkLog;
}
// Copies the host descriptor of chunk c (ring entry ce) into the device ring;
// called after a claim from the chunk succeeded, so the chunk is live and
// its entry stable.  The sequence number is written last.
__device__ __forceinline__ void serve_mirror(const ServeQueue &q, int ce, long long c) {
    const ServeDesc *hd = q.desc + ce;
    ServeDesc *md = q.mdesc + ce;
    md->start = ld_vol(&hd->start);
    md->n_cells = ld_vol(&hd->n_cells);
    md->ld = ld_vol(&hd->ld);
    md->rho = ld_vol(&hd->rho);
    md->e = ld_vol(&hd->e);
    md->T_out = ld_vol(&hd->T_out);
    md->status = ld_vol(&hd->status);
    md->dt = ld_vol(&hd->dt);
    __threadfence();
    *reinterpret_cast<volatile long long *>(&md->seq) = c;
}
// Claims up to k consecutive cells of the current chunk for a warp's free
// slots: returns how many (0 when none is published or the launch's block
// budget excludes this block), the first one's virtual number in v0 and the
// chunk's ring entry in e.  The chunk's size comes from the device copy of
// its descriptor when one is there, else from host memory (the entry is
// read after `tail` shows the chunk published and holds it until all of its
// cells are done), and the first claim makes the copy.  Bounded by the
// guard; a pass claims, finds the chunk exhausted and moves on, or starts
// the entry's counter.
__device__ __forceinline__ int serve_claim(const ServeQueue &q, int k, long long &v0, int &e) {
    serve_refresh(q);
    if ((int)blockIdx.x >= ld_cg(q.dbudget)) return 0;
    long long c = (long long)ld_cg(q.chunk);
    const unsigned long long tail = (unsigned long long)ld_acquire_gpu(reinterpret_cast<const long long *>(q.dtail));
    // chunks published: the last one's real cells end at `tail`
    const long long nch = (long long)((tail + (1ULL << kServeChunkLog) - 1) >> kServeChunkLog);
#pragma unroll 1
    for (int guard = 0; guard < 64 && c < nch; ++guard) {
        const int ce = (int)(c % q.cap);
        const bool mirrored = ld_acquire_gpu(&q.mdesc[ce].seq) == c;
        long long nc;
        if (mirrored) {
            nc = ld_cg(&q.mdesc[ce].n_cells);
        } else {
            const ServeDesc *d = q.desc + ce;
            if (ld_vol(&d->seq) != c) {
                // a stale chunk number (finished, its entry reused since)
                // moves on; an entry out of order is an error
                const long long c2 = (long long)ld_cg(q.chunk);
                if (c2 != c) {
                    c = c2;
                    continue;
                }
                atomicExch(q.error, 1);
                return 0;
            }
            nc = ld_vol(&d->n_cells);
        }
        // the entry's counter: the first claim of this lap of the ring
        // starts it (the counter is never reset otherwise, so claims that
        // arrive after a chunk is handed out only find it exhausted)
        const long long lap = c / q.cap;
        constexpr unsigned long long kCount = (1ULL << kClaimLapShift) - 1;
        unsigned long long r = ld_cg(q.claimed + ce);
        if ((long long)(r >> kClaimLapShift) < lap) {
            atomicCAS(q.claimed + ce, r, (unsigned long long)lap << kClaimLapShift);
            continue;
        }
        if ((long long)(r >> kClaimLapShift) > lap) {
            // the entry has moved on: a stale chunk number
            const long long c2 = (long long)ld_cg(q.chunk);
            if (c2 != c) {
                c = c2;
                continue;
            }
            atomicExch(q.error, 1);
            return 0;
        }
        if ((long long)(r & kCount) < nc) {
            r = atomicAdd(q.claimed + ce, (unsigned long long)k);
            const long long off = (long long)(r & kCount);
            if ((long long)(r >> kClaimLapShift) != lap) {
                // only a claim through a chunk number older than a whole
                // ring of chunks gets here
                atomicExch(q.error, 1);
                return 0;
            }
            if (off < nc) {
                if (!mirrored) serve_mirror(q, ce, c);
                const long long cnt = min((long long)k, nc - off);
                v0 = (c << kServeChunkLog) + off;
                e = ce;
                return (int)cnt;
            }
        }
        // the chunk is handed out: on to the next
        atomicMax(q.chunk, (unsigned long long)(c + 1));
        ++c;
    }
    return 0;
}
// Counts a finished cell of ring entry e (lane 0 of its slot); the slot that
// finishes the request's last cell resets the entry's counters for the next
// request and publishes the completion record to the host.
__device__ __forceinline__ void serve_cell_done(const ServeQueue &q, int e) {
    __threadfence();   // the cell's results before its count
    atomicMax(q.t_last + e, globaltimer_ns());
    __threadfence();
    const unsigned long long prev = atomicAdd(q.done + e, 1ULL);
    const ServeDesc *d = q.mdesc + e;
    if ((long long)prev + 1 == ld_cg(&d->n_cells)) {
        const unsigned long long tf = atomicExch(q.t_first + e, ~0ULL);
        const unsigned long long tl = atomicExch(q.t_last + e, 0ULL);
        atomicExch(q.done + e, 0ULL);
        __threadfence_system();
        volatile ServeDone *f = q.fin + e;
        f->t_first = tf;
        f->t_last = tl;
        __threadfence_system();
        f->seq = ld_cg(&d->seq);
    }
}

// At most 10 warps per block and 102 registers per thread: 20 warps fit on
// an SM when shared memory allows it (2 blocks of 10; the mixed path at 36
// species, 11.3 KB per cell).
// Q: request-server mode, cells claimed from b.queue (each slot's request
// descriptor in host memory; its dt, buffers and completion accounting).
template <int G, typename JT, bool Q = false>
__global__ void __launch_bounds__(kMaxBlockThreads, 2) be_kernel(DeviceMech m, StepOptions o, StepBatch b) {
    extern __shared__ __align__(16) char smem[];
    constexpr int S = 32 / G;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int slot = lane / G;
    const int sl = lane - slot * G;
    const int ns = m.ns, n = ns + 1;
    const double *tab = m.exp_tab;   // 2 KB, stays in L1
    const long long sbytes = slot_stride(m, (int)sizeof(JT), G);
    SlotMem<JT> sm;
    sm.carve(smem + (size_t)(warp * S + slot) * sbytes, m);
    __syncthreads();

    int state = kFree;
    long long cell = -1;
    // request-server mode: the slot's ring entry and its request's dt
    int qe = -1;
    double sdt = b.dt;
    unsigned long long idle_since = 0;
    double T = 1500.0, T0 = 1500.0, Tin = CUDART_NAN, h = 0.0, norm_prev = CUDART_INF;
    double atol_rho = 0.0, atol_e = 0.0;
    int k = 0, level = 0, attempts = 0, iters = 0, subs = 0, fails = 0;
    long long t_units = 0;
    const long long total = 1LL << o.max_halvings;

    // per-cell outputs (lane 0 of the slot); in request-server mode the
    // request's own buffers, and the cell counted done
    auto emit = [&](int code, double Tv) {
        if (sl == 0) {
            if constexpr (Q) {
                const ServeDesc *d = b.queue.mdesc + qe;
                int *st = ld_cg(&d->status);
                double *to = ld_cg(&d->T_out);
                if (st) st[cell] = code;
                if (to) to[cell] = Tv;
                serve_cell_done(b.queue, qe);
            } else {
                if (b.status) b.status[cell] = code;
                if (b.T_out) b.T_out[cell] = Tv;
                if (b.newton_iters) b.newton_iters[cell] = iters;
                if (b.substeps) b.substeps[cell] = subs;
                if (b.failures) b.failures[cell] = fails;
            }
        }
    };
    auto write_fail = [&](int code) {
        emit(code, Tin);
        state = kFree;
    };
    auto start_substep = [&]() {
        if (attempts >= o.max_attempts) {
            write_fail(kCellTooManySteps);
            return;
        }
        while ((total >> level) > total - t_units) ++level;
        h = ldexp(sdt, -level);
        ++attempts;
#pragma unroll 1
        for (int i = sl; i < n; i += G) sm.x[i] = sm.x0[i];
        T = T0;
        k = 0;
        norm_prev = CUDART_INF;
        state = kNewtonReady;
    };
    auto substep_fail = [&]() {
        ++fails;
        ++level;
        if (level > o.max_halvings)
            write_fail(kCellNewtonFailed);
        else
            start_substep();
    };

#pragma unroll 1
    for (;;) {
        // refill free slots and settle every pending temperature recovery
        bool q_dry = false;   // request-server mode: a claim this trip found no cell
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            long long got = -1;
            bool loading;
            const double *rho_in = b.rho, *e_in = b.e;
            long long ld_in = b.ld;
            if constexpr (Q) {
                // the warp's free slots take consecutive cells of one chunk,
                // claimed by lane 0, which reads the chunk's descriptor once
                const unsigned lead = __ballot_sync(kFull, state == kFree && sl == 0);
                int cnt = 0, e = -1;
                long long v0 = 0;
                double cdt = 0.0;   // the chunk's dt (a slot's own sdt changes only when it loads)
                if (lane == 0 && lead && !q_dry) {
                    cnt = serve_claim(b.queue, __popc(lead), v0, e);
                    if (cnt > 0) {
                        const ServeDesc *d = b.queue.mdesc + e;
                        rho_in = ld_cg(&d->rho);
                        e_in = ld_cg(&d->e);
                        ld_in = ld_cg(&d->ld);
                        cdt = ld_cg(&d->dt);
                        atomicMin(b.queue.t_first + e, globaltimer_ns());
                    }
                }
                cnt = __shfl_sync(kFull, cnt, 0);
                if (lead && cnt == 0) q_dry = true;
                loading = false;
                if (cnt > 0) {
                    e = __shfl_sync(kFull, e, 0);
                    v0 = __shfl_sync(kFull, v0, 0);
                    rho_in = reinterpret_cast<const double *>(
                        __shfl_sync(kFull, reinterpret_cast<unsigned long long>(rho_in), 0));
                    e_in = reinterpret_cast<const double *>(
                        __shfl_sync(kFull, reinterpret_cast<unsigned long long>(e_in), 0));
                    ld_in = __shfl_sync(kFull, ld_in, 0);
                    cdt = __shfl_sync(kFull, cdt, 0);
                    // this slot's rank among the warp's free slots
                    const int rank = __popc(lead & ((1u << (slot * G)) - 1u));
                    loading = state == kFree && rank < cnt;
                    if (loading) {
                        qe = e;
                        sdt = cdt;
                        cell = (v0 & ((1LL << kServeChunkLog) - 1)) + rank;
                    }
                }
            } else {
                if (state == kFree && sl == 0) got = (long long)atomicAdd(b.work_counter, 1ULL);
                got = __shfl_sync(kFull, got, slot * G);
                loading = state == kFree && got < b.n_cells;
                if (state == kFree && !loading) state = kDead;
                if (loading) cell = got;
            }
            int nonfin = 0;
            double rt = 0.0, es = 0.0;
            if (loading) {
                iters = subs = fails = 0;
                Tin = CUDART_NAN;
                if (!Q && b.schedule && sl == 0) {
#pragma unroll 1
                    for (int w = 0; w < kSchedWords; ++w) b.schedule[cell * kSchedWords + w] = 0u;
                }
#pragma unroll 1
                for (int i = sl; i < n; i += G) {
                    const double v = i < ns ? rho_in[(size_t)i * ld_in + cell] : e_in[cell];
                    sm.x0[i] = v;
                    sm.x[i] = v;
                    if (!isfinite(v)) nonfin = 1;
                    if (i < ns) {
                        rt += v;
                        es += fabs(v * __ldg(m.sp + i * kSpStride + 3));
                    } else {
                        es += fabs(v);
                    }
                }
            }
            nonfin = Grp<G>::any(nonfin);
            rt = Grp<G>::sum(rt);
            es = Grp<G>::sum(es);
            if (loading) {
                atol_rho = o.atol_rel * rt;
                atol_e = o.atol_rel * es;
                T = (!Q && b.T_in) ? b.T_in[cell] : 1500.0;
                if (nonfin || !(rt > 0.0))
                    write_fail(kCellBadInput);
                else
                    state = kInitT;
            }
            __syncwarp();
            const bool needT = state == kInitT || state == kNewtonT || state == kCheckT;
            if (!__any_sync(kFull, needT)) break;
            double Tr = T;
            bool ok = false;
            recover_T<G, sizeof(JT) == 4>(m, sm.x, sl, needT, T, Tr, ok);
            int neg = 0;
#pragma unroll 1
            for (int i = sl; i < ns; i += G)
                if (bits_lt(sm.x[i], 0.0) && bits_gt(fabs(sm.x[i]), atol_rho)) neg = 1;   // x < -atol
            neg = Grp<G>::any(neg);
            __syncwarp();
            if (state == kInitT) {
                if (!ok) {
                    write_fail(kCellTFailed);
                } else {
                    T = T0 = Tin = Tr;
                    if (sdt == 0.0) {
                        emit(kCellOk, Tr);
                        state = kFree;
                    } else {
                        t_units = 0;
                        level = 0;
                        attempts = 0;
                        start_substep();
                    }
                }
            } else if (state == kNewtonT) {
                if (!ok) {
                    substep_fail();
                } else {
                    T = Tr;
                    state = kNewtonReady;
                }
            } else if (state == kCheckT) {
                if (!ok || neg) {
                    substep_fail();
                } else {
                    T = Tr;
                    // accept the substep (and record it: attempt attempts - 1
                    // < 32 kSchedWords, the budget being capped when recording)
                    if (!Q && b.schedule && sl == 0) {
                        const int a = attempts - 1;
                        b.schedule[cell * kSchedWords + (a >> 5)] |= 1u << (a & 31);
                    }
                    if (!Q && b.substep_states && subs < kSubstepStates) {
                        double *rec = b.substep_states + ((size_t)cell * kSubstepStates + subs) * n;
#pragma unroll 1
                        for (int i = sl; i < n; i += G) rec[i] = sm.x[i];
                    }
#pragma unroll 1
                    for (int i = sl; i < n; i += G) sm.x0[i] = sm.x[i];
                    T0 = T;
                    t_units += total >> level;
                    ++subs;
                    if (level > 0) --level;
                    if (t_units == total) {
                        double *rho_out = b.rho, *e_out = b.e;
                        long long ld_out = b.ld;
                        if constexpr (Q) {
                            const ServeDesc *d = b.queue.mdesc + qe;
                            rho_out = ld_cg(&d->rho);
                            e_out = ld_cg(&d->e);
                            ld_out = ld_cg(&d->ld);
                        }
#pragma unroll 1
                        for (int i = sl; i < n; i += G) {
                            if (i < ns)
                                rho_out[(size_t)i * ld_out + cell] = sm.x[i];
                            else
                                e_out[cell] = sm.x[i];
                        }
                        if constexpr (Q) {
                            // every lane's results before lane 0 counts the cell done
                            // (the slot's G lanes are converged here)
                            __syncwarp(G == 32 ? kFull : (((1u << G) - 1u) << (slot * G)));
                        }
                        emit(kCellOk, T);
                        state = kFree;
                    } else {
                        start_substep();
                    }
                }
            }
            __syncwarp();
        }
        if (!__any_sync(kFull, state == kNewtonReady)) {
            if (__all_sync(kFull, state == kDead)) break;
            if constexpr (Q) {
                // no published cell for any slot of the warp: poll for more
                // (bounded by the linger time, then the warp leaves)
                if (__all_sync(kFull, state == kFree)) {
                    const unsigned long long now = globaltimer_ns();
                    if (idle_since == 0) idle_since = now;
                    if (lane == 0) serve_refresh(b.queue);
                    __syncwarp();
                    // one decision for the whole warp
                    if (__any_sync(kFull, (int)blockIdx.x >= ld_cg(b.queue.dbudget) ||
                                              now - idle_since > (unsigned long long)b.queue.linger_ns))
                        break;
                    __nanosleep(20000);
                }
            }
            continue;
        }
        if constexpr (Q) idle_since = 0;
        // one Newton iteration of Eq. 29 for every slot
        double norm = 0.0, T_pred = T;
        bool bad = false;
        newton_iteration<G, JT>(m, tab, sm, sl, T, h, atol_rho, atol_e, o.rtol, norm, bad, T_pred);
        if (state == kNewtonReady) {
            // start the next temperature recovery from the linear prediction
            if (bits_gt(T_pred, kTlo) && bits_lt(T_pred, kThi)) T = T_pred;
            ++iters;
            if (bad) {
                substep_fail();
            } else if (o.point_implicit || !bits_gt(norm, 1.0) ||
                       (o.conv_kappa > 0.0 && k >= 1 && bits_lt(norm, norm_prev) &&
                        norm * norm <= o.conv_kappa * (norm_prev - norm))) {
                // (the contraction-rate stop theta / (1 - theta) norm <= kappa,
                // theta = norm / norm_prev < 1, multiplied out: no division)
                state = kCheckT;
            } else if (o.div_check && k >= 2 && !bits_lt(norm, norm_prev)) {
                substep_fail();
            } else {
                norm_prev = norm;
                ++k;
                if (k >= o.max_newton)
                    substep_fail();
                else
                    state = kNewtonT;
            }
        }
        __syncwarp();
    }
}

}  // namespace chem
