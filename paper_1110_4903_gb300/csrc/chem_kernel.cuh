// chem_kernel.cuh -- batched backward-Euler chemistry step (sm_103a).
//
// One warp holds 32/G cell slots; the G lanes of a slot cooperate on one
// cell.  All slots of a warp execute the same instruction stream: one Newton
// iteration of Eq. 29 for every slot per trip of the warp loop, so a slot
// whose cell finishes picks up the next cell from a global work counter
// between iterations, without stalling the other slots.  Per-cell state,
// rates, the Jacobian and its LU live in shared memory; HBM only sees the
// cell state (SoA) on load and store.  FP64 is the binding pipe on this
// part, so every FP64 phase is spread over the G lanes.
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
    __device__ __forceinline__ static double sum(double v) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        return v;
    }
    __device__ __forceinline__ static double max(double v) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
        return v;
    }
    __device__ __forceinline__ static int any(int v) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v |= __shfl_xor_sync(kFull, v, o);
        return v;
    }
    // max |value| with the lowest index on ties
    __device__ __forceinline__ static void argmax(double &v, int &i) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            double v2 = __shfl_xor_sync(kFull, v, o);
            int i2 = __shfl_xor_sync(kFull, i, o);
            if (v2 > v || (v2 == v && i2 < i)) {
                v = v2;
                i = i2;
            }
        }
    }
};

__device__ __forceinline__ double ipow3(double c, int nu) {
    // c^nu for nu in 0..3
    return nu == 0 ? 1.0 : (nu == 1 ? c : (nu == 2 ? c * c : c * c * c));
}

// NASA-7 evaluations from a 16-double thermo row (layout in chem_internal.h)
__device__ __forceinline__ void nasa_cp_h(const double *th, double T, double invT, double &cpR,
                                          double &hRT) {
    cpR = th[0] + T * (th[1] + T * (th[2] + T * (th[3] + T * th[4])));
    hRT = th[0] + T * (th[5] + T * (th[6] + T * (th[7] + T * th[8]))) + th[9] * invT;
}
__device__ __forceinline__ double nasa_s(const double *th, double T, double lnT) {
    return th[0] * lnT + T * (th[1] + T * (th[10] + T * (th[11] + T * th[12]))) + th[13];
}
__device__ __forceinline__ const double *thermo_row(const DeviceMech &m, int s, double T) {
    return m.thermo + (size_t)(s * 2 + (T > __ldg(m.tmid + s) ? 1 : 0)) * kThermoStride;
}

// Temperature recovery from (rho_s, e) for every slot whose `need` is set:
// Newton on sum_s rho_s e_s^sens(T) = e, safeguarded by bisection on
// [kTlo, kThi], stop at |dT| <= kTtol T (Eq. 3 with the kinetic energy left to
// the flux stage).  Uniform across the warp; returns ok per slot.
template <int G>
__device__ __forceinline__ void recover_T(const DeviceMech &m, const double *x, int sl, bool need,
                                          double guess, double &T_out, bool &ok) {
    const int ns = m.ns;
    double lo = kTlo, hi = kThi, T = guess;
    if (!(T > lo && T < hi)) T = 1500.0;
    bool done = !need;
    ok = false;
    const double e = x[ns];
    for (int it = 1; it <= kTmaxIter; ++it) {
        if (!__any_sync(kFull, !done)) break;
        const double invT = 1.0 / T;
        double f = 0.0, fp = 0.0;
        for (int s = sl; s < ns; s += G) {
            const double *th = thermo_row(m, s, T);
            double cpR, hRT;
            nasa_cp_h(th, T, invT, cpR, hRT);
            const double RM = __ldg(m.sp + s * kSpStride + 2);
            const double ef = __ldg(m.sp + s * kSpStride + 3);
            const double es = RM * T * (hRT - 1.0) - ef;
            const double cv = RM * (cpR - 1.0);
            f += x[s] * es;
            fp += x[s] * cv;
        }
        f = Grp<G>::sum(f) - e;
        fp = Grp<G>::sum(fp);
        if (!done) {
            if (f == 0.0) {
                done = true;
                ok = true;
            } else {
                if (f > 0.0)
                    hi = T;
                else
                    lo = T;
                double Tn = T - f / fp;
                if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
                const double dT = Tn - T;
                T = Tn;
                if (fabs(dT) <= kTtol * T) {
                    done = true;
                    ok = !(T <= kTlo * (1.0 + 1e-9) || T >= kThi * (1.0 - 1e-9));
                }
            }
        }
    }
    if (need) T_out = T;
}

template <typename JT>
struct SlotMem {
    double *x, *x0, *c, *hRT, *gRT, *es, *wd, *Q, *dQdT, *qtb;
    JT *dTdr, *w, *u, *D, *A;
    __device__ __forceinline__ void carve(char *base, int ns, int nr, int nD) {
        const int n = ns + 1;
        double *p = reinterpret_cast<double *>(base);
        x = p;
        x0 = x + n;
        c = x0 + n;
        hRT = c + ns;
        gRT = hRT + ns;
        es = gRT + ns;
        wd = es + ns;
        Q = wd + ns;
        dQdT = Q + nr;
        qtb = dQdT + nr;
        JT *q = reinterpret_cast<JT *>(qtb + nr);
        dTdr = q;
        w = dTdr + ns;
        u = w + ns;
        D = u + ns;
        A = D + nD;
    }
};

// Bytes of one slot for the kernel's carve (must match slot_smem_bytes).
__host__ __device__ inline long long slot_bytes(int ns, int nr, int nD, int jt) {
    const int n = ns + 1;
    long long dbl = 2LL * n + 5LL * ns + 3LL * nr;
    long long jtn = 3LL * ns + nD + (long long)n * (n + 1);
    return ((dbl * 8 + jtn * jt) + 15) / 16 * 16;
}

// Sources, Jacobian and one Newton update for every slot of the warp.
// Inputs per slot: x, x0, T, h.  Outputs: x <- x + delta, the scaled norm,
// and flags for a singular pivot or a non-finite update.
template <int G, typename JT>
__device__ void newton_iteration(const DeviceMech &m, SlotMem<JT> &sm, int sl, double T, double h,
                                 double atol_rho, double atol_e, double rtol, double &norm,
                                 bool &bad) {
    const int ns = m.ns, nr = m.nr, n = ns + 1, lda = n + 1;
    const double invT = 1.0 / T;
    const double lnT = log(T);
    const double lnPaRT = log(kPa / kR) - lnT;

    // concentrations and thermo (species lane-strided)
    double ctot = 0.0, rhocv = 0.0;
    for (int s = sl; s < ns; s += G) {
        const double *spr = m.sp + s * kSpStride;
        const double ci = sm.x[s] * __ldg(spr + 1);
        sm.c[s] = ci;
        ctot += ci;
        const double *th = thermo_row(m, s, T);
        double cpR, hRT;
        nasa_cp_h(th, T, invT, cpR, hRT);
        const double sR = nasa_s(th, T, lnT);
        const double RM = __ldg(spr + 2);
        sm.hRT[s] = hRT;
        sm.gRT[s] = hRT - sR;
        const double es = RM * T * (hRT - 1.0) - __ldg(spr + 3);
        sm.es[s] = es;
        rhocv += sm.x[s] * RM * (cpR - 1.0);
    }
    ctot = Grp<G>::sum(ctot);
    rhocv = Grp<G>::sum(rhocv);
    const double dTde = 1.0 / rhocv;
    for (int s = sl; s < ns; s += G) sm.dTdr[s] = (JT)(-sm.es[s] * dTde);
    __syncwarp();

    // rates, progress rates and rate derivatives (reactions lane-strided):
    // Eq. 23 forward rate, Eq. 24 equilibrium constant, Eq. 25 progress rate
    for (int r = sl; r < nr; r += G) {
        const double *rd = m.rxn_d + (size_t)r * kRxnDStride;
        const int *ri = m.rxn_i + (size_t)r * kRxnIStride;
        const double lnA = __ldg(rd + 0), beta = __ldg(rd + 1), EaR = __ldg(rd + 2),
                     dnu = __ldg(rd + 3);
        const int rs0 = __ldg(ri + 0), rs1 = __ldg(ri + 1), rs2 = __ldg(ri + 2);
        const int ps0 = __ldg(ri + 3), ps1 = __ldg(ri + 4), ps2 = __ldg(ri + 5);
        const int nup = __ldg(ri + 6), flags = __ldg(ri + 7);
        const int nr0 = nup & 3, nr1 = (nup >> 2) & 3, nr2 = (nup >> 4) & 3;
        const int np0 = (nup >> 8) & 3, np1 = (nup >> 10) & 3, np2 = (nup >> 12) & 3;
        const double lnkf = lnA + beta * lnT - EaR * invT;
        double sg = 0.0, sh = 0.0;
        double pr0 = 1.0, pr1 = 1.0, pr2 = 1.0, pp0 = 1.0, pp1 = 1.0, pp2 = 1.0;
        if (rs0 >= 0) { pr0 = ipow3(sm.c[rs0], nr0); sg -= nr0 * sm.gRT[rs0]; sh -= nr0 * sm.hRT[rs0]; }
        if (rs1 >= 0) { pr1 = ipow3(sm.c[rs1], nr1); sg -= nr1 * sm.gRT[rs1]; sh -= nr1 * sm.hRT[rs1]; }
        if (rs2 >= 0) { pr2 = ipow3(sm.c[rs2], nr2); sg -= nr2 * sm.gRT[rs2]; sh -= nr2 * sm.hRT[rs2]; }
        if (ps0 >= 0) { pp0 = ipow3(sm.c[ps0], np0); sg += np0 * sm.gRT[ps0]; sh += np0 * sm.hRT[ps0]; }
        if (ps1 >= 0) { pp1 = ipow3(sm.c[ps1], np1); sg += np1 * sm.gRT[ps1]; sh += np1 * sm.hRT[ps1]; }
        if (ps2 >= 0) { pp2 = ipow3(sm.c[ps2], np2); sg += np2 * sm.gRT[ps2]; sh += np2 * sm.hRT[ps2]; }
        const double lnKc = dnu * lnPaRT - sg;
        const double kf = exp(lnkf);
        const double kb = exp(lnkf - lnKc);
        const double Pf = pr0 * pr1 * pr2, Pb = pp0 * pp1 * pp2;
        const int tb = flags & 1;
        const int doff = (flags >> 1) & 0xFFFFF, dcnt = (flags >> 21) & 0x3FF;
        double CM = 1.0;
        if (tb) {
            CM = ctot;
            for (int j = doff; j < doff + dcnt; ++j)
                CM += __ldg(m.deff + j) * sm.c[__ldg(m.dcol + j) & 0xff];
        }
        const double fwd = kf * Pf, rev = kb * Pb, q = fwd - rev;
        sm.Q[r] = CM * q;
        sm.qtb[r] = tb ? q : 0.0;
        const double dlnkf = beta * invT + EaR * invT * invT;
        const double dlnKc = (sh - dnu) * invT;
        sm.dQdT[r] = CM * (fwd * dlnkf - rev * (dlnkf - dlnKc));
        // d Q_r / d rho_k for the species the rate depends on, without the
        // all-ones third-body part (added below as a rank-1 term)
        for (int j = doff; j < doff + dcnt; ++j) {
            const int pk = __ldg(m.dcol + j);
            const int k = pk & 0xff, rsl = (pk >> 8) & 3, psl = (pk >> 10) & 3;
            double dPf = 0.0, dPb = 0.0;
            if (rsl == 0) dPf = nr0 * ipow3(sm.c[k], nr0 - 1) * pr1 * pr2;
            else if (rsl == 1) dPf = nr1 * ipow3(sm.c[k], nr1 - 1) * pr0 * pr2;
            else if (rsl == 2) dPf = nr2 * ipow3(sm.c[k], nr2 - 1) * pr0 * pr1;
            if (psl == 0) dPb = np0 * ipow3(sm.c[k], np0 - 1) * pp1 * pp2;
            else if (psl == 1) dPb = np1 * ipow3(sm.c[k], np1 - 1) * pp0 * pp2;
            else if (psl == 2) dPb = np2 * ipow3(sm.c[k], np2 - 1) * pp0 * pp1;
            const double d = CM * (kf * dPf - kb * dPb) + __ldg(m.deff + j) * q;
            sm.D[j] = (JT)(d * __ldg(m.sp + k * kSpStride + 1));
        }
    }
    __syncwarp();

    // species sources (Eq. 26) and the two rank-1 vectors of the Jacobian
    double wde = 0.0, wE = 0.0, uE = 0.0;
    for (int s = sl; s < ns; s += G) {
        double sq = 0.0, sdq = 0.0, squ = 0.0;
        const int e0 = __ldg(m.sp_ptr + s), e1 = __ldg(m.sp_ptr + s + 1);
        for (int e = e0; e < e1; ++e) {
            const int ent = __ldg(m.sp_ent + e);
            const int r = ent >> 8;
            const double nu = (double)(signed char)(ent & 0xff);
            sq += nu * sm.Q[r];
            sdq += nu * sm.dQdT[r];
            squ += nu * sm.qtb[r];
        }
        const double M = __ldg(m.sp + s * kSpStride);
        const double ef = __ldg(m.sp + s * kSpStride + 3);
        const double wds = M * sq, ws = M * sdq, us = M * squ;
        sm.wd[s] = wds;
        sm.w[s] = (JT)ws;
        sm.u[s] = (JT)us;
        wde -= ef * wds;
        wE += ef * ws;
        uE += ef * us;
    }
    wde = Grp<G>::sum(wde);
    wE = Grp<G>::sum(wE);
    uE = Grp<G>::sum(uE);
    __syncwarp();

    // right-hand side -F = -(x - x0 - h Omega(x))
    for (int i = sl; i < n; i += G) {
        const double om = i < ns ? sm.wd[i] : wde;
        sm.A[i * lda + n] = (JT)(-(sm.x[i] - sm.x0[i] - h * om));
    }
    // species rows of A = I - h J
    const JT hj = (JT)h;
    for (int idx = sl; idx < ns * n; idx += G) {
        const int s = idx / n, k = idx - (idx / n) * n;
        JT J;
        if (k < ns) {
            J = sm.w[s] * sm.dTdr[k] + sm.u[s] * (JT)__ldg(m.sp + k * kSpStride + 1);
            const int g = __ldg(m.jmap + s * ns + k);
            if (g >= 0) {
                JT acc = 0;
                const int e0 = __ldg(m.j_ptr + g), e1 = __ldg(m.j_ptr + g + 1);
                for (int e = e0; e < e1; ++e) {
                    const int ent = __ldg(m.j_ent + e);
                    acc += (JT)(signed char)(ent & 0xff) * sm.D[ent >> 8];
                }
                J += (JT)__ldg(m.sp + s * kSpStride) * acc;
            }
        } else {
            J = sm.w[s] * (JT)dTde;
        }
        sm.A[s * lda + k] = (s == k ? (JT)1 : (JT)0) - hj * J;
    }
    // energy row: J_ek = -sum_s e_f,s J_sk, gathered per column
    for (int k = sl; k < n; k += G) {
        JT J;
        if (k < ns) {
            JT acc = 0;
            const int e0 = __ldg(m.col_ptr + k), e1 = __ldg(m.col_ptr + k + 1);
            for (int e = e0; e < e1; ++e) {
                const int j = __ldg(m.col_ent + e);
                acc += (JT)__ldg(m.dEf + j) * sm.D[j];
            }
            J = -((JT)wE * sm.dTdr[k] + (JT)uE * (JT)__ldg(m.sp + k * kSpStride + 1) + acc);
        } else {
            J = -(JT)(wE * dTde);
        }
        sm.A[ns * lda + k] = (k == ns ? (JT)1 : (JT)0) - hj * J;
    }
    __syncwarp();

    // Gaussian elimination with row partial pivoting on [A | -F] (Sec. 3.2),
    // ties to the lowest row; the pivot's reciprocal replaces the diagonal
    bool sing = false;
    for (int j = 0; j < n; ++j) {
        double best = -1.0;
        int bi = n;
        for (int i = j + sl; i < n; i += G) {
            const double v = fabs((double)sm.A[i * lda + j]);
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        Grp<G>::argmax(best, bi);
        if (!(best > 0.0) || isinf(best)) sing = true;
        if (bi != j && bi < n) {
            for (int k = j + sl; k <= n; k += G) {
                const JT t = sm.A[j * lda + k];
                sm.A[j * lda + k] = sm.A[bi * lda + k];
                sm.A[bi * lda + k] = t;
            }
        }
        __syncwarp();
        const JT inv = (JT)1 / sm.A[j * lda + j];
        for (int i = j + 1 + sl; i < n; i += G) sm.A[i * lda + j] *= inv;
        __syncwarp();
        if (sl == 0) sm.A[j * lda + j] = inv;
        const int cols = n - j;
        const int tot = (n - j - 1) * cols;
        for (int e = sl; e < tot; e += G) {
            const int i = j + 1 + e / cols, k = j + 1 + e % cols;
            sm.A[i * lda + k] -= sm.A[i * lda + j] * sm.A[j * lda + k];
        }
        __syncwarp();
    }
    // back substitution, U delta = y
    for (int j = n - 1; j >= 0; --j) {
        const JT dj = sm.A[j * lda + n] * sm.A[j * lda + j];
        __syncwarp();
        if (sl == 0) sm.A[j * lda + n] = dj;
        for (int i = sl; i < j; i += G) sm.A[i * lda + n] -= sm.A[i * lda + j] * dj;
        __syncwarp();
    }
    // update and convergence norm
    double nrm = 0.0;
    int nonfinite = 0;
    for (int i = sl; i < n; i += G) {
        const double d = (double)sm.A[i * lda + n];
        const double xi = sm.x[i] + d;
        sm.x[i] = xi;
        if (!isfinite(xi)) nonfinite = 1;
        const double at = i < ns ? atol_rho : atol_e;
        nrm = fmax(nrm, fabs(d) / (rtol * fabs(xi) + at));
    }
    nrm = Grp<G>::max(nrm);
    nonfinite = Grp<G>::any(nonfinite);
    __syncwarp();
    norm = nrm;
    bad = sing || nonfinite;
}

template <int G, typename JT>
__global__ void __launch_bounds__(256) be_kernel(DeviceMech m, StepOptions o, StepBatch b) {
    extern __shared__ __align__(16) char smem[];
    constexpr int S = 32 / G;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int slot = lane / G;
    const int sl = lane - slot * G;
    const int ns = m.ns, n = ns + 1;
    const long long sbytes = slot_bytes(ns, m.nr, m.nD, (int)sizeof(JT));
    SlotMem<JT> sm;
    sm.carve(smem + (size_t)(warp * S + slot) * sbytes, ns, m.nr, m.nD);

    int state = kFree;
    long long cell = -1;
    double T = 1500.0, T0 = 1500.0, Tin = CUDART_NAN, h = 0.0, norm_prev = CUDART_INF;
    double atol_rho = 0.0, atol_e = 0.0;
    int k = 0, level = 0, attempts = 0, iters = 0, subs = 0, fails = 0;
    long long t_units = 0;
    const long long total = 1LL << o.max_halvings;

    auto write_fail = [&](int code) {
        if (sl == 0) {
            if (b.status) b.status[cell] = code;
            if (b.T_out) b.T_out[cell] = Tin;
            if (b.newton_iters) b.newton_iters[cell] = iters;
            if (b.substeps) b.substeps[cell] = subs;
            if (b.failures) b.failures[cell] = fails;
        }
        state = kFree;
    };
    auto start_substep = [&]() {
        if (attempts >= o.max_attempts) {
            write_fail(kCellTooManySteps);
            return;
        }
        while ((total >> level) > total - t_units) ++level;
        h = ldexp(b.dt, -level);
        ++attempts;
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

    for (;;) {
        // refill free slots and settle every pending temperature recovery
        for (int pass = 0; pass < 2; ++pass) {
            long long got = -1;
            if (state == kFree && sl == 0) got = (long long)atomicAdd(b.work_counter, 1ULL);
            got = __shfl_sync(kFull, got, slot * G);
            const bool loading = state == kFree && got < b.n_cells;
            if (state == kFree && !loading) state = kDead;
            int nonfin = 0;
            double rt = 0.0, es = 0.0;
            if (loading) {
                cell = got;
                iters = subs = fails = 0;
                Tin = CUDART_NAN;
                for (int i = sl; i < n; i += G) {
                    const double v = i < ns ? b.rho[(size_t)i * b.ld + cell] : b.e[cell];
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
                T = b.T_in ? b.T_in[cell] : 1500.0;
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
            recover_T<G>(m, sm.x, sl, needT, T, Tr, ok);
            __syncwarp();
            int neg = 0;
            for (int i = sl; i < ns; i += G)
                if (sm.x[i] < -atol_rho) neg = 1;
            neg = Grp<G>::any(neg);
            if (state == kInitT) {
                if (!ok) {
                    write_fail(kCellTFailed);
                } else {
                    T = T0 = Tin = Tr;
                    if (b.dt == 0.0) {
                        if (sl == 0) {
                            if (b.status) b.status[cell] = kCellOk;
                            if (b.T_out) b.T_out[cell] = Tr;
                            if (b.newton_iters) b.newton_iters[cell] = 0;
                            if (b.substeps) b.substeps[cell] = 0;
                            if (b.failures) b.failures[cell] = 0;
                        }
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
                    // accept the substep
                    for (int i = sl; i < n; i += G) sm.x0[i] = sm.x[i];
                    T0 = T;
                    t_units += total >> level;
                    ++subs;
                    if (level > 0) --level;
                    if (t_units == total) {
                        for (int i = sl; i < n; i += G) {
                            if (i < ns)
                                b.rho[(size_t)i * b.ld + cell] = sm.x[i];
                            else
                                b.e[cell] = sm.x[i];
                        }
                        if (sl == 0) {
                            if (b.status) b.status[cell] = kCellOk;
                            if (b.T_out) b.T_out[cell] = T;
                            if (b.newton_iters) b.newton_iters[cell] = iters;
                            if (b.substeps) b.substeps[cell] = subs;
                            if (b.failures) b.failures[cell] = fails;
                        }
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
            continue;
        }
        // one Newton iteration of Eq. 29 for every slot
        double norm = 0.0;
        bool bad = false;
        newton_iteration<G, JT>(m, sm, sl, T, h, atol_rho, atol_e, o.rtol, norm, bad);
        if (state == kNewtonReady) {
            ++iters;
            if (bad) {
                substep_fail();
            } else if (o.point_implicit || norm <= 1.0) {
                state = kCheckT;
            } else if (o.div_check && k >= 2 && norm >= norm_prev) {
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
