// chem_internal.h -- device table layout and kernel parameters of libchem.
#pragma once

#include <cstdint>

#include <vector_types.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace chem {

// Physical constants of the CUDA path.
constexpr double kR = 8.314462618;     // universal gas constant, J/(mol K)
constexpr double kPa = 101325.0;       // standard pressure in K_e (Eq. 24), Pa
constexpr double kTref = 298.15;       // reference of the formation energies, K
constexpr double kTlo = 200.0;         // temperature-recovery bracket, K
constexpr double kThi = 6000.0;
constexpr int kTmaxIter = 50;          // temperature-recovery iterations
constexpr double kTtol = 1e-13;        // |dT| <= kTtol * T ends the recovery

// Thermo table row per species and range (16 doubles):
//   0..4  cp/R coefficients a1..a5
//   5..8  h/RT coefficients a2/2, a3/3, a4/4, a5/5 (a1 and a6 shared)
//   9     a6
//   10..12 s/R coefficients a3/2, a4/3, a5/4 (a1, a2 shared)
//   13    a7
constexpr int kThermoStride = 16;

// Species table row (4 doubles): M, 1/M, R/M, e_f = e_s(T_ref).
constexpr int kSpStride = 4;

// Reaction table row (4 doubles): ln A_SI, beta, Ea/R, sum nu.
constexpr int kRxnDStride = 4;

// Reaction factor words (2 ints per reaction): the reactant concentration
// factors of prod_s [X_s]^nu'_s listed with repetition (e.g. 2 O -> O, O),
// padded with the sentinel species index ns (whose concentration is 1 and
// whose g/RT and h/RT are 0), 8 bits each in bits 0..23, plus the third-body
// flag in bit 24; then the product factors the same way.
constexpr int kRxnFStride = 2;

// Species-gather chunk length (entries per work item).
constexpr int kChunk = 8;

// Entries of the exp table (2^(j/kExpTab)).
constexpr int kExpTab = 256;

// D entries: one per (reaction r, species k) pair whose concentration the
// progress rate Q_r depends on, holding dQ_r/drho_k without the all-ones
// third-body part.  They are sorted into four groups so each group is one
// uniform loop: reactant-only, product-only, both sides, efficiency-only.
//   d_i0 = r | k << 16
//   d_i1 = fa | fb << 8 | ba << 16 | bb << 24  (the remaining factors of
//          d(prod c)/dc_k on each side, sentinel ns if none)
//   d_c  = {nu'_rk / M_k, nu''_rk / M_k, (alpha_rk - 1) / M_k}
struct DeviceMech {
    int ns, nr;
    int nD, nD_F, nD_B, nD_FB;  // group ends: [0,F) [F,B) [B,FB) [FB,nD)
    int nJ;                     // Jacobian entries gathered: ns*ns species, ns energy-row
    int n_items;                // species-gather work items
    const double *thermo;       // [ns][2][16]
    const double *tmid;         // [ns]
    const double *sp;           // [ns][4]
    const double *rxn_d;        // [nr][4]
    const int *rxn_f;           // [nr][2]
    const int *eff_ptr;         // [nr+1] CSR of efficiency corrections of +M reactions
    const int *eff_sp;          //        species
    const double *eff_c;        //        alpha - 1
    const int *d_i0;            // [nD]
    const int *d_i1;            // [nD]
    const double *d_c;          // [nD][3]
    const int *j_sk;            // [nJ] s << 8 | k (s = ns: energy row), longest gather list first
    const int *j_ptr;           // [nJ+1]
    const int *j_d;             // D index of each gather term
    const double *j_c;          // nu_rs M_s of each gather term; -sum_s nu_rs M_s e_f,s in the energy row
    const int *it_ptr;          // [n_items+1] ranges of the species lists
    const int *sp_item_ptr;     // [ns+1] work items of each species
    const int *sp_r;            // reactions with nu_rs != 0, per species
    const double *sp_nu;        // nu_rs
    const double *exp_tab;      // [kExpTab] 2^(j/kExpTab)
    // FP32 copies for the mixed-precision Jacobian
    const float *rxn_df;        // [nr][4] beta, Ea/R, sum nu, 0
    const float *d_cf;          // [nD][3]
    const int2 *j_pk;           // gather terms as {D index, FP32 coefficient bits}
    const int2 *sp_pk;          // species lists as {reaction, FP32 nu_rs bits}
    const float *spf;           // [ns][4] M, 1/M, R/M, e_f in FP32
};

struct StepOptions {
    double rtol, atol_rel, conv_kappa;
    int max_newton, max_halvings, max_attempts, point_implicit, div_check;
};

struct StepBatch {
    long long n_cells, ld;
    double *rho;
    double *e;
    double dt;
    const double *T_in;
    double *T_out;
    int *status;
    int *newton_iters;
    int *substeps;
    int *failures;
    unsigned long long *work_counter;   // zeroed before the launch
};

// Per-cell status codes (same values as the public CHEM_CELL_*).
enum CellStatus { kCellOk = 0, kCellNewtonFailed = 1, kCellTFailed = 2, kCellBadInput = 3,
                  kCellTooManySteps = 4 };

// Shared memory of a block: one region per cell slot (no block header; the
// exp table is read through L1).
constexpr int kBlockHeaderBytes = 0;

// The D region of a slot holds the nD D entries (Jacobian type) and, earlier
// in each Newton iteration, the species-gather partial sums (3 doubles per
// work item); its size in 8-byte units:
__host__ __device__ inline int dreg8_for(int nD, int n_items, int jt) {
    const int a = (nD * jt + 7) / 8, b = 3 * n_items;
    return a > b ? a : b;
}

// Bytes of one cell slot, in this order:
//   doubles  x, x0 (n each); c, hRT, gRT with a sentinel (ns+1 each); es, wd (ns each)
//   JT       dTdr (ns); w, u (ns+1 each: the species rows' T-derivative and
//            third-body vectors, then the energy row's); for FP32 also c and
//            hRT copies (ns+1 each)
//   D region dreg8 * 8 bytes
//   union    the per-reaction values Q (double) and dQdT, qtb, A1, A2 (JT),
//            dead once the D entries exist, and the augmented matrix
//            n x (n+1) in JT, which is written after that
__host__ __device__ inline long long slot_small_bytes(int ns, int jt) {
    const long long cnt = 3LL * ns + 2 + (jt == 4 ? 2LL * (ns + 1) : 0);
    return (cnt * jt + 15) / 16 * 16;
}
__host__ __device__ inline long long slot_union_bytes(int ns, int nr, int jt) {
    const int n = ns + 1;
    const long long a = (long long)nr * 8 + 4LL * nr * jt, b = (long long)n * (n + 1) * jt;
    return ((a > b ? a : b) + 15) / 16 * 16;
}
__host__ __device__ inline long long slot_bytes_for(int ns, int nr, int nD, int n_items, int jt) {
    const int n = ns + 1;
    const long long dbl = (2LL * n + 3LL * (ns + 1) + 2LL * ns) * 8;
    const long long dreg = ((long long)dreg8_for(nD, n_items, jt) * 8 + 15) / 16 * 16;
    return (dbl + 15) / 16 * 16 + slot_small_bytes(ns, jt) + dreg + slot_union_bytes(ns, nr, jt);
}

}  // namespace chem
