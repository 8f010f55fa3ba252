// chem_internal.h -- device table layout and kernel parameters of libchem.
#pragma once

#include <cstdint>

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

// Reaction table row (8 doubles): ln A_SI, beta, Ea/R, sum nu, Ef_r, 0, 0, 0
// where Ef_r = sum_s nu_rs M_s e_f,s (formation energy per unit progress).
constexpr int kRxnDStride = 8;

// Reaction integer row (8 ints):
//   0..2 reactant species (-1 unused), 3..5 product species (-1 unused),
//   6    nu packing: reac nu in bits 0..5 (2 bits each), prod nu in bits 8..13
//   7    third-body flag (bit 0) | D offset << 1 (bits 1..20) | D count << 21
constexpr int kRxnIStride = 8;

// D column packing (one per (reaction, species) pair the reaction's rate
// depends on): species in bits 0..7, reactant slot in bits 8..9 (3 = none),
// product slot in bits 10..11 (3 = none).
struct DeviceMech {
    int ns, nr, nD, nnz, nsp_ent, ncol_ent;
    const double *thermo;     // [ns][2][16]
    const double *tmid;       // [ns]
    const double *sp;         // [ns][4]
    const double *rxn_d;      // [nr][8]
    const int *rxn_i;         // [nr][8]
    const int *dcol;          // [nD] packed column descriptor
    const double *deff;       // [nD] alpha_rk - 1 for +M reactions, else 0
    const double *dEf;        // [nD] Ef of the entry's reaction
    const int *sp_ptr;        // [ns+1] CSR: reactions with nu_rs != 0 per species
    const int *sp_ent;        // (r << 8) | (nu & 0xff)
    const int *jmap;          // [ns*ns] species-block entry -> gather row, -1 = none
    const int *j_ptr;         // [nnz+1]
    const int *j_ent;         // (d_index << 8) | (nu & 0xff)
    const int *col_ptr;       // [ns+1] D entries per column species (energy row)
    const int *col_ent;       // D indices
};

struct StepOptions {
    double rtol, atol_rel;
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

// Shared-memory bytes of one cell slot for a mechanism and Jacobian type size.
inline long long slot_smem_bytes(int ns, int nr, int nD, int jt_bytes) {
    const int n = ns + 1;
    long long dbl = 2LL * n + 8LL * ns + 3LL * nr;          // x, x0, species arrays, rates
    long long jt = (long long)nD + (long long)n * (n + 1);  // D and augmented A
    long long bytes = dbl * 8 + jt * jt_bytes;
    return (bytes + 15) / 16 * 16;
}

}  // namespace chem
