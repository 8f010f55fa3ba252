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
constexpr double kLnPaOverR = 9.408091968961747;   // ln(kPa / kR), rounded from 40 digits
constexpr double kTlo = 200.0;         // temperature-recovery bracket, K
constexpr double kThi = 6000.0;
constexpr int kTmaxIter = 50;          // temperature-recovery iterations
constexpr double kTtol = 1e-13;        // |dT| <= kTtol * T ends the recovery

// Polynomial tables are stored coefficient-major, so that the lanes of a
// warp, which hold consecutive species, read consecutive words: coefficient
// c of species s in temperature range rg (0: T <= T_mid, 1: above) at
// [(2 c + rg) ns + s].  (The reaction tables stay row-major: a lane reads
// a reaction's row with two 16-byte loads, which measured faster.)
//
// Thermo table, per species and range (16 coefficients):
//   0..4  cp/R coefficients a1..a5
//   5..8  h/RT coefficients a2/2, a3/3, a4/4, a5/5 (a1 and a6 shared)
//   9     a6
//   10..12 s/R coefficients a3/2, a4/3, a5/4 (a1, a2 shared)
//   13    a7
constexpr int kThermoStride = 16;

// Energy polynomials per species and range (12 coefficients), the NASA-7 forms
// multiplied out with R/M and shifted by the formation energy:
//   0..5  e_s(T) - e_f,s = c0 + c1 T + ... + c5 T^5  (c0 = R/M a6 - e_f,
//         c1 = R/M (a1 - 1), c_i = R/M a_i / i for i = 2..5)
//   6..10 c_v,s(T) = R/M (cp/R - 1) = d0 + d1 T + ... + d4 T^4
// and an FP32 copy of d0..d4 (8 coefficients).
constexpr int kTpolyStride = 12;
constexpr int kTpolyFStride = 8;

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

// Threads per block of the step kernel at most (its launch bounds: two
// such blocks per SM, at most 102 registers per thread).
constexpr int kMaxBlockThreads = 320;

// Entries of the exp table (2^(j/kExpTab)).
constexpr int kExpTab = 256;
// Intervals of the log table: kLogTab + 1 entries {1/F, ln F}, F = 1 + j/kLogTab.
constexpr int kLogTab = 128;

// D entries: one per (reaction r, species k) pair whose concentration the
// progress rate Q_r depends on, holding dQ_r/drho_k without the all-ones
// third-body part.  They are sorted into four groups so each group is one
// uniform loop: reactant-only, product-only, both sides, efficiency-only.
//   d_pk = {r | nu'_rk << 16 | nu''_rk << 20,
//           fa | fb << 8 | ba << 16 | bb << 24  (the remaining factors of
//                d(prod c)/dc_k on each side, sentinel ns if none)}
//   d_ce  = alpha_rk - 1 (FP64 kernel), d_cef the same in FP32 (FP32
//           kernel).  Both kernels' D entries are M_k dQ_r/drho_k, with the
//           orders nu'_rk, nu''_rk from the descriptor: the 1/M_k is applied
//           once per Jacobian entry in the gather
// Gather lists laid out for G lanes per cell.  List p (a Jacobian entry, or
// an item of a species list) runs in pass p / G on lane p % G; its q-th term
// sits at word base + q G + lane, where base is the pass's first word, so the
// lanes of a pass read their q-th terms from consecutive words (one cache
// line per warp load instead of one per lane).
//   The ns*ns species entries (the kernels eliminate the energy unknown, so
//   no energy row is gathered), longest list first, in both forms:
//     j_meta[p]   = {first word of entry p, k | s << 8 | terms << 16}
//     j_d, j_c    = D index and coefficient nu_rs M_s (FP64 kernel)
//     j_meta32[p] = as j_meta, with the FP32 lists' own word positions
//     j_w         = D index (bits 0..22) | the sign and exponent bits of
//                   (float)nu_rs (FP32 kernel: the row's M_s multiplies the
//                   sum; terms ordered across the lanes of a pass for
//                   distinct shared-memory banks)
//   it_meta[i] = {first word of item i, entries}
//   sp_w       = r (bits 0..19) | the sign and exponent bits of (double)nu_rs
// (nu_rs a signed power of two in the words: any other nu_rs is split into
// one term per binary digit)
struct GatherLayout {
    const int2 *j_meta;
    const int4 *j_meta32;       // FP32 lists: {first word, length, matrix offset k ldc + s, (float)(M_s / M_k)}
    const unsigned *j_w;
    const int *j_d;
    const double *j_c;
    const int2 *it_meta;
    const unsigned *sp_w;
};
constexpr int kLayouts = 5;   // G = 2, 4, 8, 16, 32
__host__ __device__ constexpr int layout_index(int G) {
    return G == 2 ? 0 : G == 4 ? 1 : G == 8 ? 2 : G == 16 ? 3 : 4;
}

struct DeviceMech {
    int ns, nr;
    int ntb;                    // third-body reactions: the first ntb (internal order)
    int nD, nD_F, nD_B, nD_FB;  // group ends: [0,F) [F,B) [B,FB) [FB,nD)
    int nJ;                     // Jacobian entries gathered: ns*ns (species rows and columns)
    int nJ_nz;                  //   of which the first nJ_nz have reaction terms (longest list first)
    int n_items;                // species-gather work items
    const double *thermo;       // [16][2][ns] (coefficient-major, above)
    const double *tmid;         // [ns] (positive: compared as integers)
    const double *tpoly;        // [12][2][ns] energy and heat-capacity polynomials
    const float *tpoly_f;       // [8][2][ns] heat-capacity polynomial in FP32
    const double *sp;           // [ns][4]
    const double *rxn_d;        // [nr][4] ln A (SI), beta, E/R, sum nu
    const int *rxn_f;           // [nr][2]
    const int *eff_ptr;         // [nr+1] CSR of efficiency corrections of +M reactions
    const int *eff_sp;          //        species
    const double *eff_c;        //        alpha - 1
    const int2 *d_pk;           // [nD]
    const double *d_ce;         // [nD] alpha - 1 (FP64 kernel)
    // Jacobian entries (species rows and columns), longest gather list
    // first, and the species lists (reactions with nu_rs != 0) cut into
    // items of at most kChunk entries; per-G layouts above
    GatherLayout gl[kLayouts];
    const int *sp_item_ptr;     // [ns+1] work items of each species
    const double *exp_tab;      // [kExpTab] 2^(j/kExpTab)
    const double2 *log_tab;     // [kLogTab + 1] {1/F, ln F}, F = 1 + j/kLogTab
    const unsigned *div16;      // [67] ceil(2^16 / c): x / c = (x div16[c]) >> 16 for x < 64
    // FP32 copies for the mixed-precision Jacobian
    const float *rxn_df;        // [nr][4] beta, Ea/R, sum nu, 0
    const float *d_cef;         // [nD] alpha - 1 in FP32
    const float *spf;           // [ns][4] M, 1/M, R/M, e_f in FP32
};

struct StepOptions {
    double rtol, atol_rel, conv_kappa;
    int max_newton, max_halvings, max_attempts, point_implicit, div_check;
};

// Device work queue of the request server: requests published in a ring of
// descriptors in host memory mapped into the device's address space.  (The
// server publishes requests in chunks of at most 2^kServeChunkLog cells, one
// descriptor each, interleaved across requests; to the kernel a chunk is a
// request.)  Chunk `seq` owns the virtual cells [seq, seq + 1) *
// 2^kServeChunkLog, of which its first n_cells are real.  Chunks are handed
// out in order: a warp's free slots take consecutive cells of the current
// chunk together, by one atomic add on the chunk's claim counter (which
// never fails, unlike a compare-and-swap on a shared position, whose
// attempts collide at millions of claims per second); a claim past the
// chunk's cells moves the current chunk on.  The slots step their cells and
// count them done; the slot that completes a chunk's last cell resets the
// entry's completion counters and publishes the chunk's completion record.
//   Reads of mapped host memory cross the chip-to-chip link, and thousands of
// warps issuing them stall one another, so the kernels keep device copies:
// of `tail` and the launch's budget, refreshed by one warp at a time at most
// every kServePollNs, and of each chunk's descriptor, copied into a device
// ring by the first warp that claims from the chunk.
constexpr long long kServePollNs = 2000;
// A claim counter holds the ring lap of the chunk it counts (chunk / cap) in
// its high bits, so a claim through a stale chunk number is recognised.
constexpr int kClaimLapShift = 40;
constexpr int kServeChunkLog = 10;
struct ServeDesc {              // host-written, one per ring entry
    long long seq;              // chunk sequence number held by the entry
    long long start, n_cells;   // its first virtual cell (seq << kServeChunkLog) and cell count
    long long ld;               // leading dimension of rho
    double *rho, *e, *T_out;    // device state and optional output
    int *status;                // optional per-cell status
    double dt;
    long long pad;
};
struct ServeDone {              // kernel-written, one per ring entry
    long long seq;              // written last: the request with this seq is done
    unsigned long long t_first; // globaltimer (ns) of its first cell's claim
    unsigned long long t_last;  // and of its last cell's completion
    long long pad;
};
struct ServeQueue {
    const ServeDesc *desc;              // [cap], mapped host memory
    ServeDone *fin;                     // [cap], mapped host memory
    const unsigned long long *tail;     // mapped host: end of the last published chunk's real cells
    unsigned long long *front;          // mapped host: the current chunk's first virtual cell, for the host's window
    const int *budget;                  // mapped host: this launch's blocks >= budget claim nothing
    ServeDesc *mdesc;                   // device [cap]: copies of the descriptors (seq -1: none)
    unsigned long long *dtail;          // device: the latest `tail` read
    int *dbudget;                       // device: the latest budget read (set before the launch)
    unsigned long long *dpoll;          // device: globaltimer of the last read of the host values
    unsigned long long *chunk;          // device: the chunk being handed out
    unsigned long long *claimed;        // device [cap]: lap << kClaimLapShift | cells claimed
    unsigned long long *done;           // device [cap]: cells done per entry
    unsigned long long *t_first;        // device [cap]
    unsigned long long *t_last;         // device [cap]
    int cap;
    long long linger_ns;                // a warp with no work waits this long for more, then exits
    int *error;                         // device: set when a claim finds a ring entry out of order
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
    // optional record of the substep schedule: kSchedWords words per cell,
    // bit a set when attempt a was accepted (the attempt budget is capped at
    // 32 kSchedWords while recording)
    unsigned *schedule;
    // optional record of the state after each of a cell's first kSubstepStates
    // accepted substeps: [cell][substep][ns + 1]
    double *substep_states;
    // request-server mode (the kernel's queue instantiation): cells come from
    // this queue instead of [0, n_cells) of the buffers above
    ServeQueue queue;
};

// Words of the per-cell substep-schedule record (256 attempts).
constexpr int kSchedWords = 8;
// Accepted substeps whose states a cell records.
constexpr int kSubstepStates = 32;

// Per-cell status codes (same values as the public CHEM_CELL_*).
enum CellStatus { kCellOk = 0, kCellNewtonFailed = 1, kCellTFailed = 2, kCellBadInput = 3,
                  kCellTooManySteps = 4 };

// Shared memory of a block: one region per cell slot (no block header; the
// exp table is read through L1).
constexpr int kBlockHeaderBytes = 0;

// Bytes of one cell slot, in this order (jt = sizeof of the Jacobian type):
//   doubles   x, x0 (n each); FP64 path also es (ns)
//   JT        FP64 path: dTdr, w, u, rhs (ns each: the reduced system's
//             temperature column factor, the T-derivative and third-body
//             vectors, the right-hand side)
//             FP32 path: w, u, rhs, es (ns each, padded to a multiple of 4)
//   D region  first Q (nr doubles) and the species-gather partial sums (per
//             item: sum nu Q in FP64, then sum nu dQ/dT and sum nu q_tb in JT),
//             which are dead once the D entries (nD in JT) are written
//   union     while the rates, sources and D entries are formed: the species
//             values with a sentinel (ns+1 each) c, em, emi (doubles), FP64
//             path hRT (double), ek (int), FP32 path cJ, hJ (float), then the
//             per-reaction values dQdT, A1, A2 (nr JT each) and qtb (ntb JT);
//             after the D entries: the augmented matrix ns x (ns+1) in JT
//             (the energy unknown is eliminated), FP64 row-major, FP32
//             column-major with columns padded to a multiple of 4 rows
__host__ __device__ inline long long align16(long long b) { return (b + 15) / 16 * 16; }

#ifdef __CUDACC__
// The coefficients of one species and range of a coefficient-major
// polynomial table, read through the read-only path: p[c].
template <typename T>
struct CoefRow {
    const T *p;
    int stride;
    __device__ __forceinline__ T operator[](int c) const { return __ldg(p + (size_t)c * stride); }
};
template <typename T>
__device__ __forceinline__ CoefRow<T> coef_row(const T *tab, int ns, int s, int rg) {
    return CoefRow<T>{tab + (size_t)rg * ns + s, 2 * ns};
}
#endif
__host__ __device__ inline long long slot_dbl_bytes(int ns, int jt) {
    const int n = ns + 1;
    return align16((2LL * n + (jt == 8 ? ns : 0)) * 8);
}
// the FP32 path's w, u, rhs and e_s arrays are padded to a multiple of four
// entries, so that the Jacobian's dense part reads them as 16-byte vectors
__host__ __device__ inline int small_stride(int ns, int jt) { return jt == 8 ? ns : (ns + 3) & ~3; }
__host__ __device__ inline long long slot_small_bytes(int ns, int jt) {
    return align16(4LL * small_stride(ns, jt) * jt);
}
// species part of the union: c, em, emi (+ hRT) doubles, ek ints (+ cJ, hJ
// floats), padded to 16 bytes so the per-reaction arrays that follow are
// aligned
__host__ __device__ inline long long slot_union_species_bytes(int ns, int jt) {
    const long long m = ns + 1;
    return align16(m * 8 * (jt == 8 ? 4 : 3) + m * 4 * (jt == 8 ? 1 : 3));
}
__host__ __device__ constexpr long long item_bytes(int jt) { return 8 + 2LL * jt; }
__host__ __device__ inline long long slot_dreg_bytes(int nr, int nD, int n_items, int jt) {
    const long long a = (long long)nD * jt, b = (long long)nr * 8 + (long long)n_items * item_bytes(jt);
    return align16(a > b ? a : b);
}
__host__ __device__ inline long long slot_union_bytes(int ns, int nr, int ntb, int jt) {
    const int n = ns + 1;
    // the matrix: FP64 ns rows of n; FP32 n columns of ns rounded up to 4
    const long long a = slot_union_species_bytes(ns, jt) + 3LL * nr * jt + (long long)ntb * jt,
                    b = jt == 8 ? (long long)ns * n * jt : (long long)n * ((ns + 3) & ~3) * jt;
    return align16(a > b ? a : b);
}
__host__ __device__ inline long long slot_bytes_for(const DeviceMech &m, int jt) {
    return slot_dbl_bytes(m.ns, jt) + slot_small_bytes(m.ns, jt) + slot_dreg_bytes(m.nr, m.nD, m.n_items, jt) +
           slot_union_bytes(m.ns, m.nr, m.ntb, jt);
}
// Stride between the cell slots of a block.  With several slots per warp
// (lanes per cell below 32) the slots' equal offsets must fall in different
// shared-memory banks, so the stride is an odd multiple of 16 bytes: the
// S = 32 / G slots of a warp then start in S distinct 16-byte bank groups
// (S <= 8).  A stride that is a multiple of 128 bytes put all eight slots
// of a 4-lane warp in the same banks and cost the 9-species mixed path 20 %.
__host__ __device__ inline long long slot_stride(const DeviceMech &m, int jt, int G) {
    long long b = slot_bytes_for(m, jt);
    if (G < 32 && ((b >> 4) & 1) == 0) b += 16;
    return b;
}

}  // namespace chem
