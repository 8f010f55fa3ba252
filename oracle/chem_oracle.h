/*
 * chem_oracle.h -- plain FP64 CPU oracle for the operator-split implicit
 * chemistry step of Le & Cambier, "Development of a Flow Solver with Complex
 * Kinetics on the Graphic Processing Units" (arXiv 1110.4903).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct reference the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library.
 *
 * Units: SI (kg, m, s, mol, K, J) except the Arrhenius pre-exponential factor,
 * which is given in CGS mol-cm-s units for the forward order of the reaction.
 *
 * Each function cites the passage of the paper it follows.  Where the paper
 * is silent, the reading taken is stated beside the function.
 */
#ifndef CHEM_ORACLE_H
#define CHEM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Mechanism, as plain arrays (all host memory, owned by the caller). */
typedef struct om_mech {
    int ns;                    /* number of species N_s                        */
    int nr;                    /* number of reversible reactions               */
    int ne;                    /* number of elements                           */
    const double *molar_mass;  /* [ns] kg/mol                                  */
    const int    *elem_comp;   /* [ns*ne] atoms of element j in species s      */
    const double *nasa7;       /* [ns][2][7] NASA-7 a1..a7: low range, high range */
    const double *t_mid;       /* [ns] range switch temperature, K             */
    const double *arr_A;       /* [nr] CGS, (cm^3/mol)^(m-1)/s, m = forward order incl. M */
    const double *arr_beta;    /* [nr] temperature exponent                     */
    const double *arr_Ea;      /* [nr] activation energy, J/mol                 */
    const int    *reac_sp;     /* [nr*3] reactant species index, -1 = unused   */
    const int    *reac_nu;     /* [nr*3] reactant stoichiometric coefficient   */
    const int    *prod_sp;     /* [nr*3] product species index, -1 = unused    */
    const int    *prod_nu;     /* [nr*3] product stoichiometric coefficient    */
    const int    *third_body;  /* [nr] 1 if the reaction has a +M partner      */
    const double *tb_eff;      /* [nr*ns] third-body efficiencies alpha_rs     */
} om_mech;

/* Integrator options (the paper gives none; these are the stated readings). */
typedef struct om_opts {
    double rtol;          /* Newton relative tolerance                          */
    double atol_rel;      /* absolute tolerance as a fraction of the cell scale */
    int max_newton;       /* Newton iterations per substep attempt              */
    int max_halvings;     /* deepest substep level: h >= dt * 2^-max_halvings   */
    int max_attempts;     /* substep attempts (accepted + failed) per cell      */
    int point_implicit;   /* 1: one linearised step per substep, Eq. 29 as printed */
    int div_check;        /* 1: abandon a substep whose Newton norm stops falling */
    double conv_kappa;    /* > 0: also accept when the contraction rate bounds the error
                             still left by conv_kappa (Hairer & Wanner's safety factor); 0 (the
                             default): the norm test alone */
} om_opts;

/* Per-cell status codes. */
enum {
    OM_OK = 0,
    OM_NEWTON_FAILED = 1,     /* substep halving limit reached                  */
    OM_T_FAILED = 2,          /* temperature of the input state not recoverable */
    OM_BAD_INPUT = 3,         /* non-finite input or non-positive total density */
    OM_TOO_MANY_STEPS = 4,    /* substep attempt budget spent                   */
    OM_REPLAY_NOT_CONVERGED = 5, /* replay: an accepted attempt did not converge */
    OM_REPLAY_MISMATCH = 6    /* replay: the schedule does not add up to dt     */
};

/* Physical constants of the oracle. */
#define OM_R      8.314462618   /* universal gas constant, J/(mol K)            */
#define OM_PA     101325.0      /* standard pressure of K_e, Pa                 */
#define OM_TREF   298.15        /* reference temperature of formation energies  */
#define OM_TLO    200.0         /* temperature-recovery bracket, K              */
#define OM_THI    6000.0

/* ---- thermodynamics (NASA-7) ---------------------------------------------- */
void   om_thermo(const om_mech *m, int s, double T,
                 double *cp_R, double *h_RT, double *s_R);
double om_species_e(const om_mech *m, int s, double T);     /* J/kg, with formation */
double om_species_cv(const om_mech *m, int s, double T);    /* J/(kg K) */
double om_species_ef(const om_mech *m, int s);              /* e_s(T_ref), J/kg */
double om_species_esens(const om_mech *m, int s, double T); /* e_s(T) - e_s(T_ref) */

/* ---- temperature recovery from (rho_s, e) --------------------------------- */
int om_recover_T(const om_mech *m, const double *rho, double e,
                 double T_guess, double *T_out, int *iters);

/* ---- rates, sources, Jacobian --------------------------------------------- */
void om_rate_constants(const om_mech *m, double T, double *kf, double *Kc, double *kb);
void om_progress(const om_mech *m, double T, const double *rho, double *Q);
void om_source(const om_mech *m, const double *rho, double T, double *wdot);
void om_jacobian(const om_mech *m, const double *rho, double T, double *J);

/* ---- dense linear solve ----------------------------------------------------- */
int om_lu_factor(int n, double *A, int *piv);
void om_lu_solve(int n, const double *LU, const int *piv, double *b);

/* ---- backward-Euler step ---------------------------------------------------- */
typedef struct om_cell_result {
    int status;
    int newton_iters;   /* all Newton iterations, accepted and failed substeps */
    int substeps;       /* accepted substeps */
    int failures;       /* failed substep attempts */
    double T;           /* temperature of the returned state */
} om_cell_result;

void om_default_opts(om_opts *o);

void om_advance_cell(const om_mech *m, const om_opts *o,
                     double *rho, double *e, double dt, double T_guess,
                     om_cell_result *res);

/* om_advance_cell that also records which substep attempts were accepted:
 * bit a of sched[0 .. sched_words) (word a / 32, bit a % 32) is set when
 * attempt a was accepted; and, with states != NULL, the state after each of
 * the first states_cap accepted substeps (N_s + 1 values each). */
void om_advance_cell_sched(const om_mech *m, const om_opts *o, double *rho, double *e,
                           double dt, double T_guess, uint32_t *sched, int sched_words,
                           double *states, int states_cap, om_cell_result *res);

/* One cell along a given schedule of accepted / rejected substep attempts
 * (bit a of `accepted` set: attempt a accepted), each accepted attempt's
 * backward-Euler system solved to the norm test; Newton for accepted substep
 * j starts from guides[j*(N_s+1) ..] when j < n_guides (guides may be NULL),
 * else from the current state.  Status OM_OK, OM_BAD_INPUT, OM_T_FAILED,
 * OM_REPLAY_NOT_CONVERGED or OM_REPLAY_MISMATCH. */
void om_advance_cell_replay(const om_mech *m, const om_opts *o, double *rho, double *e,
                            double dt, double T_guess, const uint32_t *accepted, int n_attempts,
                            const double *guides, int n_guides, om_cell_result *res);

/* The replay over an SoA batch; cell i's schedule is
 * accepted[i*sched_words ..] with n_attempts[i] attempts, its guides (may be
 * NULL) guides[i*n_guides*(N_s+1) ..]. */
void om_advance_batch_replay(const om_mech *m, const om_opts *o, long n_cells, long ld,
                             double *rho, double *e, double dt, const double *T_in,
                             const uint32_t *accepted, int sched_words, const int *n_attempts,
                             const double *guides, int n_guides, double *T_out, int *status,
                             int *newton_iters);

/* SoA batch: rho[s*ld + cell], e[cell]; in place.  T_in may be NULL (guess
 * 1500 K).  Any of the output arrays may be NULL. */
void om_advance_batch(const om_mech *m, const om_opts *o, long n_cells, long ld,
                      double *rho, double *e, double dt, const double *T_in,
                      double *T_out, int *status, int *newton_iters,
                      int *substeps, int *failures);

/* om_advance_batch that also records each cell's accepted attempts in
 * sched[i*sched_words ..] and its states after accepted substeps in
 * states[i*states_cap*(N_s+1) ..] (as om_advance_cell_sched); sched and
 * states may be NULL. */
void om_advance_batch_sched(const om_mech *m, const om_opts *o, long n_cells, long ld,
                            double *rho, double *e, double dt, const double *T_in,
                            double *T_out, int *status, int *newton_iters, int *substeps,
                            int *failures, uint32_t *sched, int sched_words, double *states,
                            int states_cap);

/* Initial states from (T, P, Y) by Dalton's law (Eq. 5) and the energy
 * definition (Eq. 3).  Y is SoA [s*ld + cell]. */
void om_state_from_tpy(const om_mech *m, long n_cells, long ld,
                       const double *T, const double *P, const double *Y,
                       double *rho, double *e);

#ifdef __cplusplus
}
#endif
#endif
