/*
 * chem_oracle.c -- plain FP64 CPU oracle for the implicit chemistry step of
 * Le & Cambier (arXiv 1110.4903), Sections 2 and 3.2.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline).  Every loop
 * here is the definition written out: no blocking, fusion or reordering.
 * Speed is not a goal; the CUDA path is checked against this file.
 *
 * Readings of points the paper leaves open (each one is listed with its
 * justification in the design notes of the repository):
 *  - R is the universal gas constant (the paper calls it Boltzmann's constant
 *    "in J/mol K", Eq. 5), P_a in K_e is 1 atm.
 *  - thermodynamics are NASA-7 polynomials, two ranges, T <= T_mid selects the
 *    low range, polynomials are extrapolated outside their fit range.
 *  - the energy variable e excludes formation energy (Eq. 3): e = sum_s rho_s
 *    (e_s(T) - e_s(T_ref)); the formation energy released by reactions enters
 *    the energy source, Omega_e = -sum_s e_s(T_ref) wdot_s.
 *  - the progress rate (Eq. 25) carries the third-body factor only for +M
 *    reactions; stoichiometric powers are integers.
 *  - the implicit system (Eq. 29) is solved as full backward Euler by Newton
 *    iteration, with row partial pivoting; max_newton = 1 with no convergence
 *    test is the point-implicit step exactly as printed.
 */
#include "chem_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------
 * Thermodynamics.  The paper reads species data from files (Sec. 3.2); the
 * NASA 7-coefficient form is taken:
 *   cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4
 *   h/RT = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5 + a6/T
 *   s/R  = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3 + a5 T^4/4 + a7
 * ------------------------------------------------------------------------- */
static const double *nasa_coeffs(const om_mech *m, int s, double T)
{
    int high = T > m->t_mid[s];
    return m->nasa7 + (size_t)s * 14 + (high ? 7 : 0);
}

void om_thermo(const om_mech *m, int s, double T, double *cp_R, double *h_RT, double *s_R)
{
    const double *a = nasa_coeffs(m, s, T);
    double T2 = T * T, T3 = T2 * T, T4 = T3 * T;
    *cp_R = a[0] + a[1] * T + a[2] * T2 + a[3] * T3 + a[4] * T4;
    *h_RT = a[0] + a[1] * T / 2.0 + a[2] * T2 / 3.0 + a[3] * T3 / 4.0 + a[4] * T4 / 5.0 + a[5] / T;
    *s_R = a[0] * log(T) + a[1] * T + a[2] * T2 / 2.0 + a[3] * T3 / 3.0 + a[4] * T4 / 4.0 + a[6];
}

/* Internal energy per unit mass, including formation energy: e = h - RT/M. */
double om_species_e(const om_mech *m, int s, double T)
{
    double cp_R, h_RT, s_R;
    om_thermo(m, s, T, &cp_R, &h_RT, &s_R);
    return OM_R / m->molar_mass[s] * T * (h_RT - 1.0);
}

/* Constant-volume heat capacity per unit mass: cv = cp - R/M. */
double om_species_cv(const om_mech *m, int s, double T)
{
    double cp_R, h_RT, s_R;
    om_thermo(m, s, T, &cp_R, &h_RT, &s_R);
    return OM_R / m->molar_mass[s] * (cp_R - 1.0);
}

/* Formation energy per unit mass, e_s(T_ref) (the part Eq. 3 leaves out). */
double om_species_ef(const om_mech *m, int s)
{
    return om_species_e(m, s, OM_TREF);
}

/* Sensible internal energy per unit mass, the e_is of Eq. 3. */
double om_species_esens(const om_mech *m, int s, double T)
{
    return om_species_e(m, s, T) - om_species_ef(m, s);
}

/* ---------------------------------------------------------------------------
 * Temperature from the conserved chemistry variables (rho_s, e), Eq. 3 with
 * no kinetic energy (operator splitting, Eq. 4, leaves momentum to the flux
 * stage).  Solves f(T) = sum_s rho_s e_s^sens(T) - e = 0 by Newton's method
 * safeguarded by bisection on the bracket [OM_TLO, OM_THI]; stops when
 * |dT| <= 1e-13 T, at most 50 iterations.  Returns 0 on success.
 * ------------------------------------------------------------------------- */
int om_recover_T(const om_mech *m, const double *rho, double e, double T_guess,
                 double *T_out, int *iters)
{
    double lo = OM_TLO, hi = OM_THI;
    double T = T_guess;
    int it;
    if (!(T > lo && T < hi))
        T = 1500.0;
    for (it = 1; it <= 50; ++it) {
        double f = -e, fp = 0.0, Tn, dT;
        int s;
        for (s = 0; s < m->ns; ++s) {
            f += rho[s] * om_species_esens(m, s, T);
            fp += rho[s] * om_species_cv(m, s, T);
        }
        if (f == 0.0) {
            *T_out = T;
            *iters = it;
            return 0;
        }
        if (f > 0.0)
            hi = T;
        else
            lo = T;
        Tn = T - f / fp;
        if (!(Tn > lo && Tn < hi))
            Tn = 0.5 * (lo + hi);
        dT = Tn - T;
        T = Tn;
        if (fabs(dT) <= 1e-13 * T) {
            *T_out = T;
            *iters = it;
            if (T <= OM_TLO * (1.0 + 1e-9) || T >= OM_THI * (1.0 - 1e-9))
                return -1;
            return 0;
        }
    }
    *T_out = T;
    *iters = it;
    return -1;
}

/* ---------------------------------------------------------------------------
 * Reaction bookkeeping.
 * ------------------------------------------------------------------------- */
/* Dense stoichiometric tables nu'[r][s] (reactants) and nu''[r][s]
 * (products), built from the three slots per side of every reaction. */
static void dense_nu(const om_mech *m, int *nuR, int *nuP)
{
    int r, j;
    memset(nuR, 0, sizeof(int) * (size_t)m->nr * m->ns);
    memset(nuP, 0, sizeof(int) * (size_t)m->nr * m->ns);
    for (r = 0; r < m->nr; ++r) {
        for (j = 0; j < 3; ++j) {
            if (m->reac_sp[r * 3 + j] >= 0)
                nuR[(size_t)r * m->ns + m->reac_sp[r * 3 + j]] += m->reac_nu[r * 3 + j];
            if (m->prod_sp[r * 3 + j] >= 0)
                nuP[(size_t)r * m->ns + m->prod_sp[r * 3 + j]] += m->prod_nu[r * 3 + j];
        }
    }
}

static double ipow(double x, int k)
{
    double p = 1.0;
    int i;
    for (i = 0; i < k; ++i)
        p *= x;
    return p;
}

/* ---------------------------------------------------------------------------
 * Rate constants.
 *   forward, Eq. 23:  K_f = A T^beta exp(-E / RT)
 *   equilibrium, Eq. 24:  K_e = K_f / K_b = (P_a / RT)^(sum nu) exp(-dG0 / RT)
 * with sum nu = sum_s (nu''_s - nu'_s) and dG0/RT = sum_s nu_rs g_s/RT.
 * A is converted from CGS to SI by (1e-6)^(m-1), m the forward order
 * including the third body.
 * ------------------------------------------------------------------------- */
void om_rate_constants(const om_mech *m, double T, double *kf, double *Kc, double *kb)
{
    int r, s, j;
    double *g_RT = (double *)malloc(sizeof(double) * (size_t)m->ns);
    int *nuR = (int *)malloc(sizeof(int) * (size_t)m->nr * m->ns);
    int *nuP = (int *)malloc(sizeof(int) * (size_t)m->nr * m->ns);
    dense_nu(m, nuR, nuP);
    for (s = 0; s < m->ns; ++s) {
        double cp_R, h_RT, s_R;
        om_thermo(m, s, T, &cp_R, &h_RT, &s_R);
        g_RT[s] = h_RT - s_R;
    }
    for (r = 0; r < m->nr; ++r) {
        int order = m->third_body[r] ? 1 : 0;
        int dnu = 0;
        double dG_RT = 0.0, A_si;
        for (j = 0; j < 3; ++j) {
            if (m->reac_sp[r * 3 + j] >= 0)
                order += m->reac_nu[r * 3 + j];
        }
        A_si = m->arr_A[r] * pow(1e-6, (double)(order - 1));
        kf[r] = A_si * pow(T, m->arr_beta[r]) * exp(-m->arr_Ea[r] / (OM_R * T));
        for (s = 0; s < m->ns; ++s) {
            int v = nuP[(size_t)r * m->ns + s] - nuR[(size_t)r * m->ns + s];
            dnu += v;
            dG_RT += v * g_RT[s];
        }
        Kc[r] = pow(OM_PA / (OM_R * T), (double)dnu) * exp(-dG_RT);
        kb[r] = kf[r] / Kc[r];
    }
    free(g_RT);
    free(nuR);
    free(nuP);
}

/* Progress rate, Eq. 25, in mol/(m^3 s), concentrations [X_s] = rho_s / M_s. */
void om_progress(const om_mech *m, double T, const double *rho, double *Q)
{
    int r, s;
    double *c = (double *)malloc(sizeof(double) * (size_t)m->ns);
    double *kf = (double *)malloc(sizeof(double) * (size_t)m->nr);
    double *Kc = (double *)malloc(sizeof(double) * (size_t)m->nr);
    double *kb = (double *)malloc(sizeof(double) * (size_t)m->nr);
    int *nuR = (int *)malloc(sizeof(int) * (size_t)m->nr * m->ns);
    int *nuP = (int *)malloc(sizeof(int) * (size_t)m->nr * m->ns);
    dense_nu(m, nuR, nuP);
    for (s = 0; s < m->ns; ++s)
        c[s] = rho[s] / m->molar_mass[s];
    om_rate_constants(m, T, kf, Kc, kb);
    for (r = 0; r < m->nr; ++r) {
        double Pf = 1.0, Pb = 1.0, CM = 1.0;
        for (s = 0; s < m->ns; ++s) {
            Pf *= ipow(c[s], nuR[(size_t)r * m->ns + s]);
            Pb *= ipow(c[s], nuP[(size_t)r * m->ns + s]);
        }
        if (m->third_body[r]) {
            CM = 0.0;
            for (s = 0; s < m->ns; ++s)
                CM += m->tb_eff[(size_t)r * m->ns + s] * c[s];
        }
        Q[r] = CM * (kf[r] * Pf - kb[r] * Pb);
    }
    free(c);
    free(kf);
    free(Kc);
    free(kb);
    free(nuR);
    free(nuP);
}

/* Source vector: wdot_s = M_s sum_r nu_rs Q_r (Eq. 26), and the energy
 * source Omega_e = -sum_s e_s(T_ref) wdot_s (Eq. 3 and the remark after it).
 * wdot has ns+1 entries. */
void om_source(const om_mech *m, const double *rho, double T, double *wdot)
{
    int r, s;
    double *Q = (double *)malloc(sizeof(double) * (size_t)m->nr);
    int *nuR = (int *)malloc(sizeof(int) * (size_t)m->nr * m->ns);
    int *nuP = (int *)malloc(sizeof(int) * (size_t)m->nr * m->ns);
    dense_nu(m, nuR, nuP);
    om_progress(m, T, rho, Q);
    wdot[m->ns] = 0.0;
    for (s = 0; s < m->ns; ++s) {
        double sum = 0.0;
        for (r = 0; r < m->nr; ++r)
            sum += (nuP[(size_t)r * m->ns + s] - nuR[(size_t)r * m->ns + s]) * Q[r];
        wdot[s] = m->molar_mass[s] * sum;
    }
    for (s = 0; s < m->ns; ++s)
        wdot[m->ns] -= om_species_ef(m, s) * wdot[s];
    free(Q);
    free(nuR);
    free(nuP);
}

/* ---------------------------------------------------------------------------
 * Analytic Jacobian d(wdot, Omega_e)/d(rho_1..rho_ns, e), the dOmega/dQ of
 * Eq. 29, at fixed volume.  T is a function of (rho, e) through Eq. 3:
 *   dT/drho_k = -e_k^sens / (rho cv),   dT/de = 1 / (rho cv),
 * so every column carries the temperature dependence of the rates:
 *   dK_f/dT = K_f (beta/T + E/(R T^2))
 *   dln K_e/dT = (-sum nu + sum_s nu_rs h_s/RT) / T
 *   dK_b/dT = K_b (dln K_f/dT - dln K_e/dT).
 * J is row-major n x n with n = ns + 1; the last row/column is energy.
 * ------------------------------------------------------------------------- */
void om_jacobian(const om_mech *m, const double *rho, double T, double *J)
{
    int ns = m->ns, n = ns + 1;
    int r, s, k;
    double rho_cv = 0.0, dTde;
    double *c = (double *)malloc(sizeof(double) * (size_t)ns);
    double *h_RT = (double *)malloc(sizeof(double) * (size_t)ns);
    double *dTdrho = (double *)malloc(sizeof(double) * (size_t)ns);
    double *ef = (double *)malloc(sizeof(double) * (size_t)ns);
    double *kf = (double *)malloc(sizeof(double) * (size_t)m->nr);
    double *Kc = (double *)malloc(sizeof(double) * (size_t)m->nr);
    double *kb = (double *)malloc(sizeof(double) * (size_t)m->nr);
    int *nuR = (int *)malloc(sizeof(int) * (size_t)m->nr * ns);
    int *nuP = (int *)malloc(sizeof(int) * (size_t)m->nr * ns);
#define NU_R(r, s) nuR[(size_t)(r) * ns + (s)]
#define NU_P(r, s) nuP[(size_t)(r) * ns + (s)]

    dense_nu(m, nuR, nuP);
    memset(J, 0, sizeof(double) * (size_t)n * n);
    for (s = 0; s < ns; ++s) {
        double cp_R, s_R;
        om_thermo(m, s, T, &cp_R, &h_RT[s], &s_R);
        c[s] = rho[s] / m->molar_mass[s];
        rho_cv += rho[s] * om_species_cv(m, s, T);
        ef[s] = om_species_ef(m, s);
    }
    for (s = 0; s < ns; ++s)
        dTdrho[s] = -om_species_esens(m, s, T) / rho_cv;
    dTde = 1.0 / rho_cv;
    om_rate_constants(m, T, kf, Kc, kb);

    for (r = 0; r < m->nr; ++r) {
        double Pf = 1.0, Pb = 1.0, CM = 1.0, fwd, rev, dlnkf, dlnKc, dQdT;
        int dnu = 0;
        double sum_nu_h = 0.0;
        for (s = 0; s < ns; ++s) {
            int v = NU_P(r, s) - NU_R(r, s);
            Pf *= ipow(c[s], NU_R(r, s));
            Pb *= ipow(c[s], NU_P(r, s));
            dnu += v;
            sum_nu_h += v * h_RT[s];
        }
        if (m->third_body[r]) {
            CM = 0.0;
            for (s = 0; s < ns; ++s)
                CM += m->tb_eff[(size_t)r * ns + s] * c[s];
        }
        fwd = kf[r] * Pf;
        rev = kb[r] * Pb;
        dlnkf = m->arr_beta[r] / T + m->arr_Ea[r] / (OM_R * T * T);
        dlnKc = (-(double)dnu + sum_nu_h) / T;
        dQdT = CM * (fwd * dlnkf - rev * (dlnkf - dlnKc));

        for (k = 0; k < ns; ++k) {
            /* d/dc_k of prod_s c_s^nu_s by the product rule */
            double dPf = 0.0, dPb = 0.0, dQdc, dQdrho;
            int vr = NU_R(r, k), vp = NU_P(r, k);
            if (vr > 0) {
                dPf = vr * ipow(c[k], vr - 1);
                for (s = 0; s < ns; ++s)
                    if (s != k)
                        dPf *= ipow(c[s], NU_R(r, s));
            }
            if (vp > 0) {
                dPb = vp * ipow(c[k], vp - 1);
                for (s = 0; s < ns; ++s)
                    if (s != k)
                        dPb *= ipow(c[s], NU_P(r, s));
            }
            dQdc = CM * (kf[r] * dPf - kb[r] * dPb);
            if (m->third_body[r])
                dQdc += m->tb_eff[(size_t)r * ns + k] * (fwd - rev);
            dQdrho = dQdc / m->molar_mass[k] + dQdT * dTdrho[k];
            for (s = 0; s < ns; ++s) {
                int v = NU_P(r, s) - NU_R(r, s);
                if (v != 0)
                    J[s * n + k] += m->molar_mass[s] * v * dQdrho;
            }
        }
        for (s = 0; s < ns; ++s) {
            int v = NU_P(r, s) - NU_R(r, s);
            if (v != 0)
                J[s * n + ns] += m->molar_mass[s] * v * dQdT * dTde;
        }
    }
    for (k = 0; k < n; ++k) {
        double sum = 0.0;
        for (s = 0; s < ns; ++s)
            sum += ef[s] * J[s * n + k];
        J[ns * n + k] = -sum;
    }
    free(c);
    free(h_RT);
    free(dTdrho);
    free(ef);
    free(kf);
    free(Kc);
    free(kb);
    free(nuR);
    free(nuP);
#undef NU_R
#undef NU_P
}

/* ---------------------------------------------------------------------------
 * Gaussian elimination (Sec. 3.2: a direct elimination of the linear system of
 * Eq. 29).  Doolittle LU with row partial pivoting on max |a_ik|; a tie keeps
 * the lowest row index.  Row-major, in place, L has a unit diagonal.
 * Returns 0, or -1 when a pivot is zero or not finite.
 * ------------------------------------------------------------------------- */
int om_lu_factor(int n, double *A, int *piv)
{
    int i, j, k;
    for (k = 0; k < n; ++k) {
        int p = k;
        double amax = fabs(A[k * n + k]);
        for (i = k + 1; i < n; ++i) {
            if (fabs(A[i * n + k]) > amax) {
                amax = fabs(A[i * n + k]);
                p = i;
            }
        }
        piv[k] = p;
        if (!(amax > 0.0) || !isfinite(amax))
            return -1;
        if (p != k) {
            for (j = 0; j < n; ++j) {
                double t = A[k * n + j];
                A[k * n + j] = A[p * n + j];
                A[p * n + j] = t;
            }
        }
        for (i = k + 1; i < n; ++i) {
            double l = A[i * n + k] / A[k * n + k];
            A[i * n + k] = l;
            for (j = k + 1; j < n; ++j)
                A[i * n + j] -= l * A[k * n + j];
        }
    }
    return 0;
}

void om_lu_solve(int n, const double *LU, const int *piv, double *b)
{
    int i, j, k;
    for (k = 0; k < n; ++k) {
        if (piv[k] != k) {
            double t = b[k];
            b[k] = b[piv[k]];
            b[piv[k]] = t;
        }
    }
    for (i = 0; i < n; ++i)
        for (j = 0; j < i; ++j)
            b[i] -= LU[i * n + j] * b[j];
    for (i = n - 1; i >= 0; --i) {
        for (j = i + 1; j < n; ++j)
            b[i] -= LU[i * n + j] * b[j];
        b[i] /= LU[i * n + i];
    }
}

/* ---------------------------------------------------------------------------
 * Backward Euler over one (sub)step h, Eq. 29 iterated to convergence:
 *   F(x) = x - x0 - h Omega(x),   (I - h J(x)) delta = -F(x),   x <- x + delta,
 * converged when max_i |delta_i| / (rtol |x_i| + atol_i) <= 1, or (with
 * conv_kappa > 0) when the observed contraction theta = norm_k / norm_(k-1) < 1
 * bounds the error still left, theta / (1 - theta) norm_k <= conv_kappa: the
 * stopping estimate of simplified Newton in Hairer & Wanner, Solving ODEs II,
 * Sec. IV.8, with their safety factor.  A factor well below 1 keeps the
 * accepted update small enough that its rounding stays below the tolerance.
 * The first iteration uses T0 = T(x0); later ones recover T at the iterate
 * with the previous T as the guess.  A converged state is accepted only if its
 * temperature is recoverable and no density is below -atol.
 * ------------------------------------------------------------------------- */
static int be_substep(const om_mech *m, const om_opts *o, const double *x0, double T0,
                      double h, const double *atol, const double *xstart, double *x,
                      double *T_out, int *iters)
{
    int ns = m->ns, n = ns + 1;
    int i, k, ti, ok = 0;
    double T = T0, norm_prev = INFINITY;
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double *J = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *b = (double *)malloc(sizeof(double) * (size_t)n);
    int *piv = (int *)malloc(sizeof(int) * (size_t)n);

    /* Newton starts from x0 (T0 = T(x0) for the first iteration), or from a
     * given state xstart (its temperature recovered first) */
    memcpy(x, xstart ? xstart : x0, sizeof(double) * (size_t)n);
    for (k = 0; k < o->max_newton; ++k) {
        double norm = 0.0;
        int finite = 1;
        if ((k > 0 || xstart) && om_recover_T(m, x, x[ns], T, &T, &ti) != 0)
            goto done;
        *iters += 1;
        om_source(m, x, T, w);
        om_jacobian(m, x, T, J);
        for (i = 0; i < n * n; ++i)
            J[i] = -h * J[i];
        for (i = 0; i < n; ++i) {
            J[i * n + i] += 1.0;
            b[i] = -(x[i] - x0[i] - h * w[i]);
        }
        if (om_lu_factor(n, J, piv) != 0)
            goto done;
        om_lu_solve(n, J, piv, b);
        for (i = 0; i < n; ++i) {
            x[i] += b[i];
            if (!isfinite(x[i]))
                finite = 0;
        }
        if (!finite)
            goto done;
        if (o->point_implicit) {
            ok = 1;
            break;
        }
        for (i = 0; i < n; ++i) {
            double r = fabs(b[i]) / (o->rtol * fabs(x[i]) + atol[i]);
            if (r > norm)
                norm = r;
        }
        if (norm <= 1.0) {
            ok = 1;
            break;
        }
        /* theta / (1 - theta) norm <= kappa with theta = norm / norm_prev in
         * [0, 1), multiplied by (1 - theta) norm_prev > 0 */
        if (o->conv_kappa > 0.0 && k >= 1 && norm < norm_prev &&
            norm * norm <= o->conv_kappa * (norm_prev - norm)) {
            ok = 1;
            break;
        }
        if (o->div_check && k >= 2 && norm >= norm_prev)
            goto done;
        norm_prev = norm;
    }
    if (ok) {
        ok = 0;
        if (om_recover_T(m, x, x[ns], T, &T, &ti) != 0)
            goto done;
        for (i = 0; i < ns; ++i)
            if (x[i] < -atol[i])
                goto done;
        *T_out = T;
        ok = 1;
    }
done:
    free(w);
    free(J);
    free(b);
    free(piv);
    return ok;
}

void om_default_opts(om_opts *o)
{
    o->rtol = 1e-10;
    o->atol_rel = 1e-12;
    o->max_newton = 12;
    o->max_halvings = 20;
    o->max_attempts = 1000;
    o->point_implicit = 0;
    o->div_check = 1;
    o->conv_kappa = 0.0;
}

/* ---------------------------------------------------------------------------
 * One cell over the fluid step dt (the chemistry half of the operator split,
 * Eq. 4).  Substeps h = dt 2^-level: a failed substep halves h (level + 1, at
 * most max_halvings), an accepted one doubles it for the next; the last
 * substep is shortened to land exactly on dt.  Time is counted in integer
 * units of dt 2^-max_halvings so the schedule is exact.  On failure the cell
 * keeps its input values.
 *
 * With sched != NULL the outcome of every substep attempt is recorded: bit a
 * (word a / 32, bit a % 32) of sched[0 .. sched_words) is set when attempt a
 * was accepted; attempts beyond 32 sched_words are not recorded.  With
 * states != NULL the state after accepted substep j < states_cap is copied to
 * states[j*(N_s+1) ..].
 * ------------------------------------------------------------------------- */
static void advance_cell(const om_mech *m, const om_opts *o, double *rho, double *e, double dt,
                         double T_guess, uint32_t *sched, int sched_words, double *states,
                         int states_cap, om_cell_result *res)
{
    int ns = m->ns, n = ns + 1;
    int s, ti, level = 0, attempts = 0;
    int64_t total, t = 0;
    double rho_tot = 0.0, e_scale, T0;
    double *x0 = (double *)malloc(sizeof(double) * (size_t)n);
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double *atol = (double *)malloc(sizeof(double) * (size_t)n);

    res->status = OM_OK;
    res->newton_iters = 0;
    res->substeps = 0;
    res->failures = 0;
    res->T = NAN;
    for (s = 0; s < sched_words; ++s)
        sched[s] = 0u;

    for (s = 0; s < ns; ++s) {
        x0[s] = rho[s];
        rho_tot += rho[s];
    }
    x0[ns] = *e;
    for (s = 0; s < n; ++s) {
        if (!isfinite(x0[s])) {
            res->status = OM_BAD_INPUT;
            goto out;
        }
    }
    if (!(rho_tot > 0.0) || !(dt >= 0.0) || !isfinite(dt)) {
        res->status = OM_BAD_INPUT;
        goto out;
    }
    if (om_recover_T(m, x0, x0[ns], T_guess, &T0, &ti) != 0) {
        res->status = OM_T_FAILED;
        goto out;
    }
    res->T = T0;
    if (dt == 0.0)
        goto out;

    e_scale = fabs(x0[ns]);
    for (s = 0; s < ns; ++s) {
        atol[s] = o->atol_rel * rho_tot;
        e_scale += fabs(x0[s] * om_species_ef(m, s));
    }
    atol[ns] = o->atol_rel * e_scale;

    total = (int64_t)1 << o->max_halvings;
    while (t < total) {
        double h, T1;
        if (attempts >= o->max_attempts) {
            res->status = OM_TOO_MANY_STEPS;
            goto out;
        }
        while ((total >> level) > total - t)
            level++;
        h = ldexp(dt, -level);
        attempts++;
        if (be_substep(m, o, x0, T0, h, atol, NULL, x, &T1, &res->newton_iters)) {
            if (sched && attempts - 1 < 32 * sched_words)
                sched[(attempts - 1) / 32] |= 1u << ((attempts - 1) % 32);
            if (states && res->substeps < states_cap)
                memcpy(states + (size_t)res->substeps * n, x, sizeof(double) * (size_t)n);
            memcpy(x0, x, sizeof(double) * (size_t)n);
            T0 = T1;
            t += total >> level;
            res->substeps++;
            if (level > 0)
                level--;
        } else {
            res->failures++;
            level++;
            if (level > o->max_halvings) {
                res->status = OM_NEWTON_FAILED;
                goto out;
            }
        }
    }
    for (s = 0; s < ns; ++s)
        rho[s] = x0[s];
    *e = x0[ns];
    res->T = T0;
out:
    free(x0);
    free(x);
    free(atol);
}

void om_advance_cell(const om_mech *m, const om_opts *o, double *rho, double *e,
                     double dt, double T_guess, om_cell_result *res)
{
    advance_cell(m, o, rho, e, dt, T_guess, NULL, 0, NULL, 0, res);
}

void om_advance_cell_sched(const om_mech *m, const om_opts *o, double *rho, double *e, double dt,
                           double T_guess, uint32_t *sched, int sched_words, double *states,
                           int states_cap, om_cell_result *res)
{
    advance_cell(m, o, rho, e, dt, T_guess, sched, sched_words, states, states_cap, res);
}

/* ---------------------------------------------------------------------------
 * Replay: one cell over dt along a GIVEN substep schedule instead of the one
 * the control above would choose.  Backward Euler has one solution per
 * sequence of substep sizes; two integrators whose accept/reject decisions
 * differ (e.g. because one solves the Newton systems of Eq. 29 in lower
 * precision) land on different, equally valid discretisations.  This
 * integrates the schedule the other integrator took, so that its result can
 * be compared element by element.
 *
 * Attempt a (0 <= a < n_attempts) is accepted when bit a of `accepted` is
 * set.  The sizes follow the same rule as om_advance_cell: h = dt 2^-level,
 * level raised until the substep fits in the time left, +1 after a rejected
 * attempt, -1 after an accepted one.  An accepted attempt solves its
 * backward-Euler system from the current state to the norm test with up to
 * o->max_newton iterations (the caller's conv_kappa and div_check apply; a
 * replay normally passes 0 for both), then requires a recoverable T and no
 * density below -atol, as om_advance_cell does.  A rejected attempt changes
 * nothing but the level.
 *
 * Where a substep's backward-Euler system has several roots, Newton's method
 * started from the current state may reach another root than the other
 * integrator did, or none (hot cells at large h, where the iteration's global
 * phase is chaotic).  `guides` (optional, n_guides states of N_s + 1 values)
 * carries the other integrator's state after each of its accepted substeps;
 * accepted substep j then starts Newton from guides[j] instead of the current
 * state.  The root is still the oracle's own, of the system set up from the
 * oracle's own previous state; the guide only selects which root.
 *
 * res->status is OM_OK, OM_BAD_INPUT / OM_T_FAILED for the input state,
 * OM_REPLAY_NOT_CONVERGED when an accepted attempt's system does not
 * converge, or OM_REPLAY_MISMATCH when the schedule is inconsistent (a level
 * beyond max_halvings, an attempt after dt is reached, or dt not reached
 * after n_attempts).  On any status but OM_OK the cell keeps its input.
 * ------------------------------------------------------------------------- */
void om_advance_cell_replay(const om_mech *m, const om_opts *o, double *rho, double *e, double dt,
                            double T_guess, const uint32_t *accepted, int n_attempts,
                            const double *guides, int n_guides, om_cell_result *res)
{
    int ns = m->ns, n = ns + 1;
    int s, a, ti, level = 0;
    int64_t total, t = 0;
    double rho_tot = 0.0, e_scale, T0;
    double *x0 = (double *)malloc(sizeof(double) * (size_t)n);
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double *atol = (double *)malloc(sizeof(double) * (size_t)n);

    res->status = OM_OK;
    res->newton_iters = 0;
    res->substeps = 0;
    res->failures = 0;
    res->T = NAN;

    for (s = 0; s < ns; ++s) {
        x0[s] = rho[s];
        rho_tot += rho[s];
    }
    x0[ns] = *e;
    for (s = 0; s < n; ++s) {
        if (!isfinite(x0[s])) {
            res->status = OM_BAD_INPUT;
            goto out;
        }
    }
    if (!(rho_tot > 0.0) || !(dt >= 0.0) || !isfinite(dt)) {
        res->status = OM_BAD_INPUT;
        goto out;
    }
    if (om_recover_T(m, x0, x0[ns], T_guess, &T0, &ti) != 0) {
        res->status = OM_T_FAILED;
        goto out;
    }
    res->T = T0;
    if (dt == 0.0) {
        if (n_attempts != 0)
            res->status = OM_REPLAY_MISMATCH;
        goto out;
    }

    e_scale = fabs(x0[ns]);
    for (s = 0; s < ns; ++s) {
        atol[s] = o->atol_rel * rho_tot;
        e_scale += fabs(x0[s] * om_species_ef(m, s));
    }
    atol[ns] = o->atol_rel * e_scale;

    total = (int64_t)1 << o->max_halvings;
    for (a = 0; a < n_attempts; ++a) {
        double h, T1;
        if (t >= total) {
            res->status = OM_REPLAY_MISMATCH;
            goto out;
        }
        while ((total >> level) > total - t)
            level++;
        h = ldexp(dt, -level);
        if ((accepted[a / 32] >> (a % 32)) & 1u) {
            const double *g =
                guides && res->substeps < n_guides ? guides + (size_t)res->substeps * n : NULL;
            if (!be_substep(m, o, x0, T0, h, atol, g, x, &T1, &res->newton_iters)) {
                res->status = OM_REPLAY_NOT_CONVERGED;
                goto out;
            }
            memcpy(x0, x, sizeof(double) * (size_t)n);
            T0 = T1;
            t += total >> level;
            res->substeps++;
            if (level > 0)
                level--;
        } else {
            res->failures++;
            level++;
            if (level > o->max_halvings) {
                res->status = OM_REPLAY_MISMATCH;
                goto out;
            }
        }
    }
    if (t != total) {
        res->status = OM_REPLAY_MISMATCH;
        goto out;
    }
    for (s = 0; s < ns; ++s)
        rho[s] = x0[s];
    *e = x0[ns];
    res->T = T0;
out:
    free(x0);
    free(x);
    free(atol);
}

void om_advance_batch(const om_mech *m, const om_opts *o, long n_cells, long ld,
                      double *rho, double *e, double dt, const double *T_in,
                      double *T_out, int *status, int *newton_iters, int *substeps,
                      int *failures)
{
    om_advance_batch_sched(m, o, n_cells, ld, rho, e, dt, T_in, T_out, status, newton_iters,
                           substeps, failures, NULL, 0, NULL, 0);
}

void om_advance_batch_sched(const om_mech *m, const om_opts *o, long n_cells, long ld,
                            double *rho, double *e, double dt, const double *T_in,
                            double *T_out, int *status, int *newton_iters, int *substeps,
                            int *failures, uint32_t *sched, int sched_words, double *states,
                            int states_cap)
{
    int ns = m->ns;
    long i;
    int s;
    double *r = (double *)malloc(sizeof(double) * (size_t)ns);
    for (i = 0; i < n_cells; ++i) {
        om_cell_result res;
        double ei = e[i];
        for (s = 0; s < ns; ++s)
            r[s] = rho[(size_t)s * ld + i];
        advance_cell(m, o, r, &ei, dt, T_in ? T_in[i] : 1500.0,
                     sched ? sched + (size_t)i * sched_words : NULL, sched ? sched_words : 0,
                     states ? states + (size_t)i * states_cap * (ns + 1) : NULL,
                     states ? states_cap : 0, &res);
        for (s = 0; s < ns; ++s)
            rho[(size_t)s * ld + i] = r[s];
        e[i] = ei;
        if (T_out)
            T_out[i] = res.T;
        if (status)
            status[i] = res.status;
        if (newton_iters)
            newton_iters[i] = res.newton_iters;
        if (substeps)
            substeps[i] = res.substeps;
        if (failures)
            failures[i] = res.failures;
    }
    free(r);
}

/* om_advance_cell_replay over an SoA batch: the schedule of cell i is
 * accepted[i*sched_words .. (i+1)*sched_words) with n_attempts[i] attempts
 * (n_attempts[i] <= 32 sched_words). */
void om_advance_batch_replay(const om_mech *m, const om_opts *o, long n_cells, long ld,
                             double *rho, double *e, double dt, const double *T_in,
                             const uint32_t *accepted, int sched_words, const int *n_attempts,
                             const double *guides, int n_guides, double *T_out, int *status,
                             int *newton_iters)
{
    int ns = m->ns;
    long i;
    int s;
    double *r = (double *)malloc(sizeof(double) * (size_t)ns);
    for (i = 0; i < n_cells; ++i) {
        om_cell_result res;
        double ei = e[i];
        for (s = 0; s < ns; ++s)
            r[s] = rho[(size_t)s * ld + i];
        if (n_attempts[i] < 0 || n_attempts[i] > 32 * sched_words) {
            res.status = OM_REPLAY_MISMATCH;
            res.newton_iters = 0;
            res.T = NAN;
        } else {
            om_advance_cell_replay(m, o, r, &ei, dt, T_in ? T_in[i] : 1500.0,
                                   accepted + (size_t)i * sched_words, n_attempts[i],
                                   guides ? guides + (size_t)i * n_guides * (ns + 1) : NULL,
                                   n_guides, &res);
        }
        for (s = 0; s < ns; ++s)
            rho[(size_t)s * ld + i] = r[s];
        e[i] = ei;
        if (T_out)
            T_out[i] = res.T;
        if (status)
            status[i] = res.status;
        if (newton_iters)
            newton_iters[i] = res.newton_iters;
    }
    free(r);
}

/* Dalton's law (Eq. 5): P = sum_s rho_s (R/M_s) T, so with mass fractions Y_s
 * the density is rho = P / (R T sum_s Y_s/M_s); e follows Eq. 3. */
void om_state_from_tpy(const om_mech *m, long n_cells, long ld, const double *T,
                       const double *P, const double *Y, double *rho, double *e)
{
    long i;
    int s;
    for (i = 0; i < n_cells; ++i) {
        double inv_W = 0.0, rho_tot, ei = 0.0;
        for (s = 0; s < m->ns; ++s)
            inv_W += Y[(size_t)s * ld + i] / m->molar_mass[s];
        rho_tot = P[i] / (OM_R * T[i] * inv_W);
        for (s = 0; s < m->ns; ++s) {
            double rs = rho_tot * Y[(size_t)s * ld + i];
            rho[(size_t)s * ld + i] = rs;
            ei += rs * om_species_esens(m, s, T[i]);
        }
        e[i] = ei;
    }
}
