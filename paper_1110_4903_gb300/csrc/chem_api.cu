// chem_api.cu -- host side of libchem: mechanism validation and derived
// tables, launch configuration, and the C ABI declared in include/chem.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/chem.h"
#include "chem_handle.h"
#include "chem_internal.h"

namespace chem {

const void *be_kernel_fp64(int G);
const void *be_kernel_mixed(int G);

static thread_local char g_errmsg[512] = "";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_errmsg, sizeof g_errmsg, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(CHEM_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// NASA-7 on the host (validation and formation energies)
static inline void host_nasa(const double *a, double T, double &cpR, double &hRT) {
    cpR = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
    hRT = a[0] + T * (a[1] / 2 + T * (a[2] / 3 + T * (a[3] / 4 + T * a[4] / 5))) + a[5] / T;
}

static int validate(const chem_mech_desc *d) {
    if (!d) return fail(CHEM_E_INVALID_ARG, "mechanism descriptor is NULL");
    const int ns = d->n_species, nr = d->n_reactions, ne = d->n_elements;
    if (ns < 1 || nr < 0 || ne < 0) return fail(CHEM_E_INVALID_ARG, "bad sizes ns=%d nr=%d ne=%d", ns, nr, ne);
    if (ns > CHEM_MAX_SPECIES) return fail(CHEM_E_UNSUPPORTED, "n_species %d > %d", ns, CHEM_MAX_SPECIES);
    if (nr > CHEM_MAX_REACTIONS) return fail(CHEM_E_UNSUPPORTED, "n_reactions %d > %d", nr, CHEM_MAX_REACTIONS);
    if (!d->molar_mass || !d->nasa7 || !d->t_mid)
        return fail(CHEM_E_INVALID_ARG, "species arrays missing");
    if (nr > 0 && (!d->arr_A || !d->arr_beta || !d->arr_Ea || !d->reac_sp || !d->reac_nu ||
                   !d->prod_sp || !d->prod_nu || !d->third_body))
        return fail(CHEM_E_INVALID_ARG, "reaction arrays missing");
    if (ne > 0 && !d->elem_comp) return fail(CHEM_E_INVALID_ARG, "elem_comp missing");
    for (int s = 0; s < ns; ++s) {
        if (!(d->molar_mass[s] > 0) || !std::isfinite(d->molar_mass[s]))
            return fail(CHEM_E_BAD_MECHANISM, "species %d: molar mass %g", s, d->molar_mass[s]);
        if (!std::isfinite(d->t_mid[s])) return fail(CHEM_E_BAD_MECHANISM, "species %d: t_mid", s);
        for (int j = 0; j < 14; ++j)
            if (!std::isfinite(d->nasa7[s * 14 + j]))
                return fail(CHEM_E_BAD_MECHANISM, "species %d: NASA-7 coefficient %d not finite", s, j);
        // cp/R > 1 (cv > 0) on the temperature-recovery bracket keeps e(T)
        // strictly increasing, so the recovery has one root
        for (int Ti = (int)kTlo; Ti <= (int)kThi; ++Ti) {
            const double T = Ti;
            const double *a = d->nasa7 + s * 14 + (T > d->t_mid[s] ? 7 : 0);
            double cpR, hRT;
            host_nasa(a, T, cpR, hRT);
            if (!(cpR > 1.0))
                return fail(CHEM_E_BAD_MECHANISM, "species %d: cp/R = %g <= 1 at %g K", s, cpR, T);
        }
    }
    for (int r = 0; r < nr; ++r) {
        if (!(d->arr_A[r] >= 0) || !std::isfinite(d->arr_A[r]) || !std::isfinite(d->arr_beta[r]) ||
            !std::isfinite(d->arr_Ea[r]))
            return fail(CHEM_E_BAD_MECHANISM, "reaction %d: bad Arrhenius data", r);
        int tot[2] = {0, 0};
        for (int side = 0; side < 2; ++side) {
            const int32_t *sp = side ? d->prod_sp : d->reac_sp;
            const int32_t *nu = side ? d->prod_nu : d->reac_nu;
            for (int j = 0; j < 3; ++j) {
                const int s = sp[r * 3 + j];
                if (s < -1 || s >= ns)
                    return fail(CHEM_E_BAD_MECHANISM, "reaction %d: species index %d", r, s);
                if (s < 0) continue;
                if (nu[r * 3 + j] < 1 || nu[r * 3 + j] > 3)
                    return fail(CHEM_E_BAD_MECHANISM, "reaction %d: coefficient %d", r, nu[r * 3 + j]);
                for (int jj = 0; jj < j; ++jj)
                    if (sp[r * 3 + jj] == s)
                        return fail(CHEM_E_BAD_MECHANISM, "reaction %d: species %d twice on one side", r, s);
                tot[side] += nu[r * 3 + j];
            }
        }
        if (tot[0] < 1 || tot[1] < 1 || tot[0] > 3 || tot[1] > 3)
            return fail(CHEM_E_BAD_MECHANISM, "reaction %d: sides of %d and %d molecules", r, tot[0], tot[1]);
        if (d->third_body[r] != 0 && d->third_body[r] != 1)
            return fail(CHEM_E_BAD_MECHANISM, "reaction %d: third_body flag", r);
        if (d->tb_eff && d->third_body[r])
            for (int s = 0; s < ns; ++s)
                if (!std::isfinite(d->tb_eff[(size_t)r * ns + s]))
                    return fail(CHEM_E_BAD_MECHANISM, "reaction %d: efficiency", r);
        for (int el = 0; el < ne; ++el) {
            long bal = 0;
            for (int j = 0; j < 3; ++j) {
                if (d->reac_sp[r * 3 + j] >= 0)
                    bal -= (long)d->reac_nu[r * 3 + j] * d->elem_comp[d->reac_sp[r * 3 + j] * ne + el];
                if (d->prod_sp[r * 3 + j] >= 0)
                    bal += (long)d->prod_nu[r * 3 + j] * d->elem_comp[d->prod_sp[r * 3 + j] * ne + el];
            }
            if (bal != 0) return fail(CHEM_E_BAD_MECHANISM, "reaction %d: element %d not balanced", r, el);
        }
    }
    return CHEM_OK;
}

// The library orders reactions internally with the third-body reactions
// first (stable otherwise): the rate loop's third-body branch then runs in the
// first passes only, and the third-body progress values need ntb slots, not
// nr.  Only internal tables see this order.
struct ReorderedMech {
    std::vector<double> A, beta, Ea, eff;
    std::vector<int32_t> rs, rn, ps, pn, tb;
    chem_mech_desc d;
    int ntb = 0;
};

static void third_body_first(const chem_mech_desc *in, ReorderedMech &o) {
    const int ns = in->n_species, nr = in->n_reactions;
    std::vector<int> perm;
    for (int pass = 0; pass < 2; ++pass)
        for (int r = 0; r < nr; ++r)
            if ((in->third_body[r] != 0) == (pass == 0)) perm.push_back(r);
    for (int r : perm) {
        o.A.push_back(in->arr_A[r]);
        o.beta.push_back(in->arr_beta[r]);
        o.Ea.push_back(in->arr_Ea[r]);
        for (int j = 0; j < 3; ++j) {
            o.rs.push_back(in->reac_sp[r * 3 + j]);
            o.rn.push_back(in->reac_nu[r * 3 + j]);
            o.ps.push_back(in->prod_sp[r * 3 + j]);
            o.pn.push_back(in->prod_nu[r * 3 + j]);
        }
        o.tb.push_back(in->third_body[r]);
        if (in->third_body[r]) ++o.ntb;
        if (in->tb_eff)
            for (int q = 0; q < ns; ++q) o.eff.push_back(in->tb_eff[(size_t)r * ns + q]);
    }
    o.d = *in;
    o.d.arr_A = o.A.data();
    o.d.arr_beta = o.beta.data();
    o.d.arr_Ea = o.Ea.data();
    o.d.reac_sp = o.rs.data();
    o.d.reac_nu = o.rn.data();
    o.d.prod_sp = o.ps.data();
    o.d.prod_nu = o.pn.data();
    o.d.third_body = o.tb.data();
    o.d.tb_eff = in->tb_eff ? o.eff.data() : nullptr;
}

// Derived tables (layouts in chem_internal.h)
struct HostTables {
    std::vector<double> thermo, tmid, tpoly, sp, rxn_d, eff_c, d_ce, j_c, exp_tab, log_tab;
    std::vector<unsigned> div16;
    std::vector<float> tpoly_f;
    std::vector<float> rxn_df, d_cef, spf;
    std::vector<int2> d_pk;
    std::vector<unsigned> j_w, sp_w;
    std::vector<int> rxn_f, eff_ptr, eff_sp, d_i0, d_i1, j_sk, j_ptr, j_d, it_ptr, sp_item_ptr, sp_r;
    std::vector<int2> j_meta;
    std::vector<int> j_nu, sp_nui, j_sk32, j_ptr32, j_d32;
    struct Layout {
        std::vector<int2> j_meta, it_meta;
        std::vector<int4> j_meta32;
        std::vector<unsigned> j_w, sp_w;
        std::vector<int> j_d;
        std::vector<double> j_c;
    } lay[kLayouts];
    int nD = 0, nD_F = 0, nD_B = 0, nD_FB = 0, nJ = 0, nJ_nz = 0, n_items = 0, ntb = 0;
};

// {1/F, ln F} at F = 1 + j/kLogTab, j = 0..kLogTab, rounded from extended
// precision (the table of the kernels' logarithm)
void fill_log_table(std::vector<double> &tab) {
    tab.resize(2 * (kLogTab + 1));
    for (int j = 0; j <= kLogTab; ++j) {
        const long double F = 1.0L + (long double)j / kLogTab;
        tab[2 * j] = (double)(1.0L / F);
        tab[2 * j + 1] = (double)std::log(F);
    }
}

static void build_tables(const chem_mech_desc *d, HostTables &t) {
    const int ns = d->n_species, nr = d->n_reactions;
    const int SENT = ns;   // sentinel species index
    t.thermo.assign((size_t)ns * 2 * kThermoStride, 0.0);
    t.tmid.assign(d->t_mid, d->t_mid + ns);
    t.sp.assign((size_t)ns * kSpStride, 0.0);
    std::vector<double> ef(ns);
    for (int s = 0; s < ns; ++s) {
        for (int rg = 0; rg < 2; ++rg) {
            const double *a = d->nasa7 + s * 14 + rg * 7;
            double *th = &t.thermo[((size_t)s * 2 + rg) * kThermoStride];
            for (int j = 0; j < 5; ++j) th[j] = a[j];
            th[5] = a[1] / 2;
            th[6] = a[2] / 3;
            th[7] = a[3] / 4;
            th[8] = a[4] / 5;
            th[9] = a[5];
            th[10] = a[2] / 2;
            th[11] = a[3] / 3;
            th[12] = a[4] / 4;
            th[13] = a[6];
        }
        const double M = d->molar_mass[s];
        const double *aref = d->nasa7 + s * 14 + (kTref > d->t_mid[s] ? 7 : 0);
        double cpR, hRT;
        host_nasa(aref, kTref, cpR, hRT);
        ef[s] = kR / M * kTref * (hRT - 1.0);
        t.sp[s * kSpStride + 0] = M;
        t.sp[s * kSpStride + 1] = 1.0 / M;
        t.sp[s * kSpStride + 2] = kR / M;
        t.sp[s * kSpStride + 3] = ef[s];
    }
    t.tpoly.assign((size_t)ns * 2 * kTpolyStride, 0.0);
    t.tpoly_f.assign((size_t)ns * 2 * kTpolyFStride, 0.0f);
    for (int s = 0; s < ns; ++s)
        for (int rg = 0; rg < 2; ++rg) {
            const double *a = d->nasa7 + s * 14 + rg * 7;
            const long double RM = (long double)kR / d->molar_mass[s];
            double *c = &t.tpoly[((size_t)s * 2 + rg) * kTpolyStride];
            c[0] = (double)(RM * a[5] - ef[s]);
            c[1] = (double)(RM * ((long double)a[0] - 1));
            for (int i = 2; i <= 5; ++i) c[i] = (double)(RM * a[i - 1] / i);
            c[6] = (double)(RM * ((long double)a[0] - 1));
            for (int i = 1; i <= 4; ++i) c[6 + i] = (double)(RM * a[i]);
            float *cf = &t.tpoly_f[((size_t)s * 2 + rg) * kTpolyFStride];
            for (int i = 0; i <= 4; ++i) cf[i] = (float)c[6 + i];
        }
    // dense stoichiometry
    std::vector<int> nuR((size_t)nr * ns, 0), nuP((size_t)nr * ns, 0);
    for (int r = 0; r < nr; ++r)
        for (int j = 0; j < 3; ++j) {
            if (d->reac_sp[r * 3 + j] >= 0) nuR[(size_t)r * ns + d->reac_sp[r * 3 + j]] += d->reac_nu[r * 3 + j];
            if (d->prod_sp[r * 3 + j] >= 0) nuP[(size_t)r * ns + d->prod_sp[r * 3 + j]] += d->prod_nu[r * 3 + j];
        }
    auto net = [&](int r, int s) { return nuP[(size_t)r * ns + s] - nuR[(size_t)r * ns + s]; };
    // per reaction: rate constants and concentration factors with repetition
    t.rxn_d.assign((size_t)nr * kRxnDStride, 0.0);
    t.rxn_f.assign((size_t)nr * kRxnFStride, 0);
    t.eff_ptr.assign(nr + 1, 0);
    std::vector<std::array<int, 3>> facR(nr), facP(nr);
    for (int r = 0; r < nr; ++r) {
        const int tb = d->third_body[r];
        int order = tb, dnu = 0;
        for (int j = 0; j < 3; ++j)
            if (d->reac_sp[r * 3 + j] >= 0) order += d->reac_nu[r * 3 + j];
        for (int s = 0; s < ns; ++s) dnu += net(r, s);
        const double A = d->arr_A[r];
        double *rd = &t.rxn_d[(size_t)r * kRxnDStride];
        rd[0] = A > 0 ? std::log(A) + (order - 1) * std::log(1e-6) : -INFINITY;
        rd[1] = d->arr_beta[r];
        rd[2] = d->arr_Ea[r] / kR;
        rd[3] = (double)dnu;
        std::array<int, 3> fr{SENT, SENT, SENT}, fp{SENT, SENT, SENT};
        int nf = 0, nb = 0;
        for (int j = 0; j < 3; ++j) {
            if (d->reac_sp[r * 3 + j] >= 0)
                for (int q = 0; q < d->reac_nu[r * 3 + j]; ++q) fr[nf++] = d->reac_sp[r * 3 + j];
            if (d->prod_sp[r * 3 + j] >= 0)
                for (int q = 0; q < d->prod_nu[r * 3 + j]; ++q) fp[nb++] = d->prod_sp[r * 3 + j];
        }
        facR[r] = fr;
        facP[r] = fp;
        t.rxn_f[2 * r] = fr[0] | (fr[1] << 8) | (fr[2] << 16) | ((tb & 1) << 24);
        t.rxn_f[2 * r + 1] = fp[0] | (fp[1] << 8) | (fp[2] << 16);
        if (tb && d->tb_eff)
            for (int s = 0; s < ns; ++s) {
                const double a = d->tb_eff[(size_t)r * ns + s];
                if (a != 1.0) {
                    t.eff_sp.push_back(s);
                    t.eff_c.push_back(a - 1.0);
                }
            }
        t.eff_ptr[r + 1] = (int)t.eff_sp.size();
    }
    // D entries: (reaction, column species) pairs, grouped by kind
    struct DEnt { int r, k, grp; int fa, fb, ba, bb, vf, vb; double alpha1; };
    std::vector<DEnt> ents;
    for (int r = 0; r < nr; ++r) {
        std::vector<int> cols;
        auto addc = [&](int s) { if (std::find(cols.begin(), cols.end(), s) == cols.end()) cols.push_back(s); };
        for (int j = 0; j < 3; ++j) if (d->reac_sp[r * 3 + j] >= 0) addc(d->reac_sp[r * 3 + j]);
        for (int j = 0; j < 3; ++j) if (d->prod_sp[r * 3 + j] >= 0) addc(d->prod_sp[r * 3 + j]);
        const int tb = d->third_body[r];
        if (tb && d->tb_eff)
            for (int s = 0; s < ns; ++s) if (d->tb_eff[(size_t)r * ns + s] != 1.0) addc(s);
        for (int k : cols) {
            DEnt e{};
            e.r = r;
            e.k = k;
            const int vf = nuR[(size_t)r * ns + k], vb = nuP[(size_t)r * ns + k];
            // remaining factors after removing one occurrence of k
            auto rest = [&](const std::array<int, 3> &f, int &x, int &y) {
                int out[3] = {SENT, SENT, SENT}, m = 0;
                bool removed = false;
                for (int q = 0; q < 3; ++q) {
                    if (!removed && f[q] == k) { removed = true; continue; }
                    if (f[q] != SENT) out[m++] = f[q];
                }
                x = out[0];
                y = out[1];
            };
            e.fa = e.fb = e.ba = e.bb = SENT;
            if (vf > 0) rest(facR[r], e.fa, e.fb);
            if (vb > 0) rest(facP[r], e.ba, e.bb);
            e.vf = vf;
            e.vb = vb;
            e.alpha1 = tb ? (d->tb_eff ? d->tb_eff[(size_t)r * ns + k] : 1.0) - 1.0 : 0.0;
            e.grp = vf > 0 && vb == 0 ? 0 : (vf == 0 && vb > 0 ? 1 : (vf > 0 ? 2 : 3));
            ents.push_back(e);
        }
    }
    std::stable_sort(ents.begin(), ents.end(), [](const DEnt &a, const DEnt &b) { return a.grp < b.grp; });
    t.nD = (int)ents.size();
    for (const auto &e : ents) {
        if (e.grp <= 0) t.nD_F++;
        if (e.grp <= 1) t.nD_B++;
        if (e.grp <= 2) t.nD_FB++;
        t.d_i0.push_back(e.r | (e.vf << 16) | (e.vb << 20));
        t.d_cef.push_back((float)e.alpha1);
        t.d_i1.push_back(e.fa | (e.fb << 8) | (e.ba << 16) | (e.bb << 24));
        t.d_ce.push_back(e.alpha1);
    }
    // gather lists: J_sk gathers nu_rs M_s D_rk over the reactions r (the
    // kernels eliminate the energy unknown, so no energy row is gathered)
    struct Term { int j; double c; int nu; };
    std::vector<std::vector<Term>> lists((size_t)ns * ns);
    // nu as signed powers of two (the packed words carry a coefficient's
    // sign and exponent bits, exact for those; any other nu, none in the
    // mechanisms at hand, becomes one term per binary digit)
    auto pow2_parts = [](int v) {
        std::vector<int> out;
        const int a = v < 0 ? -v : v;
        for (int b = 0; b < 31; ++b)
            if (a & (1 << b)) out.push_back(v < 0 ? -(1 << b) : (1 << b));
        return out;
    };
    for (int j = 0; j < t.nD; ++j) {
        const int r = ents[j].r, k = ents[j].k;
        for (int s = 0; s < ns; ++s) {
            const int v = net(r, s);
            if (v == 0) continue;
            // the FP64 lists keep nu_rs M_s whole; the FP32 lists, the parts
            lists[(size_t)s * ns + k].push_back({j, v * d->molar_mass[s], v});
        }
    }
    // the species entries, longest list first; the FP64 kernel's lists
    // carry the coefficients nu_rs M_s, the FP32 kernel's nu_rs (it
    // multiplies by M_s once per entry)
    auto longer = [&](int a, int b) { return lists[a].size() > lists[b].size(); };
    std::vector<int> order(ns * ns);
    for (int i = 0; i < ns * ns; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), longer);
    t.nJ = ns * ns;
    t.j_ptr.push_back(0);
    t.j_ptr32.push_back(0);
    for (int idx : order) {
        const int s = idx / ns, k = idx % ns;
        t.j_sk.push_back((s << 8) | k);
        t.j_sk32.push_back((s << 8) | k);
        for (const auto &tm : lists[idx]) {
            t.j_d.push_back(tm.j);
            t.j_c.push_back(tm.c);
            for (int part : pow2_parts(tm.nu)) {
                t.j_d32.push_back(tm.j);
                t.j_nu.push_back(part);
            }
        }
        t.j_ptr.push_back((int)t.j_d.size());
        t.j_ptr32.push_back((int)t.j_d32.size());
        if (!lists[idx].empty()) t.nJ_nz++;   // (the empty lists come last)
    }
    // species lists (reactions with nu_rs != 0) in chunks of kChunk
    t.sp_item_ptr.assign(ns + 1, 0);
    t.it_ptr.push_back(0);
    for (int s = 0; s < ns; ++s) {
        int cnt = 0;
        for (int r = 0; r < nr; ++r) {
            const int v = net(r, s);
            if (v == 0) continue;
            for (int part : pow2_parts(v)) {
                t.sp_r.push_back(r);
                t.sp_nui.push_back(part);
                if (++cnt == kChunk) {
                    t.it_ptr.push_back((int)t.sp_r.size());
                    cnt = 0;
                }
            }
        }
        if (cnt > 0) t.it_ptr.push_back((int)t.sp_r.size());
        t.sp_item_ptr[s + 1] = (int)t.it_ptr.size() - 1;
    }
    t.n_items = (int)t.it_ptr.size() - 1;
    // 2^(j/256), from the exponential of the exact arguments in long double
    // reciprocals for the elimination's small divisions (numerators below 64)
    t.div16.assign(67, 0u);
    for (int c = 1; c <= 66; ++c) t.div16[c] = (65536u + c - 1) / c;
    t.exp_tab.resize(kExpTab);
    for (int j = 0; j < kExpTab; ++j) t.exp_tab[j] = (double)std::exp2l((long double)j / kExpTab);
    fill_log_table(t.log_tab);
    // FP32 copies for the mixed-precision Jacobian
    t.rxn_df.assign((size_t)nr * kRxnDStride, 0.0f);
    for (int r = 0; r < nr; ++r) {
        t.rxn_df[(size_t)r * kRxnDStride + 0] = (float)t.rxn_d[(size_t)r * kRxnDStride + 1];
        t.rxn_df[(size_t)r * kRxnDStride + 1] = (float)t.rxn_d[(size_t)r * kRxnDStride + 2];
        t.rxn_df[(size_t)r * kRxnDStride + 2] = (float)t.rxn_d[(size_t)r * kRxnDStride + 3];
    }
    for (int j = 0; j < t.nD; ++j) {
        t.d_pk.push_back(make_int2(t.d_i0[j], t.d_i1[j]));
    }
    // a term's word (nu a signed power of two): the FP32 gather's carries
    // the sign and exponent bits of (float)nu over the D index (bits 0..22),
    // the species lists' those of (double)nu over the reaction (bits 0..19),
    // so one mask gives the coefficient exactly
    auto fword = [](int i, int nu) {
        const float f = (float)nu;
        unsigned b;
        memcpy(&b, &f, 4);
        return (b & 0xff800000u) | (unsigned)i;
    };
    auto dword = [](int r, int nu) {
        const double x = (double)nu;
        unsigned long long b;
        memcpy(&b, &x, 8);
        return ((unsigned)(b >> 32) & 0xfff00000u) | (unsigned)r;
    };
    for (size_t e = 0; e < t.j_d32.size(); ++e) t.j_w.push_back(fword(t.j_d32[e], t.j_nu[e]));
    for (size_t e = 0; e < t.sp_r.size(); ++e) t.sp_w.push_back(dword(t.sp_r[e], t.sp_nui[e]));
    // the gather layouts for each lane count (chem_internal.h): list p on
    // lane p % G of pass p / G, its q-th term at base(pass) + q G + lane
    // With `bank` (the shared-memory bank each term's operand sits in), the
    // terms of each list are put in an order in which the lanes of a pass
    // read distinct banks at each step where they can: the sum is the same
    // up to the order of its FP32 additions.
    auto interleave = [](int nlists, const std::vector<int> &ptr, int G, std::vector<int2> &meta,
                         std::vector<int> &pos, int tag_shift, const std::vector<int> *tags,
                         const std::vector<int> *bank = nullptr) {
        int base = 0;
        pos.assign(ptr.back(), -1);
        for (int P0 = 0; P0 < nlists; P0 += G) {
            const int P1 = std::min(nlists, P0 + G);
            int maxlen = 0;
            for (int q = P0; q < P1; ++q) maxlen = std::max(maxlen, ptr[q + 1] - ptr[q]);
            // slot[e]: the step at which term e is read
            std::vector<int> slot(ptr[P1] - ptr[P0], 0);
            for (int q = P0; q < P1; ++q)
                for (int i = 0; i < ptr[q + 1] - ptr[q]; ++i) slot[ptr[q] + i - ptr[P0]] = i;
            if (bank) {
                // greedy per step: the lists with the fewest terms left choose
                // first, each the remaining term whose bank is least used
                std::vector<std::vector<int>> left(P1 - P0);
                for (int q = P0; q < P1; ++q)
                    for (int e = ptr[q]; e < ptr[q + 1]; ++e) left[q - P0].push_back(e);
                for (int i = 0; i < maxlen; ++i) {
                    std::vector<int> act;
                    for (int l = 0; l < P1 - P0; ++l)
                        if (!left[l].empty()) act.push_back(l);
                    std::stable_sort(act.begin(), act.end(),
                                     [&](int a, int b) { return left[a].size() < left[b].size(); });
                    int load[32] = {0};
                    std::vector<int> seen;   // operands already read at this step (broadcast)
                    for (int l : act) {
                        int best = 0, best_cost = 1 << 30;
                        for (int c = 0; c < (int)left[l].size(); ++c) {
                            const int e = left[l][c], op = (*bank)[e];
                            const bool dup = std::find(seen.begin(), seen.end(), op) != seen.end();
                            const int cost = dup ? 0 : load[op & 31];
                            if (cost < best_cost) {
                                best_cost = cost;
                                best = c;
                            }
                        }
                        const int e = left[l][best];
                        left[l].erase(left[l].begin() + best);
                        slot[e - ptr[P0]] = i;
                        const int op = (*bank)[e];
                        if (std::find(seen.begin(), seen.end(), op) == seen.end()) {
                            seen.push_back(op);
                            ++load[op & 31];
                        }
                    }
                }
            }
            for (int q = P0; q < P1; ++q) {
                const int len = ptr[q + 1] - ptr[q], lane = q - P0;
                meta.push_back(make_int2(base + lane, (tags ? (*tags)[q] : 0) | (len << tag_shift)));
                for (int e = ptr[q]; e < ptr[q + 1]; ++e) pos[e] = base + slot[e - ptr[P0]] * G + lane;
            }
            base += maxlen * G;
        }
        return base;
    };
    for (int li = 0; li < kLayouts; ++li) {
        const int G = 2 << li;
        auto &L = t.lay[li];
        std::vector<int> pos;
        const int nw = interleave(t.nJ, t.j_ptr, G, L.j_meta, pos, 16, &t.j_sk);
        L.j_d.assign(std::max(nw, 1), 0);
        L.j_c.assign(std::max(nw, 1), 0.0);
        for (size_t e = 0; e < pos.size(); ++e) {
            L.j_d[pos[e]] = t.j_d[e];
            L.j_c[pos[e]] = t.j_c[e];
        }
        std::vector<int2> meta32;
        const int nw32 = interleave(ns * ns, t.j_ptr32, G, meta32, pos, 16, &t.j_sk32, &t.j_d32);
        // the FP32 entries' metadata: first word, length, offset of (s, k)
        // in the column-major matrix of columns of ldc rows, and the factor
        // M_s / M_k rounded once to FP32
        const int ldc = (ns + 3) & ~3;
        for (const int2 &mt : meta32) {
            const int s = (mt.y >> 8) & 0xff, k = mt.y & 0xff;
            float f = (float)(d->molar_mass[s] / d->molar_mass[k]);
            int fb;
            std::memcpy(&fb, &f, sizeof fb);
            L.j_meta32.push_back(make_int4(mt.x, mt.y >> 16, k * ldc + s, fb));
        }
        L.j_w.assign(std::max(nw32, 1), 0u);
        for (size_t e = 0; e < pos.size(); ++e) L.j_w[pos[e]] = t.j_w[e];
        const int ni = interleave(t.n_items, t.it_ptr, G, L.it_meta, pos, 0, nullptr);
        L.sp_w.assign(std::max(ni, 1), 0u);
        for (size_t e = 0; e < pos.size(); ++e) {
            L.sp_w[pos[e]] = t.sp_w[e];
        }
        if (L.it_meta.empty()) L.it_meta.push_back(make_int2(0, 0));
    }
    for (double v : t.sp) t.spf.push_back((float)v);
    // the polynomial tables go coefficient-major (chem_internal.h): from
    // [2 s + rg][c] to [2 c + rg][s]
    auto coef_major = [ns](auto &v, int stride) {
        auto o = v;
        for (int s = 0; s < ns; ++s)
            for (int rg = 0; rg < 2; ++rg)
                for (int c = 0; c < stride; ++c)
                    o[(size_t)(2 * c + rg) * ns + s] = v[((size_t)s * 2 + rg) * stride + c];
        v.swap(o);
    };
    coef_major(t.thermo, kThermoStride);
    coef_major(t.tpoly, kTpolyStride);
    coef_major(t.tpoly_f, kTpolyFStride);
    // keep every array non-empty so device pointers are valid
    auto pad_f = [](std::vector<float> &v) { if (v.empty()) v.push_back(0.0f); };
    pad_f(t.rxn_df); pad_f(t.d_cef);
    if (t.d_pk.empty()) t.d_pk.push_back(make_int2(0, 0));
    auto pad_u = [](std::vector<unsigned> &v) { if (v.empty()) v.push_back(0u); };
    pad_u(t.j_w); pad_u(t.sp_w);
    auto pad_i = [](std::vector<int> &v) { if (v.empty()) v.push_back(0); };
    auto pad_d = [](std::vector<double> &v) { if (v.empty()) v.push_back(0.0); };
    pad_i(t.eff_sp); pad_d(t.eff_c); pad_d(t.d_ce);
    pad_i(t.j_d); pad_d(t.j_c); pad_i(t.rxn_f); pad_d(t.rxn_d);
}

// Copies the tables into one device allocation.
static int upload(const HostTables &t, int ns, int nr, Handle *h) {
    struct Part { const void *src; size_t bytes; size_t off; };
    std::vector<Part> parts;
    size_t total = 0;
    auto add = [&](const void *src, size_t bytes) {
        total = (total + 255) / 256 * 256;
        parts.push_back({src, bytes, total});
        total += bytes;
        return parts.size() - 1;
    };
    auto addv = [&](const auto &v) { return add(v.data(), v.size() * sizeof(v[0])); };
    const size_t i_th = addv(t.thermo), i_tm = addv(t.tmid), i_tp = addv(t.tpoly), i_tpf = addv(t.tpoly_f),
                 i_sp = addv(t.sp), i_rd = addv(t.rxn_d),
                 i_rf = addv(t.rxn_f), i_ep = addv(t.eff_ptr), i_es = addv(t.eff_sp), i_ec = addv(t.eff_c),
                 i_dpk = addv(t.d_pk),
                 // a gap where FP64 coefficient triples (24 bytes per D entry)
                 // used to sit: the tables after it keep their offsets, on
                 // which the mixed kernel's cache behaviour measurably depends
                 i_gap = add(nullptr, (size_t)3 * std::max(t.nD, 1) * sizeof(double)),
                 i_sip = addv(t.sp_item_ptr),
                 i_ex = addv(t.exp_tab), i_div = addv(t.div16), i_rdf = addv(t.rxn_df), i_dcef = addv(t.d_cef),
                 i_spf = addv(t.spf), i_log = addv(t.log_tab);
    size_t i_lay[kLayouts][8];
    for (int li = 0; li < kLayouts; ++li) {
        const auto &L = t.lay[li];
        i_lay[li][7] = addv(L.j_meta32);
        i_lay[li][0] = addv(L.j_meta);
        i_lay[li][1] = addv(L.j_w);
        i_lay[li][2] = addv(L.j_d);
        i_lay[li][3] = addv(L.j_c);
        i_lay[li][4] = addv(L.it_meta);
        i_lay[li][5] = addv(L.sp_w);
    }
    const size_t i_dce = addv(t.d_ce);
    cudaError_t e = cudaMalloc(&h->dev_tables, total);
    if (e != cudaSuccess) return fail(CHEM_E_OOM, "device tables (%zu bytes): %s", total, cudaGetErrorString(e));
    h->dev_tables_bytes = total;
    std::vector<char> staging(total, 0);
    for (const auto &p : parts)
        if (p.src) memcpy(staging.data() + p.off, p.src, p.bytes);
    e = cudaMemcpy(h->dev_tables, staging.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "copying mechanism tables");
    char *b = static_cast<char *>(h->dev_tables);
    auto at = [&](size_t i) { return (const void *)(b + parts[i].off); };
    DeviceMech &m = h->mech;
    m.ns = ns;
    m.nr = nr;
    m.ntb = t.ntb;
    m.nD = t.nD;
    m.nD_F = t.nD_F;
    m.nD_B = t.nD_B;
    m.nD_FB = t.nD_FB;
    m.nJ = t.nJ;
    m.nJ_nz = t.nJ_nz;
    m.n_items = t.n_items;
    m.thermo = (const double *)at(i_th);
    m.tmid = (const double *)at(i_tm);
    m.tpoly = (const double *)at(i_tp);
    m.tpoly_f = (const float *)at(i_tpf);
    m.sp = (const double *)at(i_sp);
    m.rxn_d = (const double *)at(i_rd);
    m.rxn_f = (const int *)at(i_rf);
    m.eff_ptr = (const int *)at(i_ep);
    m.eff_sp = (const int *)at(i_es);
    m.eff_c = (const double *)at(i_ec);
    m.d_pk = (const int2 *)at(i_dpk);
    (void)i_gap;
    m.d_ce = (const double *)at(i_dce);
    for (int li = 0; li < kLayouts; ++li) {
        GatherLayout &g = m.gl[li];
        g.j_meta = (const int2 *)at(i_lay[li][0]);
        g.j_meta32 = (const int4 *)at(i_lay[li][7]);
        g.j_w = (const unsigned *)at(i_lay[li][1]);
        g.j_d = (const int *)at(i_lay[li][2]);
        g.j_c = (const double *)at(i_lay[li][3]);
        g.it_meta = (const int2 *)at(i_lay[li][4]);
        g.sp_w = (const unsigned *)at(i_lay[li][5]);
    }
    m.sp_item_ptr = (const int *)at(i_sip);

    m.exp_tab = (const double *)at(i_ex);
    m.div16 = (const unsigned *)at(i_div);
    m.rxn_df = (const float *)at(i_rdf);
    m.d_cef = (const float *)at(i_dcef);

    m.spf = (const float *)at(i_spf);
    m.log_tab = (const double2 *)at(i_log);
    return CHEM_OK;
}

// Launch shape of the backward-Euler kernel for (precision, G, warps per
// block): wpb = 0 picks the warps per block and blocks per SM that maximise
// resident warps within shared memory and registers.
int configure(Handle *h, int prec, int G, int wpb_req, LaunchCfg &cfg, bool queue) {
    const void *fn = queue ? be_kernel_queue(prec, G) : prec == CHEM_MIXED ? be_kernel_mixed(G) : be_kernel_fp64(G);
    if (!fn) return fail(CHEM_E_INVALID_ARG, "lanes_per_cell %d not available", G);
    const int S = 32 / G;
    const long long sb = slot_stride(h->mech, prec == CHEM_MIXED ? 4 : 8, G);
    int best_warps = 0;
    LaunchCfg best{};
    // the attribute is per function and shared by every handle: allow the
    // device maximum and pass each launch its own size
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)h->max_smem_optin);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    for (int wpb = kMaxBlockThreads / 32; wpb >= 1; --wpb) {
        if (wpb_req && wpb != wpb_req) continue;
        const long long smem = kBlockHeaderBytes + (long long)wpb * S * sb;
        if (smem > h->max_smem_optin) continue;
        int blocks = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, wpb * 32, (size_t)smem);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
        if (blocks * wpb > best_warps) {
            best_warps = blocks * wpb;
            best.fn = fn;
            best.block = wpb * 32;
            best.smem = (size_t)smem;
            best.grid = blocks * h->num_sms;
            best.G = G;
        }
    }
    if (best_warps == 0)
        return fail(CHEM_E_UNSUPPORTED, "one cell slot (%lld bytes) exceeds shared memory at %d lanes/cell"
                    " and %d warps per block", sb, G, wpb_req);
    cfg = best;
    return CHEM_OK;
}

int default_lanes(int ns, int prec) {
    const int n = ns + 1;
    (void)prec;
    if (n <= 12) return 4;
    if (n <= 24) return 8;
    return 32;
}

int get_cfg(Handle *h, int prec, int G, LaunchCfg **out, bool queue) {
    const int wpb = G == h->lanes[prec] ? h->wpb[prec] : 0;
    const int key = ((queue ? 2 : 0) + prec) * 64 * 16 + G * 16 + wpb;
    std::lock_guard<std::mutex> lk(h->mu);
    auto it = h->cfgs.find(key);
    if (it == h->cfgs.end()) {
        LaunchCfg c;
        int rc = configure(h, prec, G, wpb, c, queue);
        if (rc) return rc;
        it = h->cfgs.emplace(key, c).first;
    }
    *out = &it->second;
    return CHEM_OK;
}

unsigned long long *next_counter(Handle *h) {
    const unsigned idx = h->counter_idx.fetch_add(1) % kCounterRing;
    return h->counters + idx;
}

}  // namespace chem

using namespace chem;

// ---------------------------------------------------------------------------
// small kernels: state from (T, P, Y) and temperature of given states
namespace chem {

__global__ void state_from_tpy_kernel(DeviceMech m, long long n, long long ld, const double *T,
                                      const double *P, const double *Y, double *rho, double *e) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double Ti = T[i], invT = 1.0 / Ti;
    double invW = 0.0;
    for (int s = 0; s < m.ns; ++s) invW += Y[(size_t)s * ld + i] * m.sp[s * kSpStride + 1];
    const double rt = P[i] / (kR * Ti * invW);
    double ei = 0.0;
    for (int s = 0; s < m.ns; ++s) {
        const double rs = rt * Y[(size_t)s * ld + i];
        rho[(size_t)s * ld + i] = rs;
        const auto th = coef_row(m.thermo, m.ns, s, Ti > m.tmid[s] ? 1 : 0);
        const double hRT = th[0] + Ti * (th[5] + Ti * (th[6] + Ti * (th[7] + Ti * th[8]))) + th[9] * invT;
        ei += rs * (m.sp[s * kSpStride + 2] * Ti * (hRT - 1.0) - m.sp[s * kSpStride + 3]);
    }
    e[i] = ei;
}

__global__ void temperature_kernel(DeviceMech m, long long n, long long ld, const double *rho,
                                   const double *e, const double *Tg, double *Tout) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double lo = kTlo, hi = kThi, T = Tg ? Tg[i] : 1500.0;
    if (!(T > lo && T < hi)) T = 1500.0;
    const double ei = e[i];
    bool ok = false;
    for (int it = 1; it <= kTmaxIter; ++it) {
        const double invT = 1.0 / T;
        double f = 0.0, fp = 0.0;
        for (int s = 0; s < m.ns; ++s) {
            const auto th = coef_row(m.thermo, m.ns, s, T > m.tmid[s] ? 1 : 0);
            const double cpR = th[0] + T * (th[1] + T * (th[2] + T * (th[3] + T * th[4])));
            const double hRT = th[0] + T * (th[5] + T * (th[6] + T * (th[7] + T * th[8]))) + th[9] * invT;
            const double RM = m.sp[s * kSpStride + 2];
            const double r = rho[(size_t)s * ld + i];
            f += r * (RM * T * (hRT - 1.0) - m.sp[s * kSpStride + 3]);
            fp += r * RM * (cpR - 1.0);
        }
        f -= ei;
        if (f == 0.0) { ok = true; break; }
        if (f > 0.0) hi = T; else lo = T;
        double Tn = T - f / fp;
        if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
        const double dT = Tn - T;
        T = Tn;
        if (fabs(dT) <= kTtol * T) {
            ok = !(T <= kTlo * (1.0 + 1e-9) || T >= kThi * (1.0 - 1e-9));
            break;
        }
    }
    Tout[i] = ok ? T : NAN;
}

static_assert(kSchedWords == CHEM_SCHEDULE_WORDS, "schedule record size");
static_assert(kSubstepStates == CHEM_SUBSTEP_STATES, "substep-state record size");

int launch_step(Handle *h, const chem_advance_args *a, int prec, int G, unsigned long long *counter) {
    LaunchCfg *cfg = nullptr;
    int rc = get_cfg(h, prec, G, &cfg);
    if (rc) return rc;
    return launch_cfg(h, a, prec, cfg, counter);
}

StepOptions step_options(const Handle *h, int prec) {
    return StepOptions{h->opts.rtol, h->opts.atol_rel,
                       prec == CHEM_MIXED ? h->opts.conv_kappa_mixed : h->opts.conv_kappa,
                       prec == CHEM_MIXED ? h->opts.max_newton_mixed : h->opts.max_newton,
                       h->opts.max_halvings, h->opts.max_attempts, h->opts.point_implicit,
                       h->opts.div_check};
}

int launch_cfg(Handle *h, const chem_advance_args *a, int prec, const LaunchCfg *cfg,
               unsigned long long *counter) {
    cudaStream_t st = (cudaStream_t)a->stream;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "zeroing the work counter");
    StepOptions o = step_options(h, prec);
    StepBatch b{};
    b.n_cells = a->n_cells;
    b.ld = a->ld > 0 ? a->ld : a->n_cells;
    b.rho = a->rho_s;
    b.e = a->e;
    b.dt = a->dt;
    b.T_in = a->T_in;
    b.T_out = a->T_out;
    b.status = a->status;
    b.newton_iters = a->newton_iters;
    b.substeps = a->substeps;
    b.failures = a->failures;
    b.work_counter = counter;
    b.schedule = a->schedule;
    b.substep_states = a->substep_states;
    if (a->schedule) o.max_attempts = std::min(o.max_attempts, 32 * kSchedWords);
    // no more blocks than it takes to give every cell a slot
    const long long slots_per_block = (long long)(cfg->block / 32) * (32 / cfg->G);
    long long grid = std::min<long long>(cfg->grid, (b.n_cells + slots_per_block - 1) / slots_per_block);
    if (grid < 1) grid = 1;
    void *args[] = {&h->mech, &o, &b};
    e = cudaLaunchKernel(cfg->fn, dim3((unsigned)grid), dim3(cfg->block), args, cfg->smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "launching the step kernel");
    h->launches.fetch_add(1);
    return CHEM_OK;
}

}  // namespace chem

// ---------------------------------------------------------------------------
// C ABI
extern "C" {

int chem_default_options(chem_options *o) {
    if (!o) return fail(CHEM_E_INVALID_ARG, "options pointer is NULL");
    o->precision = CHEM_FP64;
    o->rtol = 1e-10;
    o->atol_rel = 1e-12;
    o->max_newton = 12;
    o->max_halvings = 20;
    o->max_attempts = 1000;
    o->point_implicit = 0;
    o->div_check = 1;
    o->lanes_per_cell = 0;
    o->autotune = 0;
    o->hbm_budget_bytes = 0;
    o->max_newton_mixed = 12;
    o->conv_kappa = 0.0;
    o->conv_kappa_mixed = 0.01;
    return CHEM_OK;
}

static int check_options(const chem_options *o) {
    if (o->precision != CHEM_FP64 && o->precision != CHEM_MIXED)
        return fail(CHEM_E_INVALID_ARG, "precision %d", o->precision);
    if (!(o->rtol > 0) || !(o->atol_rel >= 0) || !std::isfinite(o->rtol) || !std::isfinite(o->atol_rel))
        return fail(CHEM_E_INVALID_ARG, "tolerances");
    if (o->max_newton < 1 || o->max_newton > 1000) return fail(CHEM_E_INVALID_ARG, "max_newton %d", o->max_newton);
    if (o->max_newton_mixed < 1 || o->max_newton_mixed > 1000)
        return fail(CHEM_E_INVALID_ARG, "max_newton_mixed %d", o->max_newton_mixed);
    if (o->max_halvings < 0 || o->max_halvings > 40) return fail(CHEM_E_INVALID_ARG, "max_halvings %d", o->max_halvings);
    if (o->max_attempts < 1 || o->max_attempts > 1000000) return fail(CHEM_E_INVALID_ARG, "max_attempts %d", o->max_attempts);
    const int l = o->lanes_per_cell;
    if (l != 0 && l != 2 && l != 4 && l != 8 && l != 16 && l != 32)
        return fail(CHEM_E_INVALID_ARG, "lanes_per_cell %d (0, 2, 4, 8, 16 or 32)", l);
    if (o->hbm_budget_bytes < 0) return fail(CHEM_E_INVALID_ARG, "hbm_budget_bytes");
    if (!(o->conv_kappa >= 0.0 && o->conv_kappa <= 1.0)) return fail(CHEM_E_INVALID_ARG, "conv_kappa");
    if (!(o->conv_kappa_mixed >= 0.0 && o->conv_kappa_mixed <= 1.0))
        return fail(CHEM_E_INVALID_ARG, "conv_kappa_mixed");
    return CHEM_OK;
}

int chem_create(const chem_mech_desc *mech, const chem_options *opts, chem_handle_t *out) {
    if (!out) return fail(CHEM_E_INVALID_ARG, "output handle pointer is NULL");
    *out = nullptr;
    chem_options o;
    chem_default_options(&o);
    if (opts) o = *opts;
    int rc = check_options(&o);
    if (rc) return rc;
    rc = validate(mech);
    if (rc) return rc;
    Handle *h = new (std::nothrow) Handle();
    if (!h) return fail(CHEM_E_OOM, "host allocation");
    h->opts = o;
    h->ns = mech->n_species;
    h->nr = mech->n_reactions;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaGetDevice"); }
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, h->device);
    if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaGetDeviceProperties"); }
    h->num_sms = prop.multiProcessorCount;
    h->max_smem_optin = (long long)prop.sharedMemPerBlockOptin;
    ReorderedMech rm;
    third_body_first(mech, rm);
    HostTables t;
    build_tables(&rm.d, t);
    t.ntb = rm.ntb;
    h->ef_host.resize(h->ns);
    for (int s = 0; s < h->ns; ++s) h->ef_host[s] = t.sp[s * kSpStride + 3];
    rc = upload(t, h->ns, h->nr, h);
    if (rc) { chem_destroy(h); return rc; }
    e = cudaMalloc(&h->counters, sizeof(unsigned long long) * kCounterRing);
    if (e != cudaSuccess) { chem_destroy(h); return fail(CHEM_E_OOM, "work counters"); }
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { chem_destroy(h); return cuda_fail(e, "stream"); }
    for (int prec : {CHEM_FP64, CHEM_MIXED}) {
        const int G = o.lanes_per_cell ? o.lanes_per_cell : default_lanes(h->ns, prec);
        h->lanes[prec] = G;
        LaunchCfg *cfg;
        rc = get_cfg(h, prec, G, &cfg);
        // (and the request server's queue instantiation, so that a server
        // sets up this handle's lane without touching function attributes)
        if (!rc) rc = get_cfg(h, prec, G, &cfg, true);
        if (rc) { chem_destroy(h); return rc; }
    }
    *out = h;
    return CHEM_OK;
}

int chem_destroy(chem_handle_t hh) {
    Handle *h = hh;
    if (!h) return fail(CHEM_E_INVALID_ARG, "handle is NULL");
    destroy_serving(h);
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaDeviceSynchronize();
    if (h->dev_tables) cudaFree(h->dev_tables);
    if (h->counters) cudaFree(h->counters);
    if (h->host_rho) cudaFree(h->host_rho);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return CHEM_OK;
}

int chem_advance_ex(chem_handle_t hh, const chem_advance_args *a) {
    Handle *h = hh;
    if (!h || !a) return fail(CHEM_E_INVALID_ARG, "NULL handle or arguments");
    if (a->n_cells < 0) return fail(CHEM_E_INVALID_ARG, "n_cells %lld", (long long)a->n_cells);
    if (a->n_cells == 0) return CHEM_OK;
    if (!a->rho_s || !a->e) return fail(CHEM_E_INVALID_ARG, "state pointers are NULL");
    if (a->ld != 0 && a->ld < a->n_cells) return fail(CHEM_E_INVALID_ARG, "ld %lld < n_cells", (long long)a->ld);
    if (!(a->dt >= 0) || !std::isfinite(a->dt)) return fail(CHEM_E_INVALID_ARG, "dt %g", a->dt);
    const int prec = a->precision < 0 ? h->opts.precision : a->precision;
    if (prec != CHEM_FP64 && prec != CHEM_MIXED) return fail(CHEM_E_INVALID_ARG, "precision %d", prec);
    if (h->opts.autotune && !h->tuned[prec] && !a->lanes_per_cell) {
        // first call of this precision: tune on the call's own cells (synchronous)
        int lanes = 0, wpb = 0;
        const int rc = chem_autotune(h, prec, a->n_cells, a->ld, a->rho_s, a->e, a->dt, a->T_in, a->stream,
                                     &lanes, &wpb);
        if (rc) return rc;
    }
    int G = a->lanes_per_cell ? a->lanes_per_cell : h->lanes[prec];
    if (G != 2 && G != 4 && G != 8 && G != 16 && G != 32)
        return fail(CHEM_E_INVALID_ARG, "lanes_per_cell %d", G);
    return launch_step(h, a, prec, G, next_counter(h));
}

int chem_advance_segmented(chem_handle_t hh, const chem_advance_args *a, int64_t segment_cells) {
    Handle *h = hh;
    if (!h || !a) return fail(CHEM_E_INVALID_ARG, "NULL handle or arguments");
    if (segment_cells <= 0 || segment_cells >= a->n_cells) return chem_advance_ex(h, a);
    const int64_t ld = a->ld > 0 ? a->ld : a->n_cells;
    for (int64_t off = 0; off < a->n_cells; off += segment_cells) {
        chem_advance_args s = *a;
        s.n_cells = std::min<int64_t>(segment_cells, a->n_cells - off);
        s.ld = ld;
        s.rho_s = a->rho_s + off;
        s.e = a->e + off;
        s.T_in = a->T_in ? a->T_in + off : nullptr;
        s.T_out = a->T_out ? a->T_out + off : nullptr;
        s.status = a->status ? a->status + off : nullptr;
        s.newton_iters = a->newton_iters ? a->newton_iters + off : nullptr;
        s.substeps = a->substeps ? a->substeps + off : nullptr;
        s.failures = a->failures ? a->failures + off : nullptr;
        s.schedule = a->schedule ? a->schedule + off * CHEM_SCHEDULE_WORDS : nullptr;
        s.substep_states =
            a->substep_states ? a->substep_states + off * CHEM_SUBSTEP_STATES * (h->ns + 1) : nullptr;
        const int rc = chem_advance_ex(h, &s);
        if (rc) return rc;
    }
    return CHEM_OK;
}

int chem_advance(chem_handle_t h, int64_t n_cells, double *rho_s, double *e, double dt, void *stream) {
    chem_advance_args a;
    memset(&a, 0, sizeof a);
    a.n_cells = n_cells;
    a.ld = n_cells;
    a.rho_s = rho_s;
    a.e = e;
    a.dt = dt;
    a.stream = stream;
    a.precision = -1;
    return chem_advance_ex(h, &a);
}

int chem_advance_host(chem_handle_t hh, int64_t n_cells, int64_t ld, double *rho_s, double *e, double dt,
                      double *T_out, int32_t *status) {
    Handle *h = hh;
    if (!h || !rho_s || !e) return fail(CHEM_E_INVALID_ARG, "NULL argument");
    if (n_cells < 0 || (ld != 0 && ld < n_cells)) return fail(CHEM_E_INVALID_ARG, "sizes");
    if (n_cells == 0) return CHEM_OK;
    if (ld == 0) ld = n_cells;
    std::lock_guard<std::mutex> lk(h->host_mu);
    const int ns = h->ns;
    const size_t need = (size_t)n_cells * (ns + 1) * 8 + (size_t)n_cells * (8 + 4);
    if (need > h->host_bytes) {
        if (h->host_rho) cudaFree(h->host_rho);
        h->host_rho = nullptr;
        h->host_bytes = 0;
        cudaError_t e2 = cudaMalloc(&h->host_rho, need);
        if (e2 != cudaSuccess) return fail(CHEM_E_OOM, "staging buffers (%zu bytes)", need);
        h->host_bytes = need;
    }
    double *d_rho = (double *)h->host_rho;
    double *d_e = d_rho + (size_t)n_cells * ns;
    double *d_T = d_e + n_cells;
    int32_t *d_st = (int32_t *)(d_T + n_cells);
    cudaStream_t st = h->stream;
    cudaError_t ce = cudaMemcpy2DAsync(d_rho, (size_t)n_cells * 8, rho_s, (size_t)ld * 8, (size_t)n_cells * 8, ns,
                                       cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "host-to-device copy");
    ce = cudaMemcpyAsync(d_e, e, (size_t)n_cells * 8, cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "host-to-device copy");
    chem_advance_args a;
    memset(&a, 0, sizeof a);
    a.n_cells = n_cells;
    a.ld = n_cells;
    a.rho_s = d_rho;
    a.e = d_e;
    a.dt = dt;
    a.T_out = T_out ? d_T : nullptr;
    a.status = status ? d_st : nullptr;
    a.stream = st;
    a.precision = -1;
    int rc = chem_advance_ex(h, &a);
    if (rc) return rc;
    ce = cudaMemcpy2DAsync(rho_s, (size_t)ld * 8, d_rho, (size_t)n_cells * 8, (size_t)n_cells * 8, ns,
                           cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(e, d_e, (size_t)n_cells * 8, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess && T_out) ce = cudaMemcpyAsync(T_out, d_T, (size_t)n_cells * 8, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess && status)
        ce = cudaMemcpyAsync(status, d_st, (size_t)n_cells * 4, cudaMemcpyDeviceToHost, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "device-to-host copy");
    ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return cuda_fail(ce, "synchronising the step");
    return CHEM_OK;
}

int chem_state_from_tpy(chem_handle_t hh, int64_t n, int64_t ld, const double *T, const double *P,
                        const double *Y, double *rho_s, double *e, void *stream) {
    Handle *h = hh;
    if (!h || !T || !P || !Y || !rho_s || !e) return fail(CHEM_E_INVALID_ARG, "NULL argument");
    if (n < 0 || (ld != 0 && ld < n)) return fail(CHEM_E_INVALID_ARG, "sizes");
    if (n == 0) return CHEM_OK;
    if (ld == 0) ld = n;
    const int bs = 128;
    state_from_tpy_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, (cudaStream_t)stream>>>(h->mech, n, ld, T, P, Y,
                                                                                          rho_s, e);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "state_from_tpy launch");
    h->launches.fetch_add(1);
    return CHEM_OK;
}

int chem_temperature(chem_handle_t hh, int64_t n, int64_t ld, const double *rho_s, const double *e,
                     const double *T_guess, double *T_out, void *stream) {
    Handle *h = hh;
    if (!h || !rho_s || !e || !T_out) return fail(CHEM_E_INVALID_ARG, "NULL argument");
    if (n < 0 || (ld != 0 && ld < n)) return fail(CHEM_E_INVALID_ARG, "sizes");
    if (n == 0) return CHEM_OK;
    if (ld == 0) ld = n;
    const int bs = 128;
    temperature_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, (cudaStream_t)stream>>>(h->mech, n, ld, rho_s, e,
                                                                                      T_guess, T_out);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "temperature launch");
    h->launches.fetch_add(1);
    return CHEM_OK;
}

int chem_formation_energies(chem_handle_t hh, double *e_f) {
    Handle *h = hh;
    if (!h || !e_f) return fail(CHEM_E_INVALID_ARG, "NULL argument");
    for (int s = 0; s < h->ns; ++s) e_f[s] = h->ef_host[s];
    return CHEM_OK;
}

int chem_get_lanes_per_cell(chem_handle_t hh, int32_t precision, int32_t *lanes) {
    Handle *h = hh;
    if (!h || !lanes || (precision != CHEM_FP64 && precision != CHEM_MIXED))
        return fail(CHEM_E_INVALID_ARG, "bad argument");
    *lanes = h->lanes[precision];
    return CHEM_OK;
}

int chem_launch_count(chem_handle_t hh, int64_t *count) {
    Handle *h = hh;
    if (!h || !count) return fail(CHEM_E_INVALID_ARG, "bad argument");
    *count = h->launches.load();
    return CHEM_OK;
}

const char *chem_strerror(int code) {
    switch (code) {
        case CHEM_OK: return "ok";
        case CHEM_E_INVALID_ARG: return "invalid argument";
        case CHEM_E_BAD_MECHANISM: return "invalid mechanism";
        case CHEM_E_OOM: return "out of memory";
        case CHEM_E_OVER_BUDGET: return "request exceeds the HBM budget";
        case CHEM_E_CUDA: return "CUDA error";
        case CHEM_E_TIMEOUT: return "timed out";
        case CHEM_E_UNSUPPORTED: return "size beyond the kernels' limits";
        case CHEM_E_NOT_FOUND: return "unknown ticket";
        default: return "unknown error code";
    }
}

const char *chem_last_error_message(void) { return g_errmsg; }

}  // extern "C"
