"""Hand-built mechanisms with closed-form answers, for pinning the oracle.

Each mechanism is made of species whose NASA-7 polynomials reduce to
constants, so thermodynamics, equilibrium constants and whole backward-Euler
steps have textbook closed forms that do not go through the oracle.
"""
import numpy as np

from paper_1110_4903_gb300 import synth

R = 8.314462618
PA = 101325.0
TREF = 298.15


def const_cp(a1, a6, a7, a1_high=None):
    """NASA-7 pair for cp/R = a1 (constant); a1_high gives a different
    constant above T_mid (used to pin range selection)."""
    lo = [a1, 0.0, 0.0, 0.0, 0.0, a6, a7]
    hi = [a1 if a1_high is None else a1_high, 0.0, 0.0, 0.0, 0.0, a6, a7]
    return np.array([lo, hi], np.float64)


def isomer_pair(kf=1.0e4, a7A=5.0, a7B=5.7, a1=3.5, a6=-1000.0):
    """A <=> B, isomers (same composition, same mass), same cp and a6, so
    dH = 0 and K_c = exp(a7_B - a7_A) exactly; first order, beta = E = 0,
    so K_f = kf (s^-1) at every T."""
    nasa = np.stack([const_cp(a1, a6, a7A), const_cp(a1, a6, a7B)])
    comps = {"A": {"H": 1, "O": 1}, "B": {"H": 1, "O": 1}}
    return synth.make_mechanism("isomer", ["A", "B"], comps, ["H", "O"],
                                [(("A",), ("B",), 0)], nasa,
                                arr_A=[kf], arr_beta=[0.0], arr_Ea=[0.0])


def dimer_pair(A_cgs=1.0e10, a1A=3.0, a6A=-500.0, a7A=4.0, a7B=3.0):
    """2 A <=> B with B = A2.  cp_B/R = 2 cp_A/R - 1 and a6_B = 2 a6_A make
    the per-mass energies of A and B identical functions of T, so T stays
    constant while e is constant, and K_c = (R e / P_a) exp(a7_B - 2 a7_A)
    (independent of T; e = Euler's number).  Second order, beta = E = 0,
    so K_f = A_cgs * 1e-6 m^3/(mol s)."""
    nasa = np.stack([const_cp(a1A, a6A, a7A), const_cp(2 * a1A - 1.0, 2 * a6A, a7B)])
    comps = {"A": {"H": 1}, "B": {"H": 2}}
    return synth.make_mechanism("dimer", ["A", "B"], comps, ["H"],
                                [(("A", "A"), ("B",), 0)], nasa,
                                arr_A=[A_cgs], arr_beta=[0.0], arr_Ea=[0.0])


def const_cp_mixture(a1s=(2.5, 3.5, 4.5), a6s=(0.0, -2000.0, 1500.0)):
    """Inert species with constant cp (no reactions used): the sensible
    energy is e_s = (R/M_s)(a1_s - 1)(T - T_ref) exactly."""
    nasa = np.stack([const_cp(a, b, 10.0) for a, b in zip(a1s, a6s)])
    names = ["X0", "X1", "X2"]
    comps = {"X0": {"H": 1}, "X1": {"H": 2}, "X2": {"O": 1}}
    return synth.make_mechanism("constcp", names, comps, ["H", "O"],
                                [((names[0],), (names[0],), 0)], nasa,
                                arr_A=[0.0], arr_beta=[0.0], arr_Ea=[0.0])


def two_range_species():
    """One species with cp/R = 3.5 below T_mid and 4.5 above it."""
    nasa = np.stack([const_cp(3.5, 0.0, 10.0, a1_high=4.5)])
    return synth.make_mechanism("tworange", ["A"], {"A": {"H": 1}}, ["H"],
                                [(("A",), ("A",), 0)], nasa,
                                arr_A=[0.0], arr_beta=[0.0], arr_Ea=[0.0])


def third_body_twin(A_cgs=1.0e12):
    """A + B => AB twice: once plain, once with +M (all efficiencies 1) and
    A scaled so both have the same SI rate constant.  Q_M / Q_plain must
    equal the total concentration, P/(R T) by Dalton's law (Eq. 5)."""
    nasa = np.stack([const_cp(2.5, 1000.0, 15.0), const_cp(2.5, 1200.0, 16.0),
                     const_cp(4.0, -3000.0, 20.0)])
    comps = {"A": {"H": 1}, "B": {"O": 1}, "AB": {"H": 1, "O": 1}}
    return synth.make_mechanism("tbtwin", ["A", "B", "AB"], comps, ["H", "O"],
                                [(("A", "B"), ("AB",), 0), (("A", "B"), ("AB",), 1)], nasa,
                                arr_A=[A_cgs, A_cgs * 1e6], arr_beta=[0.3, 0.3],
                                arr_Ea=[2e4, 2e4])


def trimer_chain(A2_cgs=1.0e10, A3_cgs=1.0e12, A3d_cgs=1.0e16, a1=3.0, a6=-800.0):
    """A, A2, A3 with 2 A <=> A2, A2 + A <=> A3 and 3 A <=> A3: the last gives
    A a net coefficient of -3, not a power of two.  cp/R = k a1 - (k - 1) and
    a6 = k a6_A for A_k make every species' per-mass energy the same function
    of T, so T stays constant.  (The default rates react within a 1e-6 s step
    but leave Newton's decisions insensitive to rounding: with 1e4 times
    faster rates a 1-ulp change of the input changed the oracle's own
    iteration counts in a third of the cells.)"""
    nasa = np.stack([const_cp(a1, a6, 4.0), const_cp(2 * a1 - 1.0, 2 * a6, 3.0),
                     const_cp(3 * a1 - 2.0, 3 * a6, 2.5)])
    comps = {"A": {"H": 1}, "A2": {"H": 2}, "A3": {"H": 3}}
    return synth.make_mechanism("trimer", ["A", "A2", "A3"], comps, ["H"],
                                [(("A", "A"), ("A2",), 0), (("A2", "A"), ("A3",), 0),
                                 (("A", "A", "A"), ("A3",), 0)], nasa,
                                arr_A=[A2_cgs, A3_cgs, A3d_cgs], arr_beta=[0.0, 0.5, 0.0],
                                arr_Ea=[0.0, 1.0e4, 0.0])
