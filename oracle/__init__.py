"""ctypes binding of the plain FP64 CPU oracle (chem_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it.  The CUDA library never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "chem_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

R = 8.314462618
PA = 101325.0
TREF = 298.15

OK, NEWTON_FAILED, T_FAILED, BAD_INPUT, TOO_MANY_STEPS = 0, 1, 2, 3, 4
REPLAY_NOT_CONVERGED, REPLAY_MISMATCH = 5, 6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no FMA contraction, portable)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "chem_oracle.h"))):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class _Mech(C.Structure):
    _fields_ = [("ns", C.c_int), ("nr", C.c_int), ("ne", C.c_int),
                ("molar_mass", C.c_void_p), ("elem_comp", C.c_void_p),
                ("nasa7", C.c_void_p), ("t_mid", C.c_void_p),
                ("arr_A", C.c_void_p), ("arr_beta", C.c_void_p), ("arr_Ea", C.c_void_p),
                ("reac_sp", C.c_void_p), ("reac_nu", C.c_void_p),
                ("prod_sp", C.c_void_p), ("prod_nu", C.c_void_p),
                ("third_body", C.c_void_p), ("tb_eff", C.c_void_p)]


class Opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol_rel", C.c_double),
                ("max_newton", C.c_int), ("max_halvings", C.c_int),
                ("max_attempts", C.c_int), ("point_implicit", C.c_int),
                ("div_check", C.c_int), ("conv_kappa", C.c_double)]


class _CellResult(C.Structure):
    _fields_ = [("status", C.c_int), ("newton_iters", C.c_int), ("substeps", C.c_int),
                ("failures", C.c_int), ("T", C.c_double)]


_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            d, i, p = C.c_double, C.c_int, C.c_void_p
            L.om_species_e.restype = d
            L.om_species_e.argtypes = [p, i, d]
            L.om_species_cv.restype = d
            L.om_species_cv.argtypes = [p, i, d]
            L.om_species_ef.restype = d
            L.om_species_ef.argtypes = [p, i]
            L.om_species_esens.restype = d
            L.om_species_esens.argtypes = [p, i, d]
            L.om_thermo.argtypes = [p, i, d, p, p, p]
            L.om_recover_T.restype = i
            L.om_recover_T.argtypes = [p, p, d, d, p, p]
            L.om_rate_constants.argtypes = [p, d, p, p, p]
            L.om_progress.argtypes = [p, d, p, p]
            L.om_source.argtypes = [p, p, d, p]
            L.om_jacobian.argtypes = [p, p, d, p]
            L.om_lu_factor.restype = i
            L.om_lu_factor.argtypes = [i, p, p]
            L.om_lu_solve.argtypes = [i, p, p, p]
            L.om_default_opts.argtypes = [p]
            L.om_advance_cell.argtypes = [p, p, p, p, d, d, p]
            L.om_advance_batch.argtypes = [p, p, C.c_long, C.c_long, p, p, d, p, p, p, p, p, p]
            L.om_advance_batch_sched.argtypes = [p, p, C.c_long, C.c_long, p, p, d, p, p, p, p, p,
                                                 p, p, i, p, i]
            L.om_advance_cell_sched.argtypes = [p, p, p, p, d, d, p, i, p, i, p]
            L.om_advance_cell_replay.argtypes = [p, p, p, p, d, d, p, i, p, i, p]
            L.om_advance_batch_replay.argtypes = [p, p, C.c_long, C.c_long, p, p, d, p, p, i, p,
                                                  p, i, p, p, p]
            L.om_state_from_tpy.argtypes = [p, C.c_long, C.c_long, p, p, p, p, p]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data if a is not None else None


class OracleMech:
    """Holds contiguous copies of a synth.Mechanism and the C struct over them."""

    def __init__(self, mech):
        self.mech = mech
        self._keep = dict(
            molar_mass=np.ascontiguousarray(mech.molar_mass, np.float64),
            elem_comp=np.ascontiguousarray(mech.elem_comp, np.int32),
            nasa7=np.ascontiguousarray(mech.nasa7, np.float64),
            t_mid=np.ascontiguousarray(mech.t_range[:, 1], np.float64),
            arr_A=np.ascontiguousarray(mech.arr_A, np.float64),
            arr_beta=np.ascontiguousarray(mech.arr_beta, np.float64),
            arr_Ea=np.ascontiguousarray(mech.arr_Ea, np.float64),
            reac_sp=np.ascontiguousarray(mech.reac_sp, np.int32),
            reac_nu=np.ascontiguousarray(mech.reac_nu, np.int32),
            prod_sp=np.ascontiguousarray(mech.prod_sp, np.int32),
            prod_nu=np.ascontiguousarray(mech.prod_nu, np.int32),
            third_body=np.ascontiguousarray(mech.third_body, np.int32),
            tb_eff=np.ascontiguousarray(mech.tb_eff, np.float64),
        )
        k = self._keep
        self.c = _Mech(mech.ns, mech.nr, mech.ne, *[_ptr(k[f]) for f in (
            "molar_mass", "elem_comp", "nasa7", "t_mid", "arr_A", "arr_beta", "arr_Ea",
            "reac_sp", "reac_nu", "prod_sp", "prod_nu", "third_body", "tb_eff")])
        self.ns, self.nr = mech.ns, mech.nr
        self.n = mech.ns + 1

    @property
    def ref(self):
        return C.byref(self.c)

    # -- thermo ----------------------------------------------------------------
    def thermo(self, s, T):
        cp, h, sr = C.c_double(), C.c_double(), C.c_double()
        lib().om_thermo(self.ref, s, T, C.byref(cp), C.byref(h), C.byref(sr))
        return cp.value, h.value, sr.value

    def species_e(self, s, T):
        return lib().om_species_e(self.ref, s, T)

    def species_cv(self, s, T):
        return lib().om_species_cv(self.ref, s, T)

    def species_ef(self, s):
        return lib().om_species_ef(self.ref, s)

    def species_esens(self, s, T):
        return lib().om_species_esens(self.ref, s, T)

    def ef(self):
        return np.array([self.species_ef(s) for s in range(self.ns)])

    def recover_T(self, rho, e, T_guess=1500.0):
        rho = np.ascontiguousarray(rho, np.float64)
        T, it = C.c_double(), C.c_int()
        rc = lib().om_recover_T(self.ref, _ptr(rho), float(e), float(T_guess), C.byref(T), C.byref(it))
        return rc, T.value, it.value

    # -- rates -----------------------------------------------------------------
    def rate_constants(self, T):
        kf, Kc, kb = (np.zeros(self.nr) for _ in range(3))
        lib().om_rate_constants(self.ref, float(T), _ptr(kf), _ptr(Kc), _ptr(kb))
        return kf, Kc, kb

    def progress(self, T, rho):
        rho = np.ascontiguousarray(rho, np.float64)
        Q = np.zeros(self.nr)
        lib().om_progress(self.ref, float(T), _ptr(rho), _ptr(Q))
        return Q

    def source(self, rho, T):
        rho = np.ascontiguousarray(rho, np.float64)
        w = np.zeros(self.n)
        lib().om_source(self.ref, _ptr(rho), float(T), _ptr(w))
        return w

    def jacobian(self, rho, T):
        rho = np.ascontiguousarray(rho, np.float64)
        J = np.zeros((self.n, self.n))
        lib().om_jacobian(self.ref, _ptr(rho), float(T), _ptr(J))
        return J

    # -- integration -----------------------------------------------------------
    def advance_cell(self, rho, e, dt, T_guess=1500.0, opts=None):
        o = opts if opts is not None else default_opts()
        r = np.ascontiguousarray(rho, np.float64).copy()
        ev = C.c_double(float(e))
        res = _CellResult()
        lib().om_advance_cell(self.ref, C.byref(o), _ptr(r), C.byref(ev), float(dt),
                              float(T_guess), C.byref(res))
        return r, ev.value, dict(status=res.status, newton_iters=res.newton_iters,
                                 substeps=res.substeps, failures=res.failures, T=res.T)

    def advance_cell_sched(self, rho, e, dt, T_guess=1500.0, opts=None, words=8):
        """advance_cell that also returns the accepted-attempt bits (uint32
        words: bit a set when substep attempt a was accepted)."""
        o = opts if opts is not None else default_opts()
        r = np.ascontiguousarray(rho, np.float64).copy()
        ev = C.c_double(float(e))
        sched = np.zeros(words, np.uint32)
        res = _CellResult()
        lib().om_advance_cell_sched(self.ref, C.byref(o), _ptr(r), C.byref(ev), float(dt),
                                    float(T_guess), _ptr(sched), words, None, 0, C.byref(res))
        return r, ev.value, sched, dict(status=res.status, newton_iters=res.newton_iters,
                                        substeps=res.substeps, failures=res.failures, T=res.T)

    def advance_cell_replay(self, rho, e, dt, accepted, n_attempts, T_guess=1500.0, opts=None,
                            guides=None):
        """One cell along the given schedule (om_advance_cell_replay);
        guides: optional [k, ns+1] states after the other integrator's
        accepted substeps, Newton's starting points."""
        o = opts if opts is not None else replay_opts()
        r = np.ascontiguousarray(rho, np.float64).copy()
        ev = C.c_double(float(e))
        acc = np.ascontiguousarray(accepted, np.uint32)
        g = None if guides is None else np.ascontiguousarray(guides, np.float64)
        res = _CellResult()
        lib().om_advance_cell_replay(self.ref, C.byref(o), _ptr(r), C.byref(ev), float(dt),
                                     float(T_guess), _ptr(acc), int(n_attempts), _ptr(g),
                                     0 if g is None else g.shape[0], C.byref(res))
        return r, ev.value, dict(status=res.status, newton_iters=res.newton_iters,
                                 substeps=res.substeps, failures=res.failures, T=res.T)

    def advance_batch_replay(self, rho, e, dt, accepted, n_attempts, T_in=None, opts=None,
                             threads=1, guides=None):
        """The replay over a batch: accepted [n, words] uint32, n_attempts [n],
        guides optional [n, k, ns+1].  Returns new rho, e and dict(T, status,
        newton_iters)."""
        o = opts if opts is not None else replay_opts()
        rho = np.ascontiguousarray(rho, np.float64).copy()
        e = np.ascontiguousarray(e, np.float64).copy()
        n = e.shape[0]
        ld = rho.shape[1]
        acc = np.ascontiguousarray(accepted, np.uint32)
        words = acc.shape[1]
        na = np.ascontiguousarray(n_attempts, np.int32)
        g = None if guides is None else np.ascontiguousarray(guides, np.float64)
        ng = 0 if g is None else g.shape[1]
        T_out = np.zeros(n)
        status = np.zeros(n, np.int32)
        iters = np.zeros(n, np.int32)
        T_in = None if T_in is None else np.ascontiguousarray(T_in, np.float64)

        def run(a, b):
            off8, off4 = a * 8, a * 4
            lib().om_advance_batch_replay(self.ref, C.byref(o), b - a, ld,
                                          rho.ctypes.data + off8, e.ctypes.data + off8, float(dt),
                                          None if T_in is None else T_in.ctypes.data + off8,
                                          acc.ctypes.data + a * words * 4, words,
                                          na.ctypes.data + off4,
                                          None if g is None else g.ctypes.data + a * ng * self.n * 8,
                                          ng, T_out.ctypes.data + off8,
                                          status.ctypes.data + off4, iters.ctypes.data + off4)

        if threads <= 1 or n < 2 * threads:
            run(0, n)
        else:
            chunk = max(1, (n + 4 * threads - 1) // (4 * threads))
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(lambda a: run(a, min(n, a + chunk)), range(0, n, chunk)))
        return rho, e, dict(T=T_out, status=status, newton_iters=iters)

    def advance_batch(self, rho, e, dt, T_in=None, opts=None, threads=1, schedule=False, words=8,
                      states_cap=0):
        """rho [ns, n] and e [n] float64 (copied); returns new arrays and the
        per-cell outputs.  threads > 1 splits the cells over host threads.
        schedule=True adds each cell's accepted-attempt bits ([n, words]
        uint32) to the outputs; states_cap > 0 adds its states after the
        first states_cap accepted substeps ([n, states_cap, ns+1])."""
        o = opts if opts is not None else default_opts()
        rho = np.ascontiguousarray(rho, np.float64).copy()
        e = np.ascontiguousarray(e, np.float64).copy()
        n = e.shape[0]
        ld = rho.shape[1]
        T_out = np.zeros(n)
        status = np.zeros(n, np.int32)
        iters = np.zeros(n, np.int32)
        subs = np.zeros(n, np.int32)
        fails = np.zeros(n, np.int32)
        sched = np.zeros((n, words), np.uint32) if schedule else None
        states = np.zeros((n, states_cap, self.n)) if states_cap > 0 else None
        T_in = None if T_in is None else np.ascontiguousarray(T_in, np.float64)

        def run(a, b):
            off8 = a * 8
            off4 = a * 4
            lib().om_advance_batch_sched(self.ref, C.byref(o), b - a, ld,
                                         rho.ctypes.data + off8, e.ctypes.data + off8, float(dt),
                                         None if T_in is None else T_in.ctypes.data + off8,
                                         T_out.ctypes.data + off8, status.ctypes.data + off4,
                                         iters.ctypes.data + off4, subs.ctypes.data + off4,
                                         fails.ctypes.data + off4,
                                         None if sched is None else sched.ctypes.data + a * words * 4,
                                         words if schedule else 0,
                                         None if states is None else
                                         states.ctypes.data + a * states_cap * self.n * 8,
                                         states_cap)

        if threads <= 1 or n < 2 * threads:
            run(0, n)
        else:
            chunk = max(1, (n + 4 * threads - 1) // (4 * threads))
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(lambda a: run(a, min(n, a + chunk)), range(0, n, chunk)))
        out = dict(T=T_out, status=status, newton_iters=iters, substeps=subs, failures=fails)
        if schedule:
            out["schedule"] = sched
        if states is not None:
            out["states"] = states
        return rho, e, out

    def state_from_tpy(self, T, P, Y):
        T = np.ascontiguousarray(T, np.float64)
        P = np.ascontiguousarray(P, np.float64)
        Y = np.ascontiguousarray(Y, np.float64)
        n = T.shape[0]
        rho = np.zeros_like(Y)
        e = np.zeros(n)
        lib().om_state_from_tpy(self.ref, n, Y.shape[1], _ptr(T), _ptr(P), _ptr(Y),
                                _ptr(rho), _ptr(e))
        return rho, e


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().om_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def replay_opts(**kw) -> Opts:
    """Options of a replay: every accepted attempt's backward-Euler system is
    solved to the norm test alone (no contraction-rate stop, no divergence
    check) with up to 50 Newton iterations."""
    o = default_opts(conv_kappa=0.0, div_check=0, max_newton=50)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def lu_factor(A):
    A = np.ascontiguousarray(A, np.float64).copy()
    n = A.shape[0]
    piv = np.zeros(n, np.int32)
    rc = lib().om_lu_factor(n, _ptr(A), _ptr(piv))
    return rc, A, piv


def lu_solve(LU, piv, b):
    b = np.ascontiguousarray(b, np.float64).copy()
    lib().om_lu_solve(LU.shape[0], _ptr(np.ascontiguousarray(LU)), _ptr(np.ascontiguousarray(piv, np.int32)), _ptr(b))
    return b
