"""ctypes binding of libchem (include/chem.h): argument marshalling only.

Every step of the chemistry path runs in the library's CUDA kernels; this
module converts PyTorch device tensors and numpy arrays to plain pointers.
It raises if the compiled library is missing -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchem.so")

FP64, MIXED = 0, 1
CELL_OK, CELL_NEWTON_FAILED, CELL_T_FAILED, CELL_BAD_INPUT, CELL_TOO_MANY_STEPS = range(5)
E_CODES = {0: "ok", -1: "INVALID_ARG", -2: "BAD_MECHANISM", -3: "OOM", -4: "OVER_BUDGET",
           -5: "CUDA", -6: "TIMEOUT", -7: "UNSUPPORTED", -8: "NOT_FOUND"}


class ChemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (E_CODES.get(code, "?"), code, msg))
        self.code = code


class MechDesc(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("n_reactions", C.c_int32), ("n_elements", C.c_int32),
                ("molar_mass", C.c_void_p), ("elem_comp", C.c_void_p), ("nasa7", C.c_void_p),
                ("t_mid", C.c_void_p), ("arr_A", C.c_void_p), ("arr_beta", C.c_void_p),
                ("arr_Ea", C.c_void_p), ("reac_sp", C.c_void_p), ("reac_nu", C.c_void_p),
                ("prod_sp", C.c_void_p), ("prod_nu", C.c_void_p), ("third_body", C.c_void_p),
                ("tb_eff", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("rtol", C.c_double), ("atol_rel", C.c_double),
                ("max_newton", C.c_int32), ("max_halvings", C.c_int32), ("max_attempts", C.c_int32),
                ("point_implicit", C.c_int32), ("div_check", C.c_int32),
                ("lanes_per_cell", C.c_int32), ("autotune", C.c_int32),
                ("hbm_budget_bytes", C.c_int64), ("max_newton_mixed", C.c_int32),
                ("conv_kappa", C.c_double), ("conv_kappa_mixed", C.c_double)]


class AdvanceArgs(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("ld", C.c_int64), ("rho_s", C.c_void_p), ("e", C.c_void_p),
                ("dt", C.c_double), ("T_in", C.c_void_p), ("T_out", C.c_void_p),
                ("status", C.c_void_p), ("newton_iters", C.c_void_p), ("substeps", C.c_void_p),
                ("failures", C.c_void_p), ("stream", C.c_void_p), ("precision", C.c_int32),
                ("lanes_per_cell", C.c_int32), ("schedule", C.c_void_p),
                ("substep_states", C.c_void_p)]


SCHEDULE_WORDS = 8   # CHEM_SCHEDULE_WORDS
SUBSTEP_STATES = 32  # CHEM_SUBSTEP_STATES


class ServerOptions(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_inflight", C.c_int32),
                ("queue_capacity", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("mech", C.c_void_p), ("n_cells", C.c_int64), ("ld", C.c_int64),
                ("rho_s", C.c_void_p), ("e", C.c_void_p), ("host", C.c_int32),
                ("precision", C.c_int32), ("dt", C.c_double), ("T_out", C.c_void_p),
                ("status", C.c_void_p), ("ready_event", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("state", C.c_int32), ("error", C.c_int32), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_done", C.c_double), ("dev_first_ns", C.c_uint64),
                ("dev_last_ns", C.c_uint64)]


class ServerStats(C.Structure):
    _fields_ = [("queued", C.c_int64), ("running", C.c_int64), ("completed", C.c_int64),
                ("failed", C.c_int64), ("bytes_in_use", C.c_int64), ("budget_bytes", C.c_int64),
                ("launches", C.c_int64), ("kernel_instances", C.c_int64), ("queue_errors", C.c_int64)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED = range(5)
LU_GLOBAL, LU_ONCHIP, LU_GLOBAL_FMA = 0, 1, 2

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libchem.so is not built (run __graft_entry__.build()); "
                              "there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        p, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "chem_default_options": [p],
            "chem_create": [p, p, p],
            "chem_destroy": [p],
            "chem_advance": [p, i64, p, p, d, p],
            "chem_advance_ex": [p, p],
            "chem_advance_segmented": [p, p, i64],
            "chem_advance_host": [p, i64, i64, p, p, d, p, p],
            "chem_advance_host_static": [p, i64, i64, p, p, d, p, p],
            "chem_static_scratch_bytes": [p],
            "chem_state_from_tpy": [p, i64, i64, p, p, p, p, p, p],
            "chem_temperature": [p, i64, i64, p, p, p, p, p],
            "chem_get_lanes_per_cell": [p, i32, p],
            "chem_formation_energies": [p, p],
            "chem_launch_count": [p, p],
            "chem_autotune": [p, i32, i64, i64, p, p, d, p, p, p, p],
            "chem_graph_create": [p, p, p],
            "chem_graph_launch": [p, p],
            "chem_graph_destroy": [p],
            "chem_server_default_options": [p],
            "chem_server_create": [p, p],
            "chem_server_destroy": [p],
            "chem_submit": [p, p, p],
            "chem_poll": [p, C.c_uint64, p],
            "chem_wait": [p, C.c_uint64, i64, p],
            "chem_cancel": [p, C.c_uint64],
            "chem_release": [p, C.c_uint64],
            "chem_server_stats": [p, p],
            "chem_batched_solve": [i32, i32, i64, p, p, p, p, p],
            "chem_selftest_math": [i64, p, p, p, p, p, p],
            "chem_selftest_log": [i64, p, p, p, p],
            "chem_selftest_scaled_exp": [i64, p, p, p, p, p, p, p],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.chem_strerror.argtypes = [C.c_int]
        L.chem_strerror.restype = C.c_char_p
        L.chem_last_error_message.argtypes = []
        L.chem_last_error_message.restype = C.c_char_p
        _lib = L
    return _lib


def check(rc):
    if rc != 0:
        raise ChemError(rc, lib().chem_last_error_message().decode())
    return rc


def default_options(**kw) -> Options:
    o = Options()
    check(lib().chem_default_options(C.byref(o)))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(t):
    """Device pointer of a torch tensor, or None."""
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class StepGraph:
    """A captured chemistry step (chem_graph_*)."""

    def __init__(self, g):
        self.g = g

    def launch(self, stream=None):
        check(lib().chem_graph_launch(self.g, _stream_ptr(stream)))

    def close(self):
        if self.g:
            check(lib().chem_graph_destroy(self.g))
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Chem:
    """One mechanism on the current CUDA device (chem_create / chem_destroy)."""

    def __init__(self, mech, **opts):
        self.mech = mech
        self._keep = [np.ascontiguousarray(a) for a in (
            mech.molar_mass.astype(np.float64), mech.elem_comp.astype(np.int32),
            mech.nasa7.astype(np.float64), mech.t_range[:, 1].astype(np.float64),
            mech.arr_A.astype(np.float64), mech.arr_beta.astype(np.float64),
            mech.arr_Ea.astype(np.float64), mech.reac_sp.astype(np.int32),
            mech.reac_nu.astype(np.int32), mech.prod_sp.astype(np.int32),
            mech.prod_nu.astype(np.int32), mech.third_body.astype(np.int32),
            mech.tb_eff.astype(np.float64))]
        k = self._keep
        self.desc = MechDesc(mech.ns, mech.nr, mech.ne, *[a.ctypes.data for a in k])
        self.opts = default_options(**opts)
        h = C.c_void_p()
        check(lib().chem_create(C.byref(self.desc), C.byref(self.opts), C.byref(h)))
        self.h = h
        self.ns = mech.ns

    def close(self):
        if getattr(self, "h", None):
            check(lib().chem_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def advance(self, rho, e, dt, *, n_cells=None, T_in=None, T_out=None, status=None,
                newton_iters=None, substeps=None, failures=None, precision=-1, lanes=0,
                stream=None, schedule=None, substep_states=None):
        """In-place step of device tensors rho [ns, ld] and e [>= n] (float64).
        schedule: optional int32 device tensor [n, SCHEDULE_WORDS] that receives
        each cell's accepted-attempt bits; substep_states: optional float64
        device tensor [n, SUBSTEP_STATES, ns+1] that receives its states after
        accepted substeps."""
        n = int(e.shape[0]) if n_cells is None else int(n_cells)
        a = AdvanceArgs(n, int(rho.stride(0)), rho.data_ptr(), e.data_ptr(), float(dt),
                        _ptr(T_in), _ptr(T_out), _ptr(status), _ptr(newton_iters), _ptr(substeps),
                        _ptr(failures), _stream_ptr(stream), int(precision), int(lanes),
                        _ptr(schedule), _ptr(substep_states))
        check(lib().chem_advance_ex(self.h, C.byref(a)))

    def advance_segmented(self, rho, e, dt, segment_cells, *, n_cells=None, T_in=None, T_out=None,
                          status=None, newton_iters=None, substeps=None, failures=None,
                          precision=-1, stream=None, schedule=None, substep_states=None):
        """chem_advance_segmented: the same step in launches of at most
        segment_cells cells."""
        n = int(e.shape[0]) if n_cells is None else int(n_cells)
        a = AdvanceArgs(n, int(rho.stride(0)), rho.data_ptr(), e.data_ptr(), float(dt),
                        _ptr(T_in), _ptr(T_out), _ptr(status), _ptr(newton_iters), _ptr(substeps),
                        _ptr(failures), _stream_ptr(stream), int(precision), 0, _ptr(schedule),
                        _ptr(substep_states))
        check(lib().chem_advance_segmented(self.h, C.byref(a), int(segment_cells)))

    def advance_simple(self, n_cells, rho, e, dt, stream=None):
        check(lib().chem_advance(self.h, int(n_cells), rho.data_ptr(), e.data_ptr(), float(dt),
                                 _stream_ptr(stream)))

    def advance_host(self, rho, e, dt, T_out=None, status=None):
        """Step of HOST numpy arrays rho [ns, ld] and e [n] (synchronous)."""
        n = e.shape[0]
        check(lib().chem_advance_host(self.h, n, rho.shape[1], rho.ctypes.data, e.ctypes.data,
                                      float(dt), None if T_out is None else T_out.ctypes.data,
                                      None if status is None else status.ctypes.data))

    def advance_host_static(self, rho, e, dt, T_out=None, status=None):
        """Like advance_host, but staged in the library's fixed device array:
        no device allocation per call; raises ChemError(UNSUPPORTED) when the
        request does not fit."""
        n = e.shape[0]
        check(lib().chem_advance_host_static(self.h, n, rho.shape[1], rho.ctypes.data, e.ctypes.data,
                                             float(dt), None if T_out is None else T_out.ctypes.data,
                                             None if status is None else status.ctypes.data))

    def state_from_tpy(self, T, P, Y, rho, e, stream=None):
        n = int(T.shape[0])
        check(lib().chem_state_from_tpy(self.h, n, int(Y.stride(0)), _ptr(T), _ptr(P), _ptr(Y),
                                        _ptr(rho), _ptr(e), _stream_ptr(stream)))

    def temperature(self, rho, e, T_out, T_guess=None, stream=None):
        n = int(e.shape[0])
        check(lib().chem_temperature(self.h, n, int(rho.stride(0)), _ptr(rho), _ptr(e),
                                     _ptr(T_guess), _ptr(T_out), _stream_ptr(stream)))

    def autotune(self, rho, e, dt, *, n_cells=None, T_in=None, precision=FP64, stream=None):
        """Times the launch shapes on a sample of these cells (not modified)
        and keeps the fastest; returns (lanes_per_cell, warps_per_block)."""
        n = int(e.shape[0]) if n_cells is None else int(n_cells)
        lanes, wpb = C.c_int32(), C.c_int32()
        check(lib().chem_autotune(self.h, int(precision), n, int(rho.stride(0)), rho.data_ptr(),
                                  e.data_ptr(), float(dt), _ptr(T_in), _stream_ptr(stream),
                                  C.byref(lanes), C.byref(wpb)))
        return lanes.value, wpb.value

    def graph(self, rho, e, dt, *, n_cells=None, T_in=None, T_out=None, status=None,
              newton_iters=None, substeps=None, failures=None, precision=-1, lanes=0):
        """Captures one step of these buffers as a CUDA graph (StepGraph)."""
        n = int(e.shape[0]) if n_cells is None else int(n_cells)
        a = AdvanceArgs(n, int(rho.stride(0)), rho.data_ptr(), e.data_ptr(), float(dt),
                        _ptr(T_in), _ptr(T_out), _ptr(status), _ptr(newton_iters), _ptr(substeps),
                        _ptr(failures), None, int(precision), int(lanes))
        g = C.c_void_p()
        check(lib().chem_graph_create(self.h, C.byref(a), C.byref(g)))
        return StepGraph(g)

    def formation_energies(self):
        """e_f,s = e_s(298.15 K), J/kg, as the library uses them."""
        out = np.zeros(self.ns)
        check(lib().chem_formation_energies(self.h, out.ctypes.data))
        return out

    def lanes(self, precision=FP64):
        v = C.c_int32()
        check(lib().chem_get_lanes_per_cell(self.h, precision, C.byref(v)))
        return v.value

    def launch_count(self):
        v = C.c_int64()
        check(lib().chem_launch_count(self.h, C.byref(v)))
        return v.value


class Server:
    """Request server (chem_server_*): continuous batching of chemistry steps."""

    def __init__(self, budget_bytes=0, max_inflight=64, queue_capacity=100000):
        o = ServerOptions()
        check(lib().chem_server_default_options(C.byref(o)))
        o.hbm_budget_bytes = int(budget_bytes)
        o.max_inflight = int(max_inflight)
        o.queue_capacity = int(queue_capacity)
        s = C.c_void_p()
        check(lib().chem_server_create(C.byref(o), C.byref(s)))
        self.s = s
        self._events = {}

    def submit(self, ch, rho, e, dt, *, n_cells=None, host=False, precision=-1, T_out=None,
               status=None, stream=None):
        """rho/e: torch device tensors (host=False) or numpy host arrays
        (host=True).  Device requests wait for an event recorded now on
        `stream` (default: the current stream), so work queued there before
        the submit -- e.g. the writes that produced the state -- is finished
        before the request reads its buffers."""
        ev = None
        if host:
            n = e.shape[0] if n_cells is None else n_cells
            r = Request(ch.h, n, rho.shape[1], rho.ctypes.data, e.ctypes.data, 1, int(precision),
                        float(dt), None if T_out is None else T_out.ctypes.data,
                        None if status is None else status.ctypes.data, None)
        else:
            import torch
            ev = torch.cuda.Event()
            ev.record(stream if stream is not None else torch.cuda.current_stream())
            n = int(e.shape[0]) if n_cells is None else int(n_cells)
            r = Request(ch.h, n, int(rho.stride(0)), rho.data_ptr(), e.data_ptr(), 0, int(precision),
                        float(dt), _ptr(T_out), _ptr(status), C.c_void_p(ev.cuda_event))
        t = C.c_uint64()
        check(lib().chem_submit(self.s, C.byref(r), C.byref(t)))
        if ev is not None:
            self._events[t.value] = ev      # kept alive until the request is finished
        return t.value

    def _finished(self, ticket, r):
        if r.state in (REQ_DONE, REQ_FAILED, REQ_CANCELLED):
            self._events.pop(ticket, None)
        return r

    def poll(self, ticket):
        r = Result()
        check(lib().chem_poll(self.s, C.c_uint64(ticket), C.byref(r)))
        return self._finished(ticket, r)

    def wait(self, ticket, timeout_us=-1):
        r = Result()
        rc = lib().chem_wait(self.s, C.c_uint64(ticket), int(timeout_us), C.byref(r))
        if rc == -6:
            return None
        check(rc)
        return self._finished(ticket, r)

    def cancel(self, ticket):
        check(lib().chem_cancel(self.s, C.c_uint64(ticket)))

    def release(self, ticket):
        check(lib().chem_release(self.s, C.c_uint64(ticket)))

    def stats(self):
        st = ServerStats()
        check(lib().chem_server_stats(self.s, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "s", None):
            check(lib().chem_server_destroy(self.s))
            self.s = None
            self._events.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batched_solve(method, A, b, pivots=None, info=None, stream=None):
    """In-place batched solve of device tensors (chem_batched_solve):
    LU_GLOBAL and LU_GLOBAL_FMA: A [n, n, n_sys], b [n, n_sys]; LU_ONCHIP:
    A [n_sys, n, n], b [n_sys, n]."""
    if method in (LU_GLOBAL, LU_GLOBAL_FMA):
        n, n_sys = int(A.shape[0]), int(A.shape[2])
    else:
        n_sys, n = int(A.shape[0]), int(A.shape[1])
    check(lib().chem_batched_solve(int(method), n, n_sys, A.data_ptr(), b.data_ptr(), _ptr(pivots),
                                   _ptr(info), _stream_ptr(stream)))
