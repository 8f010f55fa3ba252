"""chem_advance_host_static (the allocation-free host-buffer step) gives the
same cells as chem_advance_host, the allocating entry point, on two calls in
a row, allocates no device memory per call, takes a call of exactly its
stated cell limit, and refuses requests larger than its static device array.

Kept in a file of its own that pytest collects last."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_1110_4903_gb300 import chem, synth
    return torch, oracle, chem, synth


def _inputs(oracle, synth, mech, n, seed):
    f = synth.uniform_field(mech.ns, n, 900.0, 2800.0, seed=seed)
    rho, e = oracle.OracleMech(mech).state_from_tpy(f.T, f.P, f.Y)
    return np.ascontiguousarray(rho), np.ascontiguousarray(e)


def _both(L, h, rho, e, dt):
    """Runs the allocating and the static entry point on copies of the same
    host inputs through the C ABI."""
    n = e.shape[0]
    outs = []
    for fn in ("chem_advance_host", "chem_advance_host_static"):
        r, ev = rho.copy(), e.copy()
        T = np.zeros(n)
        st = np.full(n, -1, np.int32)
        rc = getattr(L, fn)(h, n, r.shape[1], r.ctypes.data, ev.ctypes.data, float(dt),
                            T.ctypes.data, st.ctypes.data)
        assert rc == 0, L.chem_last_error_message().decode()
        outs.append((r, ev, T, st))
    return outs


@pytest.mark.parametrize("builder,dt,precision", [("h2_air_9sp", 1e-6, 0), ("hydrocarbon_36sp", 1e-6, 0),
                                                   ("hydrocarbon_36sp", 1e-6, 1)])
def test_static_matches_allocating_entry_point_twice(env, builder, dt, precision):
    # (the same kernel in the same launch shape on the same cells: the two
    # entry points agree bit for bit, FP64 and mixed alike)
    torch, oracle, chem, synth = env
    mech = getattr(synth, builder)()
    ch = chem.Chem(mech, precision=precision)
    sizes = (3000, 1700) if mech.ns > 9 else (20000, 7777)
    for call, n in enumerate(sizes):
        rho, e = _inputs(oracle, synth, mech, n, seed=100 + call)
        (ra, ea, Ta, sa), (rb, eb, Tb, sb) = _both(chem.lib(), ch.h, rho, e, dt)
        assert np.array_equal(sa, sb)
        assert (sa == 0).mean() > 0.999
        assert np.array_equal(rb, ra) and np.array_equal(eb, ea) and np.array_equal(Tb, Ta)
    ch.close()


def test_static_calls_allocate_no_device_memory(env):
    """Free device memory is the same before and after several static calls
    on a fresh handle (after one warm-up call, which looks up the array's
    device address), on both precisions, and a call at exactly the stated
    cell limit succeeds while one cell more is refused."""
    torch, oracle, chem, synth = env
    mech = synth.hydrocarbon_36sp()
    lib = chem.lib()
    cap = C.c_int64()
    assert lib.chem_static_scratch_bytes(C.byref(cap)) == 0
    limit = (cap.value - 256) // (mech.ns * 8 + 8 + 8 + 4)
    for precision in (0, 1):
        ch = chem.Chem(mech, precision=precision)
        rho, e = _inputs(oracle, synth, mech, 2000, seed=7)
        T = np.zeros(2000)
        st = np.zeros(2000, np.int32)

        def call(r, ev, n, Tb, sb):
            return lib.chem_advance_host_static(ch.h, n, r.shape[1], r.ctypes.data, ev.ctypes.data, 1e-6,
                                                Tb.ctypes.data, sb.ctypes.data)

        assert call(rho.copy(), e.copy(), 2000, T, st) == 0
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for k in range(4):
            assert call(rho.copy(), e.copy(), 2000, T, st) == 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        ch.close()
    ch = chem.Chem(mech, precision=1)
    rho, e = _inputs(oracle, synth, mech, limit + 1, seed=8)
    T = np.zeros(limit + 1)
    st = np.full(limit + 1, -1, np.int32)
    r, ev = rho.copy(), e.copy()
    rc = lib.chem_advance_host_static(ch.h, limit + 1, r.shape[1], r.ctypes.data, ev.ctypes.data, 1e-6,
                                      T.ctypes.data, st.ctypes.data)
    assert rc == -7 and np.array_equal(r, rho)
    rc = lib.chem_advance_host_static(ch.h, limit, r.shape[1], r.ctypes.data, ev.ctypes.data, 1e-6,
                                      T.ctypes.data, st.ctypes.data)
    assert rc == 0, lib.chem_last_error_message().decode()
    assert (st[:limit] == 0).mean() > 0.999 and (st[limit] == -1)
    ch.close()


def test_static_rejects_oversize_request(env):
    torch, oracle, chem, synth = env
    mech = synth.hydrocarbon_36sp()
    ch = chem.Chem(mech)
    cap = C.c_int64()
    assert chem.lib().chem_static_scratch_bytes(C.byref(cap)) == 0
    n = int(cap.value // (mech.ns * 8 + 20)) + 10
    rho = np.full((mech.ns, n), 1e-3)
    e = np.zeros(n)
    rc = chem.lib().chem_advance_host_static(ch.h, n, n, rho.ctypes.data, e.ctypes.data, 1e-6, None, None)
    assert rc == -7
    assert "split" in chem.lib().chem_last_error_message().decode()
    assert np.all(rho == 1e-3)        # nothing was touched
    ch.close()
