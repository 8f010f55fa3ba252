"""chem_advance_host_static (the allocation-free host-buffer step) gives the
same cells as chem_advance_host, the allocating entry point, on two calls in
a row, and refuses requests larger than its static device array.

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


@pytest.mark.parametrize("builder,dt", [("h2_air_9sp", 1e-6), ("hydrocarbon_36sp", 1e-6)])
def test_static_matches_allocating_entry_point_twice(env, builder, dt):
    torch, oracle, chem, synth = env
    mech = getattr(synth, builder)()
    ch = chem.Chem(mech)
    sizes = (3000, 1700) if mech.ns > 9 else (20000, 7777)
    for call, n in enumerate(sizes):
        rho, e = _inputs(oracle, synth, mech, n, seed=100 + call)
        (ra, ea, Ta, sa), (rb, eb, Tb, sb) = _both(chem.lib(), ch.h, rho, e, dt)
        assert np.array_equal(sa, sb)
        assert (sa == 0).mean() > 0.999
        floor = 1e-12 * rho.sum(0)
        rel = np.abs(rb - ra) / np.maximum(np.abs(ra), floor[None, :])
        assert rel.max() <= 1e-10
        assert np.abs(Tb - Ta).max() <= 1e-10 * Ta.max()
        assert np.abs(eb - ea).max() <= 1e-10 * (np.abs(ea).max() + 1e6 * rho.sum(0).max())
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
