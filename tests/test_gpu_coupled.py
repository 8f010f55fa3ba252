"""The operator-split loop (Eq. 4) with the chemistry half on the GPU: mass
and U = e + sum rho_s e_f conserved over the domain, no failed cells, and the
chemistry half against the oracle -- the whole FP64 loop against the same
loop with the oracle for chemistry, and every mixed-precision chemistry half
against the oracle's replay of its own substep schedule."""
import os
import types

import numpy as np
import pytest

import parity as P

pytestmark = pytest.mark.gpu
THREADS = min(16, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return t


def test_coupled_demo_conserves(torch):
    from paper_1110_4903_gb300 import coupled_demo
    out = coupled_demo.run(cells=2048, steps=8)
    assert out["mass_drift"] < 1e-13 and out["energy_drift"] < 1e-12
    assert all(h["failed_cells"] == 0 for h in out["history"])
    assert out["history"][-1]["T_max"] > 1500.0


def test_coupled_fp64_loop_against_oracle_loop(torch):
    """The FP64 loop (GPU chemistry, captured graph) against the loop with the
    oracle's chemistry and the same advection in numpy (identical IEEE
    operations): the advection is a convex combination, so the per-step
    chemistry differences (at most a few 1e-12) do not grow beyond the sum
    over steps; 1e-10 over 8 steps."""
    from paper_1110_4903_gb300 import coupled_demo, synth
    out = coupled_demo.run(cells=2048, steps=8, precision=0, dx=1e-3)   # dt = 1 us
    mech = synth.h2_air_9sp()
    rho, e = out["rho0"].copy(), out["e0"].copy()
    for _ in range(8):
        coupled_demo.advect(rho, e, out["c"], lambda a, s, ax: np.roll(a, s, axis=ax))
        # (the demo's graph steps start every temperature recovery at 1500 K)
        rho, e, oo = P.oracle_reference(mech, rho, e, out["dt"], None, threads=THREADS, schedule=False)
        assert (oo["status"] == 0).all()
    T = oo["T"]
    rel = P.rel_species(out["rho"], rho, out["rho0"].sum(0))
    assert rel.max() <= 1e-10, rel.max()
    np.testing.assert_allclose(out["T"], T, rtol=1e-10)
    scale = np.abs(e) + np.abs(out["rho0"]).sum(0) * 1e6
    assert (np.abs(out["e"] - e) / scale).max() <= 1e-10


def test_coupled_mixed_chemistry_halves_against_replay(torch):
    """Each mixed-precision chemistry half of the loop against the oracle
    integrating the same post-advection state along the GPU's own substep
    schedule (1e-6, the mixed path's bar)."""
    from paper_1110_4903_gb300 import chem, coupled_demo, synth
    mech = synth.h2_air_9sp()
    cells, cfl, dx, u = 2048, 0.5, 1e-3, 500.0
    dt, c = cfl * dx / u, cfl
    T0, Pp, Y = coupled_demo.initial_field(mech, cells)
    rho, e = P.initial_state(mech, types.SimpleNamespace(T=T0, P=Pp, Y=Y))
    ch = chem.Chem(mech, precision=chem.MIXED)
    T_in = T0
    for step in range(6):
        coupled_demo.advect(rho, e, c, lambda a, s, ax: np.roll(a, s, axis=ax))
        rg, eg, og = P.gpu_run(torch, ch, rho, e, dt, T_in=T_in)
        assert (og["status"] == 0).all()
        st = P.replay_check(mech, rho, e, dt, T_in, rg, eg, og, P.TOL_MIXED, floor=P.FLOOR_MIXED,
                            threads=THREADS)
        assert st["replayed"] == cells
        rho, e, T_in = rg, eg, og["T"]
    ch.close()
