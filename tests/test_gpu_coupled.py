"""The operator-split loop (Eq. 4) with the chemistry half on the GPU:
mass and U = e + sum rho_s e_f conserved over the domain, no failed cells."""
import pytest

pytestmark = pytest.mark.gpu


def test_coupled_demo_conserves():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1110_4903_gb300 import coupled_demo
    out = coupled_demo.run(cells=2048, steps=8)
    assert out["mass_drift"] < 1e-13 and out["energy_drift"] < 1e-12
    assert all(h["failed_cells"] == 0 for h in out["history"])
    assert out["history"][-1]["T_max"] > 1500.0
