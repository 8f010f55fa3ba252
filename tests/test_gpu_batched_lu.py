"""Batched dense solves (the kinetics-only experiment of Sec. 5.2) against
the oracle's elimination: pivots and LU factors bit-identical, solutions
equal to the oracle's (bit for bit on the global kernel, to rounding on the
on-chip one), for sizes up to 200."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1110_4903_gb300 import chem
    return torch, chem


def _systems(n, n_sys, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n_sys, n, n)) + 0.5 * np.sqrt(n) * np.eye(n)[None]
    b = rng.standard_normal((n_sys, n))
    return A, b


@pytest.mark.parametrize("n,n_sys", [(1, 7), (10, 1000), (37, 333), (64, 100), (100, 40), (150, 9),
                                     (200, 5), (10, 200000), (25, 80000)])
@pytest.mark.parametrize("method", ["global", "onchip"])
def test_bitwise_against_oracle(env, n, n_sys, method):
    torch, chem = env
    if method == "onchip" and n * (n + 1) * 8 > 227 * 1024:
        pytest.skip("does not fit on chip")
    A, b = _systems(n, n_sys, seed=n)
    dev = torch.device("cuda")
    piv = torch.zeros((n_sys, n), dtype=torch.int32, device=dev)
    info = torch.full((n_sys,), -1, dtype=torch.int32, device=dev)
    if method == "global":
        Ad = torch.tensor(np.ascontiguousarray(A.transpose(1, 2, 0)), device=dev)
        bd = torch.tensor(np.ascontiguousarray(b.T), device=dev)
        chem.batched_solve(chem.LU_GLOBAL, Ad, bd, piv, info)
        LU = Ad.cpu().numpy().transpose(2, 0, 1)
        x = bd.cpu().numpy().T
    else:
        Ad = torch.tensor(A, device=dev)
        bd = torch.tensor(b, device=dev)
        chem.batched_solve(chem.LU_ONCHIP, Ad, bd, piv, info)
        LU = Ad.cpu().numpy()
        x = bd.cpu().numpy()
    torch.cuda.synchronize()
    piv = piv.cpu().numpy()
    assert (info.cpu().numpy() == 0).all()
    for k in range(0, n_sys, max(1, n_sys // 25)):
        rc, LUo, pivo = oracle.lu_factor(A[k])
        assert rc == 0
        assert np.array_equal(piv[k], pivo)
        assert np.array_equal(LU[k], LUo)                  # bit for bit
        xo = oracle.lu_solve(LUo, pivo, b[k])
        if method == "global":
            assert np.array_equal(x[k], xo)
        else:   # column-ordered back substitution: equal to rounding
            assert np.abs(x[k] - xo).max() <= 1e-13 * n * np.abs(xo).max()


@pytest.mark.parametrize("n,n_sys", [(1, 7), (10, 1000), (37, 333), (100, 40), (200, 5), (10, 200000),
                                     (25, 80000)])
def test_contracted_against_oracle(env, n, n_sys):
    """The contracted global elimination (reciprocal multipliers, FMA
    updates): same pivots as the oracle, factors and x equal to rounding."""
    torch, chem = env
    A, b = _systems(n, n_sys, seed=n + 1)
    dev = torch.device("cuda")
    piv = torch.zeros((n_sys, n), dtype=torch.int32, device=dev)
    info = torch.full((n_sys,), -1, dtype=torch.int32, device=dev)
    Ad = torch.tensor(np.ascontiguousarray(A.transpose(1, 2, 0)), device=dev)
    bd = torch.tensor(np.ascontiguousarray(b.T), device=dev)
    chem.batched_solve(chem.LU_GLOBAL_FMA, Ad, bd, piv, info)
    torch.cuda.synchronize()
    LU = Ad.cpu().numpy().transpose(2, 0, 1)
    x = bd.cpu().numpy().T
    piv = piv.cpu().numpy()
    assert (info.cpu().numpy() == 0).all()
    eps = np.finfo(np.float64).eps
    for k in range(0, n_sys, max(1, n_sys // 25)):
        rc, LUo, pivo = oracle.lu_factor(A[k])
        assert rc == 0 and np.array_equal(piv[k], pivo)
        assert np.abs(LU[k] - LUo).max() <= 8 * n * eps * np.abs(LUo).max()
        xo = oracle.lu_solve(LUo, pivo, b[k])
        assert np.abs(x[k] - xo).max() <= 1e-13 * n * np.abs(xo).max()


@pytest.mark.parametrize("n_sys", [5, 100000])
@pytest.mark.parametrize("method", ["global", "global_fma"])
def test_nan_and_singular_pivots_as_the_oracle(env, n_sys, method):
    """Pivot choice around NaN and zero columns as in the oracle's search
    (start from |a_jj|, take a row only if strictly larger): a NaN diagonal
    stays the pivot and its column is singular; a NaN below the diagonal is
    never the pivot; an all-zero column is singular.  Both global-memory
    variants: a block of warps per 32 systems (few) and a thread per system
    (many)."""
    torch, chem = env
    method = {"global": chem.LU_GLOBAL, "global_fma": chem.LU_GLOBAL_FMA}[method]
    n = 4
    A, b = _systems(n, n_sys, seed=3)
    A[0, 0, 0] = np.nan
    A[1, 2, 0] = np.nan
    A[2, :, 1] = 0.0
    dev = torch.device("cuda")
    piv = torch.zeros((n_sys, n), dtype=torch.int32, device=dev)
    info = torch.full((n_sys,), -1, dtype=torch.int32, device=dev)
    Ad = torch.tensor(np.ascontiguousarray(A.transpose(1, 2, 0)), device=dev)
    bd = torch.tensor(np.ascontiguousarray(b.T), device=dev)
    chem.batched_solve(method, Ad, bd, piv, info)
    torch.cuda.synchronize()
    piv, info = piv.cpu().numpy(), info.cpu().numpy()
    assert piv[0, 0] == 0 and info[0] == 1
    rc, _, pivo = oracle.lu_factor(A[1])
    assert pivo[0] != 2 and piv[1, 0] == pivo[0]
    assert (rc != 0) == (info[1] != 0)
    rc, _, pivo = oracle.lu_factor(A[2])
    assert rc != 0 and piv[2, 0] == pivo[0] and info[2] == 2
    assert (info[3:] == 0).all()


def test_singular_and_unsupported(env):
    torch, chem = env
    dev = torch.device("cuda")
    A = np.ones((3, 4, 4))
    A[1] = np.eye(4)
    b = np.ones((3, 4))
    Ad = torch.tensor(A, device=dev)
    bd = torch.tensor(b, device=dev)
    info = torch.full((3,), -1, dtype=torch.int32, device=dev)
    chem.batched_solve(chem.LU_ONCHIP, Ad, bd, None, info)
    torch.cuda.synchronize()
    inf = info.cpu().numpy()
    assert inf[1] == 0 and inf[0] == 2 and inf[2] == 2       # rank-1 all-ones: column 1 has no pivot
    with pytest.raises(chem.ChemError) as ei:
        big = torch.zeros((1, 250, 250), dtype=torch.float64, device=dev)
        chem.batched_solve(chem.LU_ONCHIP, big, torch.zeros((1, 250), dtype=torch.float64, device=dev))
    assert ei.value.code == -7
