"""Pins for the oracle's Gaussian elimination (Sec. 3.2: direct elimination of
the Eq. 29 system), against a hand-worked system and LAPACK."""
import numpy as np
import pytest


def test_hand_worked_3x3_pivots_and_solution(oracle_mod):
    # Worked by hand: column 0 pivots on row 1 (|4| largest); after
    # elimination column 1 holds 4 and 4 -- a tie, which keeps the lower index.
    A = np.array([[2.0, 1.0, 1.0], [4.0, -6.0, 0.0], [-2.0, 7.0, 2.0]])
    b = np.array([5.0, -2.0, 9.0])
    rc, LU, piv = oracle_mod.lu_factor(A)
    assert rc == 0
    assert list(piv) == [1, 1, 2]
    U = np.triu(LU)
    L = np.tril(LU, -1) + np.eye(3)
    np.testing.assert_array_equal(U, [[4.0, -6.0, 0.0], [0.0, 4.0, 1.0], [0.0, 0.0, 1.0]])
    np.testing.assert_array_equal(L, [[1.0, 0.0, 0.0], [0.5, 1.0, 0.0], [-0.5, 1.0, 1.0]])
    x = oracle_mod.lu_solve(LU, piv, b)
    np.testing.assert_array_equal(x, [1.0, 1.0, 2.0])


def test_tie_keeps_lowest_row(oracle_mod):
    A = np.array([[1.0, 2.0, 0.0], [-1.0, 3.0, 1.0], [1.0, 0.0, 4.0]])
    rc, LU, piv = oracle_mod.lu_factor(A)
    assert rc == 0 and piv[0] == 0


def test_singular_reports_failure(oracle_mod):
    A = np.array([[1.0, 2.0], [2.0, 4.0]])
    rc, _, _ = oracle_mod.lu_factor(A)
    assert rc == -1
    # a NaN anywhere ends in a non-finite pivot: on the diagonal it poisons
    # the search, below it the elimination carries it into the next pivot
    for A in ([[np.nan, 1.0], [1.0, 1.0]], [[1.0, 1.0], [np.nan, 1.0]], [[1.0, np.inf], [1.0, 1.0]]):
        rc, _, _ = oracle_mod.lu_factor(np.array(A))
        assert rc == -1


@pytest.mark.parametrize("n", [2, 10, 37, 65])
def test_random_systems_against_lapack(oracle_mod, n):
    rng = np.random.default_rng(n)
    for trial in range(5):
        A = rng.standard_normal((n, n)) + n ** 0.5 * np.eye(n) * (trial % 2)
        b = rng.standard_normal(n)
        rc, LU, piv = oracle_mod.lu_factor(A)
        assert rc == 0
        # P A = L U
        P = np.eye(n)
        for k in range(n):
            P[[k, piv[k]]] = P[[piv[k], k]]
        L = np.tril(LU, -1) + np.eye(n)
        U = np.triu(LU)
        assert np.abs(P @ A - L @ U).max() <= 1e-13 * np.abs(A).max() * n
        assert np.all(np.abs(np.tril(LU, -1)) <= 1.0)  # partial pivoting bound
        x = oracle_mod.lu_solve(LU, piv, b)
        ref = np.linalg.solve(A, b)
        cond = np.linalg.cond(A)
        assert np.abs(x - ref).max() <= 1e-15 * cond * n * max(1.0, np.abs(ref).max())
        assert np.abs(A @ x - b).max() <= 1e-13 * n * np.abs(A).max() * np.abs(x).max()
