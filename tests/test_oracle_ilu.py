"""Pins of the oracle's incomplete interior factorisation (Section 5: an
incomplete LU with tolerance tolA = 1e-4 for the (1,1) blocks).

Reading (the paper gives only the tolerance): right-looking band LU with
partial pivoting; at step k, after the row exchange, a pivot-row entry u_kj
(j > k) is dropped when |u_kj| < tau |A(:, j)|_2 and a multiplier l_ik when
|l_ik| < tau |A(:, k)|_2 / |u_kk|, before either is used; the diagonal is kept.

The pins: tau = 0 is the exact LU bit for bit; hand-worked 3 x 3 factorisations
(with and without a row exchange); an infinite tolerance on a diagonally
dominant band matrix leaves the diagonal only (x = b / diag(A)); and the
preconditioner built with it still drives FGMRES to the tolerance.
"""
import numpy as np
import pytest

import oracle as O
from paper_1104_3349_gb300 import workload as W


def _band(n, kl, ku, seed, dominant=False):
    rng = np.random.default_rng(seed)
    a = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - kl), min(n, i + ku + 1)):
            a[i, j] = rng.uniform(-1, 1)
    if dominant:
        a += np.diag(np.abs(a).sum(1) + 1.0)
    return a


def test_zero_tolerance_is_the_exact_lu():
    a = _band(40, 3, 2, 1)
    b = np.random.default_rng(2).uniform(-1, 1, 40)
    x0, p0, r0 = O.band_lu_solve(a, 3, 2, b)
    x1, p1, r1 = O.band_ilu_solve(a, 3, 2, b, 0.0)
    assert r0 == r1 == 0
    assert np.array_equal(p0, p1)
    assert np.array_equal(x0.view(np.uint64), x1.view(np.uint64))


def test_tridiagonal_by_hand():
    # A = tridiag(1, 4, 1); column norms sqrt(17), sqrt(18), sqrt(17).
    # tau = 0.24: u01 = 1 < 0.24 sqrt(18) dropped, l10 = 1/4 >= 0.24 sqrt(17)/4
    # kept, u12 = 1 >= 0.24 sqrt(17) kept, l21 = 1/4 < 0.24 sqrt(18)/4 dropped:
    # L = [1; 1/4 1; 0 0 1], U = [4 0 0; 0 4 1; 0 0 4]; b = (1, 2, 3) gives
    # z = (1, 7/4, 3), x = (1/4, 1/4, 3/4).
    a = np.array([[4.0, 1, 0], [1, 4, 1], [0, 1, 4]])
    x, piv, rc = O.band_ilu_solve(a, 1, 1, np.array([1.0, 2, 3]), 0.24)
    assert rc == 0 and list(piv) == [0, 1, 2]
    np.testing.assert_allclose(x, [0.25, 0.25, 0.75], rtol=0, atol=1e-15)
    # tau = 0.25 drops every off-diagonal entry: x = b / 4
    x, _, _ = O.band_ilu_solve(a, 1, 1, np.array([1.0, 2, 3]), 0.25)
    np.testing.assert_allclose(x, [0.25, 0.5, 0.75], rtol=0, atol=1e-15)


def test_pivoting_case_by_hand():
    # A = [1 2 0; 3 1 1; 0 1 5], tau = 0.3.  Step 0 exchanges rows 0 and 1
    # (|3| > |1|): pivot row (3, 1, 1); u01 = 1 >= 0.3 sqrt(6) kept, u02 = 1 <
    # 0.3 sqrt(26) dropped; l10 = 1/3 >= 0.3 sqrt(10)/3 kept; row 1 becomes
    # (5/3, 0).  Step 1: no exchange, l21 = 3/5 >= 0.3 sqrt(6)/(5/3) kept,
    # a22 = 5.  b = (1, 2, 3): after the exchange (2, 1, 3), forward
    # (2, 1/3, 14/5), back x = (3/5, 1/5, 14/25).
    a = np.array([[1.0, 2, 0], [3, 1, 1], [0, 1, 5]])
    x, piv, rc = O.band_ilu_solve(a, 1, 1, np.array([1.0, 2, 3]), 0.3)
    assert rc == 0 and list(piv) == [1, 1, 2]
    np.testing.assert_allclose(x, [0.6, 0.2, 0.56], rtol=0, atol=1e-15)


def test_infinite_tolerance_keeps_the_diagonal():
    a = _band(50, 4, 3, 3, dominant=True)
    b = np.random.default_rng(4).uniform(-1, 1, 50)
    x, piv, rc = O.band_ilu_solve(a, 4, 3, b, 1e300)
    assert rc == 0 and np.array_equal(piv, np.arange(50))
    np.testing.assert_allclose(x, b / np.diag(a), rtol=1e-15, atol=0)


def test_ilu_preconditioner_zero_tolerance_matches_exact():
    w = W.cavity32()
    y = W.uniform(1, w.A.n)
    R0 = O.OracleDD(w.A, w.part, w.m, O.MSCE_INF, perm=w.perm, agg_offsets=w.agg)
    R1 = O.OracleDD(w.A, w.part, w.m, O.MSCE_INF, perm=w.perm, agg_offsets=w.agg, ilu_tol=0.0)
    x0, x1 = R0.apply(y), R1.apply(y)
    assert np.array_equal(x0.view(np.uint64), x1.view(np.uint64))


@pytest.mark.parametrize("tol", [1e-4, 1e-2])
def test_ilu_preconditioner_converges(tol):
    w = W.cavity32()
    R = O.OracleDD(w.A, w.part, w.m, O.MSCE_INF, perm=w.perm, agg_offsets=w.agg, ilu_tol=tol)
    E = O.OracleDD(w.A, w.part, w.m, O.MSCE_INF, perm=w.perm, agg_offsets=w.agg)
    y = W.uniform(1, w.A.n)
    # an inexact interior solve changes the preconditioner, by more for a
    # larger tolerance
    d = np.linalg.norm(R.apply(y) - E.apply(y)) / np.linalg.norm(E.apply(y))
    assert 0 < d < (1e-2 if tol == 1e-4 else 1.0)
    r = R.fgmres(w.b, tol=1e-8, restart=50, maxit=400)
    assert r["status"] == 0
    res = np.linalg.norm(w.b - O.spmv(w.A, r["x"])) / np.linalg.norm(w.b)
    assert res <= 1e-8
