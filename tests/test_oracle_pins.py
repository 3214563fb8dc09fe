"""Pins for the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle (oracle/dd_oracle.c) against something other than
itself: brute-force dense linear algebra in numpy, scipy's LU, the
Banachiewicz form of B (Lemma 1), the spectral theorem for C B^-1 (Theorem 2
and the right-preconditioning remark), the paper's worked MSCN example
(Section 3.2), and textbook special cases.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_1104_3349_gb300 import workload as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(20240601)


# --------------------------------------------------------------------------
# LU
# --------------------------------------------------------------------------
def _unpack(lu, piv):
    n = lu.shape[0]
    L = np.tril(lu, -1) + np.eye(n)
    U = np.triu(lu)
    perm = np.arange(n)
    for k in range(n):
        perm[[k, piv[k]]] = perm[[piv[k], k]]
    return L, U, perm


@pytest.mark.parametrize("n", [1, 7, 40])
def test_dense_lu_backward_error_and_scipy(n):
    A = rng.standard_normal((n, n))
    lu, piv, rc = O.dense_lu(A)
    assert rc == 0
    L, U, perm = _unpack(lu, piv)
    assert np.abs(A[perm] - L @ U).max() <= 1e-14 * n * np.abs(A).max()
    P, Ls, Us = sla.lu(A)
    assert np.allclose(L, Ls, atol=1e-12) and np.allclose(U, Us, atol=1e-12)
    assert np.array_equal(P.T @ np.arange(n), perm.astype(float))


def test_dense_lu_first_max_pivot_and_singular():
    A = np.array([[1.0, 2.0], [-1.0, 0.0]])
    _, piv, rc = O.dense_lu(A)
    assert rc == 0 and piv[0] == 0  # |1| == |-1|: the first row wins
    S = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [0.0, 0.0, 1.0]])
    _, _, rc = O.dense_lu(S)
    assert rc == 2  # column 1 has no acceptable pivot


@pytest.mark.parametrize("n,kl,ku", [(60, 3, 2), (120, 9, 5), (50, 1, 7)])
def test_band_lu_equals_dense_lu(n, kl, ku):
    A = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - kl), min(n, i + ku + 1)):
            A[i, j] = rng.standard_normal()
    A[np.arange(n), np.arange(n)] *= 0.1  # force pivoting
    b = rng.standard_normal(n)
    x, piv_b, rc = O.band_lu_solve(A, kl, ku, b)
    assert rc == 0
    lu, piv_d, rc2 = O.dense_lu(A)
    assert rc2 == 0
    assert np.array_equal(piv_b, piv_d)
    xd = O.dense_lu_solve(lu, piv_d, b)
    assert np.abs(x - xd).max() <= 1e-12 * np.abs(xd).max()
    assert np.abs(x - np.linalg.solve(A, b)).max() <= 1e-10 * np.abs(xd).max()


# --------------------------------------------------------------------------
# Blocks of P^T C P and brute-force Schur complements
# --------------------------------------------------------------------------
def _small(n=8, m=4, nu=0.02, wind=W.WIND_FOURIER, seed=9, sz=16):
    A, _ = W.mac_system(n, nu=nu, wind=wind, wind_seed=seed)
    part, perm, _ = W.partition(A, m)
    agg = W.aggregates(A, part, perm, sz)
    return A, part, perm, agg


def _perm_blocks(A, part, perm):
    C = A.to_dense()
    Cp = C[np.ix_(perm, perm)]
    nI = int((part >= 0).sum())
    return Cp, nI, Cp[:nI, :nI], Cp[:nI, nI:], Cp[nI:, :nI], Cp[nI:, nI:]


def _brute_S(D, E, F, G):
    return G - F @ np.linalg.solve(D, E)


def _brute_blocks(kind, D, E, F, G, agg):
    S = _brute_S(D, E, F, G)
    out = []
    for i in range(len(agg) - 1):
        a, e = agg[i], agg[i + 1]
        if kind in (O.MSCE_INF, O.EXACT):
            out.append(S[a:e, a:e])
        elif kind == O.LUM:
            out.append(G[a:e, a:e])
        else:
            Dii, Eii, Fii = D[a:e, a:e], E[a:e, a:e], F[a:e, a:e]
            if not Eii.any() or not Fii.any():
                out.append(G[a:e, a:e].copy())
                continue
            X = np.linalg.solve(Dii, Eii)
            if kind == O.MSCN:
                out.append(G[a:e, a:e] - Fii @ X)
            else:
                out.append(G[a:e, a:e] - np.diag(Fii @ X @ np.ones(e - a)))
    return out


def test_exact_schur_equals_brute_force():
    A, part, perm, agg = _small()
    Cp, nI, D, E, F, G = _perm_blocks(A, part, perm)
    P = O.OracleDD(A, part, 4, O.EXACT, perm=perm)
    S = P.schur_block(0)
    Sb = _brute_S(D, E, F, G)
    assert np.abs(S - Sb).max() <= 1e-12 * np.abs(Sb).max()


@pytest.mark.parametrize("kind", [O.MSCE_INF, O.MSCN, O.MSCNR, O.LUM])
def test_schur_blocks_equal_brute_force(kind):
    A, part, perm, agg = _small(n=10, m=4, sz=12)
    Cp, nI, D, E, F, G = _perm_blocks(A, part, perm)
    P = O.OracleDD(A, part, 4, kind, perm=perm, agg_offsets=agg)
    ref = _brute_blocks(kind, D, E, F, G, agg)
    for i, Sb in enumerate(ref):
        S = P.schur_block(i)
        assert np.abs(S - Sb).max() <= 1e-11 * max(1.0, np.abs(Sb).max()), (kind, i)


def test_mscn_paper_example_index_mapping():
    """Section 3.2 worked example: aggregate {10,11} of G pairs with D-local
    {10,11}, i.e. C_4 is built from global rows/columns {10,11,26,27}."""
    g = json.load(open(os.path.join(GOLDEN, "mscn_toy_example.json")))
    nD, nG = g["n_D"], g["n_G"]
    n = nD + nG
    C = rng.standard_normal((n, n)) * 0.3 + np.eye(n) * 4.0
    rows, cols = np.nonzero(C)
    A = W.CSR(n, np.concatenate([[0], np.cumsum(np.count_nonzero(C, axis=1))]).astype(np.int32),
              cols.astype(np.int32), C[rows, cols])
    part = np.array([0] * nD + [-1] * nG, np.int32)
    sizes = [len(a) for a in g["aggregates_1based"]]
    agg = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    k = g["checked_aggregate_1based"] - 1
    idx = np.array(g["C4_global_rows_cols_1based"]) - 1
    C4 = C[np.ix_(idx, idx)]
    D4, E4, F4, G4 = C4[:2, :2], C4[:2, 2:], C4[2:, :2], C4[2:, 2:]
    P = O.OracleDD(A, part, 1, O.MSCN, agg_offsets=agg)
    assert np.abs(P.schur_block(k) - (G4 - F4 @ np.linalg.solve(D4, E4))).max() <= 1e-13
    P = O.OracleDD(A, part, 1, O.MSCNR, agg_offsets=agg)
    ref = G4 - np.diag(F4 @ np.linalg.solve(D4, E4) @ np.ones(2))
    assert np.abs(P.schur_block(k) - ref).max() <= 1e-13
    P = O.OracleDD(A, part, 1, O.LUM, agg_offsets=agg)
    assert np.abs(P.schur_block(k) - G4).max() == 0.0


# --------------------------------------------------------------------------
# Apply (Algorithm 2) against the factored form of B
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind", [O.EXACT, O.MSCE_INF, O.MSCN, O.MSCNR, O.LUM])
def test_apply_equals_inverse_of_factored_B(kind):
    A, part, perm, agg = _small(n=8, m=4, sz=14)
    Cp, nI, D, E, F, G = _perm_blocks(A, part, perm)
    P = O.OracleDD(A, part, 4, kind, perm=perm, agg_offsets=None if kind == O.EXACT else agg)
    a = P.agg_offsets()
    Sh = sla.block_diag(*[P.schur_block(i) for i in range(len(a) - 1)])
    nG = G.shape[0]
    Z = np.zeros
    L1 = np.block([[D, Z((nI, nG))], [F, Sh]])
    M = np.block([[np.linalg.inv(D), Z((nI, nG))], [Z((nG, nI)), np.linalg.inv(Sh)]])
    U1 = np.block([[D, E], [Z((nG, nI)), Sh]])
    Bp = L1 @ M @ U1
    # B = [D E; F, F D^-1 E + S_hat] (the product of the three factors)
    assert np.abs(Bp[nI:, nI:] - (F @ np.linalg.solve(D, E) + Sh)).max() <= 1e-10 * np.abs(Bp).max()
    y = W.uniform(1, A.n)
    x = P.apply(y)
    xp = np.linalg.solve(Bp, y[perm])
    ref = np.zeros(A.n)
    ref[perm] = xp
    assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref)


def test_apply_solves_B_with_F_forward_and_E_backward():
    """Algorithm 2 printed with (E z1) forward and (F x2) backward is not even
    well-typed (E is n_I x n_G); with F forward and E backward the apply
    solves B x = y for B = C with its (2,2) block replaced by F D^-1 E + S_hat."""
    A, part, perm, agg = _small(n=8, m=2, sz=10)
    Cp, nI, D, E, F, G = _perm_blocks(A, part, perm)
    P = O.OracleDD(A, part, 2, O.LUM, perm=perm, agg_offsets=agg)
    C = A.to_dense()
    y = W.uniform(2, A.n)
    x = P.apply(y)
    # B x = y with B = C except its (2,2) block is F D^-1 E + S_hat
    a = P.agg_offsets()
    Sh = sla.block_diag(*[P.schur_block(i) for i in range(len(a) - 1)])
    Bp = Cp.copy()
    Bp[nI:, nI:] = F @ np.linalg.solve(D, E) + Sh
    r = Bp @ x[perm] - y[perm]
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(y)


# --------------------------------------------------------------------------
# Spectrum: eig(C B^-1) = {1 (n_I times)} U eig(S S_hat^-1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind", [O.MSCE_INF, O.MSCN, O.LUM])
def test_right_preconditioned_spectrum(kind):
    A, part, perm, agg = _small(n=7, m=2, sz=12, seed=4)
    Cp, nI, D, E, F, G = _perm_blocks(A, part, perm)
    P = O.OracleDD(A, part, 2, kind, perm=perm, agg_offsets=agg)
    C = A.to_dense()
    Binv = np.column_stack([P.apply(e) for e in np.eye(A.n)])
    ev = np.linalg.eigvals(C @ Binv)
    a = P.agg_offsets()
    Sh = sla.block_diag(*[P.schur_block(i) for i in range(len(a) - 1)])
    S = _brute_S(D, E, F, G)
    ev_s = np.linalg.eigvals(S @ np.linalg.inv(Sh))
    expect = np.concatenate([np.ones(nI), ev_s])
    # match each expected eigenvalue to a distinct computed one
    remaining = list(ev)
    for lam in sorted(expect, key=lambda z: (z.real, z.imag)):
        d = [abs(lam - mu) for mu in remaining]
        k = int(np.argmin(d))
        assert d[k] <= 1e-8 * max(1.0, abs(lam)), (lam, d[k])
        remaining.pop(k)


# --------------------------------------------------------------------------
# GMRES
# --------------------------------------------------------------------------
def test_exact_schur_converges_in_one_iteration():
    w = W.cavity32()
    P = O.OracleDD(w.A, w.part, w.m, O.EXACT, perm=w.perm)
    r = P.fgmres(w.b, tol=1e-8, restart=50)
    assert r["status"] == 0 and r["iters"] == 1 and r["relres"] <= 1e-8


def test_single_aggregate_msce_is_exact():
    A, part, perm, agg = _small(n=8, m=4)
    nG = int((part < 0).sum())
    b = W.uniform(0, A.n)
    r1 = O.OracleDD(A, part, 4, O.EXACT, perm=perm).fgmres(b)
    r2 = O.OracleDD(A, part, 4, O.MSCE_INF, perm=perm, sz=nG).fgmres(b)
    assert r1["iters"] == r2["iters"] == 1
    assert np.abs(r1["x"] - r2["x"]).max() <= 1e-12 * np.abs(r1["x"]).max()


def test_unpreconditioned_gmres_terminates_in_n_steps():
    A, _ = W.mac_system(4, nu=0.05, wind=W.WIND_POLY)
    part = np.zeros(A.n, np.int32)
    P = O.OracleDD(A, part, 1, O.IDENTITY)
    b = W.uniform(3, A.n)
    r = P.fgmres(b, tol=1e-12, restart=A.n, maxit=A.n)
    assert r["status"] == 0 and r["iters"] <= A.n
    x = np.linalg.solve(A.to_dense(), b)
    assert np.abs(r["x"] - x).max() <= 1e-8 * np.abs(x).max()


@pytest.mark.parametrize("kind", [O.MSCE_INF, O.MSCN, O.LUM])
def test_gmres_solution_matches_dense_solve(kind):
    w = W.cavity32()
    P = O.OracleDD(w.A, w.part, w.m, kind, perm=w.perm, agg_offsets=w.agg)
    r = P.fgmres(w.b, tol=1e-8, restart=50)
    assert r["status"] == 0 and r["relres"] <= 1e-8
    C = w.A.to_dense()
    x = np.linalg.solve(C, w.b)
    cond = np.linalg.cond(C)
    assert np.linalg.norm(r["x"] - x) <= cond * 1e-8 * np.linalg.norm(x)
    assert np.linalg.norm(w.b - C @ r["x"]) <= 1e-8 * np.linalg.norm(w.b)
    h = r["history"]
    assert np.all(np.diff(h[: min(len(h), 50)]) <= 1e-15)  # non-increasing within a cycle


def test_lum_equals_mscn_when_coupling_blocks_vanish():
    """Section 5 observation: with E_ii, F_ii zero, MSCN reduces to LUM."""
    w = W.cavity32()
    r_l = O.OracleDD(w.A, w.part, w.m, O.LUM, perm=w.perm, agg_offsets=w.agg).fgmres(w.b)
    r_n = O.OracleDD(w.A, w.part, w.m, O.MSCN, perm=w.perm, agg_offsets=w.agg).fgmres(w.b)
    assert abs(r_l["iters"] - r_n["iters"]) <= 1


def test_stokes_pressure_schur_is_spd():
    """m = 1, interface = all pressures, w = 0: D is SPD (Theorem 1 applies) and
    S = G - F D^-1 E is the (pinned) pressure Schur complement, SPD."""
    n = 6
    A, _ = W.mac_system(n, nu=0.05, wind=W.WIND_NONE, scale=False)
    kind, _ = W.mac_layout(n)
    part = np.where(kind == 0, -1, 0).astype(np.int32)
    P = O.OracleDD(A, part, 1, O.EXACT)
    S = P.schur_block(0)
    assert np.abs(S - S.T).max() <= 1e-12 * np.abs(S).max()
    assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > 0


def test_invalid_partition_detected():
    A, part, perm, agg = _small(n=8, m=4)
    bad = part.copy()
    bad[perm[-1]] = 0  # an interface node joins subdomain 0 although it couples others
    with pytest.raises(O.OracleError) as e:
        O.OracleDD(A, bad, 4, O.LUM)
    assert e.value.status == 2


def test_singular_lum_block_reported():
    """LUM with plain chunks can hit a zero row of G_ii (a pressure node whose
    interface neighbours fall in another chunk): reported, not shifted."""
    A, _ = W.mac_system(16, nu=0.01, wind=W.WIND_POLY)
    kind, _ = W.mac_layout(16)
    part = np.where(kind == 0, -1, 0).astype(np.int32)
    with pytest.raises(O.OracleError) as e:
        O.OracleDD(A, part, 1, O.LUM, sz=8)
    assert e.value.status == 4 and e.value.bad_block == 0


# --------------------------------------------------------------------------
# Restarted GMRES(R): the restart path
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cav32_dense():
    w = W.cavity32()
    C = w.A.to_dense()
    return w, C, np.linalg.solve(C, w.b), np.linalg.cond(C)


@pytest.mark.parametrize("kind,restart", [(O.MSCE_INF, 5), (O.MSCE_INF, 13), (O.LUM, 25), (O.MSCN, 30)])
def test_restarted_gmres_reaches_dense_solution(cav32_dense, kind, restart):
    """Short restart lengths force several cycles (Section 5's restarted GMRES):
    the final iterate still matches the dense solve of C x = b to cond * 1e-8
    and its true residual, recomputed here, is below the tolerance."""
    w, C, x, cond = cav32_dense
    P = O.OracleDD(w.A, w.part, w.m, kind, perm=w.perm, agg_offsets=w.agg)
    r = P.fgmres(w.b, tol=1e-8, restart=restart, maxit=3000)
    assert r["status"] == 0 and r["restarts"] > 0, r["restarts"]
    assert np.linalg.norm(w.b - C @ r["x"]) <= 1e-8 * np.linalg.norm(w.b)
    assert abs(r["relres"] - np.linalg.norm(w.b - C @ r["x"]) / np.linalg.norm(w.b)) <= 1e-12
    assert np.linalg.norm(r["x"] - x) <= cond * 1e-8 * np.linalg.norm(x)


def _dense_Binv(A, part, perm, agg, kind):
    """B^-1 in the original numbering, from the factored form of B (Definition
    of B_MSCN) with brute-force Schur blocks: no part of the oracle is used."""
    Cp, nI, D, E, F, G = _perm_blocks(A, part, perm)
    Sh = sla.block_diag(*_brute_blocks(kind, D, E, F, G, agg))
    Bp = Cp.copy()
    Bp[nI:, nI:] = F @ np.linalg.solve(D, E) + Sh
    Binv_p = np.linalg.inv(Bp)
    Binv = np.zeros_like(Binv_p)
    Binv[np.ix_(perm, perm)] = Binv_p
    return Binv


def _gmres_by_definition(C, Binv, b, R, steps):
    """Right-preconditioned GMRES(R) written from its definition: every cycle
    starts from the true residual r = b - C x of the current iterate and adds
    B^-1 u, where u minimises ||r - C B^-1 u|| over the Krylov space
    K_k(C B^-1, r) (k = R, or the steps left); an orthonormal basis of the
    Krylov matrix comes from a QR factorisation."""
    M = C @ Binv
    x = np.zeros_like(b)
    left = steps
    while left > 0:
        k = min(R, left)
        r = b - C @ x
        K = np.empty((len(b), k))
        v = r / np.linalg.norm(r)
        for q in range(k):
            K[:, q] = v
            v = M @ v
            v /= np.linalg.norm(v)
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(M @ Q, r, rcond=None)
        x = x + Binv @ (Q @ y)
        left -= k
    return x


@pytest.mark.parametrize("kind,restart,maxit", [(O.LUM, 5, 10), (O.LUM, 5, 13), (O.MSCE_INF, 4, 11)])
def test_restart_cycles_match_gmres_definition(kind, restart, maxit):
    """The iterate after whole and partial cycles equals GMRES(R) computed from
    its definition with dense linear algebra: a restart from anything but the
    true residual of the accumulated iterate, or an iterate not accumulated
    over the cycles, fails this."""
    A, part, perm, agg = _small(n=6, m=2, sz=9)
    C = A.to_dense()
    b = W.uniform(11, A.n)
    P = O.OracleDD(A, part, 2, kind, perm=perm, agg_offsets=agg)
    r = P.fgmres(b, tol=1e-15, restart=restart, maxit=maxit)
    assert r["status"] == 5 and r["iters"] == maxit
    assert r["restarts"] == (maxit - 1) // restart
    x = _gmres_by_definition(C, _dense_Binv(A, part, perm, agg, kind), b, restart, maxit)
    assert np.linalg.norm(r["x"] - x) <= 1e-8 * np.linalg.norm(x)
    assert abs(r["relres"] - np.linalg.norm(b - C @ x) / np.linalg.norm(b)) <= 1e-8


# --------------------------------------------------------------------------
# Overlapped aggregates (OMSCN, OMSCNR, OLUM) and MSCE with a finite radius
# --------------------------------------------------------------------------
PLAIN_OF = {O.OMSCN: O.MSCN, O.OMSCNR: O.MSCNR, O.OLUM: O.LUM}


def _brute_overlapped(kind, D, E, F, G, agg, w):
    """S_hat of an overlapped kind from its definition: block i is MSCN /
    MSCNR / LUM on indices agg[i] .. agg[i+1]-1+w[i] (Algorithm 1), placed in
    aggregate order with a later block overwriting the overlap."""
    nG = G.shape[0]
    Sh = np.zeros((nG, nG))
    blocks = []
    for i in range(len(agg) - 1):
        a, e = agg[i], agg[i + 1] + w[i]
        Dii, Eii, Fii, Gii = D[a:e, a:e], E[a:e, a:e], F[a:e, a:e], G[a:e, a:e]
        if kind == O.OLUM or not Eii.any() or not Fii.any():
            S = Gii.copy()
        elif kind == O.OMSCN:
            S = Gii - Fii @ np.linalg.solve(Dii, Eii)
        else:
            S = Gii - np.diag(Fii @ np.linalg.solve(Dii, Eii) @ np.ones(e - a))
        blocks.append(S)
        Sh[a:e, a:e] = S
    return Sh, blocks


@pytest.mark.parametrize("kind", [O.OMSCN, O.OMSCNR, O.OLUM])
def test_zero_overlap_reproduces_the_plain_kind(kind):
    w = W.cavity32()
    P = O.OracleDD(w.A, w.part, w.m, kind, perm=w.perm, agg_offsets=w.agg, overlap=0)
    Q = O.OracleDD(w.A, w.part, w.m, PLAIN_OF[kind], perm=w.perm, agg_offsets=w.agg)
    y = W.uniform(1, w.A.n)
    x, xq = P.apply(y), Q.apply(y)
    assert np.linalg.norm(x - xq) <= 1e-12 * np.linalg.norm(xq)


@pytest.mark.parametrize("kind", [O.OMSCN, O.OMSCNR, O.OLUM])
@pytest.mark.parametrize("ov", [3, 7])
def test_overlapped_schur_equals_brute_force(kind, ov):
    A, part, perm, agg = _small(n=10, m=4, sz=12)
    Cp, nI, D, E, F, G = _perm_blocks(A, part, perm)
    P = O.OracleDD(A, part, 4, kind, perm=perm, agg_offsets=agg, overlap=ov)
    w = P.overlaps()
    assert w[-1] == 0 and all(w[i] == min(ov, agg[i + 2] - agg[i + 1]) for i in range(len(agg) - 2))
    Sh, blocks = _brute_overlapped(kind, D, E, F, G, agg, w)
    for i, Sb in enumerate(blocks):
        assert np.abs(P.schur_block(i) - Sb).max() <= 1e-11 * max(1.0, np.abs(Sb).max()), (kind, i)
    assert np.abs(P.schur_dense() - Sh).max() <= 1e-11 * max(1.0, np.abs(Sh).max())


def test_overlapped_schur_is_not_block_diagonal():
    """The Remark on overlapped aggregation: S_hat is no longer block diagonal
    over the aggregates; its entries stay inside the extended blocks."""
    A, part, perm, agg = _small(n=10, m=4, sz=12)
    P = O.OracleDD(A, part, 4, O.OMSCN, perm=perm, agg_offsets=agg, overlap=5)
    Sh, w = P.schur_dense(), P.overlaps()
    nG = Sh.shape[0]
    in_agg = np.zeros((nG, nG), bool)
    in_ext = np.zeros((nG, nG), bool)
    for i in range(len(agg) - 1):
        in_agg[agg[i]:agg[i + 1], agg[i]:agg[i + 1]] = True
        in_ext[agg[i]:agg[i + 1] + w[i], agg[i]:agg[i + 1] + w[i]] = True
    assert np.abs(Sh[~in_agg]).max() > 0
    assert np.abs(Sh[~in_ext]).max() == 0


def test_olum_takes_g_on_the_extended_blocks():
    A, part, perm, agg = _small(n=10, m=4, sz=12)
    Cp, nI, D, E, F, G = _perm_blocks(A, part, perm)
    P = O.OracleDD(A, part, 4, O.OLUM, perm=perm, agg_offsets=agg, overlap=6)
    w = P.overlaps()
    mask = np.zeros(G.shape, bool)
    for i in range(len(agg) - 1):
        mask[agg[i]:agg[i + 1] + w[i], agg[i]:agg[i + 1] + w[i]] = True
    assert np.array_equal(P.schur_dense(), np.where(mask, G, 0.0))


@pytest.mark.parametrize("kind", [O.OMSCN, O.OLUM])
def test_overlapped_apply_and_spectrum(kind):
    """The apply inverts B = [D E; F, F D^-1 E + S_hat] with the assembled
    S_hat (Lemma 1), and eig(C B^-1) = {1 (n_I times)} U eig(S S_hat^-1)."""
    A, part, perm, agg = _small(n=8, m=4, sz=14)
    Cp, nI, D, E, F, G = _perm_blocks(A, part, perm)
    P = O.OracleDD(A, part, 4, kind, perm=perm, agg_offsets=agg, overlap=5)
    Sh, _ = _brute_overlapped(kind, D, E, F, G, agg, P.overlaps())
    Bp = Cp.copy()
    Bp[nI:, nI:] = F @ np.linalg.solve(D, E) + Sh
    y = W.uniform(1, A.n)
    ref = np.zeros(A.n)
    ref[perm] = np.linalg.solve(Bp, y[perm])
    assert np.linalg.norm(P.apply(y) - ref) <= 1e-10 * np.linalg.norm(ref)
    lam = np.linalg.eigvals(Cp @ np.linalg.inv(Bp))
    mu = np.linalg.eigvals(_brute_S(D, E, F, G) @ np.linalg.inv(Sh))
    expect = np.concatenate([np.ones(nI), mu])
    for v in expect:
        k = np.argmin(np.abs(lam - v))
        assert abs(lam[k] - v) <= 1e-6 * max(1.0, abs(v))
        lam = np.delete(lam, k)


def test_overlap_beyond_the_next_aggregate_is_refused():
    A, part, perm, agg = _small(n=10, m=4, sz=12)
    bad = np.zeros(len(agg) - 1, np.int32)
    bad[0] = agg[2] - agg[1] + 1
    with pytest.raises(O.OracleError) as e:
        O.OracleDD(A, part, 4, O.OMSCN, perm=perm, agg_offsets=agg, overlaps=bad)
    assert e.value.status == 1


def _reach_set(Cp, nI, a, e, r):
    """Interior nodes within path length r of the aggregate [a, e), by
    boolean matrix powers of the interior pattern, closed by the neighbours
    of zero-diagonal nodes (the reading of D_r for MSCE)."""
    Dpat = (Cp[:nI, :nI] != 0) | (Cp[:nI, :nI] != 0).T
    np.fill_diagonal(Dpat, False)
    seed = ((Cp[nI + a:nI + e, :nI] != 0).any(axis=0)) | ((Cp[:nI, nI + a:nI + e] != 0).any(axis=1))
    reach = seed.copy()
    frontier = seed.copy()
    for _ in range(r - 1):
        frontier = (Dpat[frontier].any(axis=0)) & ~reach
        reach |= frontier
    zero_diag = np.diag(Cp[:nI, :nI]) == 0
    closure = Dpat[reach & zero_diag].any(axis=0) if (reach & zero_diag).any() else np.zeros(nI, bool)
    return np.nonzero(reach | closure)[0]


@pytest.mark.parametrize("r", [1, 2, 3])
def test_msce_radius_blocks_equal_brute_force(r):
    A, part, perm, agg = _small(n=10, m=4, sz=12)
    Cp, nI, D, E, F, G = _perm_blocks(A, part, perm)
    P = O.OracleDD(A, part, 4, O.MSCE, perm=perm, agg_offsets=agg, radius=r)
    for i in range(len(agg) - 1):
        a, e = agg[i], agg[i + 1]
        idx = _reach_set(Cp, nI, a, e, r)
        Sb = G[a:e, a:e] - F[a:e][:, idx] @ np.linalg.solve(D[np.ix_(idx, idx)], E[idx][:, a:e])
        assert np.abs(P.schur_block(i) - Sb).max() <= 1e-11 * max(1.0, np.abs(Sb).max()), (r, i)


def test_msce_radius_limits_are_lum_and_msce_inf():
    """r = 0 keeps no interior node (LUM); a radius beyond every interior's
    diameter reaches the whole adjacent interiors (MSCE_INF)."""
    w = W.cavity32()
    P0 = O.OracleDD(w.A, w.part, w.m, O.MSCE, perm=w.perm, agg_offsets=w.agg, radius=0)
    PL = O.OracleDD(w.A, w.part, w.m, O.LUM, perm=w.perm, agg_offsets=w.agg)
    Pr = O.OracleDD(w.A, w.part, w.m, O.MSCE, perm=w.perm, agg_offsets=w.agg, radius=10 ** 6)
    PI = O.OracleDD(w.A, w.part, w.m, O.MSCE_INF, perm=w.perm, agg_offsets=w.agg)
    for i in range(len(w.agg) - 1):
        assert np.array_equal(P0.schur_block(i), PL.schur_block(i))
        Si = PI.schur_block(i)
        assert np.abs(Pr.schur_block(i) - Si).max() <= 1e-12 * np.abs(Si).max()
