"""Pins for the seeded workload generator (MAC Oseen assembly and partition).

The generator is input-only; these tests check it against facts fixed by the
mathematics of the discretisation and of vertex separators, not against
itself.
"""
import numpy as np
import pytest

from paper_1104_3349_gb300 import workload as W

MASK64 = (1 << 64) - 1


def _splitmix64(x):
    x = (x + 0x9E3779B97F4A7C15) & MASK64
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return x, z ^ (z >> 31)


def _xoshiro_stream(seed, n):
    """xoshiro256** from its published definition (Blackman & Vigna, 2018)."""
    rotl = lambda v, k: ((v << k) | (v >> (64 - k))) & MASK64
    s, x = [], seed
    for _ in range(4):
        x, z = _splitmix64(x)
        s.append(z)
    out = []
    for _ in range(n):
        out.append((rotl((s[1] * 5) & MASK64, 7) * 9) & MASK64)
        t = (s[1] << 17) & MASK64
        s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3]; s[2] ^= t
        s[3] = rotl(s[3], 45)
    return out


def test_rng_matches_published_definition():
    for seed in (0, 1, 12345):
        got = [int(v) for v in W.raw_stream(seed, 16)]
        assert got == _xoshiro_stream(seed, 16)
    u = W.uniform(0, 1000, -1.0, 1.0)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.1


def _geom_widths(n, r):
    k = np.arange(n)
    d = np.minimum(k, n - 1 - k)
    h = r ** d.astype(float)
    return h / h.sum()


@pytest.mark.parametrize("r", [1.0, 1.1])
def test_spacing(r):
    assert np.allclose(W.spacing(12, r), _geom_widths(12, r), rtol=0, atol=1e-15)


def _blocks(n, **kw):
    A, rhs = W.mac_system(n, **kw)
    C = A.to_dense()
    kind, cell = W.mac_layout(n)
    return C, kind, cell


@pytest.mark.parametrize("r", [1.0, 1.15])
def test_div_grad_is_pressure_laplacian(r):
    """Div_FV M^-1 Div_FV^T equals the two-point-flux Neumann pressure Laplacian."""
    n = 6
    C, kind, cell = _blocks(n, nu=0.05, stretch=r, wind=W.WIND_FOURIER, wind_seed=7, pin=False, scale=False)
    P = np.where(kind == 0)[0]
    Vel = np.where(kind != 0)[0]
    Div = C[np.ix_(P, Vel)]
    h = _geom_widths(n, r)
    hx, hy = h, h
    # face control volume = face length * centre distance
    vol = np.empty(len(Vel))
    for q, k in enumerate(Vel):
        i, j = cell[k] % n, cell[k] // n
        if kind[k] == 1:
            vol[q] = hy[j] * 0.5 * (hx[i] + hx[i + 1])
        else:
            vol[q] = hx[i] * 0.5 * (hy[j] + hy[j + 1])
    Lap_from_div = Div @ np.diag(1.0 / vol) @ Div.T
    # Neumann Laplacian assembled cell by cell, transmissibility A_f / dist
    L = np.zeros((n * n, n * n))
    for j in range(n):
        for i in range(n):
            c = j * n + i
            if i + 1 < n:
                t = hy[j] / (0.5 * (hx[i] + hx[i + 1]))
                L[c, c] += t; L[c + 1, c + 1] += t; L[c, c + 1] -= t; L[c + 1, c] -= t
            if j + 1 < n:
                t = hx[i] / (0.5 * (hy[j] + hy[j + 1]))
                L[c, c] += t; L[c + n, c + n] += t; L[c, c + n] -= t; L[c + n, c] -= t
    pidx = cell[P]
    L = L[np.ix_(pidx, pidx)]
    assert np.abs(Lap_from_div - L).max() <= 1e-13 * np.abs(L).max()


def test_saddle_structure_and_constant_pressure():
    """C = [D, Grad; Div, 0] with Grad = -Div^T; C (0, 1_p) = 0 without the pin."""
    n = 7
    C, kind, cell = _blocks(n, nu=0.01, wind=W.WIND_FOURIER, wind_seed=3, pin=False, scale=False)
    P = kind == 0
    V = ~P
    assert np.all(C[np.ix_(P, P)] == 0)
    assert np.abs(C[np.ix_(V, P)] + C[np.ix_(P, V)].T).max() == 0.0
    ones_p = P.astype(float)
    assert np.abs(C @ ones_p).max() <= 1e-15


@pytest.mark.parametrize("n", [4, 6, 8])
def test_pin_removes_null_space(n):
    C, kind, cell = _blocks(n, nu=0.02, wind=W.WIND_POLY, pin=True, scale=True)
    s = np.linalg.svd(C, compute_uv=False)
    assert s.min() > 1e-6 * s.max()
    C0, _, _ = _blocks(n, nu=0.02, wind=W.WIND_POLY, pin=False, scale=False)
    s0 = np.linalg.svd(C0, compute_uv=False)
    assert s0.min() < 1e-12 * s0.max()


def test_stokes_block_symmetric_and_upwind_dominant():
    n = 6
    C, kind, _ = _blocks(n, nu=0.03, wind=W.WIND_NONE, pin=False, scale=False)
    V = kind != 0
    D = C[np.ix_(V, V)]
    assert np.abs(D - D.T).max() <= 1e-15
    C2, kind, _ = _blocks(n, nu=0.001, wind=W.WIND_FOURIER, wind_seed=11, pin=False, scale=False)
    D2 = C2[np.ix_(V, V)]
    off = D2 - np.diag(np.diag(D2))
    assert off.max() <= 0.0
    assert np.all(np.diag(D2) + 1e-15 >= np.abs(off).sum(axis=1))


def test_convective_fluxes_balance():
    """With nu = 0 every interior control volume's upwind row sums to sum F_f = 0."""
    n = 8
    C, kind, cell = _blocks(n, nu=0.0, wind=W.WIND_FOURIER, wind_seed=5, pin=False, scale=False)
    V = np.where(kind != 0)[0]
    P = kind == 0
    D = C[np.ix_(V, V)]
    checked = 0
    for q, k in enumerate(V):
        i, j = cell[k] % n, cell[k] // n
        if kind[k] == 1 and (1 <= i <= n - 3) and (1 <= j <= n - 2):
            assert abs(D[q].sum()) <= 1e-15
            checked += 1
        if kind[k] == 2 and (1 <= j <= n - 3) and (1 <= i <= n - 2):
            assert abs(D[q].sum()) <= 1e-15
            checked += 1
    assert checked > 20


def test_row_scaling():
    A, _ = W.mac_system(8, nu=0.01, wind=W.WIND_POLY)
    C = A.to_dense()
    assert np.allclose(np.abs(C).max(axis=1), 1.0, rtol=0, atol=1e-15)


def _check_partition(A, part, perm, m):
    n = A.n
    assert sorted(perm.tolist()) == list(range(n))
    nI = int((part >= 0).sum())
    ps = part[perm[:nI]]
    assert np.all(np.diff(ps) >= 0) and ps.min() >= 0 and ps.max() < m
    assert np.all(part[perm[nI:]] == -1)
    assert np.all(np.diff(perm[nI:]) > 0)
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    pr, pc = part[rows], part[A.col]
    bad = (pr >= 0) & (pc >= 0) & (pr != pc) & (A.val != 0)
    assert not bad.any(), "an entry couples two different interiors"


@pytest.mark.parametrize("n,m", [(8, 2), (12, 4), (16, 8), (32, 4)])
def test_partition_is_vertex_separator(n, m):
    A, _ = W.mac_system(n, nu=0.01, wind=W.WIND_POLY)
    part, perm, _ = W.partition(A, m)
    _check_partition(A, part, perm, m)
    part2, perm2, _ = W.partition(A, m)
    assert np.array_equal(part, part2) and np.array_equal(perm, perm2)


@pytest.mark.parametrize("n,m", [(8, 2), (12, 4), (16, 4), (32, 4)])
def test_interior_blocks_nonsingular(n, m):
    """The enclosed-pressure repair leaves every A_jj of full rank."""
    A, _ = W.mac_system(n, nu=0.01, wind=W.WIND_FOURIER, wind_seed=n)
    part, perm, _ = W.partition(A, m)
    C = A.to_dense()
    for j in range(m):
        idx = perm[part[perm] == j]
        B = C[np.ix_(idx, idx)]
        s = np.linalg.svd(B, compute_uv=False)
        assert s.min() > 1e-10 * s.max(), f"A_{j} singular"


def test_aggregates_cover_interface():
    w = W.cavity32()
    a = w.agg
    assert a[0] == 0 and a[-1] == w.n_interface and np.all(np.diff(a) > 0)
    C = w.A.to_dense()
    nI = w.A.n - w.n_interface
    G = C[np.ix_(w.perm[nI:], w.perm[nI:])]
    for i in range(len(a) - 1):
        Gi = G[a[i]:a[i + 1], a[i]:a[i + 1]]
        assert np.all(np.abs(Gi).sum(axis=1) > 0)
