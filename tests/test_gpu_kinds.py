"""GPU parity of the approximations beyond the five plain kinds: the
overlapped aggregates OMSCN / OMSCNR / OLUM (the Remark on overlapped
aggregation, Algorithm 1) and MSCE with a finite radius r (Algorithm 1's
mini Schur complements on edge connectivity), against the oracle.

Bars as for the plain kinds: FP64 dd_apply relative 2-norm <= 1e-10, FP32
<= 1e-4; FGMRES(50) iterations within +-1 of the oracle and true residual
<= 1e-8.
"""
import numpy as np
import pytest

import oracle as O
from paper_1104_3349_gb300 import workload as W

pytestmark = pytest.mark.gpu

KIND_O = {"omscn": O.OMSCN, "omscnr": O.OMSCNR, "olum": O.OLUM, "msce": O.MSCE}


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1104_3349_gb300 import dd
    dd.build()
    dd.load()
    return torch, dd, torch.device("cuda:0")


def _pair(dd, w, kind, prec=0, overlap=0, radius=0):
    P = dd.DD(w.A, w.part, w.m, kind, perm=w.perm, agg_offsets=w.agg, prec=prec, overlap=overlap, radius=radius)
    R = O.OracleDD(w.A, w.part, w.m, KIND_O[kind], perm=w.perm, agg_offsets=w.agg, overlap=overlap, radius=radius)
    return P, R


def _apply_err(torch, dev, P, R, n, seed=1):
    y = W.uniform(seed, n)
    yd = torch.from_numpy(y).to(dev)
    xd = torch.full_like(yd, float("nan"))
    P.apply(yd, xd)
    assert P.check_status() == 0
    x = xd.cpu().numpy()
    xr = R.apply(y)
    assert np.all(np.isfinite(x))
    return np.linalg.norm(x - xr) / np.linalg.norm(xr)


CASES = [("cav32", None), ("t20", (20, 4, 33)), ("t12", (12, 8, 16))]


def _workload(name, spec):
    if spec is None:
        return W.cavity32()
    grid, m, sz = spec
    return W.make_workload("t", grid, 0.02, 1.0, W.WIND_FOURIER, grid, m, sz=sz)


@pytest.mark.parametrize("name,spec", CASES)
@pytest.mark.parametrize("kind", ["omscn", "omscnr", "olum"])
@pytest.mark.parametrize("overlap", [0, 5, 64])
def test_overlapped_apply_fp64(env, name, spec, kind, overlap):
    torch, dd, dev = env
    w = _workload(name, spec)
    try:
        P, R = _pair(dd, w, kind, overlap=overlap)
    except (O.OracleError, dd.DDError) as e:
        # both sides must refuse alike (a singular assembled S_hat)
        with pytest.raises((O.OracleError, dd.DDError)):
            O.OracleDD(w.A, w.part, w.m, KIND_O[kind], perm=w.perm, agg_offsets=w.agg, overlap=overlap)
        with pytest.raises(dd.DDError):
            dd.DD(w.A, w.part, w.m, kind, perm=w.perm, agg_offsets=w.agg, overlap=overlap)
        return
    err = _apply_err(torch, dev, P, R, w.A.n)
    assert err <= 1e-10, (name, kind, overlap, err)


@pytest.mark.parametrize("name,spec", CASES)
@pytest.mark.parametrize("radius", [0, 1, 2, 4, 10 ** 6])
def test_msce_radius_apply_fp64(env, name, spec, radius):
    torch, dd, dev = env
    w = _workload(name, spec)
    P, R = _pair(dd, w, "msce", radius=radius)
    err = _apply_err(torch, dev, P, R, w.A.n)
    assert err <= 1e-10, (name, radius, err)


@pytest.mark.parametrize("kind,kw", [("omscn", dict(overlap=64)), ("olum", dict(overlap=64)),
                                     ("msce", dict(radius=1)), ("msce", dict(radius=3))])
def test_new_kinds_fp32_and_gmres(env, kind, kw):
    torch, dd, dev = env
    w = W.cavity32()
    P32, R = _pair(dd, w, kind, prec=1, **kw)
    err = _apply_err(torch, dev, P32, R, w.A.n)
    print(f"{kind} {kw}: FP32 apply relative error vs FP64 oracle {err:.3e}")
    assert err <= 1e-4
    ro = R.fgmres(w.b, tol=1e-8, restart=50)
    for P in (_pair(dd, w, kind, prec=0, **kw)[0], P32):
        bd = torch.from_numpy(w.b).to(dev)
        xd = torch.zeros_like(bd)
        r = P.gmres(bd, xd, tol=1e-8, restart=50)
        assert r["status"] == 0 and r["relres"] <= 1e-8
        assert abs(r["iters"] - ro["iters"]) <= 1, (kind, kw, r["iters"], ro["iters"])
        x = xd.cpu().numpy()
        assert np.linalg.norm(w.b - O.spmv(w.A, x)) <= 1e-8 * np.linalg.norm(w.b)


def test_msce_radius_limits_on_the_gpu(env):
    """r = 0 is LUM and a radius beyond the interiors is MSCE_INF, on the GPU too."""
    torch, dd, dev = env
    w = W.cavity32()
    y = torch.from_numpy(W.uniform(1, w.A.n)).to(dev)
    out = {}
    for name, kind, kw in (("r0", "msce", dict(radius=0)), ("lum", "lum", {}),
                           ("rinf", "msce", dict(radius=10 ** 6)), ("inf", "msce_inf", {})):
        P = dd.DD(w.A, w.part, w.m, kind, perm=w.perm, agg_offsets=w.agg, **kw)
        x = torch.empty_like(y)
        P.apply(y, x)
        out[name] = x.cpu().numpy()
    assert np.array_equal(out["r0"], out["lum"])
    assert np.linalg.norm(out["rinf"] - out["inf"]) <= 1e-12 * np.linalg.norm(out["inf"])


def test_overlapped_kinds_refused_in_a_batch(env):
    torch, dd, dev = env
    ws = W.batch_small(count=3)
    with pytest.raises(dd.DDError) as e:
        dd.DDBatch([(q.A, q.part, q.m, q.perm, q.agg) for q in ws], "olum")
    assert e.value.status == 1
