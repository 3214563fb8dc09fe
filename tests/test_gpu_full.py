"""Parity at the full size of the 256x256 workload, in the launch configuration
the benchmark times: 196 096 unknowns, 64 subdomains, MSCE_INF aggregates of
nominal size 2048 (six Schur blocks of 630-2049 rows), FGMRES(50) to 1e-8.

- FP64 dd_apply against the oracle's apply: relative 2-norm <= 1e-10.
- FGMRES iteration counts of the FP64 and the FP32 preconditioner within +-1
  of the oracle's, true residual <= 1e-8 (recomputed on the host).
- The setup is deterministic: two handles built from the same input give
  bitwise-equal solutions.
"""
import numpy as np
import pytest

import oracle as O
from paper_1104_3349_gb300 import workload as W

pytestmark = pytest.mark.gpu

SZ = 2048


@pytest.fixture(scope="module")
def full():
    import torch
    from paper_1104_3349_gb300 import dd
    dd.build()
    dd.load()
    w = W.fourier256()
    agg = W.aggregates(w.A, w.part, w.perm, SZ)
    R = O.OracleDD(w.A, w.part, w.m, O.MSCE_INF, perm=w.perm, agg_offsets=agg)
    y = W.uniform(1, w.A.n)
    xr = R.apply(y)
    ro = R.fgmres(w.b, tol=1e-8, restart=50, maxit=3000)
    R.close()
    assert ro["status"] == 0
    return torch, dd, torch.device("cuda:0"), w, agg, y, xr, ro


def _handle(dd, w, agg, prec):
    return dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=agg, prec=prec)


@pytest.mark.parametrize("cl", [1, 2])
def test_apply_fp64_full_size(full, cl):
    torch, dd, dev, w, agg, y, xr, ro = full
    P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=agg, prec=dd.DD_FP64, sweep_cluster=cl)
    assert P.stats()["sweep_cluster"] == cl
    st = P.stats()
    assert st["n_agg"] == len(agg) - 1 and st["max_agg"] >= 630
    yd = torch.from_numpy(y).to(dev)
    xd = torch.full_like(yd, float("nan"))
    P.apply(yd, xd)
    assert P.check_status() == 0
    err = np.linalg.norm(xd.cpu().numpy() - xr) / np.linalg.norm(xr)
    print(f"FP64 apply at 256x256 ({cl} CTA per subdomain), relative error vs oracle: {err:.3e}")
    assert err <= 1e-10, err
    P.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_fgmres_full_size_iterations(full, prec):
    torch, dd, dev, w, agg, y, xr, ro = full
    P = _handle(dd, w, agg, prec)
    bd = torch.from_numpy(w.b).to(dev)
    xd = torch.zeros_like(bd)
    r = P.gmres(bd, xd, tol=1e-8, restart=50, maxit=3000)
    P.close()
    print(f"prec {prec}: {r['iters']} iterations ({r['restarts']} restarts), oracle {ro['iters']}")
    assert r["status"] == 0 and r["relres"] <= 1e-8
    assert abs(r["iters"] - ro["iters"]) <= 1, (r["iters"], ro["iters"])
    x = xd.cpu().numpy()
    assert np.linalg.norm(w.b - O.spmv(w.A, x)) <= 1e-8 * np.linalg.norm(w.b)


@pytest.mark.parametrize("prec", [0, 1])
def test_setup_is_deterministic(full, prec):
    torch, dd, dev, w, agg, y, xr, ro = full
    bd = torch.from_numpy(w.b).to(dev)
    xs, its = [], []
    for _ in range(2):
        P = _handle(dd, w, agg, prec)
        xd = torch.zeros_like(bd)
        r = P.gmres(bd, xd, tol=1e-8, restart=50, maxit=3000)
        P.close()
        xs.append(xd.cpu().numpy())
        its.append(r["iters"])
    assert its[0] == its[1]
    assert np.array_equal(xs[0].view(np.uint64), xs[1].view(np.uint64))


def test_lookahead_fp32_full_size(full):
    """The lookahead split of the sweeps at full size, FP32 (in FP64 its ring
    stages and message buffers do not fit beside the vectors): the apply
    agrees with one CTA per subdomain to FP32 rounding and with the oracle
    within 1e-4; FGMRES takes the oracle's iterations +-1."""
    torch, dd, dev, w, agg, y, xr, ro = full
    yd = torch.from_numpy(y).to(dev)
    xs = []
    for mode in (1, 3):
        P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=agg, prec=dd.DD_FP32, sweep_cluster=mode)
        assert P.stats()["sweep_cluster"] == mode
        xd = torch.full_like(yd, float("nan"))
        P.apply(yd, xd)
        assert P.check_status() == 0
        xs.append(xd.cpu().numpy())
        if mode == 3:
            bd = torch.from_numpy(w.b).to(dev)
            r = P.gmres(bd, torch.zeros_like(bd), tol=1e-8, restart=50, maxit=3000)
            assert r["status"] == 0 and abs(r["iters"] - ro["iters"]) <= 1, (r["iters"], ro["iters"])
        P.close()
    assert np.linalg.norm(xs[0] - xs[1]) <= 1e-5 * np.linalg.norm(xs[0])
    assert np.linalg.norm(xs[1] - xr) <= 1e-4 * np.linalg.norm(xr)


def test_tf32_full_size_iterations(full):
    """DD_FP32_TF32 at full size: FGMRES(50) reaches 1e-8 within +-2
    iterations of the oracle's count (true residual recomputed on the host)."""
    torch, dd, dev, w, agg, y, xr, ro = full
    P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=agg, prec=dd.DD_FP32_TF32)
    bd = torch.from_numpy(w.b).to(dev)
    xd = torch.zeros_like(bd)
    r = P.gmres(bd, xd, tol=1e-8, restart=50, maxit=3000)
    P.close()
    print(f"DD_FP32_TF32: {r['iters']} iterations, oracle {ro['iters']}")
    assert r["status"] == 0 and abs(r["iters"] - ro["iters"]) <= 2, (r["iters"], ro["iters"])
    assert np.linalg.norm(w.b - O.spmv(w.A, xd.cpu().numpy())) <= 1e-8 * np.linalg.norm(w.b)
