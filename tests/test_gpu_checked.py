"""The checked build (libdd_checked.so, -DDD_CHECKED) on the small parity
cases: its device checks of indices, sizes and bulk-copy alignment record
DD_ERR_CHECK instead of faulting.  On correct inputs none may fire, and the
results must equal the oracle's as in the plain build.  The library is
loaded in a child process (a process loads one libdd)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
import oracle as O
from paper_1104_3349_gb300 import dd, workload as W
dd.build(checked=True)
lib = dd.load()
assert lib._name.endswith("libdd_checked.so"), lib._name
dev = torch.device("cuda:0")
cases = [("msce_inf", O.MSCE_INF, {{}}), ("lum", O.LUM, {{}}), ("exact", O.EXACT, {{}}),
         ("omscn", O.OMSCN, dict(overlap=64)), ("msce", O.MSCE, dict(radius=2))]
for grid, m, sz in ((32, 4, 64), (20, 4, 33), (12, 8, 16)):
    w = W.make_workload("t", grid, 0.02, 1.0, W.WIND_FOURIER, grid, m, sz=sz) if grid != 32 else W.cavity32()
    y = W.uniform(1, w.A.n)
    yd = torch.from_numpy(y).to(dev)
    for name, ko, kw in cases:
        agg = None if name == "exact" else w.agg
        try:
            R = O.OracleDD(w.A, w.part, w.m, ko, perm=w.perm, agg_offsets=agg, **kw)
        except O.OracleError:
            continue
        xr = R.apply(y)
        for prec in (0, 1):
            for cl in (1, 2, 3):
                P = dd.DD(w.A, w.part, w.m, name, perm=w.perm, agg_offsets=agg, prec=prec, sweep_cluster=cl, **kw)
                xd = torch.full_like(yd, float("nan"))
                P.apply(yd, xd)
                st = P.check_status()
                assert st == 0, (grid, name, prec, cl, st, lib.dd_last_error(P._h))
                err = np.linalg.norm(xd.cpu().numpy() - xr) / np.linalg.norm(xr)
                assert err <= (1e-10 if prec == 0 else 1e-4), (grid, name, prec, cl, err)
                P.close()
w = W.cavity32()
P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=w.agg)
bd = torch.from_numpy(w.b).to(dev)
r = P.gmres(bd, torch.zeros_like(bd), tol=1e-8, restart=50)
assert r["status"] == 0 and r["relres"] <= 1e-8, r
ys = torch.empty_like(bd)
P.spmv(bd, ys)
assert P.check_status() == 0
assert np.abs(ys.cpu().numpy() - O.spmv(w.A, w.b)).max() <= 1e-14 * np.abs(w.b).max() * 10
print("CHECKED OK")
'''


def test_checked_build_runs_the_parity_cases_clean():
    env = dict(os.environ, DD_CHECKED="1")
    p = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=900)
    assert p.returncode == 0 and "CHECKED OK" in p.stdout, (p.stdout[-2000:], p.stderr[-3000:])
