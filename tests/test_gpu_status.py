"""The device status word and the timeout path of the apply's bounded waits.

The sweep kernels wait on their own bulk copies with bounded mbarrier waits.
A test hook (dd_set_wait_limit) makes the first wait of every sweep CTA give
up at once; the drain of the copies in flight keeps its full bound, so no CTA
leaves with a copy outstanding and the context stays usable.  The tests check
that the timeout is reported (dd_check_status, gmres_solve), that the word is
cleared, and that the next normal apply and solve again match the oracle.
"""
import numpy as np
import pytest

import oracle as O
from paper_1104_3349_gb300 import workload as W

pytestmark = pytest.mark.gpu

DD_ERR_TIMEOUT = 7


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1104_3349_gb300 import dd
    dd.build()
    dd.load()
    w = W.cavity32()
    R = O.OracleDD(w.A, w.part, w.m, O.MSCE_INF, perm=w.perm, agg_offsets=w.agg)
    return torch, dd, torch.device("cuda:0"), w, R


@pytest.mark.parametrize("cl", [1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1])
def test_timeout_is_reported_and_cleared(env, prec, cl):
    """cl = 2: both CTAs of every cluster stop after the same cluster barrier;
    cl = 3 (the lookahead split): both finish the task's message exchange,
    agree on the outcome at its end, and the next apply is unaffected."""
    torch, dd, dev, w, R = env
    P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=w.agg, prec=prec, sweep_cluster=cl)
    y = W.uniform(1, w.A.n)
    yd = torch.from_numpy(y).to(dev)
    xd = torch.zeros_like(yd)
    assert P.check_status() == 0
    P.set_wait_limit(0)
    P.apply(yd, xd)  # asynchronous: the failure is recorded, not returned
    assert P.check_status() == DD_ERR_TIMEOUT
    assert P.check_status() == 0  # read and cleared
    bd = torch.from_numpy(w.b).to(dev)
    with pytest.raises(dd.DDError) as e:
        P.gmres(bd, torch.zeros_like(bd), tol=1e-8, restart=50)
    assert e.value.status == DD_ERR_TIMEOUT
    # the normal bound again: the apply and the solve are unaffected
    P.set_wait_limit(0xFFFFFFFF)
    xd.fill_(float("nan"))
    P.apply(yd, xd)
    assert P.check_status() == 0
    xr = R.apply(y)
    err = np.linalg.norm(xd.cpu().numpy() - xr) / np.linalg.norm(xr)
    assert err <= (1e-10 if prec == 0 else 1e-4), err
    r = P.gmres(bd, torch.zeros_like(bd), tol=1e-8, restart=50)
    assert r["status"] == 0 and r["relres"] <= 1e-8
    P.close()


def test_timeout_in_noalloc_apply(env):
    torch, dd, dev, w, R = env
    P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=w.agg)
    yd = torch.from_numpy(W.uniform(1, w.A.n)).to(dev)
    xd = torch.zeros_like(yd)
    P.set_wait_limit(0)
    P.apply_noalloc(yd, xd)
    assert P.check_status() == DD_ERR_TIMEOUT
    P.set_wait_limit(0xFFFFFFFF)
    P.apply_noalloc(yd, xd)
    assert P.check_status() == 0
    xr = R.apply(W.uniform(1, w.A.n))
    assert np.linalg.norm(xd.cpu().numpy() - xr) <= 1e-10 * np.linalg.norm(xr)
    P.close()
