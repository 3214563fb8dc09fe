"""Batching, CUDA graphs and the autotuner against the CPU oracle.

A batch is set up as one block-diagonal system.  Its B is then block
diagonal with one block B_q per system, so the batched apply must equal every
system's own oracle apply, concatenated.  The lock-step batched FGMRES must
give each system the iterations of a solve of that system alone: the
oracle's count +-1, with true residual <= 1e-8.

The small batch has 48 systems and 1664 subdomains.  That is more subdomains
than resident sweep CTAs, so the sweeps run from the persistent
longest-first task lists.  The graph path replays the same kernels, so its
residual history matches the plain launches.  The autotuner only chooses
launch parameters, so the apply stays at the FP64 bar.
"""
import numpy as np
import pytest

import oracle as O
from paper_1104_3349_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1104_3349_gb300 import dd
    dd.build()
    dd.load()
    return torch, dd, torch.device("cuda:0")


@pytest.fixture(scope="module")
def small_batch():
    return W.batch_small()


def _systems(ws):
    return [(w.A, w.part, w.m, w.perm, w.agg) for w in ws]


@pytest.mark.parametrize("cl", [1, 2, 3])
def test_batched_apply_matches_each_oracle(env, small_batch, cl):
    """1664 subdomains on persistent task lists, one CTA or a 2-CTA cluster each."""
    torch, dd, dev = env
    ws = small_batch
    P = dd.DDBatch(_systems(ws), "msce_inf", sweep_cluster=cl)
    st = P.stats()
    assert st["sweep_cluster"] == cl
    assert st["batch"] == len(ws) and st["m"] == sum(w.m for w in ws)
    assert st["sweep_grid"] < st["m"]  # the persistent task lists are in use
    ys = [W.uniform(1 + q, w.A.n) for q, w in enumerate(ws)]
    yd = torch.from_numpy(np.concatenate(ys)).to(dev)
    xd = torch.full_like(yd, float("nan"))
    P.apply(yd, xd)
    torch.cuda.synchronize()
    x = xd.cpu().numpy()
    off = 0
    for q, w in enumerate(ws):
        R = O.OracleDD(w.A, w.part, w.m, O.MSCE_INF, perm=w.perm, agg_offsets=w.agg)
        xr = R.apply(ys[q])
        xs = x[off:off + w.A.n]
        off += w.A.n
        assert np.all(np.isfinite(xs))
        assert np.linalg.norm(xs - xr) <= 1e-10 * np.linalg.norm(xr), q
    P.close()


@pytest.mark.parametrize("use_graph,cl", [(False, 0), (True, 0), (False, 3)])
def test_batched_gmres_matches_each_oracle(env, small_batch, use_graph, cl):
    """cl = 3: the lookahead sweeps on persistent task lists, with the
    systems that have converged skipped by both CTAs of every pair."""
    torch, dd, dev = env
    ws = small_batch
    P = dd.DDBatch(_systems(ws), "msce_inf", max_restart=30, use_graph=use_graph, sweep_cluster=cl)
    if cl:
        assert P.stats()["sweep_cluster"] == cl
    bs = [torch.from_numpy(w.b).to(dev) for w in ws]
    xs = [torch.zeros_like(b) for b in bs]
    rc, out = P.gmres(bs, xs, tol=1e-8, restart=30)
    assert rc == 0
    for q, w in enumerate(ws):
        R = O.OracleDD(w.A, w.part, w.m, O.MSCE_INF, perm=w.perm, agg_offsets=w.agg)
        ro = R.fgmres(w.b, tol=1e-8, restart=30)
        assert out[q]["status"] == 0
        assert abs(out[q]["iters"] - ro["iters"]) <= 1, (q, out[q]["iters"], ro["iters"])
        x = xs[q].cpu().numpy()
        r = w.b - O.spmv(w.A, x)
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(w.b) * (1 + 1e-6), q
    if use_graph:
        assert P.stats()["graphs"] == 30
    P.close()


def test_batched_fp32_preconditioner_converges(env, small_batch):
    torch, dd, dev = env
    ws = small_batch
    P = dd.DDBatch(_systems(ws), "msce_inf", prec=dd.DD_FP32, max_restart=30)
    bs = [torch.from_numpy(w.b).to(dev) for w in ws]
    xs = [torch.zeros_like(b) for b in bs]
    rc, out = P.gmres(bs, xs, tol=1e-8, restart=30)
    assert rc == 0
    for q, w in enumerate(ws):
        assert out[q]["relres"] <= 1e-8
        r = w.b - O.spmv(w.A, xs[q].cpu().numpy())
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(w.b) * (1 + 1e-6), q
    P.close()


def test_batched_exact_converges_in_one_step(env):
    torch, dd, dev = env
    ws = W.batch_small(count=6, seed=4200)
    P = dd.DDBatch(_systems(ws), "exact", max_restart=10)
    bs = [torch.from_numpy(w.b).to(dev) for w in ws]
    xs = [torch.zeros_like(b) for b in bs]
    rc, out = P.gmres(bs, xs, tol=1e-8, restart=10)
    assert rc == 0
    assert [o["iters"] for o in out] == [1] * len(ws)
    P.close()


def test_batched_rejects_mscn(env, small_batch):
    torch, dd, dev = env
    with pytest.raises(dd.DDError) as ei:
        dd.DDBatch(_systems(small_batch[:3]), "mscn")
    assert ei.value.status == 1


def test_graph_gmres_equals_plain(env):
    # LUM: its setup has no atomic accumulation, so two handles hold
    # bit-identical factors and the two solves can be compared bit for bit
    torch, dd, dev = env
    w = W.cavity32()
    b = torch.from_numpy(w.b).to(dev)
    res = []
    for g in (False, True):
        P = dd.DD(w.A, w.part, w.m, "lum", perm=w.perm, agg_offsets=w.agg, use_graph=g)
        x = torch.zeros_like(b)
        r1 = P.gmres(b, x)
        x2 = torch.zeros_like(b)
        r2 = P.gmres(b, x2)  # second solve replays the graphs captured by the first
        assert r1["status"] == 0 and r2["iters"] == r1["iters"]
        res.append((r1, x.cpu().numpy()))
        if g:
            st = P.stats()
            assert st["graphs"] == min(50, r1["iters"])
        P.close()
    (a, xa), (b_, xb) = res
    assert a["iters"] == b_["iters"]
    np.testing.assert_array_equal(a["history"], b_["history"])
    np.testing.assert_array_equal(xa, xb)


@pytest.mark.parametrize("prec", [0, 1])
def test_autotuned_apply_matches_oracle(env, prec):
    torch, dd, dev = env
    w = W.cavity32()
    P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=w.agg, prec=prec, autotune=True)
    st = P.stats()
    assert st["tuned"] >= 1 and st["tuned_us"] > 0 and st["stage_bytes"] > 0
    R = O.OracleDD(w.A, w.part, w.m, O.MSCE_INF, perm=w.perm, agg_offsets=w.agg)
    y = W.uniform(1, w.A.n)
    yd = torch.from_numpy(y).to(dev)
    xd = torch.full_like(yd, float("nan"))
    P.apply(yd, xd)
    torch.cuda.synchronize()
    xr = R.apply(y)
    err = np.linalg.norm(xd.cpu().numpy() - xr) / np.linalg.norm(xr)
    assert err <= (1e-10 if prec == 0 else 1e-4), err
    P.close()
