"""dd_apply_noalloc, the apply for callers that cannot allocate device memory.

Some callers cannot allocate device memory when they apply the
preconditioner. One example is code whose memory is all held by another
pool. Another is code in a phase where an allocation could fail or stall
the device. dd_apply_noalloc runs the same three kernels as dd_apply, but
keeps its intermediate vectors in the library's fixed device array instead
of handle buffers. These tests call it through the C ABI twice in a row and
compare each result with dd_apply's within the FP64 apply tolerance (1e-10
relative). They also check that a system larger than the array is refused.
The file sorts last, so a run that stops at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1104_3349_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1104_3349_gb300 import dd
    dd.build()
    dd.load()
    return torch, dd, torch.device("cuda:0")


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_apply_twice(env, prec):
    torch, dd, dev = env
    w = W.cavity32()
    P = dd.DD(w.A, w.part, w.m, "msce_inf", perm=w.perm, agg_offsets=w.agg, prec=prec)
    lib = dd.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (1, 2):  # two calls in a row; the second sees the first's leftovers
        y = torch.from_numpy(W.uniform(seed, w.A.n)).to(dev)
        x_ref = torch.full_like(y, float("nan"))
        x_new = torch.full_like(y, float("nan"))
        assert lib.dd_apply(P._h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x_ref.data_ptr()), stream) == 0
        rc = lib.dd_apply_noalloc(P._h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x_new.data_ptr()), stream)
        assert rc == 0, lib.dd_last_error(P._h)
        torch.cuda.synchronize()
        a, b = x_new.cpu().numpy(), x_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)
    P.close()


def test_noalloc_rejects_systems_beyond_the_scratch(env):
    torch, dd, dev = env
    n = dd.NOALLOC_MAX_ELEMS + 1
    m = 1024  # a diagonal system split into small interiors, so that setup succeeds
    A = W.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    P = dd.DD(A, (np.arange(n) % m).astype(np.int32), m, "lum", max_restart=2)
    y = torch.ones(n, dtype=torch.float64, device=dev)
    x = torch.empty_like(y)
    lib = dd.load()
    rc = lib.dd_apply_noalloc(P._h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1
    assert b"exceeds the scratch limit" in lib.dd_last_error(P._h)
    P.close()
