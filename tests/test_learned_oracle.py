"""Pins of the learned-correction oracle (oracle/learned.py) on the CPU.

- Backpropagation is checked against central finite differences (h = 1e-6)
  on every one of the 1025 parameters, in FP64.
- The sparse feature and pattern construction is checked against dense
  numpy products of the permuted blocks of C on a tiny grid.
- The targets are checked against the brute-force Schur complement
  G - F solve(D, E), restricted to each aggregate block.
- BF16 rounding is checked against hand-picked ties and against torch's
  float32 -> bfloat16 conversion (round to nearest even).
- The weight-file format is checked across its two independent
  implementations (the package writer, the oracle reader), with a
  corrupted byte rejected.
- replace_block with the G block reproduces the oracle's own LUM apply.
"""
import os

import numpy as np
import pytest

import oracle as O
from oracle import learned as L
from paper_1104_3349_gb300 import workload as W


@pytest.fixture(scope="module")
def tiny():
    A, _ = W.mac_system(8, 1e-2, 1.02, W.WIND_FOURIER, 77)
    part, perm, _ = W.partition(A, 2)
    agg = W.aggregates(A, part, perm, 8)
    return A, part, perm, agg


def _dense_blocks(A, part, perm):
    C = np.zeros((A.n, A.n))
    for i in range(A.n):
        for k in range(A.rowptr[i], A.rowptr[i + 1]):
            C[i, A.col[k]] += A.val[k]
    Cp = C[np.ix_(perm, perm)]
    nI = int((part >= 0).sum())
    return Cp[:nI, :nI], Cp[:nI, nI:], Cp[nI:, :nI], Cp[nI:, nI:]


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(3)
    p = rng.normal(0, 0.5, L.NPARAM)
    X = rng.normal(0, 1, (24, L.N_IN))
    y = rng.normal(0, 1, 24)
    _, g = L.loss_grad(p, X, y)
    h = 1e-6
    fd = np.zeros_like(p)
    for q in range(L.NPARAM):
        e = np.zeros_like(p)
        e[q] = h
        fd[q] = (L.loss_grad(p + e, X, y)[0] - L.loss_grad(p - e, X, y)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))


def test_features_match_dense_products(tiny):
    A, part, perm, agg = tiny
    D, E, F, G = _dense_blocks(A, part, perm)
    d = np.diag(D)
    dinv = np.where(d != 0, 1.0 / np.where(d != 0, d, 1), 0.0)
    FE = F @ E
    FDE = F @ np.diag(dinv) @ E
    SFE = (F != 0).astype(float) @ (E != 0).astype(float)
    ents, X = L.features(A, part, perm, agg)
    want = []
    for a in range(len(agg) - 1):
        g0, g1 = agg[a], agg[a + 1]
        for r in range(g0, g1):
            for c in range(g0, g1):
                if G[r, c] != 0 or SFE[r, c] > 0 or r == c:
                    want.append((a, r - g0, c - g0))
    assert [tuple(e) for e in ents.tolist()] == want
    for (a, r, c), x in zip(ents, X):
        R, Cc = agg[a] + r, agg[a] + c
        ref = [G[R, Cc], G[Cc, R], FE[R, Cc], FDE[R, Cc], float(r == c), float(G[R, R] == 0),
               float(G[Cc, Cc] == 0), G[R, R], G[Cc, Cc], np.abs(F[R]).sum(), np.abs(E[:, Cc]).sum(),
               np.count_nonzero(F[R]) / 8, np.count_nonzero(E[:, Cc]) / 8, FDE[R, R]]
        np.testing.assert_allclose(x, ref, rtol=1e-12, atol=1e-14)


def test_targets_match_bruteforce_schur(tiny):
    A, part, perm, agg = tiny
    D, E, F, G = _dense_blocks(A, part, perm)
    S = G - F @ np.linalg.solve(D, E)
    m = int(part.max()) + 1
    R = O.OracleDD(A, part, m, O.MSCE_INF, perm=perm, agg_offsets=agg)
    ents, _ = L.features(A, part, perm, agg)
    t = L.targets(R, ents, A, part, perm, agg)
    for (a, r, c), tv in zip(ents, t):
        Rr, Cc = agg[a] + r, agg[a] + c
        assert abs(tv - (S[Rr, Cc] - G[Rr, Cc])) <= 1e-10 * (1 + abs(S[Rr, Cc]))
    R.close()


def test_bf16_rounding():
    one = 1.0
    assert L.bf16([one])[0] == 1.0
    assert L.bf16([1 + 2 ** -8])[0] == 1.0                    # tie, even neighbour below
    assert L.bf16([1 + 3 * 2 ** -8])[0] == 1 + 2 ** -6        # tie, even neighbour above
    assert L.bf16([1 + 2 ** -8 + 2 ** -20])[0] == 1 + 2 ** -7  # just above the tie
    torch = pytest.importorskip("torch")
    v = np.random.default_rng(5).normal(0, 10, 4096).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(L.bf16(v), ref)


def test_weight_file_formats_agree(tmp_path):
    from paper_1104_3349_gb300 import train_mlp as T
    rng = np.random.default_rng(9)
    p = rng.normal(0, 1, L.NPARAM).astype(np.float32)
    mean, std = rng.normal(0, 1, 14).astype(np.float32), rng.uniform(0.5, 2, 14).astype(np.float32)
    f = tmp_path / "w.bin"
    T.write_weights(str(f), 0.75, mean, std, p, p * 2, p * 3, 17)
    w = L.read_weights(str(f))
    assert w["out_scale"] == np.float32(0.75) and w["step"] == 17
    np.testing.assert_array_equal(w["params"], p.astype(np.float64))
    np.testing.assert_array_equal(w["adam_v"], (p * 3).astype(np.float64))
    np.testing.assert_array_equal(w["std"], std.astype(np.float64))
    raw = bytearray(f.read_bytes())
    raw[100] ^= 1
    f.write_bytes(bytes(raw))
    with pytest.raises(ValueError):
        L.read_weights(str(f))


def test_replace_block_with_g_reproduces_lum():
    w = W.cavity32()
    R = O.OracleDD(w.A, w.part, w.m, O.MSCE_INF, perm=w.perm, agg_offsets=w.agg)
    Lm = O.OracleDD(w.A, w.part, w.m, O.LUM, perm=w.perm, agg_offsets=w.agg)
    for i in range(len(w.agg) - 1):
        assert R.replace_block(i, Lm.schur_block(i))
    y = W.uniform(1, w.A.n)
    np.testing.assert_allclose(R.apply(y), Lm.apply(y), rtol=0, atol=1e-12 * np.abs(Lm.apply(y)).max())
    # a singular block is refused and the previous one kept
    p = w.agg[1] - w.agg[0]
    assert not R.replace_block(0, np.zeros((p, p)))
    np.testing.assert_allclose(R.apply(y), Lm.apply(y), rtol=0, atol=1e-12 * np.abs(Lm.apply(y)).max())


def _packed(W1, b1, w2, b2):
    """Parameters in the layout of the weight file: W1 (64 x 14, row-major), b1, w2, b2."""
    return np.concatenate([np.asarray(W1, np.float64).ravel(), b1, w2, [b2]])


def test_forward_matches_torch_modules():
    """The network's forward pass against torch.nn.Linear / ReLU modules built
    from the same parameters, with BF16 rounding done by torch's own
    float32 -> bfloat16 conversion."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(21)
    W1 = rng.normal(0, 0.4, (L.N_HID, L.N_IN))
    b1, w2, b2 = rng.normal(0, 0.3, L.N_HID), rng.normal(0, 0.3, L.N_HID), 0.37
    X = rng.normal(0, 1.5, (300, L.N_IN))

    def tb(a):  # BF16 round trip in torch
        return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64)
    net = torch.nn.Sequential(torch.nn.Linear(L.N_IN, L.N_HID), torch.nn.ReLU(),
                              torch.nn.Linear(L.N_HID, 1)).double()
    with torch.no_grad():
        net[0].weight.copy_(tb(W1))
        net[0].bias.copy_(tb(b1))
        net[2].weight.copy_(tb(w2).reshape(1, -1))
        net[2].bias.copy_(tb([b2]))
        ref = net(tb(X)).numpy().ravel()
    out, _ = L.forward(L.bf16(_packed(W1, b1, w2, b2)), L.bf16(X))
    assert np.abs(out - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_predict_worked_example():
    """Two entries worked by hand: standardisation (mean 0.5, std 0.25), then
    BF16 rounding of the standardised features and of the weights, the
    14 -> 64 (ReLU) -> 1 network and the output scale 10.
      W1[0,0] = 1 + 2^-8 rounds to 1;  W1[1,1] = -(1 + 3*2^-8) to -(1 + 2^-6);
      b1 = (0.5, 0.25), w2 = (2, -4), b2 = 0.125, everything else 0.
    Entry A: x0 = 0.75 + 5*2^-11 standardises to 1 + 5*2^-9, which rounds to
      1 + 2^-7 (rounding the raw feature first would give 1 + 2^-6);
      x1 = 1 standardises to 2.  h = (1.5078125, relu(-1.78125) = 0),
      out = 3.140625, Delta = 31.40625.
    Entry B: x0 = 0.25 -> -1, x1 = 0.125 -> -1.5.  h = (relu(-0.5) = 0,
      1.7734375), out = -6.96875, Delta = -69.6875."""
    W1 = np.zeros((L.N_HID, L.N_IN))
    W1[0, 0] = 1 + 2.0 ** -8
    W1[1, 1] = -(1 + 3 * 2.0 ** -8)
    b1, w2 = np.zeros(L.N_HID), np.zeros(L.N_HID)
    b1[:2] = (0.5, 0.25)
    w2[:2] = (2.0, -4.0)
    wts = dict(out_scale=10.0, mean=np.full(L.N_IN, 0.5), std=np.full(L.N_IN, 0.25),
               params=_packed(W1, b1, w2, 0.125))
    X = np.full((2, L.N_IN), 0.5)
    X[0, :2] = (0.75 + 5 * 2.0 ** -11, 1.0)
    X[1, :2] = (0.25, 0.125)
    np.testing.assert_array_equal(L.predict(wts, X), [31.40625, -69.6875])
