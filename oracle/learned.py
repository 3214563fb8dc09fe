"""Oracle of the learned Schur correction (TEST INFRASTRUCTURE ONLY).

The paper has no learned part.  This module is the plain FP64 reference of
the extension built on the paper's lumped approximation (LUM, Ŝ = blkDiag(G_ii),
Definition of B_LUM) and of its MSCE_INF blocks (Algorithm 1, "exact"
Schur complement restricted to each aggregate).  Only tests, smoke() and
bench.py's CPU-baseline leg import it.

Definitions (P^T C P = [D E; F G] as in Section 1):
  - an aggregate R_i (Section 3.2, consecutive interface indices);
  - the pattern P_i = {(r, c) in R_i x R_i : G(r, c) != 0, or F(r, k) E(k, c)
    != 0 for some interior k, or r == c};
  - the learned block Ŝ_L(R_i, R_i) = G(R_i, R_i) + Δ, where Δ is nonzero on P_i
    only and Δ(r, c) = out_scale * MLP(normalise(x(r, c)));
  - the training target on P_i is the MSCE_INF correction S_ii(r, c) - G(r, c),
    where S_ii = G_ii - sum_j F_ij A_j^-1 E_ji is the exact local block.

Features x(r, c), 14 per entry.  They are scale-free because every row of C
is scaled by its largest magnitude.  d_k = D(k, k), and Dinv_k = 1 / d_k
where d_k != 0, else 0.
   0 G(r,c)            1 G(c,r)            2 (F E)(r,c)        3 (F Dinv E)(r,c)
   4 [r == c]          5 [G(r,r) == 0]     6 [G(c,c) == 0]     7 G(r,r)
   8 G(c,c)            9 sum_k |F(r,k)|   10 sum_k |E(k,c)|   11 #{k: F(r,k)!=0}/8
  12 #{k: E(k,c)!=0}/8 13 (F Dinv E)(r,r)

The network is 14 -> 64 (ReLU) -> 1, with parameters packed as
[W1 (64 x 14, row-major), b1 (64), w2 (64), b2 (1)].  It uses BF16 weights
and BF16 inputs: every weight and every normalised feature is rounded to
BF16, round to nearest even.  The arithmetic here is FP64.  The loss is the
mean of (out - t / out_scale)^2 over the entries.

Weight file, all little-endian:
  magic "DDMLPW01" | u32 version = 1 | u32 n_in = 14 | u32 n_hidden = 64 |
  f32 out_scale | f32 mean[14] | f32 std[14] | f32 params[1025] |
  f32 adam_m[1025] | f32 adam_v[1025] | i64 step |
  u64 FNV-1a hash of all preceding bytes.
"""
from __future__ import annotations

import struct

import numpy as np
import scipy.sparse as sp

N_IN, N_HID = 14, 64
NPARAM = N_HID * N_IN + 2 * N_HID + 1
MAGIC = b"DDMLPW01"


# ---------------------------------------------------------------------------
# blocks of P^T C P and the features
# ---------------------------------------------------------------------------
def permuted_blocks(A, part, perm):
    """D's diagonal, and F, E, G as scipy CSR matrices in the permuted numbering."""
    C = sp.csr_matrix((np.asarray(A.val, np.float64), np.asarray(A.col), np.asarray(A.rowptr)),
                      shape=(A.n, A.n))
    perm = np.asarray(perm)
    nI = int((np.asarray(part) >= 0).sum())
    Cp = C[perm][:, perm].tocsr()
    Cp.eliminate_zeros()
    d = Cp[:nI, :nI].diagonal()
    F = Cp[nI:, :nI].tocsr()
    E = Cp[:nI, nI:].tocsc()
    G = Cp[nI:, nI:].tocsr()
    return d, F, E, G


def features(A, part, perm, agg):
    """Entries (aggregate, local row, local column) of every P_i, in that order,
    and their 14 raw features (FP64)."""
    d, F, E, G = permuted_blocks(A, part, perm)
    agg = np.asarray(agg, np.int64)
    dinv = np.where(d != 0, 1.0 / np.where(d != 0, d, 1.0), 0.0)
    Er = E.tocsr()
    Fb = F.copy()
    Fb.data[:] = 1.0
    Eb = Er.copy()
    Eb.data[:] = 1.0
    gdiag = G.diagonal()
    fabs = np.asarray(abs(F).sum(axis=1)).ravel()
    eabs = np.asarray(abs(E).sum(axis=0)).ravel()
    fcnt = np.diff(F.indptr).astype(np.float64)
    ecnt = np.diff(E.indptr).astype(np.float64)
    FDE = (F @ sp.diags(dinv) @ Er).tocsr()
    fde_diag = FDE.diagonal()
    ents, rows = [], []
    for a in range(len(agg) - 1):
        g0, g1 = int(agg[a]), int(agg[a + 1])
        p = g1 - g0
        Gb = G[g0:g1, g0:g1].toarray()
        FEb = (F[g0:g1] @ Er[:, g0:g1]).toarray()
        FDEb = FDE[g0:g1, g0:g1].toarray()
        struct_fe = (Fb[g0:g1] @ Eb[:, g0:g1]).toarray() > 0
        mask = (Gb != 0) | struct_fe | np.eye(p, dtype=bool)
        r, c = np.nonzero(mask)
        R_, C_ = g0 + r, g0 + c
        X = np.stack([Gb[r, c], Gb[c, r], FEb[r, c], FDEb[r, c], (r == c).astype(np.float64),
                      (gdiag[R_] == 0).astype(np.float64), (gdiag[C_] == 0).astype(np.float64),
                      gdiag[R_], gdiag[C_], fabs[R_], eabs[C_], fcnt[R_] / 8.0, ecnt[C_] / 8.0,
                      fde_diag[R_]], axis=1)
        ents.append(np.stack([np.full(len(r), a), r, c], axis=1))
        rows.append(X)
    if not ents:
        return np.zeros((0, 3), np.int32), np.zeros((0, N_IN))
    return np.concatenate(ents).astype(np.int32), np.concatenate(rows)


def targets(R, ents, A, part, perm, agg):
    """S_ii(r, c) - G(r, c) on the entries, from the oracle's MSCE_INF blocks R."""
    _, _, _, G = permuted_blocks(A, part, perm)
    agg = np.asarray(agg, np.int64)
    t = np.zeros(len(ents))
    for a in range(len(agg) - 1):
        sel = np.nonzero(ents[:, 0] == a)[0]
        if len(sel) == 0:
            continue
        S = R.schur_block(a)
        g0 = int(agg[a])
        r, c = ents[sel, 1], ents[sel, 2]
        t[sel] = S[r, c] - np.asarray(G[g0 + r, g0 + c]).ravel()
    return t


# ---------------------------------------------------------------------------
# the network (FP64 reference of the BF16-weight forward and its backprop)
# ---------------------------------------------------------------------------
def bf16(x):
    """Round to BF16, nearest even (the value returned as float64)."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def unpack(params):
    p = np.asarray(params, np.float64)
    W1 = p[:N_HID * N_IN].reshape(N_HID, N_IN)
    b1 = p[N_HID * N_IN:N_HID * N_IN + N_HID]
    w2 = p[N_HID * N_IN + N_HID:N_HID * N_IN + 2 * N_HID]
    b2 = p[-1]
    return W1, b1, w2, b2


def forward(params, X):
    """out(e) = w2 . relu(W1 x_e + b1) + b2 for every row x_e of X."""
    W1, b1, w2, b2 = unpack(params)
    Z = X @ W1.T + b1
    H = np.maximum(Z, 0.0)
    return H @ w2 + b2, (Z, H)


def loss_grad(params, X, y):
    """Mean squared error and its gradient by backpropagation, packed like params."""
    W1, b1, w2, b2 = unpack(params)
    out, (Z, H) = forward(params, X)
    n = len(y)
    r = out - y
    loss = float(np.mean(r * r))
    dout = 2.0 * r / n
    gw2 = H.T @ dout
    gb2 = dout.sum()
    dZ = np.outer(dout, w2) * (Z > 0)
    gW1 = dZ.T @ X
    gb1 = dZ.sum(axis=0)
    return loss, np.concatenate([gW1.ravel(), gb1, gw2, [gb2]])


def normalise(X, mean, std):
    return (np.asarray(X, np.float64) - mean) / std


def predict(wts, X):
    """Δ on raw features X with the weights of a file (BF16 inputs and weights)."""
    Xn = bf16(normalise(X, wts["mean"], wts["std"]))
    out, _ = forward(bf16(wts["params"]), Xn)
    return wts["out_scale"] * out


# ---------------------------------------------------------------------------
# weight file
# ---------------------------------------------------------------------------
def fnv1a64(data: bytes) -> int:
    h = 0xCBF29CE484222325
    for b in data:
        h ^= b
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def read_weights(path):
    raw = open(path, "rb").read()
    body, tail = raw[:-8], raw[-8:]
    if struct.unpack("<Q", tail)[0] != fnv1a64(body):
        raise ValueError("weight file checksum mismatch")
    if body[:8] != MAGIC:
        raise ValueError("not a weight file")
    ver, nin, nh = struct.unpack_from("<III", body, 8)
    if (ver, nin, nh) != (1, N_IN, N_HID):
        raise ValueError("unsupported weight file version or shape")
    off = 20
    out_scale = struct.unpack_from("<f", body, off)[0]
    off += 4

    def take(k):
        nonlocal off
        v = np.frombuffer(body, np.float32, k, off).astype(np.float64)
        off += 4 * k
        return v
    mean, std, params, m, v = take(N_IN), take(N_IN), take(NPARAM), take(NPARAM), take(NPARAM)
    step = struct.unpack_from("<q", body, off)[0]
    return dict(out_scale=float(out_scale), mean=mean, std=std, params=params, adam_m=m, adam_v=v, step=step)


# ---------------------------------------------------------------------------
# the learned preconditioner (oracle): MSCE_INF blocks as the fallback, each
# replaced by G_ii + Delta when that block passes the pivot test
# ---------------------------------------------------------------------------
def learned_oracle(A, part, m, perm, agg, wts, pivtol=1e-14):
    """(OracleDD, entries, Delta, indices of the aggregates that fell back)."""
    import oracle as O
    _, _, _, G = permuted_blocks(A, part, perm)
    R = O.OracleDD(A, part, m, O.MSCE_INF, perm=perm, agg_offsets=agg, pivtol=pivtol)
    ents, X = features(A, part, perm, agg)
    delta = predict(wts, X)
    agg = np.asarray(agg, np.int64)
    fell = []
    for a in range(len(agg) - 1):
        g0, g1 = int(agg[a]), int(agg[a + 1])
        blk = G[g0:g1, g0:g1].toarray()
        sel = ents[:, 0] == a
        blk[ents[sel, 1], ents[sel, 2]] += delta[sel]
        if not R.replace_block(a, blk, pivtol):
            fell.append(a)
    return R, ents, delta, fell
