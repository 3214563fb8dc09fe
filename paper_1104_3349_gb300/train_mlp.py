"""Training of the learned Schur correction's network on the GPU (dd_mlp_*),
and the weight file it writes (the format in include/dd.h; dd_setup with
DD_LEARNED reads it).

The data set is a file of raw features X (n x 14) and targets t (n).  Rows
carry the index of the problem they come from, and the last `val_frac` of
the problems are held out.  Features are standardised with the training
rows' mean and standard deviation.  Targets are divided by out_scale, the
training targets' standard deviation.  Training is Adam on mini-batches of a
seeded permutation of the training rows, with a cosine learning-rate decay.
Every gradient is summed in a fixed order on the device, so a run is
reproducible.

  python -m paper_1104_3349_gb300.train_mlp --data data.npz --out weights.bin
      [--epochs 30] [--batch 16384] [--lr 3e-3] [--resume weights.bin]
"""
from __future__ import annotations

import argparse
import json
import math
import struct
import sys
import time

import numpy as np

from . import dd

MAGIC = b"DDMLPW01"


def fnv1a64(data: bytes) -> int:
    h = 0xCBF29CE484222325
    for b in data:
        h ^= b
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def write_weights(path, out_scale, mean, std, params, adam_m=None, adam_v=None, step=0):
    z = np.zeros(dd.MLP_NPARAM, np.float32)
    body = bytearray(MAGIC)
    body += struct.pack("<III", 1, dd.MLP_IN, dd.MLP_HIDDEN)
    body += struct.pack("<f", float(out_scale))
    for arr, k in ((mean, dd.MLP_IN), (std, dd.MLP_IN), (params, dd.MLP_NPARAM),
                   (z if adam_m is None else adam_m, dd.MLP_NPARAM), (z if adam_v is None else adam_v, dd.MLP_NPARAM)):
        a = np.ascontiguousarray(arr, np.float32)
        if a.shape != (k,):
            raise ValueError("bad array size for the weight file")
        body += a.tobytes()
    body += struct.pack("<q", int(step))
    body += struct.pack("<Q", fnv1a64(bytes(body)))
    with open(path, "wb") as f:
        f.write(bytes(body))


def read_weights(path):
    raw = open(path, "rb").read()
    body = raw[:-8]
    if struct.unpack("<Q", raw[-8:])[0] != fnv1a64(body) or body[:8] != MAGIC:
        raise ValueError("bad weight file")
    if struct.unpack_from("<III", body, 8) != (1, dd.MLP_IN, dd.MLP_HIDDEN):
        raise ValueError("unsupported weight file")
    o = 20
    out_scale = struct.unpack_from("<f", body, o)[0]
    o += 4
    arrs = []
    for k in (dd.MLP_IN, dd.MLP_IN, dd.MLP_NPARAM, dd.MLP_NPARAM, dd.MLP_NPARAM):
        arrs.append(np.frombuffer(body, np.float32, k, o).copy())
        o += 4 * k
    step = struct.unpack_from("<q", body, o)[0]
    return dict(out_scale=out_scale, mean=arrs[0], std=arrs[1], params=arrs[2], adam_m=arrs[3], adam_v=arrs[4],
                step=step)


def init_params(seed=0):
    """He-normal first layer, small second layer, zero biases."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, math.sqrt(2.0 / dd.MLP_IN), (dd.MLP_HIDDEN, dd.MLP_IN))
    w2 = rng.normal(0.0, math.sqrt(1.0 / dd.MLP_HIDDEN), dd.MLP_HIDDEN)
    return np.concatenate([W1.ravel(), np.zeros(dd.MLP_HIDDEN), w2, [0.0]]).astype(np.float32)


def train(X, t, problem, epochs=30, batch=16384, lr=3e-3, val_frac=0.1, seed=0, resume=None, log=None):
    """Returns (weights dict, history list).  X, t, problem: numpy arrays."""
    nprob = int(problem.max()) + 1
    nval = max(1, int(round(val_frac * nprob)))
    tr = problem < nprob - nval
    Xtr, ttr = X[tr].astype(np.float64), t[tr].astype(np.float64)
    mean = Xtr.mean(axis=0)
    std = Xtr.std(axis=0)
    std = np.where(std > 1e-12, std, 1.0)
    out_scale = float(ttr.std()) or 1.0
    if resume is not None:
        mean, std, out_scale = resume["mean"].astype(np.float64), resume["std"].astype(np.float64), resume["out_scale"]
    rng = np.random.default_rng(seed)
    order = rng.permutation(int(tr.sum()))
    Xn_tr = ((Xtr - mean) / std)[order].astype(np.float32)
    y_tr = (ttr / out_scale)[order].astype(np.float32)
    Xn_va = ((X[~tr].astype(np.float64) - mean) / std).astype(np.float32)
    y_va = (t[~tr].astype(np.float64) / out_scale).astype(np.float32)
    ntr, nva = len(y_tr), len(y_va)
    M = dd.MLP(resume["params"] if resume is not None else init_params(seed))
    if resume is not None:
        M.set_adam(resume["adam_m"], resume["adam_v"], resume["step"])
    M.set_data(np.concatenate([Xn_tr, Xn_va]), np.concatenate([y_tr, y_va]))
    hist = []
    nb = (ntr + batch - 1) // batch
    total = epochs * nb
    k = 0
    t0 = time.time()
    base_val = float(np.mean(y_va.astype(np.float64) ** 2))
    for ep in range(epochs):
        for q in range(nb):
            lr_k = 0.5 * lr * (1.0 + math.cos(math.pi * k / total))
            M.adam_step(q * batch, min(ntr, (q + 1) * batch), lr_k)
            k += 1
        ltr, _ = M.loss_grad(0, ntr)
        lva, _ = M.loss_grad(ntr, ntr + nva)
        hist.append(dict(epoch=ep + 1, train_loss=ltr, val_loss=lva, seconds=round(time.time() - t0, 2)))
        if log:
            print(json.dumps(hist[-1]), file=log, flush=True)
    p, m, v, step = M.get()
    M.close()
    w = dict(out_scale=out_scale, mean=mean.astype(np.float32), std=std.astype(np.float32), params=p, adam_m=m,
             adam_v=v, step=step, val_zero_loss=base_val, n_train=ntr, n_val=nva)
    return w, hist


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--data", required=True)
    ap.add_argument("--out", required=True)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--resume", default=None)
    a = ap.parse_args(argv)
    dd.build()
    dd.load()
    z = np.load(a.data)
    resume = read_weights(a.resume) if a.resume else None
    w, hist = train(z["X"], z["t"], z["problem"], epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed,
                    resume=resume, log=sys.stdout)
    write_weights(a.out, w["out_scale"], w["mean"], w["std"], w["params"], w["adam_m"], w["adam_v"], w["step"])
    print(json.dumps(dict(out=a.out, n_train=w["n_train"], n_val=w["n_val"], val_zero_loss=w["val_zero_loss"],
                          final=hist[-1] if hist else None, steps=int(w["step"]))), flush=True)


if __name__ == "__main__":
    main()
