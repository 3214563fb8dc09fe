"""Training set of the learned Schur correction, written by the oracle
(TEST INFRASTRUCTURE: a committed script that calls only oracle/ and the
seeded input generator).

Problem i, with seed = seed0 + i:
  - a 64 x 64 MAC Oseen system, nu log-uniform in [1e-3, 1e-2];
  - wall stretching ratio r uniform in [1, 1.03];
  - the seeded 8-mode Fourier wind, 4 subdomains, aggregates of nominal size 64.
The two uniforms come from the workload's xoshiro stream with that seed.
For every entry of every pattern P_i the file holds its 14 raw features
(oracle.learned.features) and its target S_ii(r, c) - G(r, c) from the
oracle's MSCE_INF blocks.

  python -m oracle.learned_data --count 2000 --out data.npz [--procs 16]
"""
from __future__ import annotations

import argparse
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)


def problem_spec(seed: int):
    from paper_1104_3349_gb300 import workload as W
    u = W.uniform(seed, 2, 0.0, 1.0)
    nu = math.exp(math.log(1e-3) + (math.log(1e-2) - math.log(1e-3)) * float(u[0]))
    return dict(grid=64, nu=nu, stretch=1.0 + 0.03 * float(u[1]), m=4, sz=64, wind_seed=seed)


def one_problem(seed: int):
    """(features, targets) of every learned-pattern entry of problem `seed`."""
    import oracle as O
    from oracle import learned as L
    from paper_1104_3349_gb300 import workload as W
    sp = problem_spec(seed)
    A, _ = W.mac_system(sp["grid"], sp["nu"], sp["stretch"], W.WIND_FOURIER, sp["wind_seed"])
    part, perm, _ = W.partition(A, sp["m"])
    agg = W.aggregates(A, part, perm, sp["sz"])
    R = O.OracleDD(A, part, sp["m"], O.MSCE_INF, perm=perm, agg_offsets=agg)
    ents, X = L.features(A, part, perm, agg)
    t = L.targets(R, ents, A, part, perm, agg)
    R.close()
    return X.astype(np.float32), t.astype(np.float32)


def _init():
    import oracle as O
    O.set_threads(1)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=2000)
    ap.add_argument("--seed0", type=int, default=5000)
    ap.add_argument("--out", required=True)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args(argv)
    import oracle as O
    O.build()
    from paper_1104_3349_gb300 import workload as W
    W.build()
    t0 = time.time()
    seeds = list(range(a.seed0, a.seed0 + a.count))
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.procs, initializer=_init) as pool:
        res = pool.map(one_problem, seeds, chunksize=4)
    X = np.concatenate([r[0] for r in res])
    t = np.concatenate([r[1] for r in res])
    prob = np.concatenate([np.full(len(r[1]), i, np.int32) for i, r in enumerate(res)])
    np.savez(a.out, X=X, t=t, problem=prob, seeds=np.asarray(seeds, np.int32))
    print(f"{a.count} problems, {len(t)} entries, {time.time() - t0:.1f} s -> {a.out}", flush=True)


if __name__ == "__main__":
    main()
