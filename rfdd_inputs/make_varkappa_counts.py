"""Writes ``varkappa_counts.json``: exact eigenvalue counts of the 3-D variable-coefficient pencils
of the serving stream on a grid of shifts, from which the stream draws its intervals.

For each pencil (N, seed) of ``VARKAPPA_POOL`` the script finds a shift whose count is about
``TOP_COUNT`` by doubling or halving, then counts the eigenvalues below ``GRID`` shifts
beta_i = beta_top (i / GRID)^(2/3) (the count of a 3-D Laplacian-like pencil grows like
beta^(3/2), so the grid steps hold similar numbers of eigenvalues).  Each count is Sylvester's
inertia of A - beta M through a sparse symmetric factorisation (``sym_inertia_count``).  The
counts are problem data (where the intervals lie), computed without any RF-DDES arithmetic.

    python -m rfdd_inputs.make_varkappa_counts [--jobs J]

Run time on 8 cores: about 15 minutes (the 48^3 factorisations dominate).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "varkappa_counts.json")
GRID = 24
TOP_COUNT = (700, 1400)


def _count(args):
    from rfdd_inputs import sym_inertia_count, varkappa7_pencil
    N, seed, beta = args
    A, M = varkappa7_pencil(N, seed)
    return N, seed, beta, sym_inertia_count(A, M, beta)


def _top_shift(N, seed, pool):
    beta = 400.0
    for _ in range(30):
        _, _, _, c = pool.apply(_count, ((N, seed, beta),))
        if c < TOP_COUNT[0]:
            beta *= 2.0 if c < TOP_COUNT[0] / 3 else 1.3
        elif c > TOP_COUNT[1]:
            beta /= 2.0 if c > 3 * TOP_COUNT[1] else 1.3
        else:
            return beta, c
    raise RuntimeError(f"no shift with a count in {TOP_COUNT} for N={N} seed={seed}")


def main():
    from rfdd_inputs import VARKAPPA_POOL
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 4)
    args = ap.parse_args()
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.jobs) as pool:
        tops = {}
        for N, seed in VARKAPPA_POOL:
            tops[(N, seed)] = _top_shift(N, seed, pool)
        work = [(N, seed, tops[(N, seed)][0] * (i / GRID) ** (2.0 / 3.0))
                for N, seed in VARKAPPA_POOL for i in range(1, GRID + 1)]
        res = pool.map(_count, work, chunksize=1)
    table = []
    for N, seed in VARKAPPA_POOL:
        rows = sorted((b, c) for n_, s_, b, c in res if n_ == N and s_ == seed)
        counts = [c for _, c in rows]
        assert all(a <= b for a, b in zip(counts, counts[1:])), (N, seed, counts)
        table.append({"N": N, "seed": seed, "beta": [b for b, _ in rows], "count": counts})
    with open(OUT, "w") as f:
        json.dump({"pencils": table, "grid": GRID,
                   "note": "count[i] = number of eigenvalues of varkappa7_pencil(N, seed) below beta[i]"},
                  f, indent=1)
    print(f"wrote {OUT}")


if __name__ == "__main__":
    main()
