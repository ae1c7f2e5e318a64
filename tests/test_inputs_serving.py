"""The generated serving stream (rfdd_inputs): the inertia count that places the windows of the
variable-coefficient requests is checked against dense eigenvalues, the stored count grid against
recounting, and the stream against its own description (seeded, window counts exact, block sizes
bounded)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import rfdd_inputs as I


@pytest.mark.parametrize("N,seed", [(7, 1), (8, 3)])
def test_sym_inertia_count_matches_dense_eigenvalues(N, seed):
    A, M = I.varkappa7_pencil(N, seed)
    ev = sla.eigh(A.to_scipy().toarray(), M.to_scipy().toarray(), eigvals_only=True)
    for q in (0, 5, len(ev) // 3, len(ev) - 2):
        b = 0.5 * (ev[q] + ev[q + 1])
        assert I.sym_inertia_count(A, M, b) == q + 1
    assert I.sym_inertia_count(A, M, 0.5 * ev[0]) == 0


def test_sym_inertia_count_on_the_q1_closed_form():
    A, M = I.q1_pencil(30, 2)
    ev = I.q1_eigenvalues(30, 2)
    for q in (10, 101, 400):
        f, l = I.snap_to_gaps(ev, q, q)
        b = 0.5 * (ev[l - 1] + ev[l])
        assert I.sym_inertia_count(A, M, b) == l


def test_stored_count_grid_recounts():
    path = os.path.join(os.path.dirname(I.__file__), "varkappa_counts.json")
    table = json.load(open(path))["pencils"]
    assert {(e["N"], e["seed"]) for e in table} == set(I.VARKAPPA_POOL)
    for e in table:
        assert all(a < b for a, b in zip(e["beta"], e["beta"][1:]))
        assert all(a <= b for a, b in zip(e["count"], e["count"][1:]))
    e = next(e for e in table if e["N"] == 24 and e["seed"] == 1)
    A, M = I.varkappa7_pencil(24, 1)
    for i in (0, 11, 23):
        assert I.sym_inertia_count(A, M, e["beta"][i]) == e["count"][i]


def test_serving_stream_matches_its_description():
    s = I.serving_stream(64, seed=7)
    assert s == I.serving_stream(64, seed=7)
    kinds = {q["kind"] for q in s}
    assert kinds == {"q1_2d", "varkappa7_3d"}
    for q in s:
        p = math.prod(q["splits"])
        assert p in (4, 8, 16) and q["n"] / p <= I.MAX_BLOCK and q["n_nodes"] == 8
        assert 20 <= q["nev"] <= 400 and q["alpha"] < q["beta"]
        if q["kind"] == "q1_2d":
            assert 64 <= q["N"] <= 256
            ev = I.q1_eigenvalues(q["N"], 2)
            assert np.count_nonzero((ev > q["alpha"]) & (ev < q["beta"])) == q["nev"]
        else:
            assert (q["N"], q["seed"]) in I.VARKAPPA_POOL
    A, M, part, p = I.serving_pencil(s[0])
    assert A.n == s[0]["n"] and len(part) == A.n and p == math.prod(s[0]["splits"])
