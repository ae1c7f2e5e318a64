"""Parity at the full size of the timed workload: 3D Q1 pencil on a 40^3 grid (n = 64000), 2x2x2
partition (p = 8), eigenvalues 300..501 (nev = 202), 8 midpoint nodes, mixed precision, default
options -- the configuration bench.py times.

The dense oracle cannot hold this size, so:
* a2-a5: sampled columns of S(zeta_l) (first and last interface index among them) at two nodes
  against the oracle's evaluation of the same definition with sparse LUs (schur_columns), to the
  mixed factor-level tolerance of the small cases (3e-4 of the largest entry; an FP32 sparse LU
  of these blocks is off by about 5e-8);
* a0-a10: the whole solve against what holds at any size: the number of eigenvalues and their
  values against the closed-form Q1 spectrum (1e-9), every residual recomputed on the host from
  the CSR pencil (<= 1e-10), and M-orthonormality of the eigenvectors (1e-9).
"""
import gc

import numpy as np
import pytest

import rfdd_inputs as I
from oracle import rfdd_oracle as O

pytestmark = pytest.mark.gpu

NAME = "q1_3d_40"


@pytest.fixture(scope="module")
def R():
    from paper_1711_09487_gb300 import build
    build.build()
    import paper_1711_09487_gb300 as pkg
    pkg.load()
    return pkg


@pytest.fixture(scope="module")
def W():
    return I.workload(NAME)


def test_full_size_schur_columns(R, W):
    w = W
    z, wt = O.quadrature(w.alpha, w.beta, w.n_nodes, w.rule)
    opts = R.rfdd_default_options(precision=R.RFDD_MIXED, quad_rule=R.RFDD_MIDPOINT, keep_schur=1)
    h = R.rfdd_setup(w.A, w.M, w.part, w.p, opts)
    R.rfdd_factor(h, z, wt)
    _, _, s = R.rfdd_layout(h)
    cols = [0, 1, s // 2, s - 2, s - 1]
    for l in (0, w.n_nodes // 2):
        Sg = R.rfdd_schur_copy(h, l)[:, cols]
        So = O.schur_columns(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p, z[l], cols)
        err = np.abs(Sg - So).max() / np.abs(So).max()
        assert err <= 3e-4, (l, err)
    del h
    gc.collect()


def test_full_size_solve(R, W):
    w = W
    ev, X, rs, info = R.solve(w.A, w.M, w.part, w.p, w.alpha, w.beta, w.n_nodes, precision=R.RFDD_MIXED,
                              quad_rule=R.RFDD_MIDPOINT)
    ex = w.exact[(w.exact > w.alpha) & (w.exact < w.beta)]
    assert info["status"] == 0, info
    assert len(ev) == len(ex) == w.expected_nev == 202
    assert np.max(np.abs(ev - ex) / ex) <= 1e-9
    assert rs.max() <= 1e-10
    A, M = w.A.to_scipy(), w.M.to_scipy()
    MX = M @ X
    res = np.linalg.norm(A @ X - MX * ev, axis=0) / (np.abs(ev) * np.linalg.norm(MX, axis=0))
    assert res.max() <= 1e-10, res.max()
    assert np.abs(X.T @ MX - np.eye(len(ev))).max() <= 1e-9
