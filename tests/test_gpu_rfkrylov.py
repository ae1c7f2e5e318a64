"""RF-KRYLOV (Algorithm 1) on the GPU through the C ABI: the Ritz values of its Krylov basis
against the oracle's Algorithm 1 from the same counter-based start block, and the pairs after the
completion passes against the closed-form spectra (5-point FD Laplacian with M = I, the paper's
FDmesh pencils; Q1 with a mass matrix)."""
import numpy as np
import pytest

import rfdd_inputs as I
from oracle import rfdd_oracle as O

pytestmark = pytest.mark.gpu

RULES = {"midpoint": 0, "gauss_legendre": 1}
TOL_EV = {0: 1e-10, 1: 1e-9}


@pytest.fixture(scope="module")
def R():
    from paper_1711_09487_gb300 import build
    build.build()
    import paper_1711_09487_gb300 as pkg
    pkg.load()
    return pkg


def run(R, w, prec, **kw):
    opts = R.rfdd_default_options(precision=prec, quad_rule=RULES[w.rule], **kw)
    h = R.rfdd_setup(w.A, w.M, w.part, w.p, opts)
    r = R.rfdd_rfkrylov(h, w.alpha, w.beta, w.n_nodes)
    ev, X, rs = R.rfdd_result_get(r)
    return ev, X, rs, R.rfdd_result_info(r), R.rfdd_result_pre_evals(r)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["fd5_32", "fd5_40_p16", "q1_2d_24", "q1_3d_12"])
def test_pairs_against_the_closed_form(R, name, prec):
    w = I.workload(name)
    ev, X, rs, info, pre = run(R, w, prec)
    ex = w.exact[(w.exact > w.alpha) & (w.exact < w.beta)]
    assert info["status"] == 0 and len(ev) == len(ex) == w.expected_nev
    assert np.max(np.abs(ev - ex) / ex) <= TOL_EV[prec]
    assert rs.max() <= 1e-10
    M = w.M.to_scipy()
    assert np.abs(X.T @ (M @ X) - np.eye(len(ev))).max() <= (1e-10 if prec == 0 else 1e-9)
    assert info["mu"] > 0 and len(pre) == len(ex)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["fd5_32", "q1_2d_24"])
def test_krylov_ritz_values_against_the_oracle(R, name, prec):
    """Lines 0-16 on both sides from the same start block (block 4): the same Krylov dimension in
    FP64, and Ritz values inside [alpha, beta] that agree to rounding (FP64) or to the filter's
    refinement level (mixed)."""
    w = I.workload(name)
    blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
    z, wt = O.quadrature(w.alpha, w.beta, w.n_nodes, w.rule)
    fac = O.Factors(blk, z)
    out = O.rf_krylov(blk.Ap, blk.Mp, lambda Q: O.filter_full(fac, wt, blk.Mp @ Q), w.alpha, w.beta,
                      tol=1e-6, block=4, seed=1)
    th_o = out["theta"][out["inside"]]
    ev, X, rs, info, pre = run(R, w, prec, block=4)
    if prec == 0:
        assert info["mu"] == out["mu"], (info["mu"], out["mu"])
    assert len(pre) == len(th_o)
    rel = np.max(np.abs(np.sort(pre) - th_o) / np.abs(th_o))
    assert rel <= (1e-10 if prec == 0 else 1e-8), rel


def test_max_dim_caps_the_basis(R):
    w = I.workload("fd5_32")
    opts = R.rfdd_default_options(precision=1, block=4)
    h = R.rfdd_setup(w.A, w.M, w.part, w.p, opts)
    r = R.rfdd_rfkrylov(h, w.alpha, w.beta, w.n_nodes, max_dim=24)
    info = R.rfdd_result_info(r)
    assert info["mu"] == 24
    ev, X, rs = R.rfdd_result_get(r)
    # a 24-dimensional Krylov basis cannot resolve all 20 pairs, the completion passes do
    assert len(ev) == w.expected_nev and rs.max() <= 1e-10
    with pytest.raises(R.RfddError):
        R.rfdd_rfkrylov(h, w.alpha, w.beta, w.n_nodes, max_dim=2)
