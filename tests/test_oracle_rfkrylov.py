"""Pins for the oracle's RF-KRYLOV (Algorithm 1, Section 2.2):

* lines 15-16 against the closed-form spectra of a 5-point finite-difference Laplacian with M = I
  (the paper's FDmesh pencils) and of a Q1 pencil (M != I): every eigenvalue inside [alpha, beta],
  none missing, none extra;
* lines 2-12: Q M-orthonormal, and H_mu equal to Q^T M rho(M^{-1}A) Q formed directly from
  ``apply_rho`` (so H is the projected filter, symmetric in the M inner product);
* line 13 on a filter whose Krylov space is exhausted at a known step: the stop comes exactly one
  check period after the sum of the eigenvalues >= 1/2 settles; eigenvalues below 1/2 do not
  count (with the trace instead, a filter with many small eigenvalues never stops early).

Planted mistakes (a Euclidean inner product with M != I, the trace in line 13) must fail a pin.
"""
import inspect
import textwrap

import numpy as np
import pytest

import rfdd_inputs as I
from oracle import rfdd_oracle as O


def plant(fns, old, new):
    """Copies of oracle functions ``fns`` (a list, sharing one namespace) with ``old`` replaced by
    ``new`` in their source; returns the namespace."""
    ns = dict(vars(O))
    hit = False
    for fn in fns:
        src = textwrap.dedent(inspect.getsource(fn))
        hit |= old in src
        exec(compile(src.replace(old, new), "<planted>", "exec"), ns)
    assert hit, old
    return ns


_cache = {}


def case(name):
    if name not in _cache:
        w = I.workload(name)
        blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
        z, wt = O.quadrature(w.alpha, w.beta, w.n_nodes, w.rule)
        fac = O.Factors(blk, z)
        _cache[name] = (w, blk, lambda Q: O.filter_full(fac, wt, blk.Mp @ Q))
    return _cache[name]


def inside_exact(w):
    return w.exact[(w.exact > w.alpha) & (w.exact < w.beta)]


@pytest.mark.parametrize("name,b", [("fd5_32", 1), ("fd5_32", 4), ("q1_2d_24", 1), ("q1_2d_24", 3)])
def test_ritz_values_match_the_closed_form(name, b):
    w, blk, rho = case(name)
    out = O.rf_krylov(blk.Ap, blk.Mp, rho, w.alpha, w.beta, block=b)
    th = out["theta"][out["inside"]]
    ex = inside_exact(w)
    assert len(th) == len(ex) == w.expected_nev
    assert np.max(np.abs(th - ex) / ex) <= 1e-12
    X = out["X"][:, out["inside"]]
    res = O.residuals(blk.Ap, blk.Mp, th, X)
    assert res.max() <= 1e-10


@pytest.mark.parametrize("name", ["fd5_32", "q1_2d_24"])
def test_basis_and_projected_filter(name):
    w, blk, rho = case(name)
    out = O.rf_krylov(blk.Ap, blk.Mp, rho, w.alpha, w.beta, block=2)
    Q, H = out["Q"], out["H"]
    assert np.abs(Q.T @ (blk.Mp @ Q) - np.eye(Q.shape[1])).max() <= 1e-12
    Hd = Q.T @ (blk.Mp @ rho(Q))
    assert np.abs(H - Hd).max() <= 1e-12
    assert np.abs(Hd - Hd.T).max() <= 1e-12           # rho(M^{-1}A) is M-self-adjoint
    # eigenvalues of H >= 1/2 <-> eigenvalues of the pencil inside [alpha, beta] (Section 2.1)
    assert np.count_nonzero(np.linalg.eigvalsh(H) >= 0.5) == w.expected_nev


def test_planted_euclidean_inner_product_fails():
    w, blk, rho = case("q1_2d_24")
    ns = plant([O._m_orth_against, O._m_cholqr, O.rf_krylov], "Mp @ W", "W")
    out = ns["rf_krylov"](blk.Ap, blk.Mp, rho, w.alpha, w.beta, block=2)
    Q, H = out["Q"], out["H"]
    Hd = Q.T @ (blk.Mp @ rho(Q))
    assert np.abs(Q.T @ (blk.Mp @ Q) - np.eye(Q.shape[1])).max() > 1e-6 or np.abs(H - Hd).max() > 1e-6


# ----------------------------------------------------------------------------------------
# line 13 on diagonal operators (A = diag(lam), M = I, rho(A) Q = f * Q)
# ----------------------------------------------------------------------------------------

N_DIAG, RANK = 120, 13


def diag_case(small):
    """f: RANK distinct values in [0.6, 1.0]; the rest 0, or (small=True) distinct values in
    [0.01, 0.3] that Krylov keeps finding one by one."""
    f = np.zeros(N_DIAG)
    f[:RANK] = np.linspace(0.6, 1.0, RANK)
    if small:
        f[RANK:] = np.linspace(0.01, 0.3, N_DIAG - RANK)
    lam = np.arange(1.0, N_DIAG + 1.0)
    import scipy.sparse as sp
    return sp.diags(lam).tocsr(), sp.identity(N_DIAG, format="csr"), (lambda Q: f[:, None] * Q), f


def expected_mu(b, check_every=10):
    t0 = -(-(RANK + b) // b)        # block step at which the Krylov space of a rank-RANK f is exhausted
    spc = max(1, -(-check_every // b))
    tc = spc
    while tc - spc < t0:
        tc += spc
    return tc * b


@pytest.mark.parametrize("b", [1, 2, 5])
def test_stop_one_check_after_the_half_sum_settles(b):
    A, M, rho, f = diag_case(False)
    out = O.rf_krylov(A, M, rho, 0.0, 1.0, tol=1e-9, block=b)
    assert out["mu"] == expected_mu(b), (out["mu"], expected_mu(b))
    assert abs(out["sums"][-1] - f[:RANK].sum()) <= 1e-12 * f[:RANK].sum()


def test_small_eigenvalues_do_not_delay_the_stop():
    A, M, rho, f = diag_case(True)
    out = O.rf_krylov(A, M, rho, 0.0, 1.0, tol=1e-8, block=1)
    assert out["mu"] < N_DIAG // 2
    assert abs(out["sums"][-1] - f[:RANK].sum()) <= 1e-7 * f[:RANK].sum()
    ns = plant([O.rf_krylov], "ev[ev >= 0.5].sum()", "ev.sum()")
    bad = ns["rf_krylov"](A, M, rho, 0.0, 1.0, tol=1e-8, block=1)
    assert bad["mu"] >= N_DIAG // 2
