"""What the mixed precision costs, result by result.  The mixed path factors in complex FP32 on
the tensor cores (3xTF32 products) and keeps FP64 for the refinement residuals, the
orthonormalisation of the filtered bases and the projected eigensolve.  For each of those results
this file measures the deviation of the mixed path from the FP64 oracle (or from the FP64 GPU path
on the same inputs, where the two follow the same steps), asserts a bound, and prints the measured
value on a line starting with ``PRECISION`` so that a run with ``-s`` records it:

* refinement: the backward error of a refined shifted solve (A - zeta M) x = b, Eq. (inv_dd2),
  against the FP64 unit roundoff;
* orthonormalisation: the interface Krylov basis Q (Algorithm 2, Euclidean) -- its loss of
  orthonormality and the principal angles between its span and the span of the FP64 oracle's basis
  from the same start block;
* Rayleigh-Ritz (Section 5, step 7): Ritz values on a well-conditioned basis Z against the oracle
  on the same Z, and the Ritz values inside [alpha, beta] before the completion passes against the
  FP64 GPU path's;
* final pairs: eigenvalues against the oracle's, eigenvectors by the angles between the M-spans of
  each cluster of equal eigenvalues, M-orthonormality.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import rfdd_inputs as I
from oracle import rfdd_oracle as O

pytestmark = pytest.mark.gpu

MIXED, FP64 = 1, 0
RULES = {"midpoint": 0, "gauss_legendre": 1}


@pytest.fixture(scope="module")
def R():
    from paper_1711_09487_gb300 import build
    build.build()
    import paper_1711_09487_gb300 as pkg
    pkg.load()
    return pkg


_cache = {}


def case(name):
    if name not in _cache:
        w = I.workload(name)
        blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
        z, wt = O.quadrature(w.alpha, w.beta, w.n_nodes, w.rule)
        _cache[name] = (w, blk, z, wt, O.Factors(blk, z))
    return _cache[name]


def handle(R, w, precision, **kw):
    opts = R.rfdd_default_options(precision=precision, quad_rule=RULES[w.rule], **kw)
    return R.rfdd_setup(w.A, w.M, w.part, w.p, opts)


def report(what, name, value):
    print(f"PRECISION {what} {name} {value:.3e}")


def cluster_angles(lam, X, Xo, M, rtol=1e-8):
    """Largest sine of the angles between span(X[:, c]) and span(Xo[:, c]) in the M inner product,
    over the clusters c of (numerically) equal eigenvalues."""
    worst, i = 0.0, 0
    while i < len(lam):
        j = i + 1
        while j < len(lam) and abs(lam[j] - lam[i]) <= rtol * abs(lam[i]):
            j += 1
        sv = np.linalg.svd(X[:, i:j].T @ (M @ Xo[:, i:j]), compute_uv=False)
        worst = max(worst, float(np.sqrt(max(0.0, 1.0 - sv.min() ** 2))))
        i = j
    return worst


@pytest.mark.parametrize("name", ["q1_2d_24", "q1_3d_12"])
def test_refinement_backward_error(R, name):
    w, blk, z, wt, fac = case(name)
    h = handle(R, w, MIXED)
    R.rfdd_factor(h, z, wt)
    rng = np.random.default_rng(5)
    worst = 0.0
    for l in range(len(z)):
        K = (blk.Ap - z[l] * blk.Mp).tocsr()
        nK = sla.norm(K.toarray(), 1)
        b = rng.standard_normal((blk.n, 3)) + 1j * rng.standard_normal((blk.n, 3))
        x = R.rfdd_shifted_solve(h, l, 2, 0, b)
        be = np.linalg.norm(K @ x - b, 1, axis=0) / (nK * np.linalg.norm(x, 1, axis=0) + np.linalg.norm(b, 1, axis=0))
        worst = max(worst, float(be.max()))
    report("refined_solve_backward_error", name, worst)
    assert worst <= 64 * np.finfo(float).eps, worst


@pytest.mark.parametrize("name", ["q1_2d_33_p9", "q1_3d_12"])
def test_interface_basis_against_fp64_oracle(R, name):
    w, blk, z, wt, fac = case(name)
    h = handle(R, w, MIXED, block=4)
    R.rfdd_factor(h, z, wt)
    Q, _ = R.rfdd_lanczos(h)
    orth = float(np.abs(Q.T @ Q - np.eye(Q.shape[1])).max())
    lz = O.lanczos_interface(lambda V: O.filter_interface(fac, wt, V), blk.s, 1e-6, block=4, seed=1)
    c = min(Q.shape[1], lz["mu"], 16)
    sv = np.linalg.svd(Q[:, :c].T @ lz["Q"][:, :c], compute_uv=False)
    ang = float(np.sqrt(max(0.0, 1.0 - sv.min() ** 2)))
    report("lanczos_Q_orthonormality", name, orth)
    report("lanczos_Q_first16_span_sine_vs_oracle", name, ang)
    assert orth <= 1e-12
    assert ang <= 1e-3, ang


@pytest.mark.parametrize("name", ["q1_2d_24", "q1_3d_12"])
def test_rayleigh_ritz_values(R, name):
    w, blk, z, wt, fac = case(name)
    # on a well-conditioned Z: the same Z in both, the projected problem solved by each
    h = handle(R, w, MIXED, nev_b=4, psi=1, block=4)
    R.rfdd_factor(h, z, wt)
    R.rfdd_lanczos(h)
    Z, k, _ = R.rfdd_interior(h, 0.5 * (w.alpha + w.beta))
    th_g = R.rfdd_rayleigh_ritz(h)
    th_o, _ = O.rayleigh_ritz(blk.Ap, blk.Mp, Z)
    rr = float(np.max(np.abs(th_g - th_o) / np.abs(th_o)))
    report("rr_values_same_Z_vs_oracle", name, rr)
    assert rr <= 1e-9, rr
    # before the completion passes: mixed vs FP64 GPU path, same steps, same seeds
    pre = {}
    for prec in (MIXED, FP64):
        hp = handle(R, w, prec)
        r = R.rfdd_solve(hp, w.alpha, w.beta, w.n_nodes)
        pre[prec] = np.sort(R.rfdd_result_pre_evals(r))
    assert len(pre[MIXED]) == len(pre[FP64])
    d = float(np.max(np.abs(pre[MIXED] - pre[FP64]) / np.abs(pre[FP64])))
    report("pre_completion_ritz_values_mixed_vs_fp64", name, d)
    assert d <= 1e-4, d


@pytest.mark.parametrize("name", ["q1_2d_24", "q1_3d_12"])
def test_final_pairs_against_fp64_oracle(R, name):
    w, blk, z, wt, fac = case(name)
    ev, X, rs, info = R.solve(w.A, w.M, w.part, w.p, w.alpha, w.beta, w.n_nodes, precision=MIXED,
                              quad_rule=RULES[w.rule])
    ro = O.rfdd_solve(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p, w.alpha, w.beta, w.n_nodes, w.rule)
    assert len(ev) == len(ro["evals"])
    o = np.argsort(ro["evals"])
    lam_o, X_o = ro["evals"][o], ro["evecs"][:, o]
    M = w.M.to_scipy()
    dl = float(np.max(np.abs(ev - lam_o) / np.abs(lam_o)))
    ang = cluster_angles(ev, X, X_o, M)
    orth = float(np.abs(X.T @ (M @ X) - np.eye(len(ev))).max())
    report("final_eigenvalues_vs_oracle", name, dl)
    report("final_eigenvector_cluster_sine_vs_oracle", name, ang)
    report("final_M_orthonormality", name, orth)
    report("final_max_residual", name, float(rs.max()))
    assert dl <= 1e-9 and ang <= 1e-6 and orth <= 1e-9 and rs.max() <= 1e-10
