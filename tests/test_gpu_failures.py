"""Failure paths the host sees, on the GPU, with no device fault or hang involved:

* admission: a solve whose factors exceed opt.mem_budget is refused with RFDD_EADMIT before any
  device work, and a budget that covers rfdd_memory_estimate admits it;
* RFDD_NOT_CONVERGED: a solve stopped by max_passes still returns its pairs with residuals;
* the interior shift guard (reading A10): sigma exactly on an eigenvalue of a subdomain pencil
  (B_j, M_B^(j)) is moved (FP64: by 1e-6 (beta - alpha), as the oracle does; mixed: further, since
  FP32 factors resolve B_sigma only to about 1e-7) and the solve still returns the brute-force
  eigenpairs -- the GPU twin of the oracle's test of the same guard.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import rfdd_inputs as I
from oracle import rfdd_oracle as O
from tests.test_oracle_dd import random_pencil, dense_eig

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1711_09487_gb300 import build
    build.build()
    import paper_1711_09487_gb300 as pkg
    pkg.load()
    return pkg


@pytest.mark.parametrize("prec", [0, 1])
def test_admission_by_memory_budget(R, prec):
    w = I.workload("q1_2d_24")
    tiny = 1 << 20
    h = R.rfdd_setup(w.A, w.M, w.part, w.p, R.rfdd_default_options(precision=prec, mem_budget=tiny))
    need = R.rfdd_memory_estimate(h, w.n_nodes, w.expected_nev)
    assert need > tiny
    launches = R.rfdd_kernel_launches()
    with pytest.raises(R.RfddError) as e:
        R.rfdd_solve(h, w.alpha, w.beta, w.n_nodes)
    assert e.value.code == R.RFDD_EADMIT
    assert R.rfdd_kernel_launches() == launches   # refused before any device work
    h2 = R.rfdd_setup(w.A, w.M, w.part, w.p, R.rfdd_default_options(precision=prec, mem_budget=need))
    r = R.rfdd_solve(h2, w.alpha, w.beta, w.n_nodes)
    ev, _, rs = R.rfdd_result_get(r, vectors=False)
    assert r.status == R.RFDD_OK and len(ev) == w.expected_nev and rs.max() <= 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_not_converged_returns_pairs_and_residuals(R, prec):
    w = I.workload("q1_2d_24")
    h = R.rfdd_setup(w.A, w.M, w.part, w.p,
                     R.rfdd_default_options(precision=prec, max_passes=1, res_tol=1e-15))
    r = R.rfdd_solve(h, w.alpha, w.beta, w.n_nodes)
    assert r.status == R.RFDD_NOT_CONVERGED
    info = R.rfdd_result_info(r)
    assert info["status"] == R.RFDD_NOT_CONVERGED and info["passes"] == 1
    ev, X, rs = R.rfdd_result_get(r)
    assert len(ev) == len(rs) == X.shape[1] > 0
    # the returned residuals are the pairs' own
    A, M = w.A.to_scipy(), w.M.to_scipy()
    res = np.linalg.norm(A @ X - (M @ X) * ev, axis=0) / (np.abs(ev) * np.linalg.norm(M @ X, axis=0))
    np.testing.assert_allclose(rs, res, rtol=1e-6, atol=1e-15)
    assert rs.max() > 1e-15 and info["max_resid"] == rs.max()


@pytest.mark.parametrize("prec", [0, 1])
def test_sigma_guard_moves_a_shift_on_a_subdomain_eigenvalue(R, prec):
    A, M, part, p = random_pencil(N=12, splits=(3, 2), seed=11)
    lam, _ = dense_eig(A, M)
    alpha, beta = 0.5 * (lam[40] + lam[41]), 0.5 * (lam[60] + lam[61])
    blk = O.Blocks(A, M, part, p)
    d0 = sla.eigh(blk.B[0], blk.MB[0], eigvals_only=True)
    sig = float(d0[np.argmin(np.abs(d0 - 0.5 * (alpha + beta)))])
    ev, X, rs, info = R.solve(A, M, part, p, alpha, beta, 6, precision=prec, sigma=sig, nev_b=10, block=2)
    # moved once: FP64 by 1e-6 (beta - alpha); mixed (FP32 factors resolve B_sigma to about 1e-7)
    # by max(1e-3 (beta - alpha), 2e-5 max(1, |sigma|))
    step = 1e-6 * (beta - alpha) if prec == 0 else max(1e-3 * (beta - alpha), 2e-5 * max(1.0, abs(sig)))
    assert abs(info["sigma"] - (sig + step)) <= 1e-12 * abs(sig), (info["sigma"], sig, step)
    assert info["status"] == R.RFDD_OK and rs.max() <= 1e-10
    np.testing.assert_allclose(ev, lam[41:61], rtol=1e-10 if prec == 0 else 1e-9)
    # a shift away from every subdomain spectrum is kept as given
    far = 0.5 * (alpha + beta)
    _, _, _, info2 = R.solve(A, M, part, p, alpha, beta, 6, precision=prec, sigma=far, nev_b=10, block=2)
    assert info2["sigma"] == far
