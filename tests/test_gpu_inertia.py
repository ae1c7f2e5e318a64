"""Eigenvalue counts by Sylvester inertia on the GPU (rfdd_inertia) against the closed-form
spectra of the Q1 pencils, against the oracle's count, and as a completeness check of a solve:
the number of eigenpairs returned in [alpha, beta] equals count(beta) - count(alpha)."""
import numpy as np
import pytest

import rfdd_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1711_09487_gb300 import build
    build.build()
    import paper_1711_09487_gb300 as pkg
    pkg.load()
    return pkg


def shifts_between(ev, fracs):
    """(sigma, count) pairs with sigma halfway between two consecutive distinct eigenvalues."""
    ev = np.sort(ev)
    out = [(ev[0] - 1.0, 0), (ev[-1] * 1.01 + 1.0, len(ev))]
    for f in fracs:
        k = int(f * (len(ev) - 1)) + 1
        while k < len(ev) and ev[k] - ev[k - 1] <= 1e-7 * abs(ev[k]):
            k += 1  # inside a degenerate cluster: move to its end
        if k < len(ev):
            out.append((0.5 * (ev[k - 1] + ev[k]), k))
    return out


@pytest.mark.parametrize("name", ["q1_2d_24", "q1_2d_33_p9", "q1_3d_12", "q1_2d_40"])
def test_inertia_matches_closed_form(R, name):
    w = I.workload(name)
    h = R.rfdd_setup(w.A, w.M, w.part, w.p)
    for sigma, want in shifts_between(w.exact, [0.05, 0.3, 0.5, 0.77, 0.95]):
        assert R.rfdd_inertia(h, sigma) == want, (name, sigma, want)


def test_inertia_matches_oracle(R):
    from oracle import rfdd_oracle as O
    w = I.workload("q1_2d_33_p9")
    h = R.rfdd_setup(w.A, w.M, w.part, w.p)
    blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
    for sigma in (w.alpha, 0.5 * (w.alpha + w.beta), w.beta):
        assert R.rfdd_inertia(h, sigma) == O.inertia_count(blk, sigma)


@pytest.mark.parametrize("name", ["q1_2d_24", "q1_3d_16"])
def test_solve_is_complete(R, name):
    w = I.workload(name)
    h = R.rfdd_setup(w.A, w.M, w.part, w.p, R.rfdd_default_options(quad_rule=0 if w.rule == "midpoint" else 1))
    r = R.rfdd_solve(h, w.alpha, w.beta, w.n_nodes)
    ev, _, rs = R.rfdd_result_get(r, vectors=False)
    assert len(ev) == R.rfdd_inertia(h, w.beta) - R.rfdd_inertia(h, w.alpha) == w.expected_nev
