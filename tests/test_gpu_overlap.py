"""A solve starts the real factorisation of the interior blocks B_sigma^(j) (Section 4.2: the
shift-invert basis V_j and the chains Sigma / Gamma of Eq. (4.5)-(4.6)) on a second stream,
from its own host thread, while the complex factorisations run.  Repeated solves on one handle
(each interval brings a new shift sigma), an asynchronous solve, and solves in both precisions
must agree with solves on fresh handles.  Also the busy-time hook of the measurement."""
import time

import numpy as np
import pytest

import rfdd_inputs as I

pytestmark = pytest.mark.gpu

RULES = {"midpoint": 0, "gauss_legendre": 1}
EV_TOL = {0: 1e-10, 1: 1e-9}


@pytest.fixture(scope="module")
def R():
    from paper_1711_09487_gb300 import build
    build.build()
    import paper_1711_09487_gb300 as pkg
    pkg.load()
    return pkg


def intervals(w):
    """The workload's interval and a second, lower one (whole eigenvalue clusters)."""
    f, l = I.snap_to_gaps(w.exact, 3, 14)
    return [(w.alpha, w.beta, None), I.interval_from_sorted(w.exact, f, l) + ((f, l),)]


def check(w, ev, rs, exact_range, prec):
    if exact_range is None:
        ref = w.exact[(w.exact > w.alpha) & (w.exact < w.beta)]
    else:
        ref = w.exact[exact_range[0] - 1:exact_range[1]]
    assert len(ev) == len(ref)
    np.testing.assert_allclose(ev, ref, rtol=EV_TOL[prec])
    assert rs.max() <= 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_repeated_solves_on_one_handle(R, prec):
    w = I.workload("q1_2d_24")
    opts = R.rfdd_default_options(precision=prec, quad_rule=RULES[w.rule])
    h = R.rfdd_setup(w.A, w.M, w.part, w.p, opts)
    ivs = intervals(w)
    for a, b, rng in ivs + ivs[:1]:  # new shift, then back to the first one
        r = R.rfdd_solve(h, a, b, w.n_nodes)
        ev, _, rs = R.rfdd_result_get(r, vectors=False)
        check(w, ev, rs, rng, prec)
        ev_fresh, _, rs_fresh, _ = R.solve(w.A, w.M, w.part, w.p, a, b, w.n_nodes, precision=prec,
                                           quad_rule=RULES[w.rule])
        np.testing.assert_allclose(ev, ev_fresh, rtol=EV_TOL[prec])


def test_async_then_sync_solve(R):
    w = I.workload("q1_3d_12")
    opts = R.rfdd_default_options(precision=1, quad_rule=RULES[w.rule])
    h = R.rfdd_setup(w.A, w.M, w.part, w.p, opts)
    r = R.rfdd_solve_async(h, w.alpha, w.beta, w.n_nodes)
    t0 = time.time()
    while R.rfdd_result_ready(r) == 0:
        assert time.time() - t0 < 120
        time.sleep(0.005)
    assert R.rfdd_result_ready(r) == 1
    ev_a, _, rs_a = R.rfdd_result_get(r, vectors=False)
    check(w, ev_a, rs_a, None, 1)
    del r
    r2 = R.rfdd_solve(h, w.alpha, w.beta, w.n_nodes)
    ev_s, _, rs_s = R.rfdd_result_get(r2, vectors=False)
    np.testing.assert_allclose(ev_s, ev_a, rtol=1e-12)


def test_profile_busy_is_the_union_of_launch_intervals(R):
    g = np.random.default_rng(3)
    A = (g.standard_normal((1000, 96)) + 1j * g.standard_normal((1000, 96))).astype(np.complex64)
    B = (g.standard_normal((96, 700)) + 1j * g.standard_normal((96, 700))).astype(np.complex64)
    C = np.zeros((1000, 700), dtype=np.complex64)
    R.rfdd_cgemm(A, B, C, 1.0, 0.0, 1)
    R.rfdd_profile(True)
    for _ in range(3):  # launches on one stream, one after the other: union = sum
        R.rfdd_cgemm(A, B, C, 1.0, 0.0, 1)
    n, ms, _ = R.rfdd_profile_get(1)
    busy = R.rfdd_profile_busy(1)
    R.rfdd_profile(False)
    assert n == 3 and ms > 0
    assert abs(busy - ms) <= 1e-4 * ms + 1e-3
    # a solve, whose interior factorisation overlaps the complex one on a second stream
    w = I.workload("q1_2d_24")
    R.rfdd_profile(True)
    R.solve(w.A, w.M, w.part, w.p, w.alpha, w.beta, w.n_nodes, precision=1, quad_rule=RULES[w.rule])
    n, ms, _ = R.rfdd_profile_get(1)
    busy = R.rfdd_profile_busy(1)
    R.rfdd_profile(False)
    assert n > 0 and 0 < busy <= ms * (1 + 1e-6) + 1e-3
