"""The serving loop on the GPU: requests of different sizes solved alone and in a mix must give the
same eigenpairs (the results of a request do not depend on what else runs), waiting requests are
admitted as memory frees up, a request too large for the whole budget is refused at submit, and a
resident pencil serves several intervals one at a time."""
import numpy as np
import pytest

import rfdd_inputs as I

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-9}


@pytest.fixture(scope="module")
def R():
    from paper_1711_09487_gb300 import build
    build.build()
    import paper_1711_09487_gb300 as pkg
    pkg.load()
    return pkg


def mix_requests():
    """(pencil, alpha, beta, n_nodes, expected nev or None) of a small mixed stream: 2-D and 3-D Q1
    pencils with closed-form windows and a 3-D variable-coefficient pencil."""
    out = []
    for name in ("q1_2d_24", "q1_3d_12", "q1_2d_33_p9", "q1_3d_16"):
        w = I.workload(name)
        out.append((w, w.alpha, w.beta, w.n_nodes, w.expected_nev))
    w = I.workload("q1_2d_24")   # a second interval on the same pencil
    ev = w.exact
    first, last = I.snap_to_gaps(ev, 40, 70)
    a, b = I.interval_from_sorted(ev, first, last)
    out.append((w, a, b, 6, last - first + 1))
    A, M = I.varkappa7_pencil(12, seed=4)
    part, p = I.geometric_partition(12, 3, (2, 2, 2))
    c1, c2 = I.sym_inertia_count(A, M, 250.0), I.sym_inertia_count(A, M, 400.0)   # 46 and 135
    wv = I.Pencil("varkappa_12", A, M, part, p, 250.0, 400.0, 8, "midpoint", None, c2 - c1)
    out.append((wv, 250.0, 400.0, 8, c2 - c1))
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_results_are_the_same_alone_and_in_the_mix(R, prec):
    reqs = mix_requests()
    alone = []
    for w, a, b, nc, nev in reqs:
        ev, X, rs, info = R.solve(w.A, w.M, w.part, w.p, a, b, nc, precision=prec)
        assert info["status"] == R.RFDD_OK and rs.max() <= 1e-10
        if nev is not None:
            assert len(ev) == nev
        alone.append(ev)
    srv = R.Server(max_inflight=3)
    ids = [srv.submit_pencil(w.A, w.M, w.part, w.p, a, b, nc, nev_hint=nev or 0,
                             opts=R.rfdd_default_options(precision=prec)) for w, a, b, nc, nev in reqs]
    for rid, ev0 in zip(ids, alone):
        r = srv.wait(rid)
        ev, X, rs = R.rfdd_result_get(r)
        assert r.status == R.RFDD_OK and rs.max() <= 1e-10
        assert len(ev) == len(ev0)
        if len(ev):
            assert np.max(np.abs(ev - ev0) / np.abs(ev0)) <= TOL[prec]
        info = srv.request_info(rid)
        assert info["latency_ms"] >= info["run_ms"] > 0 and info["nev"] == len(ev)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["waiting"] == 0
    assert 1 <= st["peak_running"] <= 3 and st["in_use"] == 0
    srv.close()


def test_admission_waits_for_memory_and_refuses_what_never_fits(R):
    w = I.workload("q1_2d_24")
    h = R.rfdd_setup(w.A, w.M, w.part, w.p)
    need = R.rfdd_memory_estimate(h, w.n_nodes, w.expected_nev)
    del h
    srv = R.Server(max_inflight=4, mem_budget=int(need * 1.6))   # one at a time fits
    pid = srv.add_pencil(w.A, w.M, w.part, w.p)
    pid2 = srv.add_pencil(w.A, w.M, w.part, w.p)
    ids = [srv.submit(q, w.alpha, w.beta, w.n_nodes, nev_hint=w.expected_nev) for q in (pid, pid2, pid, pid2)]
    for rid in ids:
        r = srv.wait(rid)
        ev, _, rs = R.rfdd_result_get(r, vectors=False)
        assert len(ev) == w.expected_nev and rs.max() <= 1e-10
    st = srv.stats()
    assert st["completed"] == 4 and st["peak_running"] == 1 and st["peak_in_use"] <= int(need * 1.6)
    with pytest.raises(R.RfddError) as e:                          # needs more than the whole budget
        srv.submit(pid, w.alpha, w.beta, w.n_nodes, nev_hint=50 * w.n)
    assert e.value.code == R.RFDD_EADMIT
    srv.remove_pencil(pid)
    with pytest.raises(R.RfddError) as e:
        srv.submit(pid, w.alpha, w.beta, w.n_nodes)
    assert e.value.code == R.RFDD_EINVAL
    srv.close()


def test_resident_pencil_serves_intervals_in_turn(R):
    w = I.workload("q1_2d_33_p9")
    ev = w.exact
    windows = [(11, 30), (21, 40), (35, 60)]
    srv = R.Server(max_inflight=4)
    pid = srv.add_pencil(w.A, w.M, w.part, w.p)
    ids = []
    for f, l in windows:
        f, l = I.snap_to_gaps(ev, f, l)
        a, b = I.interval_from_sorted(ev, f, l)
        ids.append((srv.submit(pid, a, b, 6), ev[f - 1:l]))
    with pytest.raises(R.RfddError) as e:          # requests of it are still waiting or running
        srv.remove_pencil(pid)
    assert e.value.code == R.RFDD_ESTATE
    for rid, ex in ids:
        r = srv.wait(rid)
        got, _, rs = R.rfdd_result_get(r, vectors=False)
        np.testing.assert_allclose(got, ex, rtol=1e-9)
        assert rs.max() <= 1e-10
    assert srv.stats()["peak_running"] == 1        # one solve at a time on one handle
    srv.remove_pencil(pid)
    srv.close()
