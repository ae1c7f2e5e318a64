"""GPU parity of the two-level interface factorisation (rfdd_set_interface_groups): the block
inverse of Eq. (inv_dd2) applied to S(zeta) with subdomain groups as its subdomains.

Tolerances as in test_gpu_parity: S solves to FP64 rounding (1e-12 relative residual, FP64) or
the complex-FP32 level (3e-5); refined full solves 1e-12 / 1e-11; end to end 1e-10 / 1e-9
against the closed form, residuals <= 1e-10.  The split itself is integer work and must equal
the oracle's exactly."""
import numpy as np
import pytest

import rfdd_inputs as I
from oracle import rfdd_oracle as O
from tests.test_oracle_levels import _thick_separator_pencil

pytestmark = pytest.mark.gpu

RULES = {"midpoint": 0, "gauss_legendre": 1}
TOL = {0: dict(s_res=1e-12, solve=1e-12, ev=1e-10, orth=1e-10),
       1: dict(s_res=3e-5, solve=1e-11, ev=1e-9, orth=1e-9)}
# (workload, subdomain splits, group splits)
CASES = [("q1_2d_33_p9", (3, 3), (2, 2)), ("q1_2d_49_p16", (4, 4), (2, 2)), ("q1_3d_12", (2, 2, 2), (1, 1, 2))]


@pytest.fixture(scope="module")
def R():
    from paper_1711_09487_gb300 import build
    build.build()
    import paper_1711_09487_gb300 as pkg
    pkg.load()
    return pkg


def _handle(R, w, prec, **kw):
    opts = R.rfdd_default_options(precision=prec, quad_rule=RULES[w.rule], **kw)
    return R.rfdd_setup(w.A, w.M, w.part, w.p, opts)


@pytest.mark.parametrize("name,splits,gs", CASES + [("q1_3d_24_p64", (4, 4, 4), (2, 2, 2))])
def test_split_equals_oracle(R, name, splits, gs):
    w = I.workload(name)
    groups = I.subdomain_groups(splits, gs)
    blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
    lv = O.interface_levels(blk, groups)
    h = _handle(R, w, 1)
    R.rfdd_set_interface_groups(h, groups)
    cls, s2 = R.rfdd_interface_levels(h)
    np.testing.assert_array_equal(cls, lv.cls)
    assert s2 == len(lv.I2)
    R.rfdd_set_interface_groups(h, None)
    cls, s2 = R.rfdd_interface_levels(h)
    assert np.all(cls == -1) and s2 == blk.s


def test_split_of_a_thick_separator_equals_oracle(R):
    A, M, part, p, xs, ny = _thick_separator_pencil()
    blk = O.Blocks(A, M, part, p)
    lv = O.interface_levels(blk, [0, 0, 1, 1])
    h = R.rfdd_setup(A, M, part, p, R.rfdd_default_options())
    R.rfdd_set_interface_groups(h, [0, 0, 1, 1])
    cls, s2 = R.rfdd_interface_levels(h)
    np.testing.assert_array_equal(cls, lv.cls)
    assert s2 == len(lv.I2)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,splits,gs", CASES)
def test_two_level_S_solve(R, name, splits, gs, prec):
    """S(zeta_l)^{-1} through the level factors against the oracle's dense S (Eq. inv_dd2)."""
    w = I.workload(name)
    blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
    z, wt = O.quadrature(w.alpha, w.beta, w.n_nodes, w.rule)
    h = _handle(R, w, prec)
    R.rfdd_set_interface_groups(h, I.subdomain_groups(splits, gs))
    R.rfdd_factor(h, z, wt)
    rng = np.random.default_rng(4)
    for l in range(len(z)):
        S = O.schur(blk, z[l])
        rhs = rng.standard_normal((blk.s, 3)) + 1j * rng.standard_normal((blk.s, 3))
        y = R.rfdd_shifted_solve(h, l, 1, 0, rhs)
        res = np.linalg.norm(S @ y - rhs) / (np.linalg.norm(S, 2) * np.linalg.norm(y))
        assert res <= TOL[prec]["s_res"], (l, res)
        if prec == 0:
            yo = np.linalg.solve(S, rhs)
            assert np.abs(y - yo).max() <= 1e-10 * np.abs(yo).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_two_level_refined_full_solve(R, prec):
    """Eq. (inv_dd2) with the level factors inside, FP64 refinement, against a dense solve."""
    name, splits, gs = CASES[1]
    w = I.workload(name)
    blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
    z, wt = O.quadrature(w.alpha, w.beta, w.n_nodes, w.rule)
    h = _handle(R, w, prec)
    R.rfdd_set_interface_groups(h, I.subdomain_groups(splits, gs))
    R.rfdd_factor(h, z, wt)
    rng = np.random.default_rng(5)
    for l in range(len(z)):
        rhs = rng.standard_normal((blk.n, 2)) + 1j * rng.standard_normal((blk.n, 2))
        x = R.rfdd_shifted_solve(h, l, 2, 0, rhs)
        xo = np.linalg.solve((blk.Ap - z[l] * blk.Mp).toarray(), rhs)
        assert np.abs(x - xo).max() <= TOL[prec]["solve"] * np.abs(xo).max()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,splits,gs", CASES + [("q1_3d_24_p64", (4, 4, 4), (2, 2, 2))])
def test_two_level_solve_end_to_end(R, name, splits, gs, prec):
    w = I.workload(name)
    groups = I.subdomain_groups(splits, gs)
    ev, X, rs, info = R.solve(w.A, w.M, w.part, w.p, w.alpha, w.beta, w.n_nodes, groups=groups,
                              precision=prec, quad_rule=RULES[w.rule])
    ex = w.exact[(w.exact > w.alpha) & (w.exact < w.beta)]
    assert len(ev) == len(ex)
    assert np.max(np.abs(ev - ex) / np.abs(ex)) <= TOL[prec]["ev"]
    assert rs.max() <= 1e-10
    Mx = w.M.to_scipy() @ X
    assert np.abs(X.T @ Mx - np.eye(len(ev))).max() <= TOL[prec]["orth"]
    # the same filter as the dense factorisation: Algorithm 2 takes the same number of steps
    ev1, _, _, info1 = R.solve(w.A, w.M, w.part, w.p, w.alpha, w.beta, w.n_nodes,
                               precision=prec, quad_rule=RULES[w.rule])
    assert info["mu"] == info1["mu"]
    np.testing.assert_allclose(ev, ev1, rtol=TOL[prec]["ev"])


def test_two_level_factors_take_less_memory(R):
    w = I.workload("q1_3d_24_p64")
    h = _handle(R, w, 1)
    dense = R.rfdd_memory_estimate(h, w.n_nodes, 60)
    R.rfdd_set_interface_groups(h, I.subdomain_groups((4, 4, 4), (2, 2, 2)))
    two = R.rfdd_memory_estimate(h, w.n_nodes, 60)
    assert two < 0.7 * dense, (two, dense)


def test_set_interface_groups_rejects_bad_labels(R):
    w = I.workload("q1_2d_33_p9")
    h = _handle(R, w, 1)
    with pytest.raises(R.RfddError) as e:
        R.rfdd_set_interface_groups(h, [0, 1, 2, 3, 4, 5, 6, 7, -1])
    assert e.value.code == R.RFDD_EINVAL
    hk = _handle(R, w, 1, keep_schur=1)
    with pytest.raises(R.RfddError) as e:
        R.rfdd_set_interface_groups(hk, I.subdomain_groups((3, 3), (2, 2)))
    assert e.value.code == R.RFDD_EINVAL


def test_two_level_with_complex64_factors_only(R):
    """pack_factors = 0: the level factors stay complex64 and every solve product packs its
    block on the fly (the border products of the group blocks included)."""
    name, splits, gs = CASES[1]
    w = I.workload(name)
    groups = I.subdomain_groups(splits, gs)
    ev, X, rs, info = R.solve(w.A, w.M, w.part, w.p, w.alpha, w.beta, w.n_nodes, groups=groups,
                              precision=1, quad_rule=RULES[w.rule], pack_factors=0)
    ex = w.exact[(w.exact > w.alpha) & (w.exact < w.beta)]
    assert info["packed"] == 0
    assert len(ev) == len(ex) and np.max(np.abs(ev - ex) / np.abs(ex)) <= TOL[1]["ev"]
    assert rs.max() <= 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_rfkrylov_through_the_two_level_factors(R, prec):
    """RF-KRYLOV's full-space filter goes through Eq. (inv_dd2) and so through the level solves."""
    name, splits, gs = CASES[1]
    w = I.workload(name)
    h = _handle(R, w, prec)
    R.rfdd_set_interface_groups(h, I.subdomain_groups(splits, gs))
    r = R.rfdd_rfkrylov(h, w.alpha, w.beta, w.n_nodes)
    ev, X, rs = R.rfdd_result_get(r)
    ex = w.exact[(w.exact > w.alpha) & (w.exact < w.beta)]
    assert len(ev) == len(ex) and np.max(np.abs(ev - ex) / np.abs(ex)) <= TOL[prec]["ev"]
    assert rs.max() <= 1e-10
