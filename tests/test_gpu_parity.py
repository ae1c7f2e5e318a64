"""GPU parity: every row of the hot path through the C ABI against the FP64 oracle on the same
seeded inputs.

Tolerances (relative, max-norm unless stated):
* FP64 path: factor-level results (S(zeta), filter) 1e-10; solves 1e-12 after refinement.
* mixed path (complex-FP32 factorisations): factor-level results 3e-4 (FP32 rounding of an LU of
  order d_j amplified by the conditioning of B_j(zeta)); refined shifted solves 1e-11.
* end to end (both paths): eigenvalue relative error <= 1e-10 (FP64) / 1e-9 (mixed) against the
  closed form, every residual <= 1e-10, ||X^T M X - I||_max <= 1e-10 (FP64) / 1e-9 (mixed).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import rfdd_inputs as I
from oracle import rfdd_oracle as O

pytestmark = pytest.mark.gpu

TOL = {0: dict(fac=1e-10, solve=1e-12, ev=1e-10, orth=1e-10),
       1: dict(fac=3e-4, solve=1e-11, ev=1e-9, orth=1e-9)}
RULES = {"midpoint": 0, "gauss_legendre": 1}


@pytest.fixture(scope="module")
def R():
    from paper_1711_09487_gb300 import build
    build.build()
    import paper_1711_09487_gb300 as pkg
    pkg.load()
    return pkg


_cache = {}


def oracle_case(name):
    if name not in _cache:
        w = I.workload(name)
        blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
        z, wt = O.quadrature(w.alpha, w.beta, w.n_nodes, w.rule)
        fac = O.Factors(blk, z)
        _cache[name] = (w, blk, z, wt, fac)
    return _cache[name]


def handle(R, w, precision, **kw):
    opts = R.rfdd_default_options(precision=precision, quad_rule=RULES[w.rule], **kw)
    return R.rfdd_setup(w.A, w.M, w.part, w.p, opts)


def relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = ["q1_2d_24", "q1_2d_33_p9", "q1_3d_12"]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", CASES)
def test_layout_matches_oracle(R, name, prec):
    w, blk, z, wt, fac = oracle_case(name)
    h = handle(R, w, prec)
    off, perm, s = R.rfdd_layout(h)
    assert s == blk.s
    np.testing.assert_array_equal(off, blk.off)
    np.testing.assert_array_equal(perm, blk.perm)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", CASES)
def test_schur_complement_parity(R, name, prec):
    """a2-a5: assembled S(zeta_l) = C - z M_C - sum_j E_j^T B_j^{-1} E_j, element by element."""
    w, blk, z, wt, fac = oracle_case(name)
    h = handle(R, w, prec, keep_schur=1)
    R.rfdd_factor(h, z, wt)
    for l in range(len(z)):
        Sg = R.rfdd_schur_copy(h, l)
        So = O.schur(blk, z[l])
        assert relmax(Sg, So) <= TOL[prec]["fac"], (l, relmax(Sg, So))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", CASES)
def test_factor_solves(R, name, prec):
    """a3 (B_j(zeta) LU) and a5 (S(zeta) LU): solve residuals with the oracle's matrices."""
    w, blk, z, wt, fac = oracle_case(name)
    h = handle(R, w, prec)
    R.rfdd_factor(h, z, wt)
    rng = np.random.default_rng(7)
    eps = 1e-13 if prec == 0 else 3e-6
    for l in (0, len(z) - 1):
        Bz, Ez, Cz = O.shifted(blk, z[l])
        for j in range(blk.p):
            rhs = rng.standard_normal((blk.d[j], 3)) + 1j * rng.standard_normal((blk.d[j], 3))
            x = R.rfdd_shifted_solve(h, l, 0, j, rhs)
            res = np.linalg.norm(Bz[j] @ x - rhs) / (np.linalg.norm(Bz[j], 2) * np.linalg.norm(x))
            assert res <= eps, (l, j, res)
        S = O.schur(blk, z[l])
        rhs = rng.standard_normal((blk.s, 2)) + 1j * rng.standard_normal((blk.s, 2))
        y = R.rfdd_shifted_solve(h, l, 1, 0, rhs)
        res = np.linalg.norm(S @ y - rhs) / (np.linalg.norm(S, 2) * np.linalg.norm(y))
        assert res <= (eps if prec == 0 else 3e-5), (l, res)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["q1_2d_24", "q1_3d_12"])
def test_refined_full_solve(R, name, prec):
    """Eq. (inv_dd2) block inverse with FP64 iterative refinement vs a dense solve."""
    w, blk, z, wt, fac = oracle_case(name)
    h = handle(R, w, prec)
    R.rfdd_factor(h, z, wt)
    rng = np.random.default_rng(3)
    for l in range(len(z)):
        rhs = rng.standard_normal((blk.n, 2)) + 1j * rng.standard_normal((blk.n, 2))
        x = R.rfdd_shifted_solve(h, l, 2, 0, rhs)
        xo = np.linalg.solve((blk.Ap - z[l] * blk.Mp).toarray(), rhs)
        assert relmax(x, xo) <= TOL[prec]["solve"], (l, relmax(x, xo))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", CASES)
def test_filter_apply_parity(R, name, prec):
    """a6: W = Re sum_l w_l S_l^{-1} X (Alg. 2 line 2)."""
    w, blk, z, wt, fac = oracle_case(name)
    h = handle(R, w, prec)
    R.rfdd_factor(h, z, wt)
    X = np.random.default_rng(11).standard_normal((blk.s, 5))
    Wg = R.rfdd_filter_apply(h, X)
    Wo = O.filter_interface(fac, wt, X)
    assert relmax(Wg, Wo) <= TOL[prec]["fac"], relmax(Wg, Wo)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("block", [1, 4, 32])
def test_lanczos_basis(R, prec, block):
    """a7: orthonormal basis, trace monotone, captures the interface parts of the wanted
    eigenvectors (Eq. spann), mu <= s (Prop. lowrank)."""
    name = "q1_2d_33_p9"
    w, blk, z, wt, fac = oracle_case(name)
    h = handle(R, w, prec, block=block)
    R.rfdd_factor(h, z, wt)
    Q, tr = R.rfdd_lanczos(h)
    mu = Q.shape[1]
    assert 0 < mu <= blk.s
    np.testing.assert_allclose(Q.T @ Q, np.eye(mu), atol=1e-12)
    lam, X = sla.eigh(blk.Ap.toarray(), blk.Mp.toarray())
    Yin = X[blk.off[-1]:, (lam > w.alpha) & (lam < w.beta)]
    miss = np.linalg.norm(Yin - Q @ (Q.T @ Yin), axis=0) / np.linalg.norm(Yin, axis=0)
    assert miss.max() <= (1e-6 if prec == 0 else 1e-4), miss.max()
    # same span as the oracle's block Lanczos from the same counter-based start block (FP64)
    if prec == 0 and block == 4:
        lz = O.lanczos_interface(lambda V: O.filter_interface(fac, wt, V), blk.s, 1e-6, block=4, seed=1)
        Qo = lz["Q"][:, :min(mu, lz["mu"], 16)]
        sv = np.linalg.svd(Q.T @ Qo, compute_uv=False)
        assert sv.min() >= 1 - 1e-8


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["q1_2d_24", "q1_3d_12"])
def test_interior_chains_and_rr(R, name, prec):
    """a8: Sigma^(psi), Gamma^(psi) of Eq. (trabala2) from the GPU's Q, element by element; V_j
    M_B-orthonormal and close to the oracle's eigenvectors; a9: Ritz values of range(Z)."""
    w, blk, z, wt, fac = oracle_case(name)
    h = handle(R, w, prec, nev_b=12)
    R.rfdd_factor(h, z, wt)
    Q, _ = R.rfdd_lanczos(h)
    sigma = 0.5 * (w.alpha + w.beta)
    Z, k, kappa = R.rfdd_interior(h, sigma)
    mu, psi = Q.shape[1], 3
    Sig, Gam = O.resolvent_chains(blk, sigma, Q, psi)
    dsum = blk.off[-1]
    for j in range(blk.p):
        lo, hi = blk.off[j], blk.off[j + 1]
        S_g = -Z[lo:hi, kappa:kappa + psi * mu]
        G_g = Z[lo:hi, kappa + psi * mu:kappa + 2 * psi * mu]
        assert relmax(S_g, Sig[j]) <= TOL[prec]["fac"] * 10, (j, relmax(S_g, Sig[j]))
        assert relmax(G_g, Gam[j]) <= TOL[prec]["fac"] * 10, (j, relmax(G_g, Gam[j]))
    np.testing.assert_allclose(Z[dsum:, kappa:kappa + mu], Q, atol=1e-15)
    assert np.abs(Z[dsum:, :kappa]).max() == 0 and np.abs(Z[dsum:, kappa + mu:]).max() == 0
    # V_j: M_B-orthonormal, and spans nearly the oracle's eigenvectors closest to sigma
    Vo = O.interior_eigvecs(blk, sigma, 12)
    col = 0
    for j in range(blk.p):
        lo, hi = blk.off[j], blk.off[j + 1]
        Vg = Z[lo:hi, col:col + Vo[j].shape[1]]
        col += Vo[j].shape[1]
        np.testing.assert_allclose(Vg.T @ blk.MB[j] @ Vg, np.eye(Vg.shape[1]), atol=1e-9)
        # subspace iteration converges first for the eigenvalues nearest sigma: all but the
        # last three of the nev_B oracle directions must be captured
        sv = np.linalg.svd(Vg.T @ blk.MB[j] @ Vo[j], compute_uv=False)
        assert sv[:-3].min() >= 0.99, sv
    # a9: Ritz values on range(Z) vs the oracle's Rayleigh-Ritz on the same Z.  Z's columns are
    # numerically dependent; the oracle prunes near-null directions of Z^T M Z by its
    # eigendecomposition, the GPU by pivoted Cholesky (both at 1e-12), so the two Ritz sets agree
    # to the RF-DDES approximation level (a few 1e-6 relative here), not to rounding.  Both must be
    # equally close to the exact eigenvalues.
    th_g = R.rfdd_rayleigh_ritz(h)
    th_o, _ = O.rayleigh_ritz(blk.Ap, blk.Mp, Z)
    sel_o = th_o[(th_o > w.alpha) & (th_o < w.beta)]
    sel_g = th_g[(th_g > w.alpha) & (th_g < w.beta)]
    assert len(sel_g) == len(sel_o)
    np.testing.assert_allclose(sel_g, sel_o, rtol=1e-5)
    ex = w.exact[(w.exact > w.alpha) & (w.exact < w.beta)]
    if len(ex) == len(sel_o):
        err_o = np.max(np.abs(sel_o - ex) / ex)
        err_g = np.max(np.abs(sel_g - ex) / ex)
        assert err_g <= 3.0 * err_o + 1e-9, (err_g, err_o)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["q1_2d_24", "q1_3d_12"])
def test_rayleigh_ritz_on_a_well_conditioned_basis(R, name, prec):
    """a9 to rounding: with psi = 1 and nev_b = 4 the basis Z is far from rank deficient (the
    unit-diagonal Gram matrix Z^T M Z has its smallest eigenvalue near 1e-4..1e-2, far above the
    1e-12 pruning threshold), so both pruning rules keep every column and the Rayleigh-Ritz values
    of range(Z) are unique: the GPU's must equal the oracle's on the same Z to 1e-10 (FP64) /
    1e-9 (mixed, whose Gram matrix is formed in double-FP32 arithmetic)."""
    w, blk, z, wt, fac = oracle_case(name)
    h = handle(R, w, prec, nev_b=4, psi=1, block=4)
    R.rfdd_factor(h, z, wt)
    R.rfdd_lanczos(h)
    sigma = 0.5 * (w.alpha + w.beta)
    Z, k, kappa = R.rfdd_interior(h, sigma)
    G = Z.T @ (blk.Mp @ Z)
    dg = 1.0 / np.sqrt(np.diag(G))
    assert np.linalg.eigvalsh(G * dg[:, None] * dg[None, :])[0] >= 1e-8
    th_g = R.rfdd_rayleigh_ritz(h)
    th_o, _ = O.rayleigh_ritz(blk.Ap, blk.Mp, Z)
    assert len(th_g) == len(th_o) == k
    rel = np.abs(th_g - th_o) / np.abs(th_o)
    assert rel.max() <= (1e-10 if prec == 0 else 1e-9), rel.max()


def check_result(R, w, ev, X, rs, info, prec):
    ex = w.exact[(w.exact > w.alpha) & (w.exact < w.beta)] if w.exact is not None else None
    assert info["status"] == 0, info
    if ex is not None:
        assert len(ev) == len(ex) == w.expected_nev
        assert np.max(np.abs(ev - ex) / ex) <= TOL[prec]["ev"], np.max(np.abs(ev - ex) / ex)
    assert rs.max() <= 1e-10, rs.max()
    M = w.M.to_scipy()
    G = X.T @ (M @ X)
    assert np.abs(G - np.eye(len(ev))).max() <= TOL[prec]["orth"]
    A = w.A.to_scipy()
    res = np.linalg.norm(A @ X - (M @ X) * ev, axis=0) / (np.abs(ev) * np.linalg.norm(M @ X, axis=0))
    assert res.max() <= 1e-10, res.max()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["q1_2d_40", "q1_2d_24", "q1_2d_33_p9", "q1_3d_12", "q1_3d_16"])
def test_end_to_end(R, name, prec):
    """a0-a10: eigenpairs in [alpha, beta] against the closed form, residuals, M-orthonormality,
    and the oracle's eigenvalues."""
    w = I.workload(name)
    ev, X, rs, info = R.solve(w.A, w.M, w.part, w.p, w.alpha, w.beta, w.n_nodes, precision=prec,
                              quad_rule=RULES[w.rule])
    check_result(R, w, ev, X, rs, info, prec)
    if name in ("q1_2d_40", "q1_2d_24"):
        ro = O.rfdd_solve(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p, w.alpha, w.beta, w.n_nodes, w.rule)
        np.testing.assert_allclose(ev, ro["evals"], rtol=TOL[prec]["ev"])


@pytest.mark.parametrize("name", ["q1_2d_24", "q1_3d_12"])
def test_factor_forms_give_the_same_pairs(R, name):
    """Mixed solve with the complex64 factors only (every solve product packs its factor block on
    the fly) and with their tile copies only (packed once, complex64 freed): the same pairs."""
    w = I.workload(name)
    out = {}
    for pk in (0, 1):
        ev, X, rs, info = R.solve(w.A, w.M, w.part, w.p, w.alpha, w.beta, w.n_nodes, precision=1,
                                  quad_rule=RULES[w.rule], pack_factors=pk)
        assert info["packed"] == pk
        check_result(R, w, ev, X, rs, info, 1)
        out[pk] = ev
    np.testing.assert_allclose(out[0], out[1], rtol=1e-10)


def test_device_resident_csr_gives_the_same_pairs(R):
    """rfdd_setup with A and M in device memory (rfdd_csr.location = 1) solves the same problem as
    with host arrays; an unknown location is refused."""
    import torch

    class DevCsr:
        def __init__(self, c):
            self.rowptr = torch.from_numpy(c.rowptr.astype(np.int64)).cuda()
            self.col = torch.from_numpy(c.col.astype(np.int32)).cuda()
            self.val = torch.from_numpy(c.val.astype(np.float64)).cuda()

    w = I.workload("q1_2d_24")
    ev0, X0, rs0, _ = R.solve(w.A, w.M, w.part, w.p, w.alpha, w.beta, w.n_nodes)
    ev1, X1, rs1, info = R.solve(DevCsr(w.A), DevCsr(w.M), w.part, w.p, w.alpha, w.beta, w.n_nodes)
    np.testing.assert_array_equal(ev0, ev1)
    assert info["status"] == 0 and rs1.max() <= 1e-10
    a = R._Csr(w.A)
    a.s.location = 7
    m = R._Csr(w.M)
    out = R.C.c_void_p()
    pt = np.ascontiguousarray(w.part, dtype=np.int32)
    rc = R.load().rfdd_setup(R.C.byref(a.s), R.C.byref(m.s), pt.ctypes.data_as(R.C.POINTER(R.C.c_int32)), w.p,
                             None, R.C.byref(out))
    assert rc == R.RFDD_EINVAL


@pytest.mark.parametrize("prec", [0, 1])
def test_completion_block_grows_when_rfddes_finds_too_few(R, prec):
    """A poor RF-DDES basis (one eigenvector per subdomain, psi = 1, a loose Krylov tolerance) finds
    far fewer Ritz values inside a wide interval than it holds; the completion block, sized from
    that count without tile rounding, fills up and must grow until every eigenvalue is found."""
    w = I.workload("q1_2d_24")
    ev = w.exact
    first, last = I.snap_to_gaps(ev, 11, 90)
    a, b = I.interval_from_sorted(ev, first, last)
    got, X, rs, info = R.solve(w.A, w.M, w.part, w.p, a, b, 8, precision=prec, nev_b=1, psi=1, block=2,
                               lanczos_tol=0.5, m_align=1)
    assert info["pre_nev"] < last - first + 1          # RF-DDES alone is short here
    assert info["status"] == 0 and len(got) == last - first + 1
    assert info["m"] >= len(got) and rs.max() <= 1e-10
    np.testing.assert_allclose(got, ev[first - 1:last], rtol=TOL[prec]["ev"])


@pytest.mark.parametrize("prec", [0, 1])
def test_edge_cases_one_node_block_one(R, prec):
    """Nc = 1, Lanczos block 1 (the printed Algorithm 2), psi = 1."""
    w = I.workload("q1_2d_24")
    ev, X, rs, info = R.solve(w.A, w.M, w.part, w.p, w.alpha, w.beta, 1, precision=prec, block=1, psi=1,
                              max_passes=30)
    check_result(R, w, ev, X, rs, info, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_edge_case_single_subdomain(R, prec):
    """p = 1: one subdomain whose interface is the last grid row."""
    N = 20
    A, M = I.q1_pencil(N, 2)
    part = np.zeros(N * N, dtype=np.int32)
    part[-N:] = -1
    ex = I.q1_eigenvalues(N, 2)
    first, last = I.snap_to_gaps(ex, 5, 14)
    a, b = I.interval_from_sorted(ex, first, last)
    ev, X, rs, info = R.solve(A, M, part, 1, a, b, 6, precision=prec)
    assert len(ev) == last - first + 1
    np.testing.assert_allclose(ev, ex[first - 1:last], rtol=TOL[prec]["ev"])
    assert rs.max() <= 1e-10


def test_empty_interval(R):
    """An interval with no eigenvalue returns nev = 0."""
    w = I.workload("q1_2d_24")
    ex = w.exact
    a = ex[5] + 0.2 * (ex[6] - ex[5])
    b = ex[5] + 0.4 * (ex[6] - ex[5])
    ev, X, rs, info = R.solve(w.A, w.M, w.part, w.p, a, b, 4)
    assert len(ev) == 0 and info["nev"] == 0


def test_call_order_errors(R):
    w = I.workload("q1_2d_24")
    h = handle(R, w, 1)
    with pytest.raises(R.RfddError) as e:
        R.rfdd_filter_apply(h, np.zeros((10, 1)))
    assert e.value.code == R.RFDD_ESTATE
    with pytest.raises(R.RfddError) as e:
        R.rfdd_setup(w.A, w.M, w.part, w.p, R.rfdd_default_options(block=0))
    assert e.value.code == R.RFDD_EINVAL
