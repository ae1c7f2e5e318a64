"""Pins for the domain-decomposition pieces of the oracle (Sections 2.3, 3, 4, 5).

Each test checks the oracle against an independent mathematical fact: a dense inverse, a dense
eigendecomposition of the whole pencil, a closed-form spectrum, the paper's theorems, or an
inertia count.  Pencils: small Q1 Laplacians and random pencils with the same block pattern.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import rfdd_inputs as I
from oracle import rfdd_oracle as O


def random_pencil(N=9, splits=(2, 2), seed=0, mass_coupling=True):
    """Random symmetric A and SPD M on the 9-point pattern of an N x N grid (so a 2-D geometric
    vertex separator is valid), with random weights."""
    rng = np.random.default_rng(seed)
    A0, M0 = I.q1_pencil(N, 2)
    pat = A0.to_scipy().tocoo()
    off = pat.row != pat.col
    r, c = pat.row[off], pat.col[off]
    keep = r < c
    r, c = r[keep], c[keep]
    n = N * N
    va = rng.uniform(-1, 1, r.size)
    A = sp.coo_matrix((va, (r, c)), shape=(n, n))
    A = A + A.T + sp.diags(rng.uniform(-3, 3, n))
    if mass_coupling:
        vm = rng.uniform(-0.1, 0.1, r.size)
        Mo = sp.coo_matrix((vm, (r, c)), shape=(n, n))
        Mo = Mo + Mo.T
        M = Mo + sp.diags(np.abs(Mo).sum(1).A1 + rng.uniform(0.5, 1.5, n))
    else:
        M = sp.diags(rng.uniform(0.5, 1.5, n))
    part, p = I.geometric_partition(N, 2, splits)
    return sp.csr_matrix(A), sp.csr_matrix(M), part, p


def dense_eig(A, M):
    lam, X = sla.eigh(A.toarray(), M.toarray())
    return lam, X


# ----------------------------------------------------------------------------------------
# inputs (the generator itself is pinned by closed forms)
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("N,dim", [(7, 2), (4, 3)])
def test_q1_closed_form_against_dense(N, dim):
    A, M = I.q1_pencil(N, dim)
    lam, _ = dense_eig(A.to_scipy(), M.to_scipy())
    np.testing.assert_allclose(lam, I.q1_eigenvalues(N, dim), rtol=1e-11)


def test_config_partitions():
    w = I.workload("q1_2d_40")
    blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
    assert sorted(blk.d.tolist()) == [361, 380, 380, 400] and blk.s == 79
    assert w.expected_nev == 50
    np.testing.assert_allclose([w.alpha, w.beta], [742.987601889, 1499.74966257], rtol=1e-11)
    part, p = I.geometric_partition(40, 3, (2, 2, 2))
    counts = np.bincount(part[part >= 0])
    assert p == 8 and np.count_nonzero(part == -1) == 4681
    assert sorted(set(counts.tolist())) == [6859, 7220, 7600, 8000]


def test_varkappa_pencil_and_shifted_partition():
    A, M = I.varkappa7_pencil(10, seed=5)
    a = A.to_scipy()
    assert abs(a - a.T).max() == 0
    assert np.all(np.linalg.eigvalsh(a.toarray()) > 0)
    assert np.all(M.to_scipy().diagonal() >= 0.5) and np.all(M.to_scipy().diagonal() <= 1.5)
    part, p = I.geometric_partition(10, 3, (2, 2, 2), shift_frac=0.3, seed=3)
    O.Blocks(a, M.to_scipy(), part, p)     # raises if the separator is not valid


# ----------------------------------------------------------------------------------------
# Section 3.1: Schur complement, block inverse, identity (finalizing)
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1])
def test_block_inverse_matches_dense(seed):
    A, M, part, p = random_pencil(seed=seed)
    blk = O.Blocks(A, M, part, p)
    z = 0.3 + 0.7j
    fac = O.Factors(blk, [z])
    rng = np.random.default_rng(seed + 10)
    V = rng.standard_normal((blk.n, 3))
    X = fac.resolvent(0, V)
    dense = (blk.Ap - z * blk.Mp).toarray()
    np.testing.assert_allclose(dense @ X, V, atol=1e-10)
    # S is the (2,2) block of the inverse, inverted (Eq. inv_dd2)
    Sinv = np.linalg.inv(dense)[blk.off[-1]:, blk.off[-1]:]
    np.testing.assert_allclose(np.linalg.inv(O.schur(blk, z)), Sinv, atol=1e-10)


@pytest.mark.parametrize("rule,nc", [("midpoint", 4), ("gauss_legendre", 3), ("midpoint", 1)])
def test_finalizing_identity(rule, nc):
    # Eq. (finalizing): 2 Re sum_l omega_l S(zeta_l)^{-1} = sum_i rho(lambda_i) y_i y_i^T, with
    # y_i the interface rows of the M-orthonormal eigenvectors.
    A, M, part, p = random_pencil(seed=3)
    blk = O.Blocks(A, M, part, p)
    lam, X = dense_eig(blk.Ap, blk.Mp)
    alpha, beta = lam[20] - 0.01, lam[35] + 0.01
    z, w = O.quadrature(alpha, beta, nc, rule)
    fac = O.Factors(blk, z)
    F = 2.0 * O.filter_interface(fac, w, np.eye(blk.s))
    Y = X[blk.off[-1]:]
    want = (Y * O.filter_value(lam, z, w)) @ Y.T
    np.testing.assert_allclose(F, want, atol=1e-10 * np.abs(want).max())
    np.testing.assert_allclose(F, F.T, atol=1e-12 * np.abs(F).max())


def test_full_filter_is_spectral(tmp_path):
    # Eq. (rhoAM) with Eq. (pole_eig): 2 Re sum omega (A - zeta M)^{-1} M x_i = rho(lambda_i) x_i.
    A, M, part, p = random_pencil(seed=4)
    blk = O.Blocks(A, M, part, p)
    lam, X = dense_eig(blk.Ap, blk.Mp)
    z, w = O.quadrature(lam[10] - 0.05, lam[19] + 0.05, 6, "midpoint")
    fac = O.Factors(blk, z)
    out = O.filter_full(fac, w, blk.Mp @ X)
    np.testing.assert_allclose(out, X * O.filter_value(lam, z, w), atol=1e-9)


def test_prop_lowrank_and_lanczos():
    # Prop. (lowrank): rank([y_1..y_nev]) <= r(S) <= s; Algorithm 2 captures span{y_i}.
    w = I.workload("q1_2d_24")
    blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
    lam, X = dense_eig(blk.Ap, blk.Mp)
    z, wts = O.quadrature(w.alpha, w.beta, 8, "midpoint")
    fac = O.Factors(blk, z)
    F = O.filter_interface(fac, wts, np.eye(blk.s))
    inside = (lam > w.alpha) & (lam < w.beta)
    Yin = X[blk.off[-1]:, inside]
    rank_y = np.linalg.matrix_rank(Yin, tol=1e-8 * np.abs(Yin).max())
    sv = np.linalg.svd(F, compute_uv=False)
    r_s = int(np.count_nonzero(sv > 1e-14 * sv[0]))
    assert rank_y <= r_s <= blk.s
    for b in (1, 4):
        lz = O.lanczos_interface(lambda V: O.filter_interface(fac, wts, V), blk.s, 1e-6, block=b, seed=5)
        Q = lz["Q"]
        assert lz["mu"] <= blk.s
        np.testing.assert_allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-12)
        resid = Yin - Q @ (Q.T @ Yin)
        assert np.linalg.norm(resid, axis=0).max() < 1e-6 * np.linalg.norm(Yin, axis=0).max()
        # the trace of T_mu equals the trace of Q^T F Q (the sum of its eigenvalues)
        np.testing.assert_allclose(lz["traces"][-1], np.trace(Q.T @ F @ Q), rtol=1e-9)


# ----------------------------------------------------------------------------------------
# Section 4: Lemma (prop:error), Theorems (uuhat), (uuhat2), (all)
# ----------------------------------------------------------------------------------------

def _theorem_setup(seed=2):
    A, M, part, p = random_pencil(N=8, splits=(2, 2), seed=seed)
    blk = O.Blocks(A, M, part, p)
    lam, X = dense_eig(blk.Ap, blk.Mp)
    dsum = blk.off[-1]
    B = sla.block_diag(*blk.B)
    MB = sla.block_diag(*blk.MB)
    E = np.vstack(blk.E)
    ME = np.vstack(blk.ME)
    delta, Vb = sla.eigh(B, MB)
    return blk, lam, X, dsum, B, MB, E, ME, delta, Vb


def _mb_norm(v, MB):
    return float(np.sqrt(v @ MB @ v))


def _minv_norm(v, MB):
    return float(np.sqrt(v @ np.linalg.solve(MB, v)))


def _project(U, u, MB):
    """argmin over g in span(U) of ||u - g||_{M_B}."""
    G = U.T @ MB @ U
    c = np.linalg.lstsq(G, U.T @ MB @ u, rcond=None)[0]
    return U @ c


@pytest.mark.parametrize("psi", [1, 2, 3])
def test_theorems_uuhat(psi):
    blk, lam, X, dsum, B, MB, E, ME, delta, Vb = _theorem_setup()
    sigma = 0.5 * (lam[30] + lam[31]) + 0.013
    Bs = B - sigma * MB
    Es = E - sigma * ME
    for i in range(25, 36):
        l = lam[i]
        u, y = X[:dsum, i], X[dsum:, i]
        # Lemma (prop:error) with Eq. (prol2)
        uhat = -np.linalg.solve(Bs, Es @ y)
        Bl = B - l * MB
        lemma = -(np.linalg.inv(Bl) - np.linalg.inv(Bs)) @ Es @ y + (l - sigma) * np.linalg.solve(Bl, ME @ y)
        np.testing.assert_allclose(u - uhat, lemma, atol=1e-9 * max(1, np.abs(u).max()))
        # Theorem (uuhat2) (psi = 1 is Theorem (uuhat)'s subspace; its bound is the psi=1 case
        # of the first term plus |l-s|/|l-d| * ||M_E y||)
        U1, U2 = [], []
        x1 = np.linalg.solve(Bs, Es @ y)
        x2 = np.linalg.solve(Bs, ME @ y)
        for t in range(psi):
            U1.append(x1)
            U2.append(x2)
            x1 = np.linalg.solve(Bs, MB @ x1)
            x2 = np.linalg.solve(Bs, MB @ x2)
        U = np.column_stack(U1 + U2)
        err = _mb_norm(u - _project(U, u, MB), MB)
        ne, nm = _minv_norm(Es @ y, MB), _minv_norm(ME @ y, MB)
        den = np.abs((l - delta) * (sigma - delta) ** psi)
        bound = np.max(abs(l - sigma) ** psi / den) * ne + np.max(abs(l - sigma) ** (psi + 1) / den) * nm
        assert err <= bound * (1 + 1e-8) + 1e-12
        if psi == 1:
            # Theorem (uuhat) for the basic approximation itself
            b1 = (np.max(abs(l - sigma) / np.abs((l - delta) * (sigma - delta))) * ne
                  + np.max(abs(l - sigma) / np.abs(l - delta)) * nm)
            assert _mb_norm(u - uhat, MB) <= b1 * (1 + 1e-8)
        # Theorem (all): deflate the kappa eigenvectors of (B, M_B) closest to sigma
        kappa = 6
        near = np.argsort(np.abs(delta - sigma))[:kappa]
        far = np.setdiff1d(np.arange(len(delta)), near)
        Ud = np.column_stack([U, Vb[:, near]])
        err3 = _mb_norm(u - _project(Ud, u, MB), MB)
        den_f = den[far]
        bound3 = (np.max(abs(l - sigma) ** psi / den_f) * ne
                  + np.max(abs(l - sigma) ** (psi + 1) / den_f) * nm)
        assert err3 <= bound3 * (1 + 1e-8) + 1e-12


# ----------------------------------------------------------------------------------------
# Counting, Rayleigh-Ritz sanity case, end to end
# ----------------------------------------------------------------------------------------

def test_inertia_counts():
    w = I.workload("q1_2d_24")
    blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
    ev = w.exact
    for sig in (w.alpha, w.beta, 0.5 * (ev[3] + ev[4]), ev[-1] + 1.0):
        assert O.inertia_count(blk, sig) == int(np.count_nonzero(ev < sig))
    assert O.inertia_count(blk, w.beta) - O.inertia_count(blk, w.alpha) == w.expected_nev


def test_rr_with_full_subspace_is_exact():
    # Sanity case: nev_B = d_j and mu = s make range(Z) = R^n, so Rayleigh-Ritz is exact.
    A, M, part, p = random_pencil(N=7, seed=6)
    blk = O.Blocks(A, M, part, p)
    lam, _ = dense_eig(blk.Ap, blk.Mp)
    sigma = 0.1
    V = O.interior_eigvecs(blk, sigma, 10 ** 6)
    Q = np.linalg.qr(np.random.default_rng(0).standard_normal((blk.s, blk.s)))[0]
    Sig, Gam = O.resolvent_chains(blk, sigma, Q, 2)
    Z = O.build_Z(blk, V, Sig, Gam, Q, 2)
    th, Xr = O.rayleigh_ritz(blk.Ap, blk.Mp, Z)
    np.testing.assert_allclose(th, lam, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(Xr.T @ (blk.Mp @ Xr), np.eye(blk.n), atol=1e-9)


def test_gamma_dropped_when_me_zero():
    A, M, part, p = random_pencil(N=7, seed=7, mass_coupling=False)
    blk = O.Blocks(A, M, part, p)
    Q = np.linalg.qr(np.random.default_rng(1).standard_normal((blk.s, 4)))[0]
    V = O.interior_eigvecs(blk, 0.0, 3)
    Sig, Gam = O.resolvent_chains(blk, 0.0, Q, 3)
    assert all(np.abs(g).max() == 0 for g in Gam)
    Z = O.build_Z(blk, V, Sig, Gam, Q, 3)
    assert Z.shape[1] == 3 * p + 3 * 4          # kappa + psi*mu, no Gamma block


def test_end_to_end_config1_closed_form():
    w = I.workload("q1_2d_40")
    r = O.rfdd_solve(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p, w.alpha, w.beta, w.n_nodes, w.rule)
    ex = w.exact[(w.exact > w.alpha) & (w.exact < w.beta)]
    assert r["converged"] and len(r["evals"]) == w.expected_nev == 50
    assert np.max(np.abs(r["evals"] - ex) / ex) <= 1e-10
    assert r["resid"].max() <= 1e-10
    Xv = r["evecs"]
    G = Xv.T @ (w.M.to_scipy() @ Xv)
    assert np.abs(G - np.eye(len(ex))).max() <= 1e-10
    # the pre-completion RF-DDES error is paper-like (tbl:15/17 range), not exact
    assert r["pre"]["res"].max() > 1e-10


@pytest.mark.parametrize("seed", [11, 12])
def test_end_to_end_random_pencil_brute_force(seed):
    A, M, part, p = random_pencil(N=12, splits=(3, 2), seed=seed)
    lam, X = dense_eig(A, M)
    alpha, beta = 0.5 * (lam[40] + lam[41]), 0.5 * (lam[60] + lam[61])
    r = O.rfdd_solve(A, M, part, p, alpha, beta, 6, "midpoint", nev_b=10, block=2)
    ex = lam[41:61]
    assert r["converged"] and len(r["evals"]) == 20
    np.testing.assert_allclose(r["evals"], ex, rtol=1e-10)
    # eigenvectors: same span per cluster (all simple here) -> |cos| = 1
    Mx = M @ X[:, 41:61]
    C = r["evecs"].T @ Mx
    np.testing.assert_allclose(np.abs(np.diag(C)), 1.0, atol=1e-8)


def test_sigma_guard_moves_a_shift_on_a_subdomain_eigenvalue():
    """sigma exactly at an eigenvalue of (B_0, M_B^(0)): the guard moves it by 1e-6 (beta - alpha)
    and the solve still returns the brute-force eigenpairs; a shift away from the subdomain
    spectra is kept."""
    A, M, part, p = random_pencil(N=12, splits=(3, 2), seed=11)
    lam, _ = dense_eig(A, M)
    alpha, beta = 0.5 * (lam[40] + lam[41]), 0.5 * (lam[60] + lam[61])
    blk = O.Blocks(A, M, part, p)
    d0 = sla.eigh(blk.B[0], blk.MB[0], eigvals_only=True)
    sig = float(d0[np.argmin(np.abs(d0 - 0.5 * (alpha + beta)))])
    r = O.rfdd_solve(A, M, part, p, alpha, beta, 6, "midpoint", sigma=sig, nev_b=10, block=2)
    assert r["sigma"] == sig + 1e-6 * (beta - alpha)
    assert r["converged"]
    np.testing.assert_allclose(r["evals"], lam[41:61], rtol=1e-10)
    sub = np.concatenate([sla.eigh(blk.B[j], blk.MB[j], eigvals_only=True) for j in range(p)])
    far = 0.5 * (alpha + beta)
    assert np.abs(sub - far).min() > 1e-6 * abs(far)
    r2 = O.rfdd_solve(A, M, part, p, alpha, beta, 6, "midpoint", sigma=far, nev_b=10, block=2)
    assert r2["sigma"] == far


@pytest.mark.parametrize("name", ["q1_3d_12", "q1_2d_33_p9"])
def test_sparse_schur_columns_match_the_dense_definition(name):
    """schur_columns (sparse LUs, for pencils too large for dense blocks) is the same S(zeta)."""
    w = I.workload(name)
    blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
    z, _ = O.quadrature(w.alpha, w.beta, w.n_nodes, w.rule)
    cols = [0, 1, blk.s // 2, blk.s - 1]
    for l in (0, len(z) - 1):
        Sd = O.schur(blk, z[l])[:, cols]
        Ss = O.schur_columns(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p, z[l], cols)
        assert np.abs(Ss - Sd).max() <= 1e-12 * np.abs(Sd).max()
