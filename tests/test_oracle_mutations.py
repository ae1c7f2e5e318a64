"""The oracle's pins must catch plausible mistakes.  Each case plants one mistake in a copy of an
oracle routine (CPU only) and checks that the matching pin then fails."""
import numpy as np
import scipy.linalg as sla

import rfdd_inputs as I
from oracle import rfdd_oracle as O
from tests.test_oracle_dd import random_pencil, dense_eig


def _finalizing_error(schur_fn, quad_fn):
    A, M, part, p = random_pencil(seed=3)
    blk = O.Blocks(A, M, part, p)
    lam, X = dense_eig(blk.Ap, blk.Mp)
    z, w = quad_fn(lam[20] - 0.01, lam[35] + 0.01, 4, "midpoint")
    F = np.zeros((blk.s, blk.s))
    for l in range(len(z)):
        F += 2.0 * np.real(w[l] * np.linalg.inv(schur_fn(blk, z[l])))
    Y = X[blk.off[-1]:]
    want = (Y * O.filter_value(lam, z, w)) @ Y.T
    return np.abs(F - want).max() / np.abs(want).max()


def test_pin_catches_conjugate_transpose():
    def bad_schur(blk, z):
        Bz, Ez, Cz = O.shifted(blk, z)
        S = Cz.astype(complex).copy()
        for j in range(blk.p):
            S -= Ez[j].conj().T @ np.linalg.solve(Bz[j], Ez[j])
        return S
    assert _finalizing_error(O.schur, O.quadrature) < 1e-10
    assert _finalizing_error(bad_schur, O.quadrature) > 1e-3


def test_pin_catches_weight_sign_and_scale():
    def bad_quad(a, b, nc, rule):
        z, w = O.quadrature(a, b, nc, rule)
        return z, -w
    def bad_quad2(a, b, nc, rule):
        z, w = O.quadrature(a, b, nc, rule)
        return z, w * 2.0
    assert _finalizing_error(O.schur, bad_quad) < 1e-10      # consistent sign flips cancel here...
    z, w = bad_quad(-1.0, 1.0, 4, "midpoint")
    assert abs(O.filter_value([0.0], z, w)[0] - 1.0) > 0.5   # ...but rho(c) = 1 catches them
    z, w = bad_quad2(-1.0, 1.0, 4, "midpoint")
    assert abs(O.filter_value([1.0], z, w)[0] - 0.5) > 0.1   # rho(beta) = 1/2 catches scale


def test_pin_catches_dropped_mass_coupling_in_chains():
    # dropping -sigma M_E from Phi (Eq. trabala) breaks the full-subspace exactness pin only when
    # Gamma is also missing; drop Gamma and keep Phi wrong -> RR no longer exact
    A, M, part, p = random_pencil(N=7, seed=6)
    blk = O.Blocks(A, M, part, p)
    lam, _ = dense_eig(blk.Ap, blk.Mp)
    V = O.interior_eigvecs(blk, 0.1, 1)
    Q = np.linalg.qr(np.random.default_rng(0).standard_normal((blk.s, 3)))[0]
    good_sig, good_gam = O.resolvent_chains(blk, 0.1, Q, 2)
    bad_sig = []
    for j in range(blk.p):
        lu = sla.lu_factor(blk.B[j] - 0.1 * blk.MB[j])
        Phi = blk.E[j][:, blk.sidx[j]] @ Q[blk.sidx[j]]       # mistake: no -sigma M_E term
        X = sla.lu_solve(lu, Phi)
        bad_sig.append(np.hstack([X, sla.lu_solve(lu, blk.MB[j] @ X)]))
    Zg = O.build_Z(blk, V, good_sig, good_gam, Q, 2, with_gamma=False)
    Zb = O.build_Z(blk, V, bad_sig, good_gam, Q, 2, with_gamma=False)
    # the basic prolongation column block must equal -B_sigma^{-1} E_sigma Q (Eq. prol2)
    col0 = sum(v.shape[1] for v in V)
    dsum = blk.off[-1]
    Es = np.vstack([blk.E[j] - 0.1 * blk.ME[j] for j in range(blk.p)])
    Bs = sla.block_diag(*[blk.B[j] - 0.1 * blk.MB[j] for j in range(blk.p)])
    want = -np.linalg.solve(Bs, Es @ Q)
    assert np.abs(Zg[:dsum, col0:col0 + 3] - want).max() < 1e-10
    assert np.abs(Zb[:dsum, col0:col0 + 3] - want).max() > 1e-6


def test_pin_catches_wrong_interval_count():
    w = I.workload("q1_2d_24")
    blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
    # an inertia counter that forgot the Schur term would count only interior eigenvalues
    neg_b = sum(int(np.count_nonzero(np.linalg.eigvalsh(blk.B[j] - w.beta * blk.MB[j]) < 0))
                for j in range(blk.p))
    assert neg_b != int(np.count_nonzero(w.exact < w.beta))
    assert O.inertia_count(blk, w.beta) == int(np.count_nonzero(w.exact < w.beta))


def test_pins_catch_two_level_interface_mistakes():
    from tests.test_oracle_levels import _thick_separator_pencil
    # (1) level 1 without the demotion of C-coupled candidates of different groups: the thick
    # separator's two columns become level 1 of groups 0 and 1 while S couples them
    A, M, part, p, xs, ny = _thick_separator_pencil()
    blk = O.Blocks(A, M, part, p)
    good = O.interface_levels(blk, [0, 0, 1, 1])
    orig = np.flatnonzero
    groups = np.array([0, 0, 1, 1])
    touch = [set() for _ in range(blk.s)]
    for j in range(p):
        for a in blk.sidx[j]:
            touch[a].add(int(groups[j]))
    cls = np.array([next(iter(t)) if len(t) == 1 else -1 for t in touch])
    I1 = [orig(cls == g) for g in range(2)]
    S = O.schur(blk, 1.5 + 0.5j)
    assert np.all(S[np.ix_(good.I1[0], good.I1[1])] == 0)
    assert np.any(S[np.ix_(I1[0], I1[1])] != 0)
    # (2) S22' without the group updates S21 S11^{-1} S12: the Schur identity and the solve fail
    A, M, part, p = random_pencil(N=14, splits=(3, 3), seed=5)
    blk = O.Blocks(A, M, part, p)
    lv = O.interface_levels(blk, I.subdomain_groups((3, 3), (2, 2)))
    S = O.schur(blk, -0.2 + 0.9j)
    G = np.random.default_rng(5).standard_normal((blk.s, 3))
    ref = np.linalg.solve(S, G)
    bad = O.TwoLevelSchur(S, lv)
    bad.S22p = S[np.ix_(lv.I2, lv.I2)].copy()
    bad.lu22 = sla.lu_factor(bad.S22p)
    assert np.abs(O.TwoLevelSchur(S, lv).solve(G) - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.abs(bad.solve(G) - ref).max() > 1e-3 * np.abs(ref).max()
