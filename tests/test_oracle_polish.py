"""Pins of the oracle's interior polish (Section 3, Eqs. (schur_eigvec2) and
(compute_u_parallel)): from the interface rows of an exact eigenvector (a dense generalized
eigensolve, LAPACK), the per-subdomain solves must give back the whole eigenvector; the
decoupled solves must equal the one undecoupled solve of Eq. (schur_eigvec2); and plausible
mistakes planted in a copy of the routine must fail the first pin."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import rfdd_oracle as O
from tests.test_oracle_dd import dense_eig, random_pencil

IDX = [3, 10, 25, 40, 66]  # of the 81 eigenpairs of a 9 x 9 grid pencil


def exact_pairs(seed, mass):
    A, M, part, p = random_pencil(seed=seed, mass_coupling=mass)
    blk = O.Blocks(A, M, part, p)
    lam, Xp = dense_eig(blk.Ap, blk.Mp)  # interior-first ordering, M-orthonormal columns
    return blk, lam[IDX], blk.to_original(Xp[:, IDX])


def scramble_interior(blk, X, seed):
    """The same columns with every interior row replaced by noise (input ordering)."""
    Xp = X[blk.perm].copy()
    dsum = int(blk.off[-1])
    Xp[:dsum] = np.random.default_rng(seed).standard_normal((dsum, X.shape[1]))
    return blk.to_original(Xp)


def recovery_error(polish, seed=0, mass=True):
    blk, lam, X = exact_pairs(seed, mass)
    lam2, X2, res = polish(blk, lam, scramble_interior(blk, X, seed + 100))
    return np.abs(lam2 - lam).max() / np.abs(lam).max(), np.abs(X2 - X).max() / np.abs(X).max(), res.max()


@pytest.mark.parametrize("seed,mass", [(0, True), (4, True), (2, False)])
def test_polish_recovers_dense_eigenvectors_from_interface_rows(seed, mass):
    el, ex, res = recovery_error(O.polish_interior, seed, mass)
    assert el < 1e-12 and ex < 1e-10 and res < 1e-12


def test_polish_matches_the_undecoupled_interior_solve():
    """Eq. (schur_eigvec2) with the whole block-diagonal B - lambda M_B at once, for an arbitrary
    (not an eigenvalue) lambda and interface vector."""
    A, M, part, p = random_pencil(seed=7)
    blk = O.Blocks(A, M, part, p)
    n, dsum = blk.n, int(blk.off[-1])
    rng = np.random.default_rng(1)
    lam = np.array([0.37, -1.2])
    Xp = rng.standard_normal((n, 2))
    lam2, X2, _ = O.polish_interior(blk, lam, blk.to_original(Xp))
    Ap, Mp = blk.Ap.toarray(), blk.Mp.toarray()
    for i, li in enumerate(lam):
        x = Xp[:, i].copy()
        K = Ap[:dsum, :dsum] - li * Mp[:dsum, :dsum]
        x[:dsum] = np.linalg.solve(K, -(Ap[:dsum, dsum:] - li * Mp[:dsum, dsum:]) @ x[dsum:])
        x /= np.sqrt(x @ Mp @ x)
        np.testing.assert_allclose(X2[:, i], blk.to_original(x), rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(lam2[i], x @ Ap @ x, rtol=1e-12)


def _polish_variant(mistake):
    """A copy of the polish with one planted mistake."""
    def polish(blk, lam, X):
        Xp = np.asarray(X, dtype=float)[blk.perm]
        n, nev = Xp.shape
        dsum = int(blk.off[-1])
        lam_new, Xnew = np.empty(nev), np.empty((n, nev))
        for i in range(nev):
            li = float(lam[i])
            x = Xp[:, i].copy()
            y = x[dsum:]
            for j in range(blk.p):
                lo, hi = blk.off[j], blk.off[j + 1]
                Ez = blk.E[j] if mistake == "drop_ME" else blk.E[j] - li * blk.ME[j]
                rhs = (Ez @ y) if mistake == "rhs_sign" else -(Ez @ y)
                Bz = blk.B[j] + li * blk.MB[j] if mistake == "shift_sign" else blk.B[j] - li * blk.MB[j]
                x[lo:hi] = sla.solve(Bz, rhs)
            xMx = x @ (blk.Mp @ x)
            lam_new[i] = (x @ (blk.Ap @ x)) / xMx
            Xnew[:, i] = x / np.sqrt(xMx)
        return lam_new, blk.to_original(Xnew), O.residuals(blk.Ap, blk.Mp, lam_new, Xnew)
    return polish


@pytest.mark.parametrize("mistake", ["drop_ME", "rhs_sign", "shift_sign"])
def test_pin_catches_planted_polish_mistakes(mistake):
    el, ex, res = recovery_error(_polish_variant("none"))
    assert el < 1e-12 and ex < 1e-10 and res < 1e-12
    el, ex, res = recovery_error(_polish_variant(mistake))
    assert ex > 1e-3 and res > 1e-6
