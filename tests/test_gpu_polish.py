"""Interior polish (Section 3, Eq. (compute_u_parallel)) through the C ABI against the oracle.

Inputs: exact eigenpairs of the pencil from a dense generalized eigensolve (LAPACK), with every
interior row replaced by seeded noise; only the interface rows carry information.  The GPU
polish (FP64 throughout) must match the oracle's polish of the same inputs to 1e-10 (vectors,
relative to the largest entry) and 1e-12 (eigenvalues), and both must give back the exact
eigenvectors.  Pairs are chosen with a substantial interface part and an eigenvalue away from
the spectra of the subdomain pencils (B_j, M_B^(j)) (relative distance > 1e-3), where the solves
of Eq. (compute_u_parallel) are well conditioned.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import rfdd_inputs as I
from oracle import rfdd_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1711_09487_gb300 import build
    build.build()
    import paper_1711_09487_gb300 as pkg
    pkg.load()
    return pkg


_cache = {}


def case(name, npairs, seed=0):
    """(workload, Blocks, exact lam, exact X, scrambled X) in the input ordering."""
    key = (name, npairs, seed)
    if key not in _cache:
        w = I.workload(name)
        blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
        lam, Xp = sla.eigh(blk.Ap.toarray(), blk.Mp.toarray())
        dsum = int(blk.off[-1])
        sub = np.concatenate([sla.eigh(blk.B[j], blk.MB[j], eigvals_only=True) for j in range(blk.p)])
        ok = [i for i in range(len(lam))
              if np.linalg.norm(Xp[dsum:, i]) > 0.2 * np.linalg.norm(Xp[:, i])
              and np.abs(sub - lam[i]).min() > 1e-3 * abs(lam[i])]
        idx = np.array(ok)[np.linspace(0, len(ok) - 1, npairs).astype(int)]
        X = blk.to_original(Xp[:, idx])
        Xs = Xp[:, idx].copy()
        Xs[:dsum] = np.random.default_rng(seed).standard_normal((dsum, len(idx)))
        _cache[key] = (w, blk, lam[idx], X, blk.to_original(Xs))
    return _cache[key]


def relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("name,npairs", [("q1_2d_24", 9), ("q1_3d_12", 7), ("q1_2d_33_p9", 5)])
def test_polish_parity_with_oracle(R, name, npairs):
    w, blk, lam, X, Xs = case(name, npairs)
    h = R.rfdd_setup(w.A, w.M, w.part, w.p, R.rfdd_default_options())
    lg, Xg, rg = R.rfdd_polish(h, lam, Xs)
    lo, Xo, ro = O.polish_interior(blk, lam, Xs)
    assert relmax(lg, lo) <= 1e-12
    assert relmax(Xg, Xo) <= 1e-10
    np.testing.assert_allclose(rg, ro, rtol=1e-3, atol=1e-14)
    # both give back the exact eigenpairs
    assert relmax(lg, lam) <= 1e-12 and relmax(Xg, X) <= 1e-10 and rg.max() <= 1e-12


def test_polish_in_chunks_of_pairs_is_the_same(R):
    """A memory budget that holds the dense blocks of 3 pairs: chunks 3, 3, 3, 1 (ragged)."""
    w, blk, lam, X, Xs = case("q1_2d_24", 10, seed=1)
    h = R.rfdd_setup(w.A, w.M, w.part, w.p, R.rfdd_default_options())
    per_pair = int(sum(int(d) ** 2 for d in blk.d)) * 8
    hc = R.rfdd_setup(w.A, w.M, w.part, w.p, R.rfdd_default_options(mem_budget=2 * 3 * per_pair + 8))
    l1, X1, r1 = R.rfdd_polish(h, lam, Xs)
    l3, X3, r3 = R.rfdd_polish(hc, lam, Xs)
    np.testing.assert_array_equal(l1, l3)
    np.testing.assert_array_equal(X1, X3)
    np.testing.assert_array_equal(r1, r3)
    assert relmax(X1, X) <= 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_polish_of_a_solve_result_keeps_it_converged(R, prec):
    """Polishing converged pairs of a solve (interface parts accurate to the residual target)
    keeps them converged: the solves amplify the interface error by at most the conditioning of
    B_j - lambda M_B^(j) (relative distance of these eigenvalues to the subdomain spectra >= 5e-3
    for this workload), and the eigenvalues stay on the closed form."""
    w = I.workload("q1_2d_24")
    opts = R.rfdd_default_options(precision=prec, quad_rule=1 if w.rule == "gauss_legendre" else 0)
    h = R.rfdd_setup(w.A, w.M, w.part, w.p, opts)
    r = R.rfdd_solve(h, w.alpha, w.beta, w.n_nodes)
    ev, X, rs = R.rfdd_result_get(r)
    lp, Xp, rp = R.rfdd_polish(h, ev, X)
    ref = w.exact[(w.exact > w.alpha) & (w.exact < w.beta)]
    np.testing.assert_allclose(lp, ref, rtol=1e-10)
    assert rp.max() <= max(1e-10, 50.0 * rs.max())


def test_polish_edge_cases(R):
    w, blk, lam, X, Xs = case("q1_2d_24", 3)
    h = R.rfdd_setup(w.A, w.M, w.part, w.p, R.rfdd_default_options())
    l0, X0, r0 = R.rfdd_polish(h, lam[:0], Xs[:, :0])  # nev = 0
    assert l0.size == 0 and X0.shape == (blk.n, 0)
    bad = lam.copy()
    bad[1] = np.nan
    with pytest.raises(R.RfddError) as e:
        R.rfdd_polish(h, bad, Xs)
    assert e.value.code == R.RFDD_EINVAL
    with pytest.raises(ValueError):
        R.rfdd_polish(h, lam, Xs[:-1])
    # one pair alone gives the same as in a batch
    l1, X1, _ = R.rfdd_polish(h, lam[1:2], Xs[:, 1:2])
    lb, Xb, _ = R.rfdd_polish(h, lam, Xs)
    np.testing.assert_array_equal(X1[:, 0], Xb[:, 1])
    assert l1[0] == lb[1]
