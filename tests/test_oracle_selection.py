"""Pins for two oracle rules that the end-to-end checks cannot see:

* the choice of V_j in Algorithm 3, step 3 -- the eigenvectors of (B_sigma^(j), M_B^(j)) whose
  eigenvalues are smallest in magnitude, i.e. the eigenpairs (delta, v) of (B_j, M_B^(j)) with
  delta nearest sigma (Section 4);
* the stopping test of Algorithm 2 (line 13): every ceil(10/b) block steps the process stops
  once the trace of T_mu changed by at most tol * |tr T_mu| since the previous check (a relative
  test, so scaling F does not move the stop).

Each rule is checked against facts computed another way (a dense eigensolve of the UNshifted
pencil; a diagonal F whose Krylov space is exhausted at a known step), and a copy of the oracle
routine with a plausible mistake planted in its source must fail the same check.
"""
import inspect
import textwrap

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import rfdd_oracle as O
from tests.test_oracle_dd import random_pencil


def planted(fn, old, new):
    """A copy of oracle function ``fn`` with the source text ``old`` replaced by ``new``."""
    src = textwrap.dedent(inspect.getsource(fn))
    assert old in src, old
    ns = dict(vars(O))
    exec(compile(src.replace(old, new), "<planted>", "exec"), ns)
    return ns[fn.__name__]


# ----------------------------------------------------------------------------------------
# V_j (Algorithm 3, step 3)
# ----------------------------------------------------------------------------------------

def vj_error(V, blk, sigma, nev_b):
    """Largest deviation of V from the nev_b eigenvectors of (B_j, M_B^(j)) with eigenvalues
    nearest sigma, over all subdomains j (0 when V is exactly that choice)."""
    worst = 0.0
    for j in range(blk.p):
        delta, Y = sla.eigh(blk.B[j], blk.MB[j])      # unshifted pencil, its own eigensolve
        k = min(nev_b, blk.d[j])
        pick = np.argsort(np.abs(delta - sigma), kind="stable")[:k]
        Vj = V[j]
        assert Vj.shape == (blk.d[j], k)
        # M_B-orthonormal, and Rayleigh quotients equal to the chosen eigenvalues
        worst = max(worst, np.abs(Vj.T @ blk.MB[j] @ Vj - np.eye(k)).max())
        H = Vj.T @ blk.B[j] @ Vj
        worst = max(worst, np.abs(np.linalg.eigvalsh(0.5 * (H + H.T)) - np.sort(delta[pick])).max()
                    / np.abs(delta).max())
        # same span as the chosen eigenvectors (in the M_B inner product)
        Yp = Y[:, pick]
        sv = np.linalg.svd(Yp.T @ blk.MB[j] @ Vj, compute_uv=False)
        worst = max(worst, 1.0 - sv.min())
    return worst


def sigma_apart_from_zero(blk):
    """A shift between two eigenvalues of (B_0, M_B^(0)) in its upper spectrum, so that the
    nev_b eigenvalues nearest it differ from the nev_b nearest zero in every subdomain."""
    delta = sla.eigh(blk.B[0], blk.MB[0], eigvals_only=True)
    return 0.5 * (delta[-4] + delta[-5])


@pytest.mark.parametrize("nev_b", [3, 6])
def test_vj_are_the_eigenvectors_nearest_sigma(nev_b):
    A, M, part, p = random_pencil(N=9, seed=11)
    blk = O.Blocks(A, M, part, p)
    sigma = sigma_apart_from_zero(blk)
    for j in range(blk.p):   # the choice is not moot: nearest sigma != nearest 0
        delta = sla.eigh(blk.B[j], blk.MB[j], eigvals_only=True)
        near_s = set(np.argsort(np.abs(delta - sigma))[:nev_b].tolist())
        near_0 = set(np.argsort(np.abs(delta))[:nev_b].tolist())
        assert near_s != near_0 and nev_b < blk.d[j]
    V = O.interior_eigvecs(blk, sigma, nev_b)
    assert vj_error(V, blk, sigma, nev_b) <= 1e-10


def test_vj_pin_catches_an_unshifted_choice():
    A, M, part, p = random_pencil(N=9, seed=11)
    blk = O.Blocks(A, M, part, p)
    sigma = sigma_apart_from_zero(blk)
    bad = planted(O.interior_eigvecs, "Bs = blk.B[j] - sigma * blk.MB[j]", "Bs = blk.B[j]")
    assert vj_error(bad(blk, sigma, 4), blk, sigma, 4) > 1e-3
    bad2 = planted(O.interior_eigvecs, "np.argsort(np.abs(dl)", "np.argsort(dl")
    assert vj_error(bad2(blk, sigma, 4), blk, sigma, 4) > 1e-3


# ----------------------------------------------------------------------------------------
# Algorithm 2, line 13 (reading: relative trace test every ceil(10/b) block steps)
# ----------------------------------------------------------------------------------------

S_DIM, RANK = 100, 23


def diag_F(scale):
    """F = diag(f) of rank RANK with distinct positive entries.  From a start block of b generic
    vectors the block Krylov space is span(start) + range(F), of dimension RANK + b; it is
    exhausted at block step t0 = ceil((RANK + b) / b), where tr T reaches tr F and stays there
    (later vectors, drawn after breakdown, lie in the null space of F)."""
    f = np.zeros(S_DIM)
    f[:RANK] = scale * np.linspace(1.0, 2.0, RANK)
    return (lambda V: f[:, None] * V), float(f.sum())


def expected_mu(b, check_every=10):
    t0 = -(-(RANK + b) // b)
    spc = max(1, -(-check_every // b))
    tc = spc
    while tc - spc < t0:      # the first check whose previous check already saw tr F
        tc += spc
    return tc * b


@pytest.mark.parametrize("b", [1, 3, 4])
@pytest.mark.parametrize("scale", [1.0, 1e8, 1e-8])
def test_lanczos_stops_one_check_after_the_trace_settles(b, scale):
    F, trF = diag_F(scale)
    out = O.lanczos_interface(F, S_DIM, tol=1e-6, block=b, seed=5)
    assert out["mu"] == expected_mu(b), (out["mu"], expected_mu(b))
    assert abs(out["traces"][-1] - trF) <= 1e-12 * trF
    # the trace was still growing at the check before the last one
    spc = max(1, -(-10 // b))
    assert out["traces"][-1 - 2 * spc] < trF * (1 - 1e-6)
    Q = out["Q"]
    assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() <= 1e-12


def test_lanczos_stops_when_the_space_is_exhausted():
    """mu = s ends the process even if the trace test never fires (tol = 0); with s = 30 and
    b = 4 the last block keeps the 2 columns that still fit."""
    f = np.linspace(1.0, 3.0, 30)
    out = O.lanczos_interface(lambda V: f[:, None] * V, 30, tol=0.0, block=4, seed=2)
    assert out["mu"] == 30 and abs(out["traces"][-1] - f.sum()) <= 1e-12 * f.sum()
    assert np.abs(out["Q"].T @ out["Q"] - np.eye(30)).max() <= 1e-12


def test_stop_pin_catches_an_absolute_tolerance_and_a_wrong_check_period():
    absolute = planted(O.lanczos_interface, "<= tol * abs(trace)", "<= tol")
    F, _ = diag_F(1e-8)
    assert absolute(F, S_DIM, tol=1e-6, block=1, seed=5)["mu"] != expected_mu(1)
    per_block_step = planted(O.lanczos_interface, "steps_per_check = max(1, -(-check_every // b))",
                             "steps_per_check = check_every")
    F, _ = diag_F(1.0)
    assert per_block_step(F, S_DIM, tol=1e-6, block=3, seed=5)["mu"] != expected_mu(3)


# ----------------------------------------------------------------------------------------
# Completion (reading A17): filter gain of Ritz vectors, spurious Ritz values
# ----------------------------------------------------------------------------------------

def test_filter_gain_is_rho_on_eigenvectors_and_small_on_mirror_mixtures():
    """For exact eigenvectors the gain equals the closed-form filter value rho(lambda); a mixture
    of two eigenvectors on opposite sides of the interval (equal small rho) has a Rayleigh
    quotient inside the interval but a gain far below 1/4, so the completion discards it."""
    import rfdd_inputs as I
    w = I.workload("q1_2d_24")
    blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
    lam, Xe = sla.eigh(blk.Ap.toarray(), blk.Mp.toarray())
    z, wt = O.quadrature(w.alpha, w.beta, w.n_nodes, w.rule)
    fac = O.Factors(blk, z)
    pick = [5, 12, 25, 40, 60]
    Xp = Xe[:, pick]
    g = O.filter_gain(blk.Mp, Xp, O.filter_full(fac, wt, blk.Mp @ Xp))
    np.testing.assert_allclose(g, O.filter_value(lam[pick], z, wt), rtol=1e-9, atol=1e-13)
    # mirror pair: eigenvalues below alpha and above beta with nearly equal filter values
    c = 0.5 * (w.alpha + w.beta)
    lo = np.flatnonzero(lam < w.alpha)[-3]
    up = np.flatnonzero(lam > w.beta)
    hi = up[np.argmin(np.abs(lam[up] - (2 * c - lam[lo])))]
    v = (Xe[:, lo] + Xe[:, hi]) / np.sqrt(2.0)
    theta = (v @ (blk.Ap @ v)) / (v @ (blk.Mp @ v))
    assert w.alpha < theta < w.beta
    Xp = np.column_stack([v, Xe[:, 15]])
    g = O.filter_gain(blk.Mp, Xp, O.filter_full(fac, wt, blk.Mp @ Xp))
    assert g[0] < 0.25 and g[1] > 0.5
