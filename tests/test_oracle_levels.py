"""Pins of the oracle's two-level interface factorisation (the block inverse of Eq. inv_dd2
applied to S(zeta) with groups of subdomains as its subdomains; Section 7's recursion).

They tie it to things other than itself: the geometry of the separator grid (which interface
nodes must be level 2), the exact zeros of a dense S(zeta), the Schur-complement identity
(S^{-1})[I2, I2] = S22'^{-1}, a dense linear solve, and the closed-form Q1 spectrum through a
whole RF-DDES solve."""
import numpy as np
import scipy.sparse as sp

import rfdd_inputs as I
from oracle import rfdd_oracle as O
from tests.test_oracle_dd import random_pencil


def _q1_blocks(N, splits):
    A, M = I.q1_pencil(N, len(splits))
    part, p = I.geometric_partition(N, len(splits), splits)
    return O.Blocks(A.to_scipy(), M.to_scipy(), part, p), part


def test_level2_is_the_middle_separator_lines():
    # 2-D Q1, N = 33, 4 x 4 subdomains (planes at 7, 16, 24), groups 2 x 2: the level-2 nodes
    # are exactly the interface nodes on the middle lines x = 16 or y = 16
    N = 33
    blk, part = _q1_blocks(N, (4, 4))
    lv = O.interface_levels(blk, I.subdomain_groups((4, 4), (2, 2)))
    iface = np.flatnonzero(part == -1)
    x, y = iface // N, iface % N
    want = np.flatnonzero((x == 16) | (y == 16))
    np.testing.assert_array_equal(lv.I2, want)
    # the level-1 nodes of each group lie in that group's quadrant
    for g in range(4):
        gx, gy = divmod(g, 2)
        xs, ys = x[lv.I1[g]], y[lv.I1[g]]
        assert len(xs) > 0
        assert np.all((xs < 16) == (gx == 0)) and np.all((ys < 16) == (gy == 0))
    # the sets partition the interface
    allidx = np.sort(np.concatenate(lv.I1 + [lv.I2]))
    np.testing.assert_array_equal(allidx, np.arange(blk.s))


def _check_exact_zeros(blk, lv, z):
    S = O.schur(blk, z)
    G = len(lv.I1)
    for g in range(G):
        for h in range(G):
            if g != h and len(lv.I1[g]) and len(lv.I1[h]):
                assert np.all(S[np.ix_(lv.I1[g], lv.I1[h])] == 0)
        far = np.setdiff1d(lv.I2, lv.I2g[g])
        if len(lv.I1[g]) and len(far):
            assert np.all(S[np.ix_(lv.I1[g], far)] == 0)
            assert np.all(S[np.ix_(far, lv.I1[g])] == 0)
    return S


def test_level1_blocks_of_S_are_uncoupled_across_groups():
    # random weights on the 9-point pattern, 3 x 3 subdomains in groups of uneven shape
    A, M, part, p = random_pencil(N=14, splits=(3, 3), seed=11)
    blk = O.Blocks(A, M, part, p)
    groups = I.subdomain_groups((3, 3), (2, 2))
    lv = O.interface_levels(blk, groups)
    assert sum(len(a) for a in lv.I1) > 0 and len(lv.I2) > 0
    _check_exact_zeros(blk, lv, 0.3 + 0.7j)


def _thick_separator_pencil():
    # 5-point Laplacian on a 12 x 6 grid (x the first axis); columns x = 2, 5, 6, 9 are the
    # interface; subdomains x in [0,2), [3,5), [7,9), [10,12); the separator between subdomains
    # 1 and 2 is two columns wide
    nx, ny = 12, 6
    n = nx * ny
    rows, cols, vals = [], [], []
    for x in range(nx):
        for y in range(ny):
            i = x * ny + y
            rows.append(i); cols.append(i); vals.append(4.0)
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                xx, yy = x + dx, y + dy
                if 0 <= xx < nx and 0 <= yy < ny:
                    rows.append(i); cols.append(xx * ny + yy); vals.append(-1.0)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    M = sp.identity(n, format="csr")
    xs = np.arange(n) // ny
    part = np.full(n, -1, dtype=np.int32)
    for j, (lo, hi) in enumerate(((0, 2), (3, 5), (7, 9), (10, 12))):
        part[(xs >= lo) & (xs < hi)] = j
    return A, M, part, 4, xs, ny


def test_thick_separator_demotes_coupled_candidates():
    A, M, part, p, xs, ny = _thick_separator_pencil()
    blk = O.Blocks(A, M, part, p)
    lv = O.interface_levels(blk, [0, 0, 1, 1])
    ix = xs[part == -1]                     # x coordinate of each interface node
    # column 5 touches only subdomain 1 (group 0), column 6 only subdomain 2 (group 1), and they
    # are coupled in C: both are level 2; columns 2 and 9 are level 1 of groups 0 and 1
    np.testing.assert_array_equal(lv.I2, np.flatnonzero((ix == 5) | (ix == 6)))
    np.testing.assert_array_equal(lv.I1[0], np.flatnonzero(ix == 2))
    np.testing.assert_array_equal(lv.I1[1], np.flatnonzero(ix == 9))
    np.testing.assert_array_equal(lv.I2g[0], np.flatnonzero(ix == 5))
    np.testing.assert_array_equal(lv.I2g[1], np.flatnonzero(ix == 6))
    _check_exact_zeros(blk, lv, 1.5 + 0.5j)


def test_two_level_solve_equals_dense_solve_and_schur_identity():
    for (N, splits, gs, seed) in ((14, (3, 3), (2, 2), 5), (17, (4, 4), (2, 2), 6)):
        A, M, part, p = random_pencil(N=N, splits=splits, seed=seed)
        blk = O.Blocks(A, M, part, p)
        lv = O.interface_levels(blk, I.subdomain_groups(splits, gs))
        z = -0.2 + 0.9j
        S = O.schur(blk, z)
        two = O.TwoLevelSchur(S, lv)
        # Schur-complement identity: the (2,2) block of S^{-1} is the inverse of S22'
        Sinv = np.linalg.inv(S)
        want = np.linalg.inv(Sinv[np.ix_(lv.I2, lv.I2)])
        assert np.abs(two.S22p - want).max() <= 1e-10 * np.abs(want).max()
        G = np.random.default_rng(seed).standard_normal((blk.s, 5))
        ref = np.linalg.solve(S, G)
        got = two.solve(G)
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_two_level_solve_with_a_single_group_and_empty_level1():
    # one group: every node that touches a subdomain is level 1, S22' holds only nodes that touch
    # none (none here); a grouping with every subdomain alone still solves exactly
    A, M, part, p = random_pencil(N=11, splits=(2, 2), seed=8)
    blk = O.Blocks(A, M, part, p)
    S = O.schur(blk, 0.5 + 0.5j)
    G = np.random.default_rng(1).standard_normal((blk.s, 3))
    ref = np.linalg.solve(S, G)
    for groups in ([0, 0, 0, 0], [0, 1, 2, 3]):
        lv = O.interface_levels(blk, groups)
        got = O.TwoLevelSchur(S, lv).solve(G)
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    lv = O.interface_levels(blk, [0, 0, 0, 0])
    assert len(lv.I2) == 0 and len(lv.I1[0]) == blk.s


def test_rfdd_solve_with_two_levels_matches_closed_form():
    w = I.workload("q1_2d_33_p9")
    groups = I.subdomain_groups((3, 3), (2, 2))
    ro2 = O.rfdd_solve(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p, w.alpha, w.beta, w.n_nodes, w.rule,
                       block=4, groups=groups)
    ro1 = O.rfdd_solve(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p, w.alpha, w.beta, w.n_nodes, w.rule,
                       block=4)
    ex = w.exact[(w.exact > w.alpha) & (w.exact < w.beta)]
    assert len(ro2["evals"]) == len(ex)
    assert np.max(np.abs(ro2["evals"] - ex) / ex) <= 1e-10
    # the filter is the same operator, so Algorithm 2 takes the same number of steps
    assert ro2["mu"] == ro1["mu"]
    assert np.max(np.abs(ro2["pre"]["theta"] - ro1["pre"]["theta"]) / ro1["pre"]["theta"]) <= 1e-8
