"""Plain FP64 CPU oracle of RF-DDES (Kalantzis, Xi, Saad: "Beyond AMLS: Domain decomposition
with rational filtering", arXiv:1711.09487).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module.  The product path (the CUDA library and its Python
binding) never calls it and shares no code with it; both sides read the same seeded arrays
produced by ``rfdd_inputs``.

Every routine follows the paper's steps in its own order and notation, using numpy/scipy
primitives (dense LU, triangular solves, symmetric eigensolves, matrix products) as steps.  No
blocking, fusion or reordering beyond what the cited passage states.  Readings of passages that
are silent or ambiguous are marked "Reading:".

Pins (see tests/test_oracle_*.py): closed-form Q1 spectra, the Midpoint-filter closed form,
Gauss-Legendre exactness, the (2,2)-block identity of Eq. (finalizing), the block inverse of
Eq. (inv_dd2) against a dense inverse, Prop. (lowrank), Theorems (uuhat), (uuhat2), (all) at
tiny n, Sylvester inertia counts, the interior polish of Eq. (compute_u_parallel) recovering
dense-eigensolver eigenvectors from their interface rows, brute-force dense generalized
eigensolves, and for RF-KRYLOV (Algorithm 1) the closed-form spectra of the 5-point Laplacian
with M = I and of the Q1 pencil, the projected filter H_mu formed directly, and the stopping
step on filters whose Krylov space is exhausted at a known step.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

MASK64 = (1 << 64) - 1


# ----------------------------------------------------------------------------------------
# Counter-based random numbers (SplitMix64, S. Vigna's published finaliser)
# ----------------------------------------------------------------------------------------

def splitmix64(x: int) -> int:
    """SplitMix64 output for state ``x`` (increment already applied by the caller)."""
    z = x & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def counter_uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """Values in [-1, 1): element i of ``stream`` is
    splitmix64(seed + (stream * 2^32 + i + 1) * 0x9E3779B97F4A7C15) >> 11, scaled by 2^-52 - 1.
    Reading: the paper leaves the start vector of Algorithm 2 unspecified; both sides draw it from
    this generator so that runs are reproducible and comparable."""
    golden = np.uint64(0x9E3779B97F4A7C15)
    c = (np.uint64(stream) << np.uint64(32)) + np.arange(1, count + 1, dtype=np.uint64)
    z = np.uint64(seed & MASK64) + c * golden
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0


# ----------------------------------------------------------------------------------------
# Section 2.1: rational filter, Eq. (contour), (contour2), (contour3)
# ----------------------------------------------------------------------------------------

def quadrature(alpha: float, beta: float, n_nodes: int, rule: str = "midpoint"):
    """Poles zeta_l (Im > 0) and weights omega_l of the discretised Cauchy integral.

    Eq. (contour): I(zeta) = -1/(2 pi i) * contour integral of dnu / (zeta - nu) over the circle
    nu = c + r e^{i theta}, c = (alpha+beta)/2, r = (beta-alpha)/2, counter-clockwise.  With
    dnu = i r e^{i theta} d theta the integrand in theta is -(1/(2 pi)) r e^{i theta}/(zeta - nu).

    * ``midpoint``: the midpoint rule of order 2 Nc on [0, 2 pi] (Section 6), keeping the Nc
      nodes with positive imaginary part: theta_l = (2l-1) pi / (2 Nc), weight pi/Nc, so
      omega_l = -r e^{i theta_l} / (2 Nc).
    * ``gauss_legendre``: Nc Gauss-Legendre points t_l, w_l on [-1, 1] mapped to the upper
      half circle theta = (pi/2)(1 + t) (the lower half follows by conjugation, Eq. contour3):
      omega_l = -(r/4) w_l e^{i theta_l}.
    """
    if not (beta > alpha) or n_nodes < 1:
        raise ValueError("need alpha < beta and n_nodes >= 1")
    c = 0.5 * (alpha + beta)
    r = 0.5 * (beta - alpha)
    if rule == "midpoint":
        theta = (2.0 * np.arange(1, n_nodes + 1) - 1.0) * np.pi / (2.0 * n_nodes)
        e = np.exp(1j * theta)
        z = c + r * e
        w = -r * e / (2.0 * n_nodes)
    elif rule == "gauss_legendre":
        t, wl = np.polynomial.legendre.leggauss(n_nodes)
        theta = 0.5 * np.pi * (1.0 + t)
        e = np.exp(1j * theta)
        z = c + r * e
        w = -0.25 * r * wl * e
    else:
        raise ValueError(f"unknown rule {rule!r}")
    return z.astype(np.complex128), w.astype(np.complex128)


def filter_value(x, z, w):
    """rho(x) = 2 Re sum_l omega_l / (x - zeta_l) for real x (Eq. contour3)."""
    x = np.asarray(x, dtype=np.float64)[..., None]
    return 2.0 * np.real(np.sum(w / (x - z), axis=-1))


# ----------------------------------------------------------------------------------------
# Section 2.3: domain-decomposition ordering, Eq. (dd1), (eq1)
# ----------------------------------------------------------------------------------------

class Blocks:
    """Interior-first reordering of (A, M) and its blocks (Eq. dd1).

    Interior variables of subdomain j = 0..p-1 come first (in increasing original index), then
    the interface (label -1).  ``E[j]`` is the d_j x s coupling of subdomain j with the whole
    interface; ``sidx[j]`` lists the interface columns where E[j] or ME[j] has a nonzero
    (Reading: with a vertex separator the contiguous pattern E_j = [0, E^_j, 0] of Section 2.3 does
    not hold; E^_j is E_j restricted to the columns sidx[j]).
    """

    def __init__(self, A, M, part, p):
        A = sp.csr_matrix(A)
        M = sp.csr_matrix(M)
        part = np.asarray(part)
        n = A.shape[0]
        self.n, self.p = n, p
        groups = [np.flatnonzero(part == j) for j in range(p)]
        iface = np.flatnonzero(part == -1)
        self.d = np.array([len(g) for g in groups], dtype=np.int64)
        self.s = len(iface)
        self.perm = np.concatenate(groups + [iface]).astype(np.int64)   # new -> old
        self.iperm = np.empty(n, dtype=np.int64)
        self.iperm[self.perm] = np.arange(n)                            # old -> new
        self.off = np.concatenate([[0], np.cumsum(self.d)])
        dsum = int(self.off[-1])
        Ap = A[self.perm][:, self.perm].tocsr()
        Mp = M[self.perm][:, self.perm].tocsr()
        self.Ap, self.Mp = Ap, Mp
        self.B, self.MB, self.E, self.ME, self.sidx = [], [], [], [], []
        for j in range(p):
            lo, hi = self.off[j], self.off[j + 1]
            self.B.append(Ap[lo:hi, lo:hi].toarray())
            self.MB.append(Mp[lo:hi, lo:hi].toarray())
            Ej = Ap[lo:hi, dsum:].toarray()
            MEj = Mp[lo:hi, dsum:].toarray()
            # Eq. dd1: no couplings between different subdomains' interiors
            for k in range(p):
                if k != j:
                    klo, khi = self.off[k], self.off[k + 1]
                    if Ap[lo:hi, klo:khi].nnz or Mp[lo:hi, klo:khi].nnz:
                        raise ValueError("partition is not a vertex separator")
            cols = np.flatnonzero((np.abs(Ej).sum(0) + np.abs(MEj).sum(0)) > 0)
            self.E.append(Ej)
            self.ME.append(MEj)
            self.sidx.append(cols)
        self.C = Ap[dsum:, dsum:].toarray()
        self.MC = Mp[dsum:, dsum:].toarray()

    def to_original(self, X):
        """Permute rows back to the input ordering (Algorithm 3, step 8)."""
        return X[self.iperm]


# ----------------------------------------------------------------------------------------
# Section 3.1: shifted blocks and the Schur complement, Eq. (inv_dd2)
# ----------------------------------------------------------------------------------------

def shifted(blk: Blocks, z):
    """B_z = B - z M_B, E_z = E - z M_E, C_z = C - z M_C (Section 3.1)."""
    Bz = [blk.B[j] - z * blk.MB[j] for j in range(blk.p)]
    Ez = [blk.E[j] - z * blk.ME[j] for j in range(blk.p)]
    Cz = blk.C - z * blk.MC
    return Bz, Ez, Cz


def schur(blk: Blocks, z):
    """S_z = C_z - E_z^T B_z^{-1} E_z.

    Reading: the paper writes E^H in Eq. (inv_dd2); A - zM is complex *symmetric*, so its block
    inverse uses the plain transpose (consistent with Eq. schur_eigvec3).  Never conjugate.
    """
    Bz, Ez, Cz = shifted(blk, z)
    S = Cz.astype(np.complex128).copy()
    for j in range(blk.p):
        S -= Ez[j].T @ np.linalg.solve(Bz[j], Ez[j])
    return S


def schur_columns(A, M, part, p, z, cols):
    """Columns ``cols`` (interface indices, interior-first ordering) of S_z = C_z - E_z^T B_z^{-1} E_z
    for pencils too large for the dense ``Blocks``: the same definition as ``schur``, with each
    B_j(z) factored by a sparse LU (SuperLU, a library primitive) and applied to the columns of
    E_j(z) that are needed.  Returns an s x len(cols) complex array."""
    from scipy.sparse.linalg import splu
    A = sp.csr_matrix(A)
    M = sp.csr_matrix(M)
    part = np.asarray(part)
    groups = [np.flatnonzero(part == j) for j in range(p)]
    iface = np.flatnonzero(part == -1)
    cols = np.asarray(cols)
    Az = (A - z * M).tocsr()
    S = Az[iface][:, iface[cols]].toarray().astype(np.complex128)
    for j in range(p):
        Bz = Az[groups[j]][:, groups[j]].tocsc()
        Ez = Az[groups[j]][:, iface].tocsc()
        X = splu(Bz).solve(Ez[:, cols].toarray())
        S -= (Ez.T @ X)
    return S


class Factors:
    """LU factorisations of every B_j(zeta_l) and S(zeta_l) (Algorithm 3 step 5 needs solves with
    them; the paper uses PARDISO/MUMPS, the oracle uses dense LU with partial pivoting)."""

    def __init__(self, blk: Blocks, z, groups=None):
        """``groups`` (optional, one label in 0..G-1 per subdomain): factor each S(zeta_l) in two
        levels (``TwoLevelSchur``) instead of one dense LU."""
        self.blk = blk
        self.z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
        self.levels = None if groups is None else interface_levels(blk, groups)
        self.Blu, self.Slu, self.Ez = [], [], []
        for zl in self.z:
            Bz, Ez, Cz = shifted(blk, zl)
            lus = [sla.lu_factor(Bz[j]) for j in range(blk.p)]
            S = Cz.astype(np.complex128).copy()
            for j in range(blk.p):
                S -= Ez[j].T @ sla.lu_solve(lus[j], Ez[j])
            self.Blu.append(lus)
            self.Ez.append(Ez)
            if self.levels is None:
                self.Slu.append(sla.lu_factor(S))
            else:
                self.Slu.append(TwoLevelSchur(S, self.levels))

    def solve_S(self, l, G):
        if self.levels is not None:
            return self.Slu[l].solve(G)
        return sla.lu_solve(self.Slu[l], G.astype(np.complex128))

    def solve_B(self, l, F):
        """Block-diagonal solve with B_{zeta_l} on the interior part (d rows)."""
        blk = self.blk
        out = np.empty(F.shape, dtype=np.complex128)
        for j in range(blk.p):
            lo, hi = blk.off[j], blk.off[j + 1]
            out[lo:hi] = sla.lu_solve(self.Blu[l][j], F[lo:hi].astype(np.complex128))
        return out

    def resolvent(self, l, V):
        """(A - zeta_l M)^{-1} V through the block inverse of Eq. (inv_dd2):
        t = B^{-1} f, y = S^{-1} (g - E^T t), u = t - B^{-1} E y."""
        blk = self.blk
        dsum = int(blk.off[-1])
        f, g = V[:dsum], V[dsum:]
        t = self.solve_B(l, f)
        Et = np.vstack([self.Ez[l][j] for j in range(blk.p)])          # d x s (= E_z)
        y = self.solve_S(l, g - Et.T @ t)
        u = t - self.solve_B(l, Et @ y)
        return np.vstack([u, y])


# ----------------------------------------------------------------------------------------
# Two-level interface factorisation: the block inverse of Eq. (inv_dd2) applied once more, to
# S(zeta) itself, with groups of subdomains in the role of the subdomains (the recursive use of
# RF-DDES's decomposition that Section 7 suggests; Section 6.3 names the S solves as what limits
# RF-DDES when p grows)
# ----------------------------------------------------------------------------------------

class InterfaceLevels:
    """Split of the interface for a grouping of the subdomains.

    ``I1[g]``: level-1 nodes of group g; ``I2``: level-2 nodes; ``I2g[g]``: the level-2 nodes
    that S(zeta) can couple to ``I1[g]`` (all index arrays ascending, interface numbering)."""

    def __init__(self, I1, I2, I2g, cls):
        self.I1, self.I2, self.I2g, self.cls = I1, I2, I2g, cls


def interface_levels(blk: Blocks, groups):
    """Reading (the paper gives no recursion of the interface): S(zeta)[a, b] can be nonzero
    only when interface nodes a and b touch a common subdomain (a term of E^T B^{-1} E) or are
    coupled in C or M_C.  An interface node is level 1 of group g when every subdomain it touches
    is in group g (at least one) and no node it is coupled to in C or M_C is such a level-1
    candidate of another group; every other interface node is level 2.  S(zeta) restricted to
    the level-1 nodes is then block diagonal over the groups."""
    groups = np.asarray(groups, dtype=np.int64)
    s, p = blk.s, blk.p
    G = int(groups.max()) + 1 if p else 0
    touch = [set() for _ in range(s)]
    for j in range(p):
        for a in blk.sidx[j]:
            touch[a].add(int(groups[j]))
    cand = np.full(s, -1, dtype=np.int64)
    for a in range(s):
        if len(touch[a]) == 1:
            cand[a] = next(iter(touch[a]))
    pattern = (blk.C != 0) | (blk.MC != 0)
    cls = cand.copy()
    for a in range(s):
        if cand[a] < 0:
            continue
        nb = np.flatnonzero(pattern[a])
        if np.any((cand[nb] >= 0) & (cand[nb] != cand[a])):
            cls[a] = -1
    I1 = [np.flatnonzero(cls == g) for g in range(G)]
    I2 = np.flatnonzero(cls < 0)
    I2g = []
    for g in range(G):
        near = np.zeros(s, dtype=bool)
        for j in np.flatnonzero(groups == g):
            near[blk.sidx[j]] = True
        if len(I1[g]):
            near |= pattern[I1[g]].any(axis=0)
        near &= cls < 0
        I2g.append(np.flatnonzero(near))
    return InterfaceLevels(I1, I2, I2g, cls)


class TwoLevelSchur:
    """S = [[S11, S12], [S21, S22]] with S11 = blockdiag_g S(I1_g, I1_g) (``interface_levels``),
    factored by Eq. (inv_dd2) one level down:
        S22' = S22 - sum_g S(I2g_g, I1_g) S(I1_g, I1_g)^{-1} S(I1_g, I2g_g),
    and solved as t_g = S11_g^{-1} g1_g,  S22' y2 = g2 - sum_g S21_g t_g,
    y1_g = S11_g^{-1} (g1_g - S12_g y2[I2g_g])."""

    def __init__(self, S, lv: InterfaceLevels):
        self.lv = lv
        self.s = S.shape[0]
        pos2 = np.full(self.s, -1, dtype=np.int64)
        pos2[lv.I2] = np.arange(len(lv.I2))
        self.pos2 = pos2
        S22 = S[np.ix_(lv.I2, lv.I2)].astype(np.complex128).copy()
        self.lu11, self.S12, self.S21 = [], [], []
        for g in range(len(lv.I1)):
            I1, J = lv.I1[g], lv.I2g[g]
            lu = sla.lu_factor(S[np.ix_(I1, I1)]) if len(I1) else None
            S12 = S[np.ix_(I1, J)]
            S21 = S[np.ix_(J, I1)]
            if len(I1) and len(J):
                S22[np.ix_(pos2[J], pos2[J])] -= S21 @ sla.lu_solve(lu, S12)
            self.lu11.append(lu)
            self.S12.append(S12)
            self.S21.append(S21)
        self.S22p = S22
        self.lu22 = sla.lu_factor(S22) if len(lv.I2) else None

    def solve(self, G):
        lv = self.lv
        G = G.astype(np.complex128)
        Y = np.zeros(G.shape, dtype=np.complex128)
        g2 = G[lv.I2].copy()
        for g in range(len(lv.I1)):
            I1, J = lv.I1[g], lv.I2g[g]
            if len(I1) and len(J):
                g2[self.pos2[J]] -= self.S21[g] @ sla.lu_solve(self.lu11[g], G[I1])
        y2 = sla.lu_solve(self.lu22, g2) if len(lv.I2) else g2
        Y[lv.I2] = y2
        for g in range(len(lv.I1)):
            I1, J = lv.I1[g], lv.I2g[g]
            if len(I1):
                Y[I1] = sla.lu_solve(self.lu11[g], G[I1] - self.S12[g] @ y2[self.pos2[J]])
        return Y


def filter_interface(fac: Factors, w, X):
    """Re sum_l omega_l S(zeta_l)^{-1} X  (Algorithm 2, line 2, as printed: no factor 2)."""
    acc = np.zeros(X.shape, dtype=np.complex128)
    for l in range(len(fac.z)):
        acc += w[l] * fac.solve_S(l, X)
    return np.real(acc)


def filter_full(fac: Factors, w, MX):
    """2 Re sum_l omega_l (A - zeta_l M)^{-1} (M X)  (Eq. rhoAM), applied via Eq. (inv_dd2)."""
    acc = np.zeros(MX.shape, dtype=np.complex128)
    for l in range(len(fac.z)):
        acc += w[l] * fac.resolvent(l, MX)
    return 2.0 * np.real(acc)


# ----------------------------------------------------------------------------------------
# Section 3.2: Algorithm 2 (Krylov restricted to the interface variables)
# ----------------------------------------------------------------------------------------

def _orth_against(Qs, W, passes=2):
    for _ in range(passes):
        for Qk in Qs:
            W = W - Qk @ (Qk.T @ W)
    return W


def lanczos_interface(apply_F, s, tol=1e-6, block=1, seed=1, check_every=10, max_steps=None):
    """Algorithm 2 on F = Re sum omega_l S_l^{-1} with block size ``block`` (b = 1 is the printed
    algorithm).  Returns dict(Q (s x mu), alphas (list of b x b), betas, traces, mu).

    Readings:
    * q^(1): a counter-based uniform block, orthonormalised (the paper leaves it open).
    * lines 4-6 (one classical Gram-Schmidt pass) are run twice ("CGS2"); no effect in exact
      arithmetic, keeps ||Q^T Q - I|| at rounding level.
    * line 13: every ``check_every`` vectors (ceil(check_every / b) block steps) stop when
      |tr T_mu - tr T_(mu - check_every)| <= tol * |tr T_mu|; also stop once mu = s, the last
      block keeping only the s - mu columns that still fit.
    * breakdown (line 8): ||w|| <= 1e-14 max|a| -> new random vectors orthogonal to Q.
    """
    b = block
    start = counter_uniform(seed, 0, s * b).reshape(s, b)
    Q1, _ = np.linalg.qr(start)
    Qs = [Q1]
    Qprev = np.zeros((s, b))
    Bmu = np.zeros((b, b))
    alphas, betas, traces = [], [], []
    steps_per_check = max(1, -(-check_every // b))
    max_steps = max_steps or -(-s // b)
    trace = 0.0
    history = [0.0]
    extra = 1
    for mu in range(1, max_steps + 1):
        Qmu = Qs[-1]
        W = apply_F(Qmu) - Qprev @ Bmu.T                       # line 2
        Amu = Qmu.T @ W                                         # line 3
        Amu = 0.5 * (Amu + Amu.T)
        W = _orth_against(Qs, W)                                # lines 4-6 (twice)
        alphas.append(Amu)
        trace += float(np.trace(Amu))
        traces.append(trace)
        ncols = sum(q.shape[1] for q in Qs)
        if ncols >= s:                                          # mu = s: the space is exhausted
            break
        # Reading: a block that would pass mu = s keeps its leading s - mu columns
        bn = min(b, s - ncols)
        Wfull = W
        W = W[:, :bn]
        Qn, R = np.linalg.qr(W)                                 # lines 7-12
        amax = max(np.max(np.abs(np.diag(A_))) for A_ in alphas)
        dead = np.abs(np.diag(R)) <= 1e-14 * max(amax, 1e-300)
        if np.any(dead):
            fresh = counter_uniform(seed, extra, s * bn).reshape(s, bn)
            extra += 1
            fresh = _orth_against(Qs, fresh)
            Qf, _ = np.linalg.qr(fresh)
            Qn[:, dead] = Qf[:, dead]
            Qn = _orth_against(Qs, Qn)
            Qn, R2 = np.linalg.qr(Qn)
            R[dead, :] = 0.0
        # a vector that lost most of its norm in lines 4-6 is mostly rounding noise: one more
        # pass after normalisation restores orthogonality (the "twice is enough" rule)
        Qn = _orth_against(Qs, Qn, passes=1)
        Qn, R2 = np.linalg.qr(Qn)
        R = R2 @ R if bn == Wfull.shape[1] else Qn.T @ Wfull    # B_(mu+1) = Q_(mu+1)^T W
        betas.append(R)
        Bmu = R
        Qprev = Qmu
        Qs.append(Qn)
        if mu % steps_per_check == 0:                          # line 13
            if abs(trace - history[-1]) <= tol * abs(trace):
                break
            history.append(trace)
    Q = np.hstack(Qs[:len(alphas)])
    return dict(Q=Q, alphas=alphas, betas=betas, traces=traces, mu=Q.shape[1])


# ----------------------------------------------------------------------------------------
# Section 4 and 5: interior approximation, Eq. (prol2), (yet1), (trabala), (trabala2), (z)
# ----------------------------------------------------------------------------------------

def interior_eigvecs(blk: Blocks, sigma, nev_b):
    """V_j: eigenvectors of (B_sigma^(j), M_B^(j)) for the nev_B^(j) eigenvalues of smallest
    magnitude (Algorithm 3, step 3), M_B-normalised.  Dense generalised symmetric eigensolve."""
    V = []
    for j in range(blk.p):
        Bs = blk.B[j] - sigma * blk.MB[j]
        dl, X = sla.eigh(Bs, blk.MB[j])
        k = min(int(nev_b), blk.d[j])
        order = np.argsort(np.abs(dl), kind="stable")[:k]
        V.append(X[:, np.sort(order)])
    return V


def interface_rows(blk: Blocks, Q, j):
    """Q_j: rows of Q at subdomain j's coupled interface nodes (Eq. q; Reading: s_j = |sidx_j|)."""
    return Q[blk.sidx[j]]


def resolvent_chains(blk: Blocks, sigma, Q, psi):
    """Sigma_j^(psi) and Gamma_j^(psi) of Eq. (trabala2) with Phi_j, Psi_j of Eq. (trabala)."""
    Sig, Gam = [], []
    for j in range(blk.p):
        Bs = blk.B[j] - sigma * blk.MB[j]
        lu = sla.lu_factor(Bs)
        Qj = interface_rows(blk, Q, j)
        Ehat = blk.E[j][:, blk.sidx[j]]
        MEhat = blk.ME[j][:, blk.sidx[j]]
        Phi = (Ehat - sigma * MEhat) @ Qj
        Psi = MEhat @ Qj
        cs, cg = [], []
        X = sla.lu_solve(lu, Phi)
        Y = sla.lu_solve(lu, Psi)
        for t in range(psi):
            cs.append(X)
            cg.append(Y)
            if t + 1 < psi:
                X = sla.lu_solve(lu, blk.MB[j] @ X)
                Y = sla.lu_solve(lu, blk.MB[j] @ Y)
        Sig.append(np.hstack(cs))
        Gam.append(np.hstack(cg))
    return Sig, Gam


def build_Z(blk: Blocks, V, Sig, Gam, Q, psi, with_gamma=None):
    """Projection matrix Z of Eq. (z), rows in the interior-first ordering.

    Column blocks: [blockdiag(V_j) | -Sigma^(psi) | Gamma^(psi)]; the interface rows hold
    [Q, 0_{s,(psi-1)mu}] under the Sigma block.  Gamma is dropped when M_E == 0 (Section 5.1).
    """
    n, s = blk.n, blk.s
    mu = Q.shape[1]
    kappa = sum(v.shape[1] for v in V)
    if with_gamma is None:
        with_gamma = any(np.any(me != 0) for me in blk.ME)
    k = kappa + psi * mu * (2 if with_gamma else 1)
    Z = np.zeros((n, k))
    col = 0
    for j in range(blk.p):
        lo, hi = blk.off[j], blk.off[j + 1]
        Z[lo:hi, col:col + V[j].shape[1]] = V[j]
        col += V[j].shape[1]
    for j in range(blk.p):
        lo, hi = blk.off[j], blk.off[j + 1]
        Z[lo:hi, col:col + psi * mu] = -Sig[j]
        if with_gamma:
            Z[lo:hi, col + psi * mu:col + 2 * psi * mu] = Gam[j]
    dsum = int(blk.off[-1])
    Z[dsum:, col:col + mu] = Q
    return Z


# ----------------------------------------------------------------------------------------
# Rayleigh-Ritz (Algorithm 3, step 7) and residuals
# ----------------------------------------------------------------------------------------

def m_orthonormal_basis(Ap, Mp, Z, drop=1e-12):
    """Basis W of range(Z) with W^T M W = I.  Reading: Z may be rank deficient (its column
    blocks overlap), so the Gram matrix Z^T M Z is eigendecomposed and directions with
    eigenvalue < drop * max are pruned (this is the plain definition of Rayleigh-Ritz on
    range(Z))."""
    nrm = np.sqrt(np.maximum(np.einsum("ij,ij->j", Z, Mp @ Z), 1e-300))
    Zs = Z / nrm
    G = Zs.T @ (Mp @ Zs)
    G = 0.5 * (G + G.T)
    g, U = np.linalg.eigh(G)
    keep = g > drop * g.max()
    return Zs @ (U[:, keep] / np.sqrt(g[keep]))


def rayleigh_ritz(Ap, Mp, Z, drop=1e-12):
    """Solve Z^T A Z G = Z^T M Z G Lambda on range(Z); returns sorted (theta, X) with
    X^T M X = I."""
    W = m_orthonormal_basis(Ap, Mp, Z, drop)
    H = W.T @ (Ap @ W)
    H = 0.5 * (H + H.T)
    th, G = np.linalg.eigh(H)
    return th, W @ G


def residuals(A, M, lam, X):
    """||A x - lambda M x||_2 / (|lambda| ||M x||_2) per column."""
    AX = A @ X
    MX = M @ X
    R = AX - MX * lam
    return np.linalg.norm(R, axis=0) / (np.abs(lam) * np.linalg.norm(MX, axis=0))


# ----------------------------------------------------------------------------------------
# Section 3, Eqs. (schur_eigvec2) and (compute_u_parallel): interior part from interface part
# ----------------------------------------------------------------------------------------

def polish_interior(blk: Blocks, lam, X):
    """Interior polish of approximate eigenpairs (lam[i], X[:, i]); X is n x nev in the input
    ordering.  The interface part y of each column is kept, and the interior part of subdomain j
    is recomputed from Eq. (compute_u_parallel):
        (B_j - lam_i M_B^(j)) u_j = -(E_j - lam_i M_E^(j)) y.
    Reading (the paper stops at u): the new vector is then M-normalised and lam_i becomes its
    Rayleigh quotient x^T A x / x^T M x, with the residual of ``residuals``.
    Returns (lam', X' in the input ordering, resid)."""
    X = np.asarray(X, dtype=float)
    n, nev = X.shape
    dsum = int(blk.off[-1])
    Xp = X[blk.perm]                     # interior-first ordering (new -> old)
    lam_new = np.empty(nev)
    Xnew = np.empty((n, nev))
    for i in range(nev):
        li = float(lam[i])
        y = Xp[dsum:, i]
        x = np.empty(n)
        x[dsum:] = y
        for j in range(blk.p):
            lo, hi = blk.off[j], blk.off[j + 1]
            rhs = -((blk.E[j] - li * blk.ME[j]) @ y)
            x[lo:hi] = sla.solve(blk.B[j] - li * blk.MB[j], rhs)
        xMx = x @ (blk.Mp @ x)
        lam_new[i] = (x @ (blk.Ap @ x)) / xMx
        Xnew[:, i] = x / np.sqrt(xMx)
    resid = residuals(blk.Ap, blk.Mp, lam_new, Xnew)
    return lam_new, blk.to_original(Xnew), resid


# ----------------------------------------------------------------------------------------
# Counting: Sylvester inertia through the DD blocks (Haynsworth additivity)
# ----------------------------------------------------------------------------------------

def inertia_count(blk: Blocks, sigma):
    """Number of eigenvalues of (A, M) below sigma: nu(A - sigma M) = nu(B_sigma) + nu(S(sigma))
    (Haynsworth inertia additivity applied to the block form of Eq. eq1)."""
    neg = 0
    for j in range(blk.p):
        neg += int(np.count_nonzero(np.linalg.eigvalsh(blk.B[j] - sigma * blk.MB[j]) < 0))
    S = np.real(schur(blk, sigma))
    S = 0.5 * (S + S.T)
    neg += int(np.count_nonzero(np.linalg.eigvalsh(S) < 0))
    return neg


# ----------------------------------------------------------------------------------------
# Algorithm 3 (RF-DDES) + completion passes
# ----------------------------------------------------------------------------------------

def select_nearest(theta, alpha, beta, m):
    """Indices of the m values closest to [alpha, beta] (distance 0 inside)."""
    dist = np.maximum(np.maximum(alpha - theta, theta - beta), 0.0)
    order = np.lexsort((np.abs(theta - 0.5 * (alpha + beta)), dist))
    return np.sort(order[:m])


def rfdd_solve(A, M, part, p, alpha, beta, n_nodes=4, rule="midpoint", sigma=None, nev_b=100,
               psi=3, lanczos_tol=1e-6, block=1, seed=1, res_tol=1e-10, max_passes=8,
               guard_frac=0.3, min_guard=8, groups=None):
    """RF-DDES (Algorithm 3) followed by completion passes.

    Readings:
    * sigma defaults to (alpha+beta)/2 (the paper's default is 0; the theory favours sigma
      near the wanted eigenvalues).  Guard: while sigma lies within 1e-8 max(1, |sigma|) of an
      eigenvalue of some (B_j, M_B^(j)), B_sigma is (nearly) singular and sigma moves by
      1e-6 (beta - alpha), at most three times.
    * nev_B^(j) = min(nev_b, d_j).
    * Completion (accuracy contract beyond the paper): X <- 2 Re sum omega (A - zeta M)^{-1} M X
      through Eq. (inv_dd2) with the same factors, then M-orthonormalisation and Rayleigh-Ritz;
      X starts from the m RF-DDES Ritz vectors nearest the interval, m = n_in + max(ceil(0.3 n_in),
      8); stop when every Ritz pair inside [alpha, beta] has residual <= res_tol and the count
      inside is unchanged from the previous pass.  When some inside pairs keep large residuals
      while the number of converged ones stays the same over two passes, the next filter
      application measures the filter gain (filter_gain) of those suspects; if every suspect's
      gain is below 1/4 they are spurious and the converged pairs of that pass are the result.
      When the Ritz values inside leave fewer than max(ceil(0.3 count), 8) columns of the block,
      the block doubles with counter-based vectors (stream 5000 + growth index), at most four
      times, two more passes each; at most max_passes + 10 passes in all.
    * groups: subdomain group labels for the two-level interface factorisation (TwoLevelSchur);
      None factors each S(zeta_l) densely.
    Returns a dict with eigenvalues, eigenvectors (original ordering), residuals and diagnostics.
    """
    A = sp.csr_matrix(A)
    M = sp.csr_matrix(M)
    if sigma is None:
        sigma = 0.5 * (alpha + beta)
    blk = Blocks(A, M, part, p)                                   # step 1
    for _ in range(3):
        gap = min(np.abs(sla.eigh(blk.B[j] - sigma * blk.MB[j], blk.MB[j], eigvals_only=True)).min()
                  for j in range(p))
        if gap >= 1e-8 * max(1.0, abs(sigma)):
            break
        sigma += 1e-6 * (beta - alpha)
    z, w = quadrature(alpha, beta, n_nodes, rule)
    fac = Factors(blk, z, groups)
    V = interior_eigvecs(blk, sigma, nev_b)                       # steps 2-4
    lz = lanczos_interface(lambda X: filter_interface(fac, w, X), blk.s, lanczos_tol, block, seed)
    Q = lz["Q"]                                                   # step 5
    Sig, Gam = resolvent_chains(blk, sigma, Q, psi)
    Z = build_Z(blk, V, Sig, Gam, Q, psi)                         # step 6
    Ap, Mp = blk.Ap, blk.Mp
    theta, X = rayleigh_ritz(Ap, Mp, Z)                           # step 7
    inside = (theta >= alpha) & (theta <= beta)
    pre = dict(theta=theta[inside].copy(), res=residuals(Ap, Mp, theta[inside], X[:, inside]),
               k=Z.shape[1], mu=lz["mu"])
    n_in = int(np.count_nonzero(inside))
    m = min(n_in + max(int(math.ceil(guard_frac * n_in)), min_guard), Z.shape[1])
    X = X[:, select_nearest(theta, alpha, beta, m)]
    count_prev = n_in
    passes = 0
    converged = False
    res_in = pre["res"]
    th_in = pre["theta"]
    X_in = X
    grown, limit, good_prev, suspect = 0, max_passes, -1, None
    while passes < limit:
        passes += 1
        Y = filter_full(fac, w, Mp @ X)                           # completion pass
        if suspect is not None:
            # the last pass's inside pairs with large residuals: spurious when the filter damps
            # them below 1/4 (mixtures of eigenvectors from both sides of the interval)
            th_s, res_s, X_s = suspect
            g = filter_gain(Mp, X_s, Y)
            bad = (th_s >= alpha) & (th_s <= beta) & (res_s > res_tol)
            if np.all(g[bad] < 0.25):
                ok = (th_s >= alpha) & (th_s <= beta) & (res_s <= res_tol)
                th_in, X_in, res_in = th_s[ok], X_s[:, ok], res_s[ok]
                converged = True
                break
        theta, X = rayleigh_ritz(Ap, Mp, Y)
        inside = (theta >= alpha) & (theta <= beta)
        th_in = theta[inside]
        X_in = X[:, inside]
        res_in = residuals(Ap, Mp, th_in, X_in)
        cnt = int(np.count_nonzero(inside))
        good = int(np.count_nonzero(res_in <= res_tol))
        guard = max(int(math.ceil(guard_frac * cnt)), min_guard)
        if cnt > 0 and X.shape[1] - cnt < guard and grown < 4 and X.shape[1] < X.shape[0]:
            mn = min(max(2 * X.shape[1], cnt + 2 * guard), X.shape[0])
            extra = counter_uniform(seed, 5000 + grown, X.shape[0] * (mn - X.shape[1]))
            X = np.hstack([X, extra.reshape(X.shape[0], mn - X.shape[1])])
            grown, limit = grown + 1, min(max_passes + 10, limit + 2)
            count_prev, good_prev, suspect = -1, -1, None
            continue
        if cnt == count_prev and (cnt == 0 or res_in.max() <= res_tol):
            converged = True
            break
        suspect = None
        if 0 < good < cnt and good == good_prev:
            res_all = np.full(len(theta), np.inf)
            res_all[inside] = res_in
            suspect = (theta.copy(), res_all, X.copy())
            limit = min(max_passes + 10, max(limit, passes + 1))
        count_prev, good_prev = cnt, good
    return dict(evals=th_in, evecs=blk.to_original(X_in), resid=res_in, passes=passes,
                converged=converged, mu=lz["mu"], k=Z.shape[1], pre=pre, blocks=blk,
                z=z, w=w, sigma=sigma, lanczos=lz)


# ----------------------------------------------------------------------------------------
# Algorithm 1 (RF-KRYLOV): Krylov on rho(M^{-1} A) in the whole space, Section 2.2
# ----------------------------------------------------------------------------------------

def _m_orth_against(Mp, Qs, W, passes=2):
    """W minus its M-projection onto the columns of the blocks in Qs (classical Gram-Schmidt,
    repeated ``passes`` times); also returns the accumulated coefficients Q^T M W per block."""
    coef = [np.zeros((Qk.shape[1], W.shape[1])) for Qk in Qs]
    for _ in range(passes):
        MW = Mp @ W
        for i, Qk in enumerate(Qs):
            c = Qk.T @ MW
            W = W - Qk @ c
            coef[i] += c
    return W, coef


def _m_cholqr(Mp, W):
    """W = Q R with Q^T M Q = I, R upper triangular (Cholesky of the Gram matrix W^T M W)."""
    G = W.T @ (Mp @ W)
    R = np.linalg.cholesky(0.5 * (G + G.T)).T
    return sla.solve_triangular(R, W.T, trans="T", lower=False).T, R


def rf_krylov(Ap, Mp, apply_rho, alpha, beta, tol=1e-6, block=1, seed=1, check_every=10, max_dim=None):
    """Algorithm 1 (RF-KRYLOV) on rho(M^{-1}A), with ``apply_rho(Q)`` = 2 Re sum_l omega_l
    (A - zeta_l M)^{-1} M Q (line 2).  Returns dict(Q (n x mu), H (mu x mu), mu, sums, theta,
    X, inside): the Krylov basis, the projected matrix, the sums that line 13 compares, and the
    Ritz pairs of (A, M) from lines 15-16 (X M-orthonormal, theta ascending; ``inside`` marks
    theta in [alpha, beta]).

    Readings:
    * the inner product is M's.  rho(M^{-1}A) is self-adjoint in it, so H_mu = Q^T M rho Q is
      symmetric and the Arnoldi process of lines 3-12 is a Lanczos process with full
      orthogonalisation; with M = I (the paper's RF-KRYLOV experiments) it is the printed
      Euclidean one.
    * q^(1): ``block`` counter-based uniform vectors (stream 7000), M-orthonormalised; b = 1 is
      the printed algorithm.
    * lines 3-6 are run twice (CGS2); h_{k,mu} accumulates both passes.
    * lines 7-12: the columns of the new block are M-normalised one after another, each first
      projected (twice) off Q and the block's earlier columns; a column whose M norm is then at
      most 1e-14 max|H| (breakdown, h_{mu+1,mu} = 0) is replaced by fresh counter-based vectors
      (streams 7001, ...) projected the same way.
    * line 13: every ceil(check_every / b) block steps, stop when the sum of the eigenvalues of
      (the symmetric part of) H_mu that are >= 1/2 changed by at most tol times its magnitude
      since the previous check; also stop when mu reaches n or ``max_dim``.
    * lines 15-16: the Ritz vectors of (A, M) are those of the Rayleigh-Ritz problem on
      range(Q_mu); each one's Rayleigh quotient x^T A x / x^T M x is its Ritz value.  (The
      eigenvectors of H_mu alone are not enough where rho takes nearly equal values on several
      eigenvalues -- rho is symmetric about the centre of [alpha, beta] -- since any mixture of
      their eigenvectors is then an eigenvector of H_mu.)
    """
    n = Ap.shape[0]
    b = block
    max_dim = min(max_dim or n, n)
    Q1, _ = _m_cholqr(Mp, counter_uniform(seed, 7000, n * b).reshape(n, b))
    Qs = [Q1]
    cols = []               # H columns, one block of b columns per step
    sums = []
    steps_per_check = max(1, -(-check_every // b))
    last = None
    extra = 1
    mu = b
    while True:
        W = apply_rho(Qs[-1])                                               # line 2
        W, coef = _m_orth_against(Mp, Qs, W)                                # lines 3-6 (twice)
        cols.append(np.vstack(coef))
        t = len(cols)
        if t % steps_per_check == 0 or mu >= max_dim:                       # line 13
            H = _assemble_h(cols, Qs, b)
            ev = np.linalg.eigvalsh(H)
            cur = float(ev[ev >= 0.5].sum())
            sums.append(cur)
            if last is not None and abs(cur - last) <= tol * abs(cur):
                break
            last = cur
        if mu >= max_dim:
            break
        bn = min(b, max_dim - mu)
        # lines 7-12, column by column: normalise in the M norm what is left after the
        # projections; a column left with norm <= 1e-14 max|H| (h_{mu+1,mu} = 0) is replaced by
        # a fresh counter-based vector orthogonal to everything so far
        hmax = max(np.abs(c).max() for c in cols)
        new_cols = []
        for j in range(bn):
            v = W[:, j:j + 1]
            for attempt in range(2):
                prev = Qs + ([np.hstack(new_cols)] if new_cols else [])
                v, _ = _m_orth_against(Mp, prev, v)
                nrm = math.sqrt(max(float(v[:, 0] @ (Mp @ v[:, 0])), 0.0))
                if nrm > 1e-14 * max(hmax, 1e-300):
                    break
                v = counter_uniform(seed, 7000 + extra, n).reshape(n, 1)
                extra += 1
            new_cols.append(v / nrm)
        Qs.append(np.hstack(new_cols))
        mu += bn
    Q = np.hstack(Qs[:len(cols)])
    H = _assemble_h(cols, Qs, b)
    theta, X = rayleigh_ritz(Ap, Mp, Q)                                      # lines 15-16
    inside = (theta >= alpha) & (theta <= beta)
    return dict(Q=Q, H=H, mu=Q.shape[1], sums=sums, theta=theta, X=X, inside=inside)


def _assemble_h(cols, Qs, b):
    """H_mu = Q_mu^T M rho(M^{-1}A) Q_mu.  The block column of step t holds the coefficients of
    rho(M^{-1}A) Q_t on blocks 1..t, i.e. the blocks of H on and above the diagonal; H is
    symmetric, so the blocks below it are their transposes (the diagonal blocks are
    symmetrised)."""
    widths = [q.shape[1] for q in Qs[:len(cols)]]
    mu = sum(widths)
    U = np.zeros((mu, mu))
    c0 = 0
    for t, c in enumerate(cols):
        w = widths[t]
        U[:c.shape[0], c0:c0 + w] = c[:, :w]
        c0 += w
    D = np.zeros((mu, mu))
    c0 = 0
    for w in widths:
        blk = U[c0:c0 + w, c0:c0 + w]
        D[c0:c0 + w, c0:c0 + w] = 0.5 * (blk + blk.T)
        U[c0:c0 + w, c0:c0 + w] = 0.0
        c0 += w
    return U + U.T + D


def filter_gain(Mp, X, Y):
    """Filter gain of each column x of an M-orthonormal block X with Y = rho(A) X: the Rayleigh
    quotient x^T M rho(A) x, which is rho(lambda) when x is an eigenvector (rho >= 1/2 on
    [alpha, beta], Section 2.1)."""
    return np.einsum("ij,ij->j", Mp @ X, Y)


def brute_force(A, M, alpha=None, beta=None):
    """All eigenpairs of the pencil by a dense generalised symmetric eigensolve (small n)."""
    A = sp.csr_matrix(A).toarray()
    M = sp.csr_matrix(M).toarray()
    lam, X = sla.eigh(A, M)
    if alpha is not None:
        sel = (lam >= alpha) & (lam <= beta)
        lam, X = lam[sel], X[:, sel]
    return lam, X
