"""Seeded synthetic inputs for the RF-DDES interface-filter path.

This module builds the *problems* only: sparse symmetric pencils (A, M), vertex-separator
partitions, the closed-form spectra of the tensor-product Q1 pencils and the search
intervals [alpha, beta] derived from them.  It holds none of the eigensolver's arithmetic,
so both the CPU oracle (``oracle/``) and the GPU path consume identical arrays from here
without sharing any method code.

Pencil shapes follow the paper's model problems (Section 6: finite-difference / finite-element
Laplacians, ``M = I`` or a mass matrix) and the synthetic workloads named for this build:

* ``q1_pencil(N, dim)``: Q1 finite-element Laplacian on an N^dim interior grid, h = 1/(N+1),
  built as Kronecker sums of the 1-D pencil K1 = (1/h) tridiag(-1, 2, -1),
  M1 = (h/6) tridiag(1, 4, 1).  Its eigenvalues are sums over the axes of
  (6/h^2)(1 - cos t_k)/(2 + cos t_k), t_k = k pi/(N+1)  (``q1_eigenvalues``).
* ``varkappa7_pencil(N, seed)``: 3-D 7-point diffusion with a per-edge coefficient
  kappa_e = exp(g_e), g_e ~ N(0, 1) i.i.d., boundary edges included, and a diagonal lumped mass
  with entries uniform in [0.5, 1.5].
* ``fd5_pencil(N)``: the 2-D 5-point finite-difference Laplacian stencil (4 on the diagonal,
  -1 to each grid neighbour, Dirichlet boundary, no 1/h^2 scaling) on an N x N grid with M = I,
  the pencils the paper's distributed comparison calls FDmesh (FDmesh2: N = 500,
  n = 250,000; FDmesh3: N = 1000).  Eigenvalues 4 - 2 cos(a pi/(N+1)) - 2 cos(b pi/(N+1))
  (``fd5_eigenvalues``).
* ``geometric_partition``: axis-aligned vertex separators (planes of width one node) that split
  the grid into a product of blocks; label -1 marks the interface (the ordering of Eq. dd1 puts
  those variables last).

Matrices are returned as full (both triangles) CSR with int64 row pointers, int32 column
indices sorted within each row and float64 values.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

__all__ = [
    "Csr", "Pencil", "q1_1d", "q1_pencil", "q1_eigenvalues", "varkappa7_pencil",
    "separator_planes", "geometric_partition", "interval_from_sorted", "workload",
    "WORKLOADS", "random_rhs", "snap_to_gaps", "sym_inertia_count", "VARKAPPA_POOL", "serving_stream",
    "serving_pencil", "fd5_pencil", "fd5_eigenvalues",
]


@dataclasses.dataclass
class Csr:
    """Full symmetric CSR: ``rowptr`` int64[n+1], ``col`` int32[nnz], ``val`` float64[nnz]."""
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @staticmethod
    def from_scipy(a) -> "Csr":
        a = sp.csr_matrix(a, dtype=np.float64)
        a.sum_duplicates()
        a.sort_indices()
        return Csr(a.shape[0], a.indptr.astype(np.int64), a.indices.astype(np.int32),
                   a.data.astype(np.float64))

    def to_scipy(self):
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


@dataclasses.dataclass
class Pencil:
    """A seeded problem instance: pencil, partition, interval and quadrature choice."""
    name: str
    A: Csr
    M: Csr
    part: np.ndarray            # int32[n], -1 = interface, 0..p-1 = subdomain
    p: int
    alpha: float
    beta: float
    n_nodes: int
    rule: str                   # "midpoint" | "gauss_legendre"
    exact: np.ndarray | None    # sorted closed-form eigenvalues of the whole pencil, if known
    expected_nev: int | None    # eigenvalue count inside [alpha, beta], if known
    grid: tuple = ()
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.n


# ----------------------------------------------------------------------------------------
# Q1 tensor-product Laplacian pencils
# ----------------------------------------------------------------------------------------

def q1_1d(N: int):
    """1-D linear finite-element stiffness and mass matrices on N interior nodes."""
    h = 1.0 / (N + 1)
    e = np.ones(N)
    K1 = sp.diags([-e[:-1], 2 * e, -e[:-1]], [-1, 0, 1]) / h
    M1 = sp.diags([e[:-1], 4 * e, e[:-1]], [-1, 0, 1]) * (h / 6.0)
    return sp.csr_matrix(K1), sp.csr_matrix(M1)


def q1_pencil(N: int, dim: int) -> tuple[Csr, Csr]:
    """Q1 Laplacian pencil on an N^dim grid as a Kronecker sum (row-major grid ordering)."""
    K1, M1 = q1_1d(N)
    if dim == 2:
        A = sp.kron(K1, M1) + sp.kron(M1, K1)
        M = sp.kron(M1, M1)
    elif dim == 3:
        A = sp.kron(sp.kron(K1, M1), M1) + sp.kron(sp.kron(M1, K1), M1) + sp.kron(sp.kron(M1, M1), K1)
        M = sp.kron(sp.kron(M1, M1), M1)
    else:
        raise ValueError("dim must be 2 or 3")
    return Csr.from_scipy(A), Csr.from_scipy(M)


def q1_eigenvalues(N: int, dim: int) -> np.ndarray:
    """Sorted closed-form eigenvalues of ``q1_pencil(N, dim)``."""
    h = 1.0 / (N + 1)
    t = np.arange(1, N + 1) * np.pi / (N + 1)
    lam = (6.0 / h ** 2) * (1.0 - np.cos(t)) / (2.0 + np.cos(t))
    if dim == 2:
        ev = lam[:, None] + lam[None, :]
    else:
        ev = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    return np.sort(ev.ravel())


# ----------------------------------------------------------------------------------------
# 5-point finite-difference Laplacian with M = I (the FDmesh pencils)
# ----------------------------------------------------------------------------------------

def fd5_pencil(N: int) -> tuple[Csr, Csr]:
    """tridiag(-1, 2, -1) Kronecker-summed over two axes (row-major grid), and M = I."""
    e = np.ones(N)
    T = sp.diags([-e[:-1], 2 * e, -e[:-1]], [-1, 0, 1])
    I1 = sp.identity(N)
    A = sp.kron(T, I1) + sp.kron(I1, T)
    return Csr.from_scipy(A), Csr.from_scipy(sp.identity(N * N))


def fd5_eigenvalues(N: int) -> np.ndarray:
    """Sorted closed-form eigenvalues of ``fd5_pencil(N)``."""
    lam = 2.0 - 2.0 * np.cos(np.arange(1, N + 1) * np.pi / (N + 1))
    return np.sort((lam[:, None] + lam[None, :]).ravel())


# ----------------------------------------------------------------------------------------
# Variable-coefficient 7-point diffusion pencil
# ----------------------------------------------------------------------------------------

def varkappa7_pencil(N: int, seed: int) -> tuple[Csr, Csr]:
    """3-D 7-point diffusion, per-edge kappa = exp(g), g ~ N(0,1); lumped M ~ U[0.5, 1.5].

    A = sum_e kappa_e h^-2 (e_i - e_j)(e_i - e_j)^T over interior edges; an edge from a node to
    the Dirichlet boundary adds kappa_e h^-2 to that node's diagonal only.
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / (N + 1)
    n = N ** 3
    idx = np.arange(n).reshape(N, N, N)
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    for axis in range(3):
        # N+1 edges per grid line along this axis: boundary, N-1 interior, boundary
        shape = [N, N, N]
        shape[axis] = N + 1
        kap = np.exp(rng.standard_normal(shape)) / h ** 2
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        # edge e between node e-1 and node e along the axis (e = 0..N)
        sl_lo[axis] = slice(0, N)      # edges 0..N-1 touch node e (the node on their + side)
        sl_hi[axis] = slice(1, N + 1)  # edges 1..N touch node e-1 (the node on their - side)
        diag += kap[tuple(sl_lo)].ravel() + kap[tuple(sl_hi)].ravel()
        inner = [slice(None)] * 3
        inner[axis] = slice(1, N)
        k_in = kap[tuple(inner)]
        a_sl = [slice(None)] * 3
        b_sl = [slice(None)] * 3
        a_sl[axis] = slice(0, N - 1)
        b_sl[axis] = slice(1, N)
        ia = idx[tuple(a_sl)].ravel()
        ib = idx[tuple(b_sl)].ravel()
        kv = k_in.ravel()
        rows += [ia, ib]
        cols += [ib, ia]
        vals += [-kv, -kv]
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(diag)
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    M = sp.diags(rng.uniform(0.5, 1.5, n))
    return Csr.from_scipy(A), Csr.from_scipy(M)


def sym_inertia_count(A: Csr, M: Csr, beta: float) -> int:
    """Number of eigenvalues of the pencil (A, M) below ``beta`` (M SPD), by Sylvester's law of
    inertia: P (A - beta M) P^T = L D L^T with a fill-reducing symmetric permutation P and no
    off-diagonal pivoting (SuperLU in symmetric mode, diagonal pivots only), so the count is the
    number of negative entries of D = diag(U).  Used to place the intervals of generated
    requests; it is not the solver's eigenvalue count (that one works through the domain
    decomposition on the GPU)."""
    import scipy.sparse.linalg as sla
    K = (A.to_scipy() - beta * M.to_scipy()).tocsc()
    lu = sla.splu(K, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0, options=dict(SymmetricMode=True))
    if not np.array_equal(lu.perm_r, lu.perm_c):
        raise RuntimeError("sym_inertia_count: the factorisation pivoted off the diagonal")
    d = lu.U.diagonal()
    if not np.all(np.isfinite(d)) or np.any(d == 0):
        raise RuntimeError(f"sym_inertia_count: singular or unstable at beta={beta}")
    return int(np.count_nonzero(d < 0))


# the 3-D variable-coefficient pencils of the serving stream: (N, seed); the exact eigenvalue
# counts on a grid of shifts are stored in varkappa_counts.json (make_varkappa_counts.py)
VARKAPPA_POOL = [(24, 1), (24, 2), (32, 1), (32, 2), (40, 1), (40, 2), (48, 1), (48, 2)]


# ----------------------------------------------------------------------------------------
# Geometric vertex-separator partitions
# ----------------------------------------------------------------------------------------

def separator_planes(N: int, k: int, shift_frac: float = 0.0, rng=None) -> list[int]:
    """0-based separator indices along one axis of N nodes split k ways.

    Nominal planes sit at floor(i (N+1)/k) - 1, i = 1..k-1.  With ``shift_frac`` > 0 each plane
    moves by round(u * shift_frac * (N+1)/k), u ~ U[-1, 1]; planes stay strictly increasing with
    at least one interior node between neighbours and at both ends.
    """
    c = [(i * (N + 1)) // k - 1 for i in range(1, k)]
    if shift_frac > 0.0:
        assert rng is not None
        span = shift_frac * (N + 1) / k
        c = [ci + int(round(rng.uniform(-1.0, 1.0) * span)) for ci in c]
        lo = 1
        for i in range(len(c)):
            hi = N - 2 - 2 * (len(c) - 1 - i)
            c[i] = min(max(c[i], lo), hi)
            lo = c[i] + 2
    return c


def geometric_partition(N: int, dim: int, splits: tuple[int, ...], shift_frac: float = 0.0,
                        seed: int | None = None) -> tuple[np.ndarray, int]:
    """Label every grid node with its subdomain (row-major over axis blocks) or -1 (interface)."""
    assert len(splits) == dim
    rng = np.random.default_rng(seed) if shift_frac > 0 else None
    block_of = []
    on_sep = []
    for k in splits:
        planes = separator_planes(N, k, shift_frac, rng)
        b = np.zeros(N, dtype=np.int64)
        sep = np.zeros(N, dtype=bool)
        for c in planes:
            sep[c] = True
            b[c + 1:] += 1
        block_of.append(b)
        on_sep.append(sep)
    grids = np.meshgrid(*[np.arange(N)] * dim, indexing="ij")
    lab = np.zeros([N] * dim, dtype=np.int64)
    sep = np.zeros([N] * dim, dtype=bool)
    for ax in range(dim):
        lab = lab * splits[ax] + block_of[ax][grids[ax]]
        sep |= on_sep[ax][grids[ax]]
    lab[sep] = -1
    p = int(np.prod(splits))
    return lab.ravel().astype(np.int32), p


def subdomain_groups(splits: tuple[int, ...], group_splits: tuple[int, ...]) -> np.ndarray:
    """Group label of every subdomain of ``geometric_partition(N, dim, splits)`` when the blocks
    along each axis are gathered into ``group_splits[ax]`` contiguous runs (row-major over the
    group grid, like the subdomain ids).  Input to the two-level interface factorisation."""
    assert len(splits) == len(group_splits)
    for k, g in zip(splits, group_splits):
        assert 1 <= g <= k
    idx = np.meshgrid(*[np.arange(k) for k in splits], indexing="ij")
    lab = np.zeros(splits, dtype=np.int64)
    for ax, (k, g) in enumerate(zip(splits, group_splits)):
        lab = lab * g + (idx[ax] * g) // k
    return lab.ravel().astype(np.int32)


def interval_from_sorted(ev: np.ndarray, first: int, last: int) -> tuple[float, float]:
    """[alpha, beta] holding sorted eigenvalues first..last (1-based, inclusive), with both
    endpoints at the midpoints of the neighbouring spectral gaps."""
    alpha = 0.5 * (ev[first - 2] + ev[first - 1]) if first > 1 else ev[0] - 1.0
    beta = 0.5 * (ev[last - 1] + ev[last])
    return float(alpha), float(beta)


# ----------------------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------------------

def snap_to_gaps(ev: np.ndarray, first: int, last: int, rtol: float = 1e-10) -> tuple[int, int]:
    """Widen the 1-based window first..last so that it does not cut through a cluster of equal
    eigenvalues (multiplicities of tensor-product spectra)."""
    while first > 1 and ev[first - 1] - ev[first - 2] <= rtol * abs(ev[first - 1]):
        first -= 1
    while last < len(ev) and ev[last] - ev[last - 1] <= rtol * abs(ev[last - 1]):
        last += 1
    return first, last


def _q1_workload(name, N, dim, splits, first, last, n_nodes, rule):
    A, M = q1_pencil(N, dim)
    part, p = geometric_partition(N, dim, splits)
    ev = q1_eigenvalues(N, dim)
    first, last = snap_to_gaps(ev, first, last)
    alpha, beta = interval_from_sorted(ev, first, last)
    nev = int(np.count_nonzero((ev > alpha) & (ev < beta)))
    return Pencil(name, A, M, part, p, alpha, beta, n_nodes, rule, ev, nev,
                  grid=(N,) * dim, meta=dict(first=first, last=last, splits=splits))


def _fd5_workload(name, N, splits, first, last, n_nodes, rule):
    A, M = fd5_pencil(N)
    part, p = geometric_partition(N, 2, splits)
    ev = fd5_eigenvalues(N)
    first, last = snap_to_gaps(ev, first, last)
    alpha, beta = interval_from_sorted(ev, first, last)
    if first == 1:
        alpha = 0.0   # the smallest eigenvalues: [0, beta], as the paper's FDmesh windows
    nev = int(np.count_nonzero((ev > alpha) & (ev < beta)))
    return Pencil(name, A, M, part, p, alpha, beta, n_nodes, rule, ev, nev,
                  grid=(N, N), meta=dict(first=first, last=last, splits=splits))


def workload(name: str) -> Pencil:
    """Build one named seeded workload (see ``WORKLOADS``)."""
    if name not in WORKLOADS:
        raise KeyError(f"unknown workload {name!r}; known: {sorted(WORKLOADS)}")
    return WORKLOADS[name]()


WORKLOADS = {
    # 2-D Q1, 40x40 interior grid, 2x2 cross separator (79 nodes), eigenvalues 51..100,
    # 4 Gauss-Legendre nodes on the upper semicircle.
    "q1_2d_40": lambda: _q1_workload("q1_2d_40", 40, 2, (2, 2), 51, 100, 4, "gauss_legendre"),
    # 3-D Q1, 40^3 grid, 2x2x2 separators (8 subdomains, s = 4681), eigenvalues 300..501
    # (the window 301..500 widened to whole eigenvalue clusters), 8 midpoint nodes.
    "q1_3d_40": lambda: _q1_workload("q1_3d_40", 40, 3, (2, 2, 2), 300, 501, 8, "midpoint"),
    # Small cases for parity tests: several tiles and ragged tails, oracle in seconds.
    "q1_2d_24": lambda: _q1_workload("q1_2d_24", 24, 2, (2, 2), 11, 30, 4, "midpoint"),
    "q1_2d_33_p9": lambda: _q1_workload("q1_2d_33_p9", 33, 2, (3, 3), 21, 40, 6, "midpoint"),
    "q1_3d_12": lambda: _q1_workload("q1_3d_12", 12, 3, (2, 2, 2), 8, 27, 6, "midpoint"),
    "q1_3d_16": lambda: _q1_workload("q1_3d_16", 16, 3, (2, 2, 2), 20, 60, 8, "midpoint"),
    "q1_2d_64": lambda: _q1_workload("q1_2d_64", 64, 2, (2, 2), 40, 120, 8, "midpoint"),
    # many subdomains, for the two-level interface factorisation (groups of subdomains)
    "q1_2d_49_p16": lambda: _q1_workload("q1_2d_49_p16", 49, 2, (4, 4), 21, 60, 6, "midpoint"),
    "q1_3d_24_p64": lambda: _q1_workload("q1_3d_24_p64", 24, 3, (4, 4, 4), 30, 80, 8, "midpoint"),
    # 3-D Q1, 48^3, 4 x 4 x 4 subdomains (s = 19,467 against d_j of 1,331-1,728): the dense S(zeta)
    # dominates the factorisation; eigenvalues 100..200, 8 midpoint nodes
    "q1_3d_48_p64": lambda: _q1_workload("q1_3d_48_p64", 48, 3, (4, 4, 4), 100, 200, 8, "midpoint"),
    # FDmesh2 of the paper's RF-KRYLOV / RF-DDES comparison: 5-point FD Laplacian, M = I, 500^2
    # grid (n = 250,000), the 100 algebraically smallest eigenvalues, Nc = 2 midpoint nodes; an
    # 8 x 8 separator grid (64 subdomains of about 62^2, s = 6,951) so that the dense
    # subdomain blocks stay small.
    "fdmesh2": lambda: _fd5_workload("fdmesh2", 500, (8, 8), 1, 100, 2, "midpoint"),
    # small FD cases for parity tests
    "fd5_32": lambda: _fd5_workload("fd5_32", 32, (2, 2), 1, 20, 4, "midpoint"),
    "fd5_40_p16": lambda: _fd5_workload("fd5_40_p16", 40, (4, 4), 1, 30, 2, "midpoint"),
}


def random_rhs(n: int, b: int, seed: int) -> np.ndarray:
    """Seeded dense test block (n x b, float64, row-major) for solve/filter parity cases."""
    return np.random.default_rng(seed).standard_normal((n, b))


# ----------------------------------------------------------------------------------------
# Serving stream: requests of mixed size and kind
# ----------------------------------------------------------------------------------------

def _varkappa_counts():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "varkappa_counts.json")
    with open(path) as f:
        return {(e["N"], e["seed"]): (np.array(e["beta"]), np.array(e["count"])) for e in json.load(f)["pencils"]}


MAX_BLOCK = 8192  # largest nominal subdomain interior (unknowns) a generated request may have


def _pick_splits(rng, n: int, options: list) -> tuple:
    """A partition drawn uniformly among the options whose nominal subdomain size n / p is at most
    MAX_BLOCK (the dense blocks of a larger one would hold most of the device on their own)."""
    ok = [sp_ for sp_ in options if n / math.prod(sp_) <= MAX_BLOCK]
    return ok[int(rng.integers(0, len(ok)))]


def serving_stream(count: int = 256, seed: int = 7) -> list[dict]:
    """Seeded request descriptions of the serving stream (arrival times are drawn by the caller).

    Half the requests are 2-D Q1 Laplacian pencils on an N^2 grid, N ~ U{64..256}, with a window of
    nev ~ U[20, 400] consecutive eigenvalues starting at index U{1..200}, widened to whole clusters
    and bounded at gap midpoints (closed form).  The other half are 3-D variable-coefficient
    7-point pencils drawn from ``VARKAPPA_POOL`` (N = 24..48), with a window between two shifts of
    the stored count grid that holds 20..400 eigenvalues (exact counts by inertia).  Partitions:
    2x2, 4x2 or 4x4 (2-D) and 2x2x1, 2x2x2 or 4x2x2 (3-D), i.e. p in {4, 8, 16}, drawn among those
    whose nominal subdomain holds at most MAX_BLOCK = 8192 unknowns; 8 midpoint nodes.
    """
    rng = np.random.default_rng(seed)
    counts = None
    out = []
    for i in range(count):
        if rng.random() < 0.5:
            N = int(rng.integers(64, 257))
            splits = _pick_splits(rng, N ** 2, [(2, 2), (4, 2), (4, 4)])
            ev = q1_eigenvalues(N, 2)
            nev = int(rng.integers(20, 401))
            first = int(rng.integers(1, 201))
            first, last = snap_to_gaps(ev, first, first + nev - 1)
            alpha, beta = interval_from_sorted(ev, first, last)
            out.append(dict(index=i, kind="q1_2d", N=N, seed=0, splits=splits, alpha=alpha, beta=beta,
                            nev=last - first + 1, n_nodes=8, n=N * N))
        else:
            if counts is None:
                counts = _varkappa_counts()
            N, pseed = VARKAPPA_POOL[int(rng.integers(0, len(VARKAPPA_POOL)))]
            splits = _pick_splits(rng, N ** 3, [(2, 2, 1), (2, 2, 2), (4, 2, 2)])
            betas, cnt = counts[(N, pseed)]
            pairs = [(a, b) for a in range(len(cnt)) for b in range(a + 1, len(cnt))
                     if 20 <= cnt[b] - cnt[a] <= 400]
            a, b = pairs[int(rng.integers(0, len(pairs)))]
            out.append(dict(index=i, kind="varkappa7_3d", N=N, seed=pseed, splits=splits,
                            alpha=float(betas[a]), beta=float(betas[b]), nev=int(cnt[b] - cnt[a]), n_nodes=8,
                            n=N ** 3))
    return out


def serving_pencil(req: dict) -> tuple[Csr, Csr, np.ndarray, int]:
    """(A, M, part, p) of one request of ``serving_stream``."""
    N, splits = req["N"], tuple(req["splits"])
    if req["kind"] == "q1_2d":
        A, M = q1_pencil(N, 2)
        part, p = geometric_partition(N, 2, splits)
    else:
        A, M = varkappa7_pencil(N, req["seed"])
        part, p = geometric_partition(N, 3, splits)
    return A, M, part, p
