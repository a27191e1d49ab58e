"""Seeded synthetic KKT inputs shaped like OPF / SCOPF networks.

This module only draws inputs: CSR patterns and random values for the
components of the NCL Newton system (the Hessian H, the Jacobian J, the
barrier diagonal Sigma, the regularisation delta, the penalty rho and the
right-hand sides).  It does no factorisation, no solve and no assembly of
the KKT matrices, so both the CPU oracle and the CUDA path can be fed from
it without sharing any of the method's arithmetic.

Network model (a power-grid-like R x C grid graph with 4-neighbour edges):

* bus ``b = r*C + c``; primal variables ``4b+v`` (v = 0..3); constraint rows
  ``2b+k`` (k = 0, 1).
* Jacobian row ``2b+k`` touches the variable pair ``{4b'+2k, 4b'+2k+1}`` of
  the bus itself and of each neighbour ``b'`` (10 entries for an interior
  bus), values N(0, 1).
* Hessian ``H = sum_e Q_e diag(lambda_e) Q_e^T`` over the 8 variables of the
  two endpoints of each edge ``e``, with ``Q_e`` Haar-distributed (QR of an
  8x8 Gaussian with the sign of diag(R) folded in) and ``lambda_e ~ U[-1,1]``.
* ``Sigma_i = 10**U[-2, 2]`` (the barrier term of Section 3.1, a positive
  diagonal).
* ``delta``: 0 if positive definiteness of ``H + Sigma`` is certified,
  otherwise the smallest power of ten that certifies ``H + Sigma + delta*I``
  positive definite.  The certificate is the edge-block bound
  ``H >= -diag(c)`` with ``c_i = sum over edges e touching variable i of
  max(0, -min(lambda_e))`` (each block is ``>= min(lambda_e) * I`` on its 8
  variables).
* seeds: numpy PCG64 with ``seed = 251005885 + 1000*config + draw``.
"""
from __future__ import annotations

import dataclasses
import numpy as np

SEED_BASE = 251005885


def seed_for(config: int, draw: int) -> int:
    return SEED_BASE + 1000 * int(config) + int(draw)


@dataclasses.dataclass
class GridPattern:
    """Sparsity pattern of one grid network (no values)."""

    R: int
    C: int
    n: int                 # primal variables = 4 * buses
    m: int                 # constraint rows = 2 * buses
    edges: np.ndarray      # (E, 2) int64, b1 < b2
    H_rowptr: np.ndarray   # lower CSR of H incl. the full diagonal (int32)
    H_colind: np.ndarray
    J_rowptr: np.ndarray   # CSR of J, m x n (int32)
    J_colind: np.ndarray
    edge_pos: np.ndarray   # (E, 36) position in H_val of each lower block entry
    var_edge_count: np.ndarray  # per primal variable: incident edges

    @property
    def nnz_H(self) -> int:
        return int(self.H_rowptr[-1])

    @property
    def nnz_J(self) -> int:
        return int(self.J_rowptr[-1])


_LOW_A, _LOW_B = np.tril_indices(8)   # 36 lower entries of an 8x8 block


def grid_edges(R: int, C: int) -> np.ndarray:
    b = np.arange(R * C, dtype=np.int64).reshape(R, C)
    right = np.stack([b[:, :-1].ravel(), b[:, 1:].ravel()], axis=1)
    down = np.stack([b[:-1, :].ravel(), b[1:, :].ravel()], axis=1)
    e = np.concatenate([right, down], axis=0)
    order = np.lexsort((e[:, 1], e[:, 0]))
    return e[order]


def make_pattern(R: int, C: int, deleted: np.ndarray | None = None) -> GridPattern:
    """Pattern of H (lower CSR with diagonal) and J for an R x C grid.

    ``deleted`` lists edge indices (into ``grid_edges(R, C)``) to remove: the
    edge's Hessian block and the Jacobian coupling between its endpoints go.
    """
    N = R * C
    edges = grid_edges(R, C)
    if deleted is not None and len(deleted):
        keep = np.ones(len(edges), bool)
        keep[np.asarray(deleted, dtype=np.int64)] = False
        edges = edges[keep]
    E = len(edges)
    n, m = 4 * N, 2 * N

    # ---- H lower pattern: 4x4 lower block of every bus + 4x4 block per edge
    bb = np.arange(N, dtype=np.int64)
    la, lb = np.tril_indices(4)
    rows_d = (4 * bb[:, None] + la[None, :]).ravel()
    cols_d = (4 * bb[:, None] + lb[None, :]).ravel()
    a4, c4 = np.meshgrid(np.arange(4), np.arange(4), indexing="ij")
    rows_o = (4 * edges[:, 1][:, None] + a4.ravel()[None, :]).ravel()
    cols_o = (4 * edges[:, 0][:, None] + c4.ravel()[None, :]).ravel()
    rows = np.concatenate([rows_d, rows_o])
    cols = np.concatenate([cols_d, cols_o])
    key = np.sort(rows * n + cols)
    key = key[np.concatenate([[True], key[1:] != key[:-1]])]   # sorted, unique
    rows = key // n
    cols = key % n
    H_rowptr = np.zeros(n + 1, np.int64)
    np.add.at(H_rowptr, rows + 1, 1)
    H_rowptr = np.cumsum(H_rowptr)
    H_colind = cols

    # position of each (edge, lower local entry) in H_val
    ev = np.concatenate([4 * edges[:, :1] + np.arange(4)[None, :],
                         4 * edges[:, 1:] + np.arange(4)[None, :]], axis=1)  # (E, 8)
    gr = ev[:, _LOW_A]
    gc = ev[:, _LOW_B]
    edge_pos = np.searchsorted(key, gr * n + gc)
    assert np.all(key[edge_pos] == gr * n + gc)

    var_edge_count = np.zeros(n, np.int64)
    if E:
        np.add.at(var_edge_count, ev.ravel(), 1)

    # ---- J pattern: row 2b+k -> vars {4b'+2k, 4b'+2k+1}, b' in {b} U nbr(b)
    pairs = np.concatenate([np.stack([bb, bb], 1), edges, edges[:, ::-1]], 0)
    order = np.lexsort((pairs[:, 1], pairs[:, 0]))
    pairs = pairs[order]
    deg1 = np.bincount(pairs[:, 0], minlength=N)            # 1 + degree
    starts = np.concatenate([[0], np.cumsum(deg1)])
    row_len = np.repeat(2 * deg1, 2)                          # rows 2b, 2b+1
    J_rowptr = np.concatenate([[0], np.cumsum(row_len)])
    J_colind = np.empty(J_rowptr[-1], np.int64)
    # entries of row 2b+k, in order of b': 4b'+2k, 4b'+2k+1
    for k in range(2):
        rstart = J_rowptr[2 * bb + k]
        # offset of pair p within its bus group
        p_bus = pairs[:, 0]
        p_off = np.arange(len(pairs)) - starts[p_bus]
        base = rstart[p_bus] + 2 * p_off
        J_colind[base] = 4 * pairs[:, 1] + 2 * k
        J_colind[base + 1] = 4 * pairs[:, 1] + 2 * k + 1

    return GridPattern(R=R, C=C, n=n, m=m, edges=edges,
                       H_rowptr=H_rowptr.astype(np.int32), H_colind=H_colind.astype(np.int32),
                       J_rowptr=J_rowptr.astype(np.int32), J_colind=J_colind.astype(np.int32),
                       edge_pos=edge_pos, var_edge_count=var_edge_count)


def haar_blocks(rng: np.random.Generator, count: int, k: int = 8) -> np.ndarray:
    """``count`` Haar-distributed k x k orthogonal matrices."""
    G = rng.standard_normal((count, k, k))
    Q, Rr = np.linalg.qr(G)
    s = np.sign(np.diagonal(Rr, axis1=1, axis2=2))
    s[s == 0] = 1.0
    return Q * s[:, None, :]


def draw_H(pat: GridPattern, rng: np.random.Generator):
    """Values of H on ``pat`` and the per-variable certificate weights."""
    E = len(pat.edges)
    Hval = np.zeros(pat.nnz_H)
    cert = np.zeros(pat.n)
    if E == 0:
        return Hval, cert
    Q = haar_blocks(rng, E)
    lam = rng.uniform(-1.0, 1.0, size=(E, 8))
    B = np.einsum("eik,ek,ejk->eij", Q, lam, Q)
    np.add.at(Hval, pat.edge_pos.ravel(), B[:, _LOW_A, _LOW_B].ravel())
    neg = np.maximum(0.0, -lam.min(axis=1))                 # (E,)
    ev = np.concatenate([4 * pat.edges[:, :1] + np.arange(4)[None, :],
                         4 * pat.edges[:, 1:] + np.arange(4)[None, :]], axis=1)
    np.add.at(cert, ev.ravel(), np.repeat(neg, 8))
    return Hval, cert


def certified_delta(Sigma: np.ndarray, cert: np.ndarray) -> float:
    """Smallest delta in {0} U {10^k} with min_i(Sigma_i + delta - cert_i) > 0."""
    slack = float(np.min(Sigma - cert))
    if slack > 0:
        return 0.0
    k = int(np.floor(np.log10(-slack)))
    while not np.all(Sigma + 10.0 ** k - cert > 0):
        k += 1
    return float(10.0 ** k)


@dataclasses.dataclass
class KKTInstance:
    """One NCL KKT system: pattern + values + right-hand sides."""

    pat: GridPattern
    form: str              # "stabilized" (K2r) or "condensed" (K1)
    H_val: np.ndarray
    J_val: np.ndarray
    Sigma: np.ndarray
    delta: float
    rho: float
    b: np.ndarray          # (dim, nrhs) column-major right-hand sides
    sigma0: np.ndarray | None = None

    @property
    def n(self) -> int:
        return self.pat.n

    @property
    def m(self) -> int:
        return self.pat.m

    @property
    def dim(self) -> int:
        return self.pat.n + (self.pat.m if self.form == "stabilized" else 0)


def draw_instance(pat: GridPattern, rng: np.random.Generator, *, form: str, rho: float,
                  nrhs: int = 1, sigma0: np.ndarray | None = None) -> KKTInstance:
    """Draw H, J, Sigma, delta and b on a fixed pattern.

    With ``sigma0`` given (a Newton-step redraw), Sigma = sigma0 * U[0.5, 2].
    """
    Hval, cert = draw_H(pat, rng)
    Jval = rng.standard_normal(pat.nnz_J)
    if sigma0 is None:
        Sigma = 10.0 ** rng.uniform(-2.0, 2.0, size=pat.n)
    else:
        Sigma = sigma0 * rng.uniform(0.5, 2.0, size=pat.n)
    delta = certified_delta(Sigma, cert)
    dim = pat.n + (pat.m if form == "stabilized" else 0)
    b = rng.standard_normal((nrhs, dim)).T.copy(order="F")
    return KKTInstance(pat=pat, form=form, H_val=Hval, J_val=Jval, Sigma=Sigma,
                       delta=delta, rho=float(rho), b=b,
                       sigma0=Sigma if sigma0 is None else sigma0)


# --------------------------------------------------------------------------
# The five workloads (grid sizes, forms, penalties, batch shapes)
# --------------------------------------------------------------------------

def stabilized_20x25(draw: int = 0) -> KKTInstance:
    """20x25 grid, K2r, rho = 1e4, 1 RHS (n=2000, m=1000)."""
    rng = np.random.Generator(np.random.PCG64(seed_for(1, draw)))
    return draw_instance(make_pattern(20, 25), rng, form="stabilized", rho=1e4)


def condensed_grid(side: int = 300, rho: float = 1e5, draw: int = 0,
                   pat: GridPattern | None = None, sigma0: np.ndarray | None = None) -> KKTInstance:
    """Condensed K = H + Sigma + delta I + rho J^T J on a side x side grid.

    ``draw`` 0 draws Sigma fresh; later draws jitter it by U[0.5, 2] (fixed
    pattern, values re-drawn, as successive Newton steps do).
    """
    rng = np.random.Generator(np.random.PCG64(seed_for(2, draw)))
    pat = pat if pat is not None else make_pattern(side, side)
    return draw_instance(pat, rng, form="condensed", rho=rho, sigma0=sigma0)


def scenario_batch(count: int = 64, side: int = 100, nrhs: int = 4, draw: int = 0):
    """``count`` K2r instances of a side x side grid, each with 1-3 edges deleted."""
    rng = np.random.Generator(np.random.PCG64(seed_for(3, draw)))
    E = len(grid_edges(side, side))
    out = []
    for _ in range(count):
        k = int(rng.integers(1, 4))
        dele = rng.choice(E, size=k, replace=False)
        pat = make_pattern(side, side, np.sort(dele))
        out.append(draw_instance(pat, rng, form="stabilized", rho=1e4, nrhs=nrhs))
    return out


def adjoint_sides(count: int = 256, lo: int = 10, hi: int = 70, seed: int | None = None):
    sides = np.array([lo + int(round((hi - lo) * i / max(count - 1, 1))) for i in range(count)])
    rng = np.random.Generator(np.random.PCG64(seed_for(4, 0) if seed is None else seed))
    rng.shuffle(sides)
    return sides


def adjoint_batch(count: int = 256, lo: int = 10, hi: int = 70, draw: int = 0):
    """K2r instances on grids of side 10..70 (uneven sizes), rho = 1e4."""
    sides = adjoint_sides(count, lo, hi)
    rng = np.random.Generator(np.random.PCG64(seed_for(4, draw) + 1))
    pats = {}
    out = []
    for s in sides:
        s = int(s)
        if s not in pats:
            pats[s] = make_pattern(s, s)
        out.append(draw_instance(pats[s], rng, form="stabilized", rho=1e4))
    return out


def large_stabilized(side: int = 700, rho: float = 1e6, draw: int = 0,
                     pat: GridPattern | None = None) -> KKTInstance:
    """K2r on a side x side grid (700 -> n = 1.96M, m = 0.98M), rho = 1e6."""
    rng = np.random.Generator(np.random.PCG64(seed_for(5, draw)))
    pat = pat if pat is not None else make_pattern(side, side)
    return draw_instance(pat, rng, form="stabilized", rho=rho)


def random_instance(R: int, C: int, seed: int, *, form: str = "stabilized", rho: float = 1e4,
                    nrhs: int = 1) -> KKTInstance:
    rng = np.random.Generator(np.random.PCG64(seed))
    return draw_instance(make_pattern(R, C), rng, form=form, rho=rho, nrhs=nrhs)
