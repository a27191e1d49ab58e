"""Plain FP64 CPU oracle for the NCL KKT systems (test infrastructure only).

What it computes, and where the paper defines it:

* ``kkt_stabilized``: the stabilized system K2r of Section 3.2,
  ``[[H + Sigma + delta I, J^T], [J, -rho^{-1} I]]`` (Eq. K2r; the caller's
  scalar ``rho`` plays the role of the paper's rho-hat = rho + delta).
* ``kkt_condensed``: the condensed system of Section 3.3,
  ``K = H + Sigma + delta I + rho J^T J`` (Eq. K1).
* ``LDLT``: the LDL^T factorisation with D diagonal and static pivoting of
  Section 3.1 ("Sparse LDL^T factorization") with the zero-pivot policy of
  the same paragraph (replace a null pivot by +-eps, sign by the block of the
  index before reordering; eps = 1e-10 as in Section 4.3), computed by the
  simplicial up-looking algorithm in ``ldlt_oracle.c``.
* inertia from the signs of D (Section 3.4, Proposition on the inertia).
* ``solve_ir``: Richardson iterative refinement in FP64 (Section 4.3).
* ``backward_error``: the normwise backward error
  ``||b - K x||_inf / (||K||_inf ||x||_inf + ||b||_inf)``.
* ``kkt_condensed_slack``: the condensed system with slacks of Section 3.3
  (Eq. K1s), ``H + Sigma_t + delta I + rho J_E^T J_E + rho J_I^T Omega J_I``,
  ``Omega = Sigma_s (rho + Sigma_s)^{-1}``; rows with ``Sigma_s = +inf`` are
  the equality rows E, the others the inequality rows I.
  ``k1s_slack_step``: the eliminated slack step of the proposition's proof,
  ``Delta s = (Sigma_s + rho I)^{-1} (rho J_I Delta t + r_s)`` (0 on E rows);
  ``k1s_rhs``: the right-hand side that elimination produces,
  ``r_t + rho J_I^T (Sigma_s + rho I)^{-1} r_s`` (the statement of Eq. K1s
  prints it without the inverse; the proof's own steps give it with).
* ``newton_rhs`` / ``newton_recover``: the Newton step of Algorithm NCL
  around the factored system: the right-hand side of Eq. K2r (unknown
  ``[Delta x; -Delta y]``) or Eq. K1 (unknown ``Delta x``), and Delta y,
  Delta r (Eq. K2 elimination), Delta z_l, Delta z_u (eliminated from
  Eq. K3), Section 3.1-3.3.
* ``regularize``: the inertia correction of Section 3.1 (regularised matrix
  Eq. K2): raise the primal regularisation delta until the inertia is the
  regular one, with rho-hat = rho + delta in the matrix as the same section
  defines it; the growth schedule is the caller's (the paper fixes none).
* ``adjoint``: gradients of a loss of ``x = K^{-1} b`` with respect to b and
  to the stored values of H, J, Sigma (and delta, rho): ``g_b = K^{-1} g_x``
  and ``dl/dK = -g_b x^T`` folded onto the stored pattern.

The ordering is reverse Cuthill-McKee from scipy (a library routine), or a
caller-given permutation; any symmetric permutation of an SQD matrix has an
LDL^T factorisation (Section 3.2, citing Vanderbei), so results are compared
on the solution and the inertia, never on the factors.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig
import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import reverse_cuthill_mckee

__all__ = [
    "build_oracle", "kkt_stabilized", "kkt_condensed", "instance_matrix", "block_signs",
    "LDLT", "solve_ir", "backward_error", "solve_instance", "adjoint", "cond1_estimate", "regularize",
    "kkt_condensed_slack", "k1s_slack_step", "k1s_rhs", "newton_rhs", "newton_recover",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ldlt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libldlt_oracle.so")
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile ``ldlt_oracle.c`` into ``oracle/_build/libldlt_oracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        P = ctypes.c_void_p
        lib.oracle_ldl_symbolic.argtypes = [ctypes.c_int64, P, P, P, P, P]
        lib.oracle_ldl_symbolic.restype = None
        lib.oracle_ldl_numeric.argtypes = [ctypes.c_int64, P, P, P, P, P, P, ctypes.c_double,
                                           ctypes.c_int, P, P, P, P, P, P, P, P]
        lib.oracle_ldl_numeric.restype = ctypes.c_int
        lib.oracle_ldl_solve.argtypes = [ctypes.c_int64, P, P, P, P, P, P]
        lib.oracle_ldl_solve.restype = None
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# Matrices from their definitions
# ---------------------------------------------------------------------------

def _H_full(n, H_rowptr, H_colind, H_val):
    """Symmetric H from its lower-triangle CSR (each off-diagonal value
    stands for both (i,j) and (j,i))."""
    Hl = sp.csr_matrix((np.asarray(H_val, float), np.asarray(H_colind), np.asarray(H_rowptr)),
                       shape=(n, n))
    return Hl + sp.tril(Hl, k=-1).T


def kkt_stabilized(n, m, H_rowptr, H_colind, H_val, J_rowptr, J_colind, J_val,
                   Sigma, delta, rho) -> sp.csc_matrix:
    """K2r = [[H + Sigma + delta I, J^T], [J, -I/rho]]  (Section 3.2, Eq. K2r)."""
    H = _H_full(n, H_rowptr, H_colind, H_val)
    J = sp.csr_matrix((np.asarray(J_val, float), np.asarray(J_colind), np.asarray(J_rowptr)),
                      shape=(m, n))
    top = H + sp.diags(np.asarray(Sigma, float) + delta)
    K = sp.bmat([[top, J.T], [J, sp.diags(np.full(m, -1.0 / rho))]], format="csc")
    return K


def kkt_condensed(n, m, H_rowptr, H_colind, H_val, J_rowptr, J_colind, J_val,
                  Sigma, delta, rho) -> sp.csc_matrix:
    """K = H + Sigma + delta I + rho J^T J  (Section 3.3, Eq. K1)."""
    H = _H_full(n, H_rowptr, H_colind, H_val)
    J = sp.csr_matrix((np.asarray(J_val, float), np.asarray(J_colind), np.asarray(J_rowptr)),
                      shape=(m, n))
    K = H + sp.diags(np.asarray(Sigma, float) + delta) + rho * (J.T @ J)
    return sp.csc_matrix(K)


def kkt_condensed_slack(n, m, H_rowptr, H_colind, H_val, J_rowptr, J_colind, J_val,
                        Sigma_t, Sigma_s, delta, rho) -> sp.csc_matrix:
    """K1s = H + Sigma_t + delta I + rho J_E^T J_E + rho J_I^T Omega J_I
    (Section 3.3, Eq. K1s), Omega = Sigma_s / (rho + Sigma_s) on the rows
    with a finite Sigma_s (I), the rows with Sigma_s = +inf forming E."""
    H = _H_full(n, H_rowptr, H_colind, H_val)
    J = sp.csr_matrix((np.asarray(J_val, float), np.asarray(J_colind), np.asarray(J_rowptr)),
                      shape=(m, n))
    Ss = np.asarray(Sigma_s, float)
    eq = np.isposinf(Ss)
    JE, JI = J[np.flatnonzero(eq)], J[np.flatnonzero(~eq)]
    omega = Ss[~eq] / (rho + Ss[~eq])
    K = (H + sp.diags(np.asarray(Sigma_t, float) + delta) + rho * (JE.T @ JE)
         + rho * (JI.T @ sp.diags(omega) @ JI))
    return sp.csc_matrix(K)


def k1s_slack_step(m, J_rowptr, J_colind, J_val, n, Sigma_s, rho, dt, rs) -> np.ndarray:
    """Delta s = (Sigma_s + rho I)^{-1} (rho J_I Delta t + r_s) on the rows
    with a finite Sigma_s, 0 on the others (proof of the proposition on
    Eq. K1s, Section 3.3)."""
    J = sp.csr_matrix((np.asarray(J_val, float), np.asarray(J_colind), np.asarray(J_rowptr)),
                      shape=(m, n))
    Ss = np.asarray(Sigma_s, float)
    dt = np.asarray(dt, float).reshape(n, -1)
    rs = np.asarray(rs, float).reshape(m, -1)
    ds = np.zeros_like(rs)
    I = np.flatnonzero(~np.isposinf(Ss))
    ds[I] = (rho * (J[I] @ dt) + rs[I]) / (Ss[I] + rho)[:, None]
    return ds


def k1s_rhs(m, J_rowptr, J_colind, J_val, n, Sigma_s, rho, rt, rs) -> np.ndarray:
    """r_t + rho J_I^T (Sigma_s + rho I)^{-1} r_s: eliminating Delta s from the
    second block row of Eq. K1' (Section 3.3) and moving it to the right."""
    J = sp.csr_matrix((np.asarray(J_val, float), np.asarray(J_colind), np.asarray(J_rowptr)),
                      shape=(m, n))
    Ss = np.asarray(Sigma_s, float)
    rt = np.asarray(rt, float).reshape(n, -1)
    rs = np.asarray(rs, float).reshape(m, -1)
    I = np.flatnonzero(~np.isposinf(Ss))
    return rt + rho * (J[I].T @ (rs[I] / (Ss[I] + rho)[:, None]))


def _J(m, n, J_rowptr, J_colind, J_val):
    return sp.csr_matrix((np.asarray(J_val, float), np.asarray(J_colind), np.asarray(J_rowptr)), shape=(m, n))


def newton_rhs(form, n, m, J_rowptr, J_colind, J_val, pt, mu, rho) -> np.ndarray:
    """Right-hand side of the factored Newton system (Section 3.2, Eq. K2r;
    Section 3.3, Eq. K1).  ``pt``: dict of numpy arrays grad_phi, x, lower,
    upper (+-inf allowed), c, y, y_k; ``rho`` is the matrix's rho-hat."""
    J = _J(m, n, J_rowptr, J_colind, J_val)
    x, lo, up = pt["x"], pt["lower"], pt["upper"]
    barrier = -mu / (x - lo) + mu / (up - x)          # -(X-L)^{-1} mu e + (U-X)^{-1} mu e
    if form == "stabilized":
        top = -(pt["grad_phi"] - J.T @ pt["y"] + barrier)
        bot = -(pt["c"] - (pt["y_k"] - pt["y"]) / rho)
        return np.concatenate([top, bot])
    return J.T @ (pt["y_k"] - rho * pt["c"]) - (pt["grad_phi"] + barrier)


def newton_recover(form, n, m, J_rowptr, J_colind, J_val, pt, mu, rho, X) -> dict:
    """The Newton direction from the solution X of the factored system:
    Delta y (dual block of Eq. K2r with its sign, or Eq. K1's elimination
    -rho (J Delta x + c) + y_k - y), Delta r = (Delta y - y_k + y)/rho - r
    (Eq. K2 elimination), and the bound multipliers eliminated from Eq. K3."""
    J = _J(m, n, J_rowptr, J_colind, J_val)
    X = np.asarray(X, float)
    dx = X[:n].copy()
    if form == "stabilized":
        dy = -X[n:n + m]
    else:
        dy = -rho * (J @ dx + pt["c"]) + pt["y_k"] - pt["y"]
    dr = (dy - pt["y_k"] + pt["y"]) / rho - pt["r"]
    x, lo, up, zl, zu = pt["x"], pt["lower"], pt["upper"], pt["z_lower"], pt["z_upper"]
    dzl = -(zl * dx - mu) / (x - lo) - zl
    dzu = (zu * dx + mu) / (up - x) - zu
    return {"dx": dx, "dy": dy, "dr": dr, "dz_lower": dzl, "dz_upper": dzu}


def instance_matrix(inst) -> sp.csc_matrix:
    p = inst.pat
    f = kkt_stabilized if inst.form == "stabilized" else kkt_condensed
    return f(p.n, p.m, p.H_rowptr, p.H_colind, inst.H_val, p.J_rowptr, p.J_colind,
             inst.J_val, inst.Sigma, inst.delta, inst.rho)


def block_signs(form: str, n: int, m: int) -> np.ndarray:
    """+1 for a primal index, -1 for a dual one (K2r); all +1 for K."""
    if form == "stabilized":
        return np.concatenate([np.ones(n, np.int32), -np.ones(m, np.int32)])
    return np.ones(n, np.int32)


# ---------------------------------------------------------------------------
# LDL^T
# ---------------------------------------------------------------------------

class LDLT:
    """FP64 LDL^T of a symmetric matrix ``A`` under the permutation ``perm``
    (new index -> old index), static pivoting with the +-eps policy."""

    def __init__(self, A, sign=None, perm=None, eps: float = 1e-10, policy: int = 0,
                 ordering: str = "rcm"):
        A = sp.csc_matrix(A)
        N = A.shape[0]
        self.N = N
        if perm is None:
            if ordering == "rcm":
                perm = np.asarray(reverse_cuthill_mckee(sp.csr_matrix(A), symmetric_mode=True),
                                  dtype=np.int64)
            else:
                perm = np.arange(N, dtype=np.int64)
        self.perm = np.asarray(perm, dtype=np.int64)
        sign = np.ones(N, np.int32) if sign is None else np.asarray(sign, np.int32)
        self.sign_perm = np.ascontiguousarray(sign[self.perm], dtype=np.int32)
        B = A[self.perm][:, self.perm]
        U = sp.triu(B, format="csc")
        U.sort_indices()
        Ap = U.indptr.astype(np.int64)
        Ai = U.indices.astype(np.int64)
        Ax = U.data.astype(np.float64)
        lib = _load()
        parent = np.empty(N, np.int64)
        Lnz = np.empty(N, np.int64)
        flag = np.empty(N, np.int64)
        lib.oracle_ldl_symbolic(N, _p(Ap), _p(Ai), _p(parent), _p(Lnz), _p(flag))
        Lp = np.zeros(N + 1, np.int64)
        Lp[1:] = np.cumsum(Lnz)
        nnzL = int(Lp[-1])
        Li = np.empty(max(nnzL, 1), np.int64)
        Lx = np.empty(max(nnzL, 1), np.float64)
        D = np.empty(N, np.float64)
        Y = np.zeros(N, np.float64)
        pattern = np.empty(N, np.int64)
        counts = np.zeros(4, np.int64)
        rc = lib.oracle_ldl_numeric(N, _p(Ap), _p(Ai), _p(Ax), _p(Lp), _p(parent),
                                    _p(self.sign_perm), float(eps), int(policy), _p(Lnz), _p(Li),
                                    _p(Lx), _p(D), _p(Y), _p(pattern), _p(flag), _p(counts))
        self.ok = rc == 0
        self.parent, self.Lp, self.Lnz, self.Li, self.Lx, self.D = parent, Lp, Lnz, Li, Lx, D
        self.nnz_L = nnzL
        self.n_pos, self.n_neg, self.n_zero, self.n_perturbed = (int(c) for c in counts)
        # algorithmic flops: sum_j (c_j^2 + 3 c_j), c_j = strictly-lower count of column j
        c = Lnz.astype(np.float64)
        self.flops = float(np.sum(c * c + 3.0 * c))

    @property
    def inertia(self):
        return (self.n_pos, self.n_neg, self.n_zero)

    def L(self) -> sp.csc_matrix:
        """Unit lower-triangular factor (permuted numbering)."""
        N = self.N
        nnz = self.nnz_L
        rows = self.Li[:nnz]
        cols = np.repeat(np.arange(N), self.Lnz)
        Lm = sp.csc_matrix((self.Lx[:nnz], (rows, cols)), shape=(N, N))
        return Lm + sp.identity(N, format="csc")

    def solve(self, b: np.ndarray) -> np.ndarray:
        b = np.asarray(b, dtype=np.float64)
        one = b.ndim == 1
        B = b.reshape(self.N, -1)
        X = np.empty_like(B)
        lib = _load()
        for j in range(B.shape[1]):
            w = np.ascontiguousarray(B[self.perm, j])
            lib.oracle_ldl_solve(self.N, _p(self.Lp), _p(self.Lnz), _p(self.Li), _p(self.Lx),
                                 _p(self.D), _p(w))
            X[self.perm, j] = w
        return X[:, 0] if one else X


def backward_error(A, x: np.ndarray, b: np.ndarray) -> float:
    """Normwise backward error ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf),
    the largest over right-hand-side columns."""
    A = sp.csr_matrix(A)
    X = np.asarray(x, float).reshape(A.shape[0], -1)
    Bm = np.asarray(b, float).reshape(A.shape[0], -1)
    nA = float(np.max(np.abs(A).sum(axis=1))) if A.nnz else 0.0
    eta = 0.0
    for j in range(X.shape[1]):
        r = Bm[:, j] - A @ X[:, j]
        den = nA * np.max(np.abs(X[:, j]), initial=0.0) + np.max(np.abs(Bm[:, j]), initial=0.0)
        eta = max(eta, float(np.max(np.abs(r), initial=0.0) / den) if den > 0 else 0.0)
    return eta


def solve_ir(A, fac: LDLT, b: np.ndarray, max_steps: int = 3, tol: float = 0.0):
    """x = fac.solve(b) followed by up to ``max_steps`` FP64 Richardson steps
    x += fac.solve(b - A x) (Section 4.3).  Returns (x, steps taken, eta)."""
    A = sp.csr_matrix(A)
    x = fac.solve(b)
    steps = 0
    eta = backward_error(A, x, b)
    while steps < max_steps and eta > tol:
        r = np.asarray(b, float).reshape(x.shape) - (A @ x.reshape(A.shape[0], -1)).reshape(x.shape)
        x = x + fac.solve(r)
        steps += 1
        eta = backward_error(A, x, b)
    return x, steps, eta


def solve_instance(inst, ir_steps: int = 3, eps: float = 1e-10, policy: int = 0, perm=None):
    """Assemble, factor, solve with FP64 IR.  Returns (x, fac, eta, A)."""
    A = instance_matrix(inst)
    fac = LDLT(A, block_signs(inst.form, inst.n, inst.m), perm=perm, eps=eps, policy=policy)
    x, _, eta = solve_ir(A, fac, inst.b, max_steps=ir_steps)
    return x, fac, eta, A


def regularize(inst, delta0: float = 0.0, delta_first: float = 1e-4, growth: float = 10.0, max_tries: int = 20,
               eps: float = 1e-10, policy: int = 0, perm=None):
    """Inertia correction of Section 3.1.  ``inst.rho`` is the unregularised
    penalty rho_k; each try factors the matrix with delta and rho-hat =
    rho_k + delta (Section 3.1, the definition of rho-hat after Eq. K2), and
    while the inertia is not (n, m, 0) for K2r or (n, 0, 0) for K
    (Section 3.1: the inertia a valid search direction needs), delta is
    raised: to ``delta_first`` from zero, else multiplied by ``growth``.
    Returns (fac, A, delta, tries, regular) of the last try."""
    p = inst.pat
    want = (inst.n, inst.m if inst.form == "stabilized" else 0, 0)
    build = kkt_stabilized if inst.form == "stabilized" else kkt_condensed
    sign = block_signs(inst.form, inst.n, inst.m)
    delta = float(delta0)
    t = 0
    while True:
        t += 1
        A = build(p.n, p.m, p.H_rowptr, p.H_colind, inst.H_val, p.J_rowptr, p.J_colind, inst.J_val,
                  inst.Sigma, delta, inst.rho + delta)
        fac = LDLT(A, sign, perm=perm, eps=eps, policy=policy)
        if fac.inertia == want:
            return fac, A, delta, t, True
        if t >= max_tries:
            return fac, A, delta, t, False
        delta = delta * growth if delta > 0 else delta_first


def cond1_estimate(A, fac: LDLT) -> float:
    """kappa_1(A) = ||A||_1 ||A^{-1}||_1 with ||A^{-1}||_1 estimated by
    scipy's onenormest applying A^{-1} through the oracle factors."""
    from scipy.sparse.linalg import LinearOperator, onenormest
    N = A.shape[0]
    op = LinearOperator((N, N), matvec=lambda v: fac.solve(np.asarray(v, float).ravel()),
                        rmatvec=lambda v: fac.solve(np.asarray(v, float).ravel()), dtype=float)
    nA = float(np.max(np.abs(sp.csc_matrix(A)).sum(axis=0)))
    return nA * float(onenormest(op))


# ---------------------------------------------------------------------------
# Adjoint
# ---------------------------------------------------------------------------

def adjoint(inst, fac: LDLT, A, x: np.ndarray, gx: np.ndarray, ir_steps: int = 3) -> dict:
    """Gradients of a loss l(x), x = K^{-1} b, given g_x = dl/dx.

    g_b = K^{-1} g_x (K symmetric); dl/dK = -g_b x^T, folded onto the stored
    values: an off-diagonal lower H value stands for (i,j) and (j,i).
    For several right-hand sides the contributions of the columns add up.
    """
    p = inst.pat
    n, m = p.n, p.m
    X = np.asarray(x, float).reshape(A.shape[0], -1)
    GX = np.asarray(gx, float).reshape(A.shape[0], -1)
    GB, _, _ = solve_ir(A, fac, GX, max_steps=ir_steps)
    GB = GB.reshape(X.shape)
    rows = np.repeat(np.arange(n), np.diff(p.H_rowptr))
    cols = p.H_colind.astype(np.int64)
    Jrows = np.repeat(np.arange(m), np.diff(p.J_rowptr))
    Jcols = p.J_colind.astype(np.int64)
    gH = np.zeros(p.nnz_H)
    gJ = np.zeros(p.nnz_J)
    gS = np.zeros(n)
    gdelta = 0.0
    grho = 0.0
    for k in range(X.shape[1]):
        g, xx = GB[:, k], X[:, k]
        off = rows != cols
        gH += -(g[rows] * xx[cols] + np.where(off, g[cols] * xx[rows], 0.0))
        gS += -(g[:n] * xx[:n])
        gdelta += -float(np.dot(g[:n], xx[:n]))
        if inst.form == "stabilized":
            gJ += -(g[n + Jrows] * xx[Jcols] + g[Jcols] * xx[n + Jrows])
            grho += -float(np.dot(g[n:], xx[n:])) / inst.rho ** 2   # d(-1/rho)/drho = 1/rho^2
        else:
            J = sp.csr_matrix((inst.J_val, p.J_colind, p.J_rowptr), shape=(m, n))
            Jx = J @ xx
            Jg = J @ g
            gJ += -inst.rho * (Jg[Jrows] * xx[Jcols] + Jx[Jrows] * g[Jcols])
            grho += -float(np.dot(Jg, Jx))
    return {"g_b": GB if np.asarray(gx).ndim > 1 else GB[:, 0], "g_H": gH, "g_J": gJ,
            "g_Sigma": gS, "g_delta": gdelta, "g_rho": grho}
