"""Small shared helpers for the tests (no method arithmetic here)."""
from __future__ import annotations

import types

import numpy as np
import scipy.sparse as sp

from paper_2510_05885_gb300 import synth


def lower_csr(M):
    """Lower triangle (with the full diagonal kept structurally) as CSR arrays."""
    M = sp.csr_matrix(M)
    n = M.shape[0]
    L = sp.tril(M, format="coo")
    rows = np.concatenate([L.row, np.arange(n)])
    cols = np.concatenate([L.col, np.arange(n)])
    vals = np.concatenate([L.data, np.zeros(n)])
    C = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    C.sum_duplicates()
    C.sort_indices()
    return C.indptr.astype(np.int32), C.indices.astype(np.int32), C.data.astype(float)


def custom_instance(H, J, Sigma, delta, rho, b, form="stabilized"):
    """A KKTInstance-like object from explicit H (n x n, symmetric), J (m x n)."""
    H = sp.csr_matrix(H)
    J = sp.csr_matrix(J)
    n = H.shape[0]
    m = J.shape[0]
    Hp, Hi, Hv = lower_csr(H)
    J.sort_indices()
    pat = types.SimpleNamespace(n=n, m=m, H_rowptr=Hp, H_colind=Hi,
                                J_rowptr=J.indptr.astype(np.int32), J_colind=J.indices.astype(np.int32),
                                nnz_H=int(Hp[-1]), nnz_J=int(J.indptr[-1]))
    dim = n + (m if form == "stabilized" else 0)
    b = np.asarray(b, float).reshape(dim, -1)
    return synth.KKTInstance(pat=pat, form=form, H_val=Hv, J_val=J.data.astype(float),
                             Sigma=np.asarray(Sigma, float), delta=float(delta), rho=float(rho), b=b)


def read_golden(path):
    out = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            out[k] = [float(t) for t in v]
    return out


def newton_point(inst, seed, frac_unbounded=0.3):
    """A seeded interior point of the instance's NCL subproblem (Section 3.1):
    bounds around x (some infinite, with zero multipliers there), positive
    multipliers, and the Sigma = (X-L)^{-1} Z_l + (U-X)^{-1} Z_u they imply.
    Returns (point dict of numpy arrays, Sigma)."""
    rng = np.random.default_rng(seed)
    n, m = inst.n, inst.m
    x = rng.standard_normal(n)
    lo = x - rng.uniform(0.1, 2.0, n)
    up = x + rng.uniform(0.1, 2.0, n)
    lo[rng.random(n) < frac_unbounded] = -np.inf
    up[rng.random(n) < frac_unbounded] = np.inf
    zl = np.where(np.isinf(lo), 0.0, rng.uniform(0.01, 1.0, n))
    zu = np.where(np.isinf(up), 0.0, rng.uniform(0.01, 1.0, n))
    pt = {"grad_phi": rng.standard_normal(n), "x": x, "lower": lo, "upper": up, "z_lower": zl, "z_upper": zu,
          "c": rng.standard_normal(m), "y": rng.standard_normal(m), "y_k": rng.standard_normal(m),
          "r": rng.standard_normal(m)}
    sigma = zl / (x - lo) + zu / (up - x)
    return pt, sigma
