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
