"""Host-side tests of the library (no GPU): the C ABI loads and exports every
declared symbol, pattern errors are reported, and the symbolic analysis
(nested dissection, elimination tree, supernodes) is consistent with the
oracle's own symbolic factorisation under the same permutation.

The permutation is a free choice (any symmetric permutation of an SQD
matrix factors, Section 3.2); given it, the exact nonzero count of L is a
property of the matrix that the oracle computes independently.
"""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2510_05885_gb300 import ncl_kkt as nk
from paper_2510_05885_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "ncl_kkt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ncl_kkt_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = nk.load()
    declared = _declared_functions()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(nk.EXPORTED)


def test_status_strings():
    lib = nk.load()
    for i, name in enumerate(nk.STATUS):
        assert lib.ncl_kkt_status_string(i).decode() == name


def _host(form, pat, **kw):
    opt = nk.default_options(host_only=1, **kw)
    h = nk.ncl_kkt_analyze(form, pat.n, pat.m, pat.H_rowptr, pat.H_colind, pat.J_rowptr, pat.J_colind, opt)
    return h


def _structural(pat, form):
    """All-ones values: every stored entry is nonzero and nothing cancels,
    so the oracle sees the full structural pattern."""
    dim = pat.n + (pat.m if form == "stabilized" else 0)
    return synth.KKTInstance(pat=pat, form=form, H_val=np.ones(pat.nnz_H), J_val=np.ones(pat.nnz_J),
                             Sigma=np.ones(pat.n), delta=0.0, rho=1.0, b=np.ones((dim, 1)))


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (7, 9), (20, 25)])
def test_symbolic_counts_match_oracle(form, shape):
    pat = synth.make_pattern(*shape)
    inst = _structural(pat, "stabilized" if form == 0 else "condensed")
    h = _host(form, pat)
    try:
        ai = nk.ncl_kkt_get_analysis_info(h)
        perm = nk.ncl_kkt_get_permutation(h, ai.dim)
        assert sorted(perm.tolist()) == list(range(ai.dim))
        A = O.instance_matrix(inst)
        assert ai.dim == A.shape[0]
        fac = O.LDLT(A, O.block_signs(inst.form, inst.n, inst.m), perm=perm)
        assert ai.nnz_L == fac.nnz_L
        assert ai.flops == pytest.approx(fac.flops, rel=1e-12)
        import scipy.sparse as sp
        assert ai.nnz_A == sp.tril(A).nnz
        ns = int(ai.n_supernodes)
        col0, parent, nrow = nk.ncl_kkt_get_supernodes(h, ns)
        assert col0[0] == 0 and col0[-1] == ai.dim and np.all(np.diff(col0) > 0)
        for s in range(ns):
            assert parent[s] == -1 or parent[s] > s
            assert nrow[s] >= col0[s + 1] - col0[s]
        # every column's true structure lies inside its supernode's rows:
        # the stored (padded) entries cover nnz(L)
        assert ai.nnz_L_stored >= ai.nnz_L
    finally:
        nk.ncl_kkt_destroy(h)


def test_batch_analysis_is_block_diagonal():
    pats = [synth.make_pattern(3, 4), synth.make_pattern(5, 2), synth.make_pattern(1, 1)]
    opt = nk.default_options(host_only=1)
    h = nk.ncl_kkt_batch_analyze(0, [p.n for p in pats], [p.m for p in pats], [p.H_rowptr for p in pats],
                                 [p.H_colind for p in pats], [p.J_rowptr for p in pats],
                                 [p.J_colind for p in pats], opt)
    try:
        ai = nk.ncl_kkt_get_analysis_info(h)
        assert ai.dim == sum(p.n + p.m for p in pats)
        tot = 0
        for p in pats:
            h1 = _host(0, p)
            tot += nk.ncl_kkt_get_analysis_info(h1).nnz_L
            nk.ncl_kkt_destroy(h1)
        # fill of a block-diagonal matrix is the sum of the blocks' fills
        # (orderings may differ per block, so compare with each block's oracle count)
        perm = nk.ncl_kkt_get_permutation(h, ai.dim)
        offs = np.cumsum([0] + [p.n + p.m for p in pats])
        inst_of = np.searchsorted(offs, perm, side="right") - 1
        nnz = 0
        for i, p in enumerate(pats):
            sub = perm[inst_of == i] - offs[i]
            fac = O.LDLT(O.instance_matrix(_structural(p, "stabilized")), perm=sub)
            nnz += fac.nnz_L
        assert ai.nnz_L == nnz
        assert nk.load().ncl_kkt_instance_count(h) == 3
    finally:
        nk.ncl_kkt_destroy(h)


def _expect_pattern_error(form, n, m, Hp, Hi, Jp, Ji):
    opt = nk.default_options(host_only=1)
    with pytest.raises(nk.NclError) as e:
        nk.ncl_kkt_analyze(form, n, m, Hp, Hi, Jp, Ji, opt)
    assert e.value.status == 2


def test_pattern_errors():
    Hp, Hi = np.array([0, 1, 3]), np.array([0, 0, 1])
    # H entry above the diagonal
    _expect_pattern_error(0, 2, 1, np.array([0, 2, 3]), np.array([0, 1, 1]), np.array([0, 1]), np.array([0]))
    # unsorted J columns
    _expect_pattern_error(0, 2, 1, Hp, Hi, np.array([0, 2]), np.array([1, 0]))
    # J column out of range
    _expect_pattern_error(1, 2, 1, Hp, Hi, np.array([0, 1]), np.array([2]))
    # duplicate H column
    _expect_pattern_error(0, 2, 0, np.array([0, 1, 3]), np.array([0, 1, 1]), np.array([0]), np.array([], np.int32))


def test_invalid_arguments():
    with pytest.raises(nk.NclError) as e:
        nk.ncl_kkt_analyze(5, 1, 0, [0, 1], [0], [0], [], nk.default_options(host_only=1))
    assert e.value.status == 1
    h = _host(0, synth.make_pattern(1, 2))
    try:
        with pytest.raises(nk.NclError) as e:
            nk.ncl_kkt_factor(h, None, None, None, 0.0, 1.0, stream=_FakeStream())
        assert e.value.status == 5   # host-only handle: no numeric state
    finally:
        nk.ncl_kkt_destroy(h)


class _FakeStream:
    cuda_stream = 0


@pytest.mark.slow
def test_analysis_300x300_condensed_fill():
    """The condensed 300x300 workload: fill and flops of our ordering (the
    value is recorded in the design notes; here only sanity bounds)."""
    pat = synth.make_pattern(300, 300)
    h = _host(1, pat)
    try:
        ai = nk.ncl_kkt_get_analysis_info(h)
        assert ai.dim == 360000
        assert ai.nnz_L < 2.0e8 and ai.flops < 3e11
    finally:
        nk.ncl_kkt_destroy(h)


def test_analyze_like_copies_the_analysis():
    """A handle made from another's analysis (other options) has the same
    ordering, supernodes and statistics; the source is not needed afterwards."""
    pat = synth.make_pattern(13, 17)
    src = nk.KKT(1, pat.n, pat.m, pat.H_rowptr, pat.H_colind, pat.J_rowptr, pat.J_colind, host_only=1)
    twin = nk.KKT.like(src, host_only=1, prec="fp64", pivot_policy=1)
    assert np.array_equal(src.permutation, twin.permutation)
    for a, b in zip(src.supernodes(), twin.supernodes()):
        assert np.array_equal(a, b)
    ia, ib = src.analysis.as_dict(), twin.analysis.as_dict()
    ia.pop("analyze_ms")
    ib.pop("analyze_ms")
    assert ia == ib
    src.close()
    assert twin.analysis.dim == pat.n
    twin.close()
    with pytest.raises(nk.NclError):
        nk.ncl_kkt_analyze_like(None, nk.default_options(host_only=1))


def test_next_row_entry_points_check_their_arguments_on_the_host():
    """The entry points of the inertia correction, the slack form and the
    Newton step reject NULL handles and host-only handles before any device
    work (status codes, nothing thrown across the C ABI)."""
    lib = nk.load()
    assert lib.ncl_kkt_factor_regularize(None, None, None, None, None, None, 1e-4, 10.0, 5, None, None, None) == 1
    assert lib.ncl_kkt_factor_k1s(None, None, None, None, None, None, None, None, None) == 1
    assert lib.ncl_kkt_k1s_rhs(None, 1, None, 0, None, 0, None, 0, None) == 1
    assert lib.ncl_kkt_k1s_slack_step(None, 1, None, 0, None, 0, None, 0, None) == 1
    assert lib.ncl_kkt_newton_rhs(None, None, None, None, None) == 1
    assert lib.ncl_kkt_newton_recover(None, None, None, None, None, None, None, None, None, None) == 1
    pat = synth.make_pattern(2, 3)
    for form in (0, 1):
        h = _host(form, pat)
        try:
            d = np.zeros(1)
            r = np.ones(1)
            st = lib.ncl_kkt_factor_regularize(h, None, None, None, d.ctypes.data, r.ctypes.data, 1e-4, 10.0, 5,
                                               None, None, None)
            assert st == 5                                   # host-only: no numeric state
            st = lib.ncl_kkt_factor_k1s(h, None, None, None, None, d.ctypes.data, r.ctypes.data, None, None)
            assert st == 5
            pt = nk.NewtonPoint()
            mu = np.full(1, 0.1)
            assert lib.ncl_kkt_newton_rhs(h, nk.ctypes.byref(pt), mu.ctypes.data, None, None) == 1   # NULL B
            assert lib.ncl_kkt_k1s_slack_step(h, 1, None, 0, None, 0, None, 0, None) == 5
        finally:
            nk.ncl_kkt_destroy(h)


def _csr(rows, n_cols):
    """CSR (rowptr, colind) from a list of sorted column lists."""
    rp = np.zeros(len(rows) + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([c for r in rows for c in r], np.int32)
    return rp, ci


@pytest.mark.parametrize("form", [0, 1])
def test_symbolic_counts_on_degenerate_patterns(form):
    """Patterns outside the grids: empty constraint rows, rows of H without
    a diagonal entry, no constraints at all, and two disconnected parts; the
    library's nnz(L) under its own permutation equals the oracle's."""
    import types
    cases = [
        # n = 5, m = 3 with an empty J row and H rows without diagonal
        ([[0], [], [0, 2], [3], [1, 4]], [[0, 2], [], [3, 4]], 5),
        # no constraints
        ([[0], [0, 1], [2], [1, 3]], [], 4),
        # two disconnected parts (H and J both split)
        ([[0], [0, 1], [2], [2, 3], [4]], [[0, 1], [2, 3], [4]], 5),
        # a single variable, a single constraint
        ([[0]], [[0]], 1),
    ]
    for Hrows, Jrows, n in cases:
        Hp, Hi = _csr(Hrows, n)
        Jp, Ji = _csr(Jrows, n) if Jrows else (np.zeros(1, np.int32), np.zeros(0, np.int32))
        m = len(Jrows)
        pat = types.SimpleNamespace(n=n, m=m, H_rowptr=Hp, H_colind=Hi, J_rowptr=Jp, J_colind=Ji,
                                    nnz_H=int(Hp[-1]), nnz_J=int(Jp[-1]))
        inst = _structural(pat, "stabilized" if form == 0 else "condensed")
        h = _host(form, pat)
        try:
            ai = nk.ncl_kkt_get_analysis_info(h)
            perm = nk.ncl_kkt_get_permutation(h, ai.dim)
            assert sorted(perm.tolist()) == list(range(ai.dim))
            fac = O.LDLT(O.instance_matrix(inst), O.block_signs(inst.form, inst.n, inst.m), perm=perm)
            assert ai.nnz_L == fac.nnz_L
            assert ai.flops == pytest.approx(fac.flops, rel=1e-12)
        finally:
            nk.ncl_kkt_destroy(h)
