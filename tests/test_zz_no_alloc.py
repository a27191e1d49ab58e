"""The solve entry point that allocates no device memory.

It is meant for callers that cannot allocate at the point where they solve
(a stream being captured into a CUDA graph, real-time loops, a device whose
memory is committed elsewhere).  It runs the regular solve on a fixed static
device workspace, so its results must match ncl_kkt_solve's, call after
call, and problems too large for that workspace must be refused.
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_05885_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda:0")


@pytest.mark.parametrize("prec,eta_tol", [("fp64", 1e-12), ("fp32_ir", 1e-10)])
def test_noalloc_solve_matches_solve(prec, eta_tol):
    from paper_2510_05885_gb300 import ncl_kkt as nk
    inst = synth.random_instance(20, 25, seed=77, form="stabilized", rho=1e4, nrhs=3)
    p = inst.pat
    K = nk.KKT(0, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec=prec)
    K.factor(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), inst.delta, inst.rho)
    Bc = _t(inst.b.T.copy())                      # column-major dim x nrhs
    X_ref = torch.empty_like(Bc)
    nk.ncl_kkt_solve(K._h, 3, Bc, K.dim, X_ref, K.dim)
    ref = X_ref.cpu().numpy().T
    A = O.instance_matrix(inst)
    for _ in range(2):                             # two calls in a row share the scratch
        X = torch.full_like(Bc, float("nan"))
        info = nk.ncl_kkt_solve_noalloc(K._h, 3, Bc, K.dim, X, K.dim)
        got = X.cpu().numpy().T
        assert info.status == 0
        assert info.backward_err <= eta_tol
        assert O.backward_error(A, got, inst.b) <= eta_tol
        assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
    K.close()


def test_noalloc_solve_rejects_oversized_problem():
    from paper_2510_05885_gb300 import ncl_kkt as nk
    pat = synth.make_pattern(150, 150)
    inst = synth.condensed_grid(150, rho=1e4, draw=0, pat=pat)
    K = nk.KKT(1, pat.n, pat.m, pat.H_rowptr, pat.H_colind, pat.J_rowptr, pat.J_colind, prec="fp32_ir")
    K.factor(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), inst.delta, inst.rho)
    B = _t(np.tile(inst.b, (1, 8)).T.copy())
    X = torch.empty_like(B)
    with pytest.raises(nk.NclError) as e:
        nk.ncl_kkt_solve_noalloc(K._h, 8, B, K.dim, X, K.dim)
    assert e.value.status == 1 and "too large" in str(e.value)
    K.close()
