"""The solve entry point that allocates no memory.

It is meant for callers that cannot allocate at the point where they solve
(real-time loops that cannot afford an allocator round trip, a device whose
memory is committed elsewhere).  It runs the regular solve, FGMRES stage
included, on a fixed static device workspace, so its results must match
ncl_kkt_solve's, call after call, the handle's device memory must not grow,
problems too large for that workspace must be refused, and a stream under
graph capture must be refused (the refinement reads norms back between
steps).
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_05885_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda:0")


def _device_bytes(K):
    from paper_2510_05885_gb300 import ncl_kkt as nk
    return nk.ncl_kkt_get_analysis_info(K._h).device_bytes


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
    held = _device_bytes(K)
    for _ in range(2):                             # two calls in a row share the scratch
        X = torch.full_like(Bc, float("nan"))
        info = nk.ncl_kkt_solve_noalloc(K._h, 3, Bc, K.dim, X, K.dim)
        got = X.cpu().numpy().T
        assert info.status == 0
        assert info.backward_err <= eta_tol
        assert O.backward_error(A, got, inst.b) <= eta_tol
        assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
    assert _device_bytes(K) == held
    K.close()


def test_noalloc_fgmres_stage_allocates_nothing():
    """rho = 1e7 on the condensed 24 x 24 grid with the precision fallback
    off: Richardson refinement of the FP32 factors stagnates and the FGMRES
    stage runs.  Its Krylov vectors come from the static array: the handle
    (which has never run FGMRES before) holds no more device memory after
    two calls, and the result equals that of the regular solve, which
    allocates the same vectors in the handle on its first FGMRES use."""
    from paper_2510_05885_gb300 import ncl_kkt as nk
    inst = synth.condensed_grid(24, rho=1e7, draw=0)
    p = inst.pat
    K = nk.KKT(1, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec="fp32_ir", precision_fallback=0)
    K.factor(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), inst.delta, inst.rho)
    Bc = _t(inst.b.T.copy())
    A = O.instance_matrix(inst)
    held = _device_bytes(K)
    outs = []
    for _ in range(2):
        X = torch.full_like(Bc, float("nan"))
        info = nk.ncl_kkt_solve_noalloc(K._h, 1, Bc, K.dim, X, K.dim)
        assert info.status == 0 and info.used_fgmres == 1
        got = X.cpu().numpy().T
        assert O.backward_error(A, got, inst.b) <= 1e-10
        outs.append(got)
    assert _device_bytes(K) == held
    X_ref = torch.empty_like(Bc)
    sref = nk.ncl_kkt_solve(K._h, 1, Bc, K.dim, X_ref, K.dim)
    assert sref.status == 0 and sref.used_fgmres == 1
    assert _device_bytes(K) > held                 # the regular solve allocated its Krylov vectors
    ref = X_ref.cpu().numpy().T
    for got in outs:
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


def test_noalloc_solve_refuses_a_capturing_stream():
    from paper_2510_05885_gb300 import ncl_kkt as nk
    inst = synth.random_instance(6, 7, seed=5, form="stabilized", rho=1e3)
    p = inst.pat
    K = nk.KKT(0, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec="fp64")
    K.factor(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), inst.delta, inst.rho)
    Bc = _t(inst.b.T.copy())
    X = torch.empty_like(Bc)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            nk.ncl_kkt_solve_noalloc(K._h, 1, Bc, K.dim, X, K.dim, stream=s)
        except nk.NclError as e:
            status = e.status
        finally:
            g.capture_end()
    assert status == 5
    info = nk.ncl_kkt_solve_noalloc(K._h, 1, Bc, K.dim, X, K.dim)   # usable afterwards
    assert info.status == 0
    K.close()
