"""GPU parity: the CUDA factor/solve (through the C ABI) against the FP64 CPU
oracle on the same seeded inputs.

Tolerances (see the design notes for the derivation):
* FP64 path: backward error eta <= 1e-12 and relative solution error
  <= max(1e-9, 10 kappa u) against the oracle (two backward-stable FP64
  solves differ by about kappa u).
* FP32 + refinement: eta <= 1e-10, solution error <= max(1e-9, 10 kappa 1e-10).
* inertia: exactly (n, m, 0) for K2r and (n, 0, 0) for K (Section 3.4).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_2510_05885_gb300 import synth
from tests.helpers import custom_instance

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def nk():
    from paper_2510_05885_gb300 import ncl_kkt
    return ncl_kkt


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def gpu_solve(inst, prec, **opts):
    p = inst.pat
    form = 0 if inst.form == "stabilized" else 1
    K = nk().KKT(form, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec=prec, **opts)
    finfo = K.factor(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), inst.delta, inst.rho)
    X, sinfo = K.solve(_t(inst.b))
    torch.cuda.synchronize()
    return K, finfo, X.cpu().numpy(), sinfo


def check_against_oracle(inst, prec, X, finfo, sinfo, eta_tol):
    x_o, fac, eta_o, A = O.solve_instance(inst)
    assert eta_o <= 1e-12
    assert finfo.inertia == fac.inertia
    assert finfo.n_perturbed == fac.n_perturbed == 0
    eta = O.backward_error(A, X, inst.b)          # recomputed on the CPU, FP64
    assert eta <= eta_tol, eta
    assert sinfo.backward_err <= eta_tol * 1.0001
    kappa = O.cond1_estimate(A, fac) if A.shape[0] <= 60000 else 1e6
    # two backward-stable solves with backward errors eta_1, eta_2 differ by
    # about kappa (eta_1 + eta_2): FP64 is compared at its achieved backward
    # errors (at least u), FP32 + refinement at its target 1e-10
    u = max(2.0 ** -53, eta + eta_o) if prec == "fp64" else 1e-10
    tol = max(1e-9, 10 * kappa * u)
    err = np.max(np.abs(X - x_o)) / np.max(np.abs(x_o))
    assert err <= tol, (err, tol, kappa)
    return eta, err


@pytest.mark.parametrize("prec,eta_tol", [("fp64", 1e-12), ("fp32_ir", 1e-10)])
def test_stabilized_20x25(prec, eta_tol):
    inst = synth.stabilized_20x25()
    K, finfo, X, sinfo = gpu_solve(inst, prec)
    assert finfo.inertia == (2000, 1000, 0)
    check_against_oracle(inst, prec, X, finfo, sinfo, eta_tol)


@pytest.mark.parametrize("prec,eta_tol", [("fp64", 1e-12), ("fp32_ir", 1e-10)])
@pytest.mark.parametrize("side,rho", [(24, 1e2), (24, 1e5), (30, 1e4)])
def test_condensed_grid(prec, eta_tol, side, rho):
    inst = synth.condensed_grid(side, rho=rho, draw=1, sigma0=None)
    K, finfo, X, sinfo = gpu_solve(inst, prec)
    assert finfo.inertia == (inst.n, 0, 0)
    check_against_oracle(inst, prec, X, finfo, sinfo, eta_tol)


@pytest.mark.parametrize("prec,eta_tol", [("fp64", 1e-12), ("fp32_ir", 1e-10)])
@pytest.mark.parametrize("shape", [(1, 1), (1, 2), (3, 1), (13, 17), (40, 40)])
def test_stabilized_shapes_multi_rhs(prec, eta_tol, shape):
    inst = synth.random_instance(*shape, seed=100 + shape[0], form="stabilized", rho=1e4, nrhs=4)
    K, finfo, X, sinfo = gpu_solve(inst, prec)
    assert finfo.inertia == (inst.n, inst.m, 0)
    check_against_oracle(inst, prec, X, finfo, sinfo, eta_tol)


@pytest.mark.parametrize("nrhs", [9, 17])
def test_many_rhs(nrhs):
    """More right-hand sides than one sweep carries (8)."""
    inst = synth.random_instance(6, 7, seed=3, form="stabilized", rho=1e3, nrhs=nrhs)
    K, finfo, X, sinfo = gpu_solve(inst, "fp64")
    check_against_oracle(inst, "fp64", X, finfo, sinfo, 1e-12)


def test_no_constraints_is_cholesky():
    """m = 0: K2r reduces to H + Sigma + delta I."""
    base = synth.random_instance(5, 5, seed=8, form="stabilized")
    p = base.pat
    Hfull = O.kkt_condensed(p.n, 0, p.H_rowptr, p.H_colind, base.H_val, np.zeros(1, np.int32),
                            np.zeros(0, np.int32), np.zeros(0), np.zeros(p.n), 0.0, 1.0)
    inst = custom_instance(Hfull, sp.csr_matrix((0, p.n)), base.Sigma, base.delta, 1.0,
                           np.random.default_rng(0).standard_normal(p.n))
    K, finfo, X, sinfo = gpu_solve(inst, "fp64")
    assert finfo.inertia == (p.n, 0, 0)
    check_against_oracle(inst, "fp64", X, finfo, sinfo, 1e-12)


def test_zero_pivot_perturbation_and_stop_policy():
    """Both diagonal entries ~0: whichever is eliminated first is a zero pivot
    (Section 3.1); it is replaced by +-eps and refinement recovers x."""
    inst = custom_instance(np.array([[-1.0]]), np.array([[1.0]]), [1.0], 0.0, 1e300, [3.0, -2.0])
    K, finfo, X, sinfo = gpu_solve(inst, "fp64", ir_max_iter=10)
    assert finfo.n_perturbed == 1
    assert finfo.inertia == (1, 1, 0)
    assert np.allclose(X[:, 0], [-2.0, 3.0], rtol=1e-9)
    p = inst.pat
    K2 = nk().KKT(0, 1, 1, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec="fp64", pivot_policy=1)
    info = K2.factor(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), 0.0, 1e300)
    assert info.status == 6 and info.n_zero == 1 and info.n_perturbed == 0


def test_diag_H_identity_J_closed_form():
    from tests.helpers import read_golden
    import os
    gd = read_golden(os.path.join(os.path.dirname(__file__), "golden", "diag_H_identity_J.txt"))
    a = np.array(gd["a"])
    inst = custom_instance(np.diag(a), np.eye(2), np.zeros(2), 0.0, gd["rho"][0],
                           np.concatenate([gd["f"], gd["g"]]))
    for prec in ("fp64", "fp32_ir"):
        K, finfo, X, sinfo = gpu_solve(inst, prec)
        assert finfo.inertia == (2, 2, 0)
        assert np.allclose(X[:2, 0], gd["u"], rtol=1e-12)
        assert np.allclose(X[2:, 0], gd["v"], rtol=1e-12)


def test_refactor_same_pattern_new_values():
    """Analyze once, factor many: values redrawn on the fixed pattern."""
    pat = synth.make_pattern(18, 18)
    form = 1
    K = nk().KKT(form, pat.n, pat.m, pat.H_rowptr, pat.H_colind, pat.J_rowptr, pat.J_colind, prec="fp32_ir")
    sig0 = None
    for d in range(4):
        inst = synth.condensed_grid(18, rho=1e4, draw=d, pat=pat, sigma0=sig0)
        sig0 = inst.sigma0
        finfo = K.factor(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), inst.delta, inst.rho)
        X, sinfo = K.solve(_t(inst.b))
        check_against_oracle(inst, "fp32_ir", X.cpu().numpy(), finfo, sinfo, 1e-10)


def test_solve_before_factor_is_state_error():
    pat = synth.make_pattern(2, 2)
    K = nk().KKT(0, pat.n, pat.m, pat.H_rowptr, pat.H_colind, pat.J_rowptr, pat.J_colind, prec="fp64")
    with pytest.raises(nk().NclError) as e:
        K.solve(torch.zeros(pat.n + pat.m, dtype=torch.float64, device=DEV))
    assert e.value.status == 5


def test_device_memory_cap():
    pat = synth.make_pattern(10, 10)
    with pytest.raises(nk().NclError) as e:
        nk().KKT(0, pat.n, pat.m, pat.H_rowptr, pat.H_colind, pat.J_rowptr, pat.J_colind,
                 max_device_bytes=1000)
    assert e.value.status == 3


# ------------------------------------------------------------------ batches

@pytest.mark.parametrize("prec,eta_tol", [("fp64", 1e-12), ("fp32_ir", 1e-10)])
def test_scenario_batch(prec, eta_tol):
    """Instances with 1-3 deleted edges each (patterns differ), 4 RHS, one
    handle; each instance against its own oracle solve."""
    batch = synth.scenario_batch(count=6, side=12, nrhs=4)
    pats = [(i.n, i.m, i.pat.H_rowptr, i.pat.H_colind, i.pat.J_rowptr, i.pat.J_colind) for i in batch]
    K = nk().KKT.batch(0, pats, prec=prec)
    Hv = _t(np.concatenate([i.H_val for i in batch]))
    Jv = _t(np.concatenate([i.J_val for i in batch]))
    S = _t(np.concatenate([i.Sigma for i in batch]))
    B = _t(np.concatenate([i.b for i in batch], axis=0))
    infos = K.factor(Hv, Jv, S, [i.delta for i in batch], [i.rho for i in batch])
    X, sinfo = K.solve(B)
    X = X.cpu().numpy()
    off = 0
    for inst, fi in zip(batch, infos):
        d = inst.dim
        assert fi.inertia == (inst.n, inst.m, 0)
        check_against_oracle(inst, prec, X[off:off + d], fi, sinfo, eta_tol)
        off += d


def test_batch_factor_solve_entry_point():
    batch = synth.scenario_batch(count=3, side=8, nrhs=2)
    pats = [(i.n, i.m, i.pat.H_rowptr, i.pat.H_colind, i.pat.J_rowptr, i.pat.J_colind) for i in batch]
    K = nk().KKT.batch(0, pats, prec="fp32_ir")
    Hv = _t(np.concatenate([i.H_val for i in batch]))
    Jv = _t(np.concatenate([i.J_val for i in batch]))
    S = _t(np.concatenate([i.Sigma for i in batch]))
    B = np.concatenate([i.b for i in batch], axis=0)
    Bc = _t(B.T.copy())
    Xc = torch.empty_like(Bc)
    infos, sinfo = nk().ncl_kkt_batch_factor_solve(K._h, Hv, Jv, S, [i.delta for i in batch],
                                                   [i.rho for i in batch], 2, Bc, K.dim, Xc, K.dim)
    X = Xc.cpu().numpy().T
    off = 0
    for inst, fi in zip(batch, infos):
        check_against_oracle(inst, "fp32_ir", X[off:off + inst.dim], fi, sinfo, 1e-10)
        off += inst.dim


# ------------------------------------------------------------------ adjoint

@pytest.mark.parametrize("form", ["stabilized", "condensed"])
@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
def test_adjoint_matches_oracle(form, prec):
    inst = synth.random_instance(6, 5, seed=44, form=form, rho=1e3, nrhs=2)
    K, finfo, X, sinfo = gpu_solve(inst, prec)
    rng = np.random.default_rng(9)
    GX = rng.standard_normal(X.shape)
    p = inst.pat
    g = K.adjoint(_t(X), _t(GX), nnz_H=p.nnz_H, nnz_J=p.nnz_J, n_var=p.n)
    x_o, fac, _, A = O.solve_instance(inst)
    ref = O.adjoint(inst, fac, A, x_o, GX)
    tol = 1e-9 if prec == "fp64" else 1e-7
    for key, rk in (("b", "g_b"), ("H", "g_H"), ("J", "g_J"), ("Sigma", "g_Sigma")):
        got = g[key].cpu().numpy().reshape(-1)
        want = np.asarray(ref[rk]).reshape(-1)
        assert np.max(np.abs(got - want)) <= tol * max(1.0, np.max(np.abs(want))), key
    sc = g["scal"].cpu().numpy()
    assert abs(sc[0] - ref["g_delta"]) <= tol * max(1.0, abs(ref["g_delta"]))
    assert abs(sc[1] - ref["g_rho"]) <= tol * max(1.0, abs(ref["g_rho"]))


# ------------------------------------------------------------------ full size

@pytest.mark.parametrize("prec,rho,eta_tol", [("fp32_ir", 1e2, 1e-10), ("fp32_ir", 1e5, 1e-10),
                                              ("fp64", 1e5, 1e-12)])
def test_condensed_300x300_full_size(prec, rho, eta_tol):
    """The 300 x 300 condensed workload at full size, in the bench's
    configuration: properties that hold at any size (inertia, FP64 backward
    error recomputed on the CPU from the oracle's matrix), plus sampled
    entries of K x against b computed row by row from the oracle's matrix."""
    pat = synth.make_pattern(300, 300)
    inst = synth.condensed_grid(300, rho=rho, draw=0, pat=pat)
    K, finfo, X, sinfo = gpu_solve(inst, prec)
    assert finfo.inertia == (inst.n, 0, 0)
    assert finfo.n_perturbed == 0
    A = O.instance_matrix(inst)
    eta = O.backward_error(A, X, inst.b)
    assert eta <= eta_tol, eta
    rows = np.random.default_rng(0).choice(inst.n, 64, replace=False)
    Ar = sp.csr_matrix(A)[rows]
    scale = np.abs(Ar).sum(axis=1).A1 * np.max(np.abs(X)) + np.abs(inst.b[rows, 0])
    assert np.all(np.abs(Ar @ X[:, 0] - inst.b[rows, 0]) <= eta_tol * scale)


# ------------------------------------------------------------------ refinement beyond Richardson

def test_condensed_rho_1e7_needs_fgmres():
    """rho = 1e7: kappa(K) * u_fp32 > 1, so Richardson
    refinement of the FP32 factorisation stagnates; the FGMRES fallback (FP64
    Krylov vectors, FP32 LDL^T preconditioner) reaches 1e-10.  The precision
    fallback is off so that the FP32 factor is the one refined."""
    inst = synth.condensed_grid(24, rho=1e7, draw=0)
    K, finfo, X, sinfo = gpu_solve(inst, "fp32_ir", precision_fallback=0)
    assert finfo.fp64_fallback == 0 and sum(finfo.inertia) == inst.n
    assert sinfo.status == 0 and sinfo.used_fgmres == 1 and sinfo.fp64_fallback == 0
    A = O.instance_matrix(inst)
    assert O.backward_error(A, X, inst.b) <= 1e-10


def test_condensed_rho_1e7_without_fallback_is_honest():
    """A larger grid at rho = 1e7 with the precision fallback off: the FP32
    factor (kappa * u_fp32 >> 1) may be too poor even as an FGMRES
    preconditioner.  Whatever happens, the solve either reaches 1e-10 or
    says that it did not: it never reports success with a worse residual."""
    inst = synth.condensed_grid(40, rho=1e7, draw=0)
    K, finfo, X, sinfo = gpu_solve(inst, "fp32_ir", precision_fallback=0)
    assert finfo.fp64_fallback == 0 and sum(finfo.inertia) == inst.n
    A = O.instance_matrix(inst)
    eta = O.backward_error(A, X, inst.b)
    assert sinfo.status in (0, 8)     # NCL_OK or NCL_ERR_IR_NOT_CONVERGED
    if sinfo.status == 0:
        assert eta <= 1e-10
    else:
        assert sinfo.backward_err > 1e-10 and eta > 1e-10 * 0.5


@pytest.mark.parametrize("side", [24, 40])
def test_condensed_rho_1e7_default(side):
    """Default options at rho = 1e7: FGMRES on the FP32 factor, or the FP64
    refactorisation when the FP32 pivots' signs are not those of an SPD
    matrix; either way the regular inertia and a 1e-10 backward error."""
    inst = synth.condensed_grid(side, rho=1e7, draw=0)
    K, finfo, X, sinfo = gpu_solve(inst, "fp32_ir")
    assert finfo.inertia == (inst.n, 0, 0)
    assert sinfo.status == 0
    A = O.instance_matrix(inst)
    assert O.backward_error(A, X, inst.b) <= 1e-10


@pytest.mark.parametrize("form", ["condensed", "stabilized"])
def test_rho_1e8_fp32_falls_back_to_fp64(form):
    """rho = 1e8: in FP32 the O(1) part H + Sigma + delta I is lost against
    rho J^T J (kappa ~ 3e9 > 1/u_fp32), and the FP32 pivots' signs are not
    those of the matrix.  The FP32+IR handle detects the irregular inertia
    and refactors the same FP64 values in FP64; without that fallback it
    reports that refinement did not converge."""
    if form == "condensed":
        inst = synth.condensed_grid(24, rho=1e8, draw=0)
    else:
        inst = synth.random_instance(24, 24, seed=3, form="stabilized", rho=1e8)
    want = (inst.n, inst.m, 0) if form == "stabilized" else (inst.n, 0, 0)
    A = O.instance_matrix(inst)
    K, finfo, X, sinfo = gpu_solve(inst, "fp32_ir")
    assert finfo.fp64_fallback == 1 and finfo.inertia == want
    assert sinfo.status == 0 and sinfo.fp64_fallback == 1
    assert O.backward_error(A, X, inst.b) <= 1e-10     # the FP32+IR handle's target
    K0, f0, X0, s0 = gpu_solve(inst, "fp32_ir", precision_fallback=0)
    assert f0.fp64_fallback == 0 and f0.inertia != want
    assert s0.status == 8
    K64, f64, X64, s64 = gpu_solve(inst, "fp64")
    assert f64.inertia == want
    assert O.backward_error(A, X64, inst.b) <= 1e-12


def test_fp32_failure_penalty_is_remembered():
    """After an untrusted FP32 factor at rho = 1e8 (with regular FP64
    factors), the handle starts later factorisations at rho >= 1e8 in FP64
    directly (fp64_fallback = 2), with the same results; a smaller penalty
    tries FP32 again, and precision_fallback = 2 remembers nothing."""
    hi = synth.condensed_grid(24, rho=1e8, draw=0)
    lo = synth.condensed_grid(24, rho=1e5, draw=1)
    p = hi.pat
    want = (hi.n, 0, 0)
    for mode, second in ((1, 2), (2, 1)):
        K = nk().KKT(1, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec="fp32_ir",
                     precision_fallback=mode)
        seen = []
        for inst, rho in ((hi, hi.rho), (hi, 2 * hi.rho), (lo, lo.rho), (hi, hi.rho)):
            A = O.instance_matrix(inst) if rho == inst.rho else None
            f = K.factor(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), inst.delta, rho)
            X, si = K.solve(_t(inst.b))
            torch.cuda.synchronize()
            assert f.inertia == want and si.status == 0
            if A is not None:
                assert O.backward_error(A, X.cpu().numpy(), inst.b) <= 1e-10
            seen.append((f.fp64_fallback, si.fp64_fallback))
        assert seen == [(1, 1), (second, 1), (0, 0), (second, 1)], (mode, seen)
        K.close()


def test_batch_factor_solve_graph_replay():
    """The one-graph factor + solve of a batch, replayed with new values on
    the same patterns and buffers, against the oracle every time."""
    rng = np.random.default_rng(5)
    pats = [synth.make_pattern(10, 12, np.sort(rng.choice(len(synth.grid_edges(10, 12)), k, replace=False)))
            for k in (1, 2, 3)]
    K = nk().KKT.batch(0, [(p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind) for p in pats],
                       prec="fp32_ir")
    dim = K.dim
    Hv = torch.empty(sum(p.nnz_H for p in pats), dtype=torch.float64, device=DEV)
    Jv = torch.empty(sum(p.nnz_J for p in pats), dtype=torch.float64, device=DEV)
    S = torch.empty(sum(p.n for p in pats), dtype=torch.float64, device=DEV)
    Bc = torch.empty(3, dim, dtype=torch.float64, device=DEV)
    Xc = torch.empty_like(Bc)
    for draw in range(4):
        insts = [synth.draw_instance(p, np.random.default_rng(100 * draw + i), form="stabilized", rho=1e4, nrhs=3)
                 for i, p in enumerate(pats)]
        Hv.copy_(_t(np.concatenate([i.H_val for i in insts])))
        Jv.copy_(_t(np.concatenate([i.J_val for i in insts])))
        S.copy_(_t(np.concatenate([i.Sigma for i in insts])))
        Bc.copy_(_t(np.concatenate([i.b for i in insts], axis=0).T))
        infos, sinfo = nk().ncl_kkt_batch_factor_solve(K._h, Hv, Jv, S, [i.delta for i in insts],
                                                       [i.rho for i in insts], 3, Bc, dim, Xc, dim)
        X = Xc.cpu().numpy().T
        off = 0
        for inst, fi in zip(insts, infos):
            assert fi.inertia == (inst.n, inst.m, 0)
            check_against_oracle(inst, "fp32_ir", X[off:off + inst.dim], fi, sinfo, 1e-10)
            off += inst.dim


# ------------------------------------------------------------------ deep fronts, elementwise

@pytest.mark.parametrize("persistent", [1, 0])
@pytest.mark.parametrize("prec,eta_tol", [("fp64", 1e-12), ("fp32_ir", 1e-10)])
@pytest.mark.parametrize("form,side", [("condensed", 80), ("stabilized", 80)])
def test_deep_fronts_elementwise(prec, eta_tol, form, side, persistent):
    """Grids large enough that the top fronts hold several 128-column macro
    panels (712 pivots condensed, 528 stabilized), tensor-core updates
    (FP32) and supernodes of several 128-row block-rows in the chained
    sweeps: the whole solution against the oracle, elementwise, and the
    kernel profile showing that those paths ran -- the persistent
    large-front launch per level and the small-subtree sweeps, or one launch
    per panel step and per-level sweeps throughout."""
    if form == "condensed":
        inst = synth.condensed_grid(side, rho=1e4, draw=2)
    else:
        inst = synth.random_instance(side, side, seed=880 + side, form="stabilized", rho=1e4)
    p = inst.pat
    K = nk().KKT(0 if form == "stabilized" else 1, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind,
                 prec=prec, persistent_fronts=persistent, subtree_sweeps=persistent)
    nk().ncl_kkt_profile(K._h, 1)
    finfo = K.factor(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), inst.delta, inst.rho)
    X, sinfo = K.solve(_t(inst.b))
    torch.cuda.synchronize()
    prof = nk().ncl_kkt_profile_report(K._h)
    assert K.analysis.max_pivots > 4 * 128
    suffix = "f32" if prec == "fp32_ir" else "f64"
    if persistent:
        assert prof[f"front_dag_{suffix}"]["launches"] >= 1 and f"macro_panel_{suffix}" not in prof
        assert prof[f"subtree_fwd_{suffix}"]["launches"] >= 1 and prof[f"subtree_bwd_{suffix}"]["launches"] >= 1
    else:
        assert prof[f"macro_panel_{suffix}"]["launches"] >= 5
        assert f"subtree_fwd_{suffix}" not in prof
    assert prof[f"fwd_chain_multi_{suffix}"]["launches"] >= 1
    assert prof[f"bwd_chain_multi_{suffix}"]["launches"] >= 1
    if prec == "fp32_ir" and not persistent:
        # the trailing updates of every many-pivot front (roots included)
        assert prof["update_tc_f32"]["launches"] >= 2
    if prec == "fp32_ir" and persistent and form == "condensed":
        # the update blocks of the many-pivot fronts with rows below (the
        # trailing updates run inside the persistent launch)
        assert prof["update_tc_f32"]["launches"] >= 1
    want = (inst.n, inst.m, 0) if form == "stabilized" else (inst.n, 0, 0)
    assert finfo.inertia == want
    # the quality of the factors, not only the refined answer: at rho = 1e4
    # (kappa ~ 4e5) a sound FP32 factorisation needs at most 3 Richardson steps
    assert sinfo.used_fgmres == 0 and sinfo.ir_iters <= 3, sinfo.ir_iters
    check_against_oracle(inst, prec, X.cpu().numpy(), finfo, sinfo, eta_tol)


# ------------------------------------------------------------------ the other full-size workloads

def _sampled_rows_ok(A, X, b, eta_tol, count=64, seed=0):
    rows = np.random.default_rng(seed).choice(A.shape[0], count, replace=False)
    Ar = sp.csr_matrix(A)[rows]
    ok = True
    for r in range(X.shape[1]):
        scale = np.abs(Ar).sum(axis=1).A1 * np.max(np.abs(X[:, r])) + np.abs(b[rows, r])
        ok = ok and bool(np.all(np.abs(Ar @ X[:, r] - b[rows, r]) <= eta_tol * scale))
    return ok


@pytest.mark.parametrize("prec,eta_tol", [("fp32_ir", 1e-10), ("fp64", 1e-12)])
def test_stabilized_700x700_full_size(prec, eta_tol):
    """The 700 x 700 stabilized workload (n = 1.96M, m = 0.98M, rho = 1e6) at
    full size: inertia, the FP64 backward error recomputed on the CPU from
    the oracle's matrix, and 64 sampled rows of K x - b."""
    inst = synth.large_stabilized(700, rho=1e6, draw=0)
    K, finfo, X, sinfo = gpu_solve(inst, prec)
    assert finfo.inertia == (inst.n, inst.m, 0)
    assert finfo.n_perturbed == 0
    assert sinfo.status == 0
    A = O.instance_matrix(inst)
    eta = O.backward_error(A, X, inst.b)
    assert eta <= eta_tol, eta
    assert _sampled_rows_ok(A, X, inst.b, eta_tol)
    K.close()


def test_scenario_batch_64_full_size():
    """The 64-scenario batch of 100 x 100 grids (1-3 edges deleted each,
    4 right-hand sides) at full size, through the one-graph factor + solve:
    per instance its inertia, its FP64 backward error recomputed on the CPU
    and sampled rows."""
    batch = synth.scenario_batch(count=64, side=100, nrhs=4)
    pats = [(i.n, i.m, i.pat.H_rowptr, i.pat.H_colind, i.pat.J_rowptr, i.pat.J_colind) for i in batch]
    K = nk().KKT.batch(0, pats, prec="fp32_ir")
    Hv = _t(np.concatenate([i.H_val for i in batch]))
    Jv = _t(np.concatenate([i.J_val for i in batch]))
    S = _t(np.concatenate([i.Sigma for i in batch]))
    Bc = _t(np.concatenate([i.b for i in batch], axis=0).T.copy())
    Xc = torch.empty_like(Bc)
    for _ in range(2):      # the direct first call, then the replayed graph
        infos, sinfo = nk().ncl_kkt_batch_factor_solve(K._h, Hv, Jv, S, [i.delta for i in batch],
                                                       [i.rho for i in batch], 4, Bc, K.dim, Xc, K.dim)
        assert sinfo.status == 0
        X = Xc.cpu().numpy().T
        off = 0
        for k, (inst, fi) in enumerate(zip(batch, infos)):
            assert fi.inertia == (inst.n, inst.m, 0)
            Xi = X[off:off + inst.dim]
            A = O.instance_matrix(inst)
            assert O.backward_error(A, Xi, inst.b) <= 1e-10
            if k % 8 == 0:
                assert _sampled_rows_ok(A, Xi, inst.b, 1e-10, count=16, seed=k)
            off += inst.dim
    K.close()
