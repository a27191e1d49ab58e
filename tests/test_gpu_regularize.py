"""GPU parity of the inertia correction of Section 3.1 (through the C ABI)
against the oracle's loop on the same seeded inputs.

Both sides factor the regularised matrix with rho-hat = rho + delta, raise
delta on an irregular inertia with the same schedule, and must stop at the
same delta after the same number of factorisations.  The inertia decides an
integer, so every test first checks on the CPU (dense FP64 eigenvalues of
the Schur complement H + Sigma + delta I + rho-hat J^T J) that no tried
delta puts an eigenvalue within 1e-5 of the matrix norm of zero: there the
FP32 and FP64 decisions cannot differ.  The solution of the final system is
then held to the parity tolerances of the plain solve.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_2510_05885_gb300 import synth
from tests.helpers import custom_instance, read_golden

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SCHED = dict(delta_first=1e-2, growth=3.0, max_tries=40)


def nk():
    from paper_2510_05885_gb300 import ncl_kkt
    return ncl_kkt


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def _assert_margins(inst, last_delta, delta_first, growth):
    """Every delta of the schedule up to last_delta keeps the Schur
    complement's smallest eigenvalue away from zero."""
    p = inst.pat
    J = sp.csr_matrix((inst.J_val, p.J_colind, p.J_rowptr), shape=(p.m, p.n)).toarray()
    d = 0.0
    while True:
        A = O.kkt_condensed(p.n, 0, p.H_rowptr, p.H_colind, inst.H_val, np.zeros(1, np.int32),
                            np.zeros(0, np.int32), np.zeros(0), inst.Sigma, d, 1.0).toarray()
        ev = np.linalg.eigvalsh(A + (inst.rho + d) * J.T @ J)
        assert abs(ev[0]) > 1e-5 * np.max(np.abs(ev)), d
        if d >= last_delta:
            return
        d = d * growth if d > 0 else delta_first


def _check_solution(K, A, fac, b, prec):
    X, sinfo = K.solve(_t(b))
    torch.cuda.synchronize()
    X = X.cpu().numpy().reshape(b.shape)
    eta_tol = 1e-12 if prec == "fp64" else 1e-10
    eta = O.backward_error(A, X, b)
    assert eta <= eta_tol, eta
    x_o, _, eta_o = O.solve_ir(A, fac, b, max_steps=3)
    kappa = O.cond1_estimate(A, fac)
    u = max(2.0 ** -53, eta + eta_o) if prec == "fp64" else 1e-10
    err = np.max(np.abs(X - x_o)) / np.max(np.abs(x_o))
    assert err <= max(1e-9, 10 * kappa * u), (err, kappa)


@pytest.mark.parametrize("prec,fallback", [("fp64", 1), ("fp32_ir", 1), ("fp32_ir", 0)])
@pytest.mark.parametrize("form,R,C,rho,seed", [("stabilized", 13, 17, 1e2, 2), ("condensed", 16, 16, 1.0, 1)])
def test_regularize_matches_oracle_loop(prec, fallback, form, R, C, rho, seed):
    """fallback = 0: the FP32 inertia decides every try on its own."""
    inst = synth.random_instance(R, C, seed, form=form, rho=rho)
    fac, A, delta_o, tries_o, regular = O.regularize(inst, 0.0, **SCHED)
    assert regular and tries_o > 1                 # at least one correction happens
    _assert_margins(inst, delta_o, SCHED["delta_first"], SCHED["growth"])
    p = inst.pat
    K = nk().KKT(0 if form == "stabilized" else 1, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind,
                 prec=prec, precision_fallback=fallback)
    infos, delta, tries, st = K.factor_regularized(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), 0.0, rho,
                                                   **SCHED)
    assert st == 0
    assert not infos[0].fp64_fallback or fallback
    assert tries == tries_o and delta[0] == delta_o
    assert infos[0].inertia == fac.inertia == (inst.n, inst.m if form == "stabilized" else 0, 0)
    _check_solution(K, A, fac, inst.b, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
@pytest.mark.parametrize("form", ["stabilized", "condensed"])
def test_regularize_golden_scalar(prec, form):
    gd = read_golden(os.path.join(GOLDEN, "regularize_scalar.txt"))
    inst = custom_instance(np.array([[gd["h"][0]]]), np.array([[1.0]]), np.zeros(1), 0.0, gd["rho"][0],
                           np.ones(2 if form == "stabilized" else 1), form=form)
    p = inst.pat
    K = nk().KKT(0 if form == "stabilized" else 1, 1, 1, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind,
                 prec=prec)
    infos, delta, tries, st = K.factor_regularized(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), 0.0,
                                                   gd["rho"][0], gd["delta_first"][0], gd["growth"][0])
    assert st == 0 and tries == int(gd["tries"][0]) and delta[0] == gd["delta"][0]
    assert infos[0].inertia == tuple(int(v) for v in gd[f"inertia_{form}"])
    # the same limit with two tries: INERTIA, delta of the last try kept
    infos, delta, tries, st = K.factor_regularized(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), 0.0,
                                                   gd["rho"][0], gd["delta_first"][0], gd["growth"][0],
                                                   max_tries=2, raise_on_inertia=False)
    assert st == nk().ERR_INERTIA and tries == 2 and delta[0] == gd["delta_first"][0]


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
def test_regularize_batch_per_instance(prec):
    """Each instance of a batch is corrected on its own schedule; an
    instance that starts regular keeps its delta."""
    insts = [synth.random_instance(7, 4, s, form="stabilized", rho=10.0) for s in (1, 2, 3)]
    d0 = [0.0, 5.0, 0.0]
    want = []
    for inst, d in zip(insts, d0):
        fac, A, dl, t, regular = O.regularize(inst, d, **SCHED)
        assert regular
        _assert_margins(inst, dl, SCHED["delta_first"], SCHED["growth"])
        want.append((dl, t, fac.inertia))
    pats = [(i.n, i.m, i.pat.H_rowptr, i.pat.H_colind, i.pat.J_rowptr, i.pat.J_colind) for i in insts]
    K = nk().KKT.batch(0, pats, prec=prec)
    infos, delta, tries, st = K.factor_regularized(_t(np.concatenate([i.H_val for i in insts])),
                                                   _t(np.concatenate([i.J_val for i in insts])),
                                                   _t(np.concatenate([i.Sigma for i in insts])), d0,
                                                   [i.rho for i in insts], **SCHED)
    assert st == 0
    assert tries == max(w[1] for w in want)
    assert want[1][0] == 5.0
    for k, (dl, t, inertia) in enumerate(want):
        assert delta[k] == dl
        assert infos[k].inertia == inertia


def test_regularize_rejects_bad_schedule():
    inst = synth.random_instance(3, 3, 1, form="stabilized", rho=10.0)
    p = inst.pat
    K = nk().KKT(0, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec="fp64")
    args = (_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma))
    for bad in (dict(growth=1.0), dict(delta_first=0.0), dict(max_tries=0)):
        with pytest.raises(nk().NclError):
            K.factor_regularized(*args, 0.0, 10.0, **bad)
    with pytest.raises(nk().NclError):
        K.factor_regularized(*args, -1.0, 10.0)
