"""GPU parity of the condensed form with slacks (Section 3.3, Eq. K1s)
through the C ABI against the oracle: the weighted factorisation and solve,
the right-hand side and slack step of the proof's elimination, the batch
path, the adjoint through the row weights (central differences of the
oracle's solves) and the argument checks."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_2510_05885_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def nk():
    from paper_2510_05885_gb300 import ncl_kkt
    return ncl_kkt


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def _case(R, C, seed, rho, frac_eq=0.4):
    inst = synth.random_instance(R, C, seed, form="condensed", rho=rho)
    rng = np.random.default_rng(seed + 1000)
    Ss = 10.0 ** rng.uniform(-2, 2, inst.m)
    Ss[rng.random(inst.m) < frac_eq] = np.inf
    return inst, Ss


def _oracle_matrix(inst, Ss, rho=None, J_val=None):
    p = inst.pat
    return O.kkt_condensed_slack(p.n, p.m, p.H_rowptr, p.H_colind, inst.H_val, p.J_rowptr, p.J_colind,
                                 inst.J_val if J_val is None else J_val, inst.Sigma, Ss, inst.delta,
                                 inst.rho if rho is None else rho)


def _handle(inst, prec):
    p = inst.pat
    return nk().KKT(1, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec=prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
@pytest.mark.parametrize("R,C,seed,rho", [(12, 14, 3, 1e2), (20, 20, 4, 1e4)])
def test_k1s_factor_solve_and_slack_step(prec, R, C, seed, rho):
    inst, Ss = _case(R, C, seed, rho)
    p = inst.pat
    n, m = p.n, p.m
    K = _handle(inst, prec)
    info = K.factor_k1s(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), _t(Ss), inst.delta, rho)
    A = _oracle_matrix(inst, Ss)
    fac = O.LDLT(A)
    assert info.inertia == fac.inertia == (n, 0, 0)
    rng = np.random.default_rng(seed)
    rt, rs = rng.standard_normal((n, 2)), rng.standard_normal((m, 2))
    # right-hand side of the proof's elimination
    rhs = K.k1s_rhs(_t(rt), _t(rs)).cpu().numpy()
    rhs_o = O.k1s_rhs(m, p.J_rowptr, p.J_colind, inst.J_val, n, Ss, rho, rt, rs)
    assert np.max(np.abs(rhs - rhs_o)) <= 1e-13 * np.max(np.abs(rhs_o))
    # Delta t: parity tolerances of the plain solve
    X, sinfo = K.solve(_t(rhs_o))
    torch.cuda.synchronize()
    X = X.cpu().numpy()
    eta_tol = 1e-12 if prec == "fp64" else 1e-10
    eta = O.backward_error(A, X, rhs_o)
    assert eta <= eta_tol, eta
    x_o, _, eta_o = O.solve_ir(A, fac, rhs_o, max_steps=3)
    kappa = O.cond1_estimate(A, fac)
    u = max(2.0 ** -53, eta + eta_o) if prec == "fp64" else 1e-10
    assert np.max(np.abs(X - x_o)) / np.max(np.abs(x_o)) <= max(1e-9, 10 * kappa * u)
    # Delta s from the same Delta t on both sides
    ds = K.slack_step(_t(x_o), _t(rs)).cpu().numpy()
    ds_o = O.k1s_slack_step(m, p.J_rowptr, p.J_colind, inst.J_val, n, Ss, rho, x_o, rs)
    assert np.max(np.abs(ds - ds_o)) <= 1e-13 * max(1.0, np.max(np.abs(ds_o)))
    assert np.all(ds[np.isinf(Ss)] == 0.0)


def test_k1s_all_equality_rows_is_the_plain_condensed_factor():
    """Sigma_s = +inf on every row: the same factors and solution as Eq. K1."""
    inst, _ = _case(9, 11, 5, 1e3)
    K1 = _handle(inst, "fp64")
    K1.factor(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), inst.delta, inst.rho)
    x1, _ = K1.solve(_t(inst.b))
    K2 = _handle(inst, "fp64")
    K2.factor_k1s(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), _t(np.full(inst.m, np.inf)), inst.delta,
                  inst.rho)
    x2, _ = K2.solve(_t(inst.b))
    assert torch.equal(x1, x2)


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
def test_k1s_batch(prec):
    cases = [_case(6, 7, s, 1e2) for s in (11, 12, 13)]
    insts = [c[0] for c in cases]
    pats = [(i.n, i.m, i.pat.H_rowptr, i.pat.H_colind, i.pat.J_rowptr, i.pat.J_colind) for i in insts]
    K = nk().KKT.batch(1, pats, prec=prec)
    infos = K.factor_k1s(_t(np.concatenate([i.H_val for i in insts])), _t(np.concatenate([i.J_val for i in insts])),
                         _t(np.concatenate([i.Sigma for i in insts])), _t(np.concatenate([c[1] for c in cases])),
                         [i.delta for i in insts], [i.rho for i in insts])
    B = np.concatenate([i.b for i in insts], axis=0)
    X, sinfo = K.solve(_t(B))
    X = X.cpu().numpy()
    off = 0
    for (inst, Ss), fi in zip(cases, infos):
        A = _oracle_matrix(inst, Ss)
        fac = O.LDLT(A)
        assert fi.inertia == fac.inertia
        x_o, _, _ = O.solve_ir(A, fac, inst.b)
        xs = X[off:off + inst.n]
        assert O.backward_error(A, xs, inst.b) <= (1e-12 if prec == "fp64" else 1e-10)
        assert np.max(np.abs(xs - x_o)) / np.max(np.abs(x_o)) <= 1e-7
        off += inst.n


def test_k1s_adjoint_through_the_weights():
    """dl/dJ and dl/drho of l = 0.5 ||x||^2, x = K1s^{-1} b, against central
    differences of the oracle's FP64 solves (the weights rho Omega_r depend
    on rho and multiply J_r^T J_r)."""
    inst, Ss = _case(4, 5, 7, 10.0)
    p = inst.pat
    K = _handle(inst, "fp64")
    K.factor_k1s(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), _t(Ss), inst.delta, inst.rho)
    X, _ = K.solve(_t(inst.b))
    g = K.adjoint(X, X, nnz_H=p.nnz_H, nnz_J=p.nnz_J, n_var=p.n)
    gJ = g["J"].cpu().numpy()
    grho = float(g["scal"].cpu().numpy()[1])

    def loss(rho=inst.rho, J_val=inst.J_val):
        A = _oracle_matrix(inst, Ss, rho=rho, J_val=J_val)
        x, _, _ = O.solve_ir(A, O.LDLT(A), inst.b)
        return 0.5 * float(np.sum(x * x))

    h = 1e-6
    for q in np.random.default_rng(2).choice(p.nnz_J, 6, replace=False):
        Jp, Jm = inst.J_val.copy(), inst.J_val.copy()
        hq = h * max(1.0, abs(inst.J_val[q]))
        Jp[q] += hq
        Jm[q] -= hq
        fd = (loss(J_val=Jp) - loss(J_val=Jm)) / (2 * hq)
        assert abs(gJ[q] - fd) <= 1e-6 * max(1.0, abs(fd)), (q, gJ[q], fd)
    hr = h * inst.rho
    fd = (loss(rho=inst.rho + hr) - loss(rho=inst.rho - hr)) / (2 * hr)
    assert abs(grho - fd) <= 1e-6 * max(1.0, abs(fd)), (grho, fd)


def test_k1s_argument_checks():
    inst, Ss = _case(3, 3, 9, 10.0)
    p = inst.pat
    Ks = nk().KKT(0, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec="fp64")
    with pytest.raises(nk().NclError):          # not a condensed handle
        Ks.factor_k1s(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), _t(Ss), 0.0, 10.0)
    K = _handle(inst, "fp64")
    with pytest.raises(nk().NclError):          # no factor yet
        K.slack_step(_t(np.zeros(p.n)), _t(np.zeros(p.m)))
