"""GPU parity of the Newton step around the factorisation (Sections 3.1-3.3)
through the C ABI against the oracle: the right-hand side of Eq. K2r / K1 at
a seeded interior point, the recovery of Delta y, Delta r, Delta z_l,
Delta z_u, and the whole chain right-hand side -> refined solve -> recovery.
(The oracle's chain is itself pinned to a dense solve of Eq. K3.)"""
import numpy as np
import pytest

import oracle as O
from paper_2510_05885_gb300 import synth
from tests.helpers import newton_point

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
MU = 0.05
DELTA = 10.0      # keeps H + Sigma(point) + delta I positive definite on these grids


def nk():
    from paper_2510_05885_gb300 import ncl_kkt
    return ncl_kkt


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def _setup(form, prec, R=9, C=11, seed=61):
    inst = synth.random_instance(R, C, seed, form=form, rho=50.0)
    pt, sigma = newton_point(inst, seed)
    p = inst.pat
    K = nk().KKT(0 if form == "stabilized" else 1, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind,
                 prec=prec)
    info = K.factor(_t(inst.H_val), _t(inst.J_val), _t(sigma), DELTA, inst.rho)
    build = O.kkt_stabilized if form == "stabilized" else O.kkt_condensed
    A = build(p.n, p.m, p.H_rowptr, p.H_colind, inst.H_val, p.J_rowptr, p.J_colind, inst.J_val, sigma, DELTA,
              inst.rho)
    fac = O.LDLT(A, O.block_signs(form, p.n, p.m))
    assert info.inertia == fac.inertia == (p.n, p.m if form == "stabilized" else 0, 0)
    return inst, pt, K, A, fac


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
@pytest.mark.parametrize("form", ["stabilized", "condensed"])
def test_newton_rhs_solve_and_recovery(form, prec):
    inst, pt, K, A, fac = _setup(form, prec)
    p = inst.pat
    dpt = {k: _t(v) for k, v in pt.items()}
    b = K.newton_rhs(dpt, MU).cpu().numpy()
    b_o = O.newton_rhs(form, p.n, p.m, p.J_rowptr, p.J_colind, inst.J_val, pt, MU, inst.rho)
    assert np.max(np.abs(b - b_o)) <= 1e-13 * np.max(np.abs(b_o))
    X_o, _, _ = O.solve_ir(A, fac, b_o)
    # the recovery from the same solution on both sides
    rec = K.newton_recover(dpt, MU, _t(X_o))
    rec_o = O.newton_recover(form, p.n, p.m, p.J_rowptr, p.J_colind, inst.J_val, pt, MU, inst.rho, X_o)
    for k, want in rec_o.items():
        got = rec[k].cpu().numpy()
        assert np.max(np.abs(got - want)) <= 1e-13 * max(1.0, np.max(np.abs(want))), k
    # the whole chain: library right-hand side, refined solve, recovery
    X, sinfo = K.solve(_t(b))
    rec = K.newton_recover(dpt, MU, X)
    kappa = O.cond1_estimate(A, fac)
    tol = max(1e-9, 10 * kappa * (1e-10 if prec == "fp32_ir" else 1e-15))
    for k, want in rec_o.items():
        got = rec[k].cpu().numpy()
        assert np.max(np.abs(got - want)) <= tol * max(1.0, np.max(np.abs(want))), k
    assert np.all(rec["dz_lower"].cpu().numpy()[np.isinf(pt["lower"])] == 0.0)
    assert np.all(rec["dz_upper"].cpu().numpy()[np.isinf(pt["upper"])] == 0.0)


def test_newton_step_batch():
    insts = [synth.random_instance(5, 6, s, form="stabilized", rho=50.0) for s in (71, 72)]
    pts = [newton_point(i, 80 + k) for k, i in enumerate(insts)]
    pats = [(i.n, i.m, i.pat.H_rowptr, i.pat.H_colind, i.pat.J_rowptr, i.pat.J_colind) for i in insts]
    K = nk().KKT.batch(0, pats, prec="fp64")
    K.factor(_t(np.concatenate([i.H_val for i in insts])), _t(np.concatenate([i.J_val for i in insts])),
             _t(np.concatenate([s for _, s in pts])), [DELTA, DELTA], [i.rho for i in insts])
    keys = pts[0][0].keys()
    dpt = {k: _t(np.concatenate([pt[k] for pt, _ in pts])) for k in keys}
    mus = [0.05, 0.2]
    b = K.newton_rhs(dpt, mus).cpu().numpy()
    X, _ = K.solve(_t(b))
    rec = {k: v.cpu().numpy() for k, v in K.newton_recover(dpt, mus, X).items()}
    off_row = off_n = off_m = 0
    for inst, (pt, sigma), mu in zip(insts, pts, mus):
        p = inst.pat
        b_o = O.newton_rhs("stabilized", p.n, p.m, p.J_rowptr, p.J_colind, inst.J_val, pt, mu, inst.rho)
        assert np.max(np.abs(b[off_row:off_row + inst.dim] - b_o)) <= 1e-13 * np.max(np.abs(b_o))
        A = O.kkt_stabilized(p.n, p.m, p.H_rowptr, p.H_colind, inst.H_val, p.J_rowptr, p.J_colind, inst.J_val,
                             sigma, DELTA, inst.rho)
        X_o, _, _ = O.solve_ir(A, O.LDLT(A, O.block_signs("stabilized", p.n, p.m)), b_o)
        rec_o = O.newton_recover("stabilized", p.n, p.m, p.J_rowptr, p.J_colind, inst.J_val, pt, mu, inst.rho, X_o)
        for k, want in rec_o.items():
            sl = slice(off_n, off_n + p.n) if k in ("dx", "dz_lower", "dz_upper") else slice(off_m, off_m + p.m)
            assert np.max(np.abs(rec[k][sl] - want)) <= 1e-8 * max(1.0, np.max(np.abs(want))), k
        off_row += inst.dim
        off_n += p.n
        off_m += p.m


def test_newton_step_argument_checks():
    inst = synth.random_instance(3, 3, 5, form="stabilized", rho=50.0)
    pt, sigma = newton_point(inst, 5)
    p = inst.pat
    K = nk().KKT(0, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec="fp64")
    dpt = {k: _t(v) for k, v in pt.items()}
    with pytest.raises(nk().NclError):          # no factor yet
        K.newton_rhs(dpt, MU)
    K.factor(_t(inst.H_val), _t(inst.J_val), _t(sigma), DELTA, inst.rho)
    bad = dict(dpt)
    bad["y_k"] = None
    with pytest.raises(nk().NclError):          # a missing vector
        K.newton_rhs(bad, MU)
    with pytest.raises(nk().NclError):          # negative mu
        K.newton_rhs(dpt, -1.0)
