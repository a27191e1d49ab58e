"""The torch.autograd.Function around the hand-written adjoint, against the
oracle's adjoint and against torch autograd through a dense FP64 solve."""
import numpy as np
import pytest

import oracle as O
from paper_2510_05885_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(a, grad=False):
    t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda:0")
    return t.requires_grad_(grad)


@pytest.mark.parametrize("form", ["stabilized", "condensed"])
@pytest.mark.parametrize("prec,eta_target", [("fp64", 2.0 ** -53), ("fp32_ir", 1e-10)])
def test_autograd_matches_oracle_adjoint(form, prec, eta_target):
    """Both solves (x and g_b = K^-T g_x) are refined to the backward error
    target eta; two backward-stable answers differ by about kappa * eta, so
    the gradients are compared at max(1e-9, kappa * eta) relative to their
    largest entry, kappa estimated through the oracle's factors."""
    from paper_2510_05885_gb300 import ncl_kkt as nk
    from paper_2510_05885_gb300.autograd import kkt_solve
    inst = synth.random_instance(10, 10, seed=12, form=form, rho=1e4)
    p = inst.pat
    K = nk.KKT(0 if form == "stabilized" else 1, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind,
               prec=prec)
    Hv, Jv, S, b = _t(inst.H_val, True), _t(inst.J_val, True), _t(inst.Sigma, True), _t(inst.b[:, 0], True)
    delta = torch.tensor(inst.delta, dtype=torch.float64, requires_grad=True)
    rho = torch.tensor(inst.rho, dtype=torch.float64, requires_grad=True)
    w = np.random.default_rng(4).standard_normal(inst.dim)
    x = kkt_solve(K, Hv, Jv, S, b, delta, rho)
    (x * _t(w)).sum().backward()
    x_o, fac, _, A = O.solve_instance(inst)
    ref = O.adjoint(inst, fac, A, x_o[:, 0], w)
    tol = max(1e-9, O.cond1_estimate(A, fac) * eta_target)
    for t, key in ((Hv, "g_H"), (Jv, "g_J"), (S, "g_Sigma"), (b, "g_b")):
        got = t.grad.cpu().numpy()
        want = np.asarray(ref[key]).reshape(-1)
        assert np.max(np.abs(got - want)) <= tol * max(1.0, np.max(np.abs(want))), key
    assert abs(delta.grad.item() - ref["g_delta"]) <= tol * max(1.0, abs(ref["g_delta"]))
    assert abs(rho.grad.item() - ref["g_rho"]) <= tol * max(1.0, abs(ref["g_rho"]))


def test_autograd_matches_dense_torch_gradient():
    """10x10 grid, K2r (n+m = 600): against torch autograd through
    torch.linalg.solve on the dense FP64 matrix built from the same values."""
    from paper_2510_05885_gb300 import ncl_kkt as nk
    from paper_2510_05885_gb300.autograd import kkt_solve
    inst = synth.random_instance(10, 10, seed=31, form="stabilized", rho=1e4)
    p = inst.pat
    n, m = p.n, p.m
    K = nk.KKT(0, n, m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec="fp64")
    w = torch.as_tensor(np.random.default_rng(2).standard_normal(n + m))
    Hv, Jv, S, b = _t(inst.H_val, True), _t(inst.J_val, True), _t(inst.Sigma, True), _t(inst.b[:, 0], True)
    x = kkt_solve(K, Hv, Jv, S, b, inst.delta, inst.rho)
    (x * w.cuda()).sum().backward()
    # dense reference on the CPU
    c = lambda a: torch.tensor(np.asarray(a, float), dtype=torch.float64, requires_grad=True)
    Hc, Jc, Sc, bc = c(inst.H_val), c(inst.J_val), c(inst.Sigma), c(inst.b[:, 0])
    rows = torch.tensor(np.repeat(np.arange(n), np.diff(p.H_rowptr)))
    cols = torch.tensor(p.H_colind.astype(np.int64))
    Jr = torch.tensor(np.repeat(np.arange(m), np.diff(p.J_rowptr)))
    Jcl = torch.tensor(p.J_colind.astype(np.int64))
    Hd = torch.zeros(n, n, dtype=torch.float64).index_put((rows, cols), Hc, accumulate=True)
    off = rows != cols
    Hd = Hd.index_put((cols[off], rows[off]), Hc[off], accumulate=True) + torch.diag(Sc + inst.delta)
    Jd = torch.zeros(m, n, dtype=torch.float64).index_put((Jr, Jcl), Jc, accumulate=True)
    Kd = torch.cat([torch.cat([Hd, Jd.T], 1),
                    torch.cat([Jd, -torch.eye(m, dtype=torch.float64) / inst.rho], 1)], 0)
    (torch.linalg.solve(Kd, bc) * w).sum().backward()
    for t, r in ((Hv, Hc), (Jv, Jc), (S, Sc), (b, bc)):
        got, want = t.grad.cpu(), r.grad
        assert torch.max(torch.abs(got - want)) <= 1e-10 * max(1.0, float(torch.max(torch.abs(want))))


def test_autograd_refactor_between_forward_and_backward_raises():
    from paper_2510_05885_gb300 import ncl_kkt as nk
    from paper_2510_05885_gb300.autograd import kkt_solve
    inst = synth.random_instance(3, 3, seed=1, form="stabilized")
    p = inst.pat
    K = nk.KKT(0, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec="fp64")
    Hv = _t(inst.H_val, True)
    x = kkt_solve(K, Hv, _t(inst.J_val), _t(inst.Sigma), _t(inst.b[:, 0]), inst.delta, inst.rho)
    K.factor(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), inst.delta, inst.rho)
    with pytest.raises(RuntimeError):
        x.sum().backward()
