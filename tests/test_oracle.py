"""Pins for the CPU oracle (no GPU).

The oracle is checked against facts that do not come from itself:
dense library solves and eigenvalues on tiny inputs, the closed-form block
factorisation of Section 3.2 (Eq. ldlk2r), the K2r <-> K1 equivalence of
Section 3.3, the inertia proposition of Section 3.4, the textbook Cholesky
special case (m = 0), hand-derived golden values, finite differences and a
dense autograd gradient for the adjoint.  ``test_planted_*`` plant mistakes
in the oracle and check that a pin catches each.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_2510_05885_gb300 import synth
from tests.helpers import custom_instance, read_golden

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny(R, C, seed, form, rho=1e4, nrhs=1):
    return synth.random_instance(R, C, seed, form=form, rho=rho, nrhs=nrhs)


# ---------------------------------------------------------------- generator

def test_generator_sizes_20x25():
    inst = synth.stabilized_20x25()
    p = inst.pat
    assert (p.n, p.m, len(p.edges)) == (2000, 1000, 955)
    assert p.nnz_J == 9640                       # 4 (N + 2E)
    assert 2 * p.nnz_H - p.n == 38560            # full H: 16 (N + 2E)
    assert inst.b.shape == (3000, 1)
    assert inst.delta in (0.0, 0.1, 1.0, 10.0)
    # the certificate makes H + Sigma + delta I positive definite
    Hs = O.kkt_condensed(p.n, 0, p.H_rowptr, p.H_colind, inst.H_val, np.zeros(1, np.int32),
                         np.zeros(0, np.int32), np.zeros(0), inst.Sigma, inst.delta, 1.0)
    assert np.linalg.eigvalsh(Hs.toarray()).min() > 0


def test_generator_deterministic():
    a = synth.stabilized_20x25(draw=3)
    b = synth.stabilized_20x25(draw=3)
    c = synth.stabilized_20x25(draw=4)
    assert np.array_equal(a.H_val, b.H_val) and np.array_equal(a.b, b.b)
    assert not np.array_equal(a.H_val, c.H_val)


def test_generator_edge_deletion_keeps_sizes():
    batch = synth.scenario_batch(count=3, side=6, nrhs=4)
    full = synth.make_pattern(6, 6)
    for inst in batch:
        assert inst.n == full.n and inst.m == full.m
        assert inst.pat.nnz_J < full.nnz_J and inst.pat.nnz_H < full.nnz_H
        assert inst.b.shape == (inst.n + inst.m, 4)


# ---------------------------------------------------------------- dense pins

@pytest.mark.parametrize("form", ["stabilized", "condensed"])
@pytest.mark.parametrize("shape,seed", [((1, 1), 1), ((2, 3), 2), ((3, 3), 3), ((1, 5), 4)])
@pytest.mark.parametrize("ordering", ["rcm", "natural"])
def test_dense_solve_and_inertia(form, shape, seed, ordering):
    inst = _tiny(*shape, seed, form, nrhs=2)
    A = O.instance_matrix(inst)
    fac = O.LDLT(A, O.block_signs(form, inst.n, inst.m), ordering=ordering)
    Ad = A.toarray()
    xd = np.linalg.solve(Ad, inst.b)
    x = fac.solve(inst.b)
    assert np.max(np.abs(x - xd)) <= 1e-9 * np.max(np.abs(xd))
    ev = np.linalg.eigvalsh(Ad)
    assert fac.inertia == (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    # Section 3.4: In(K2r) = (n, m, 0) and In(K) = (n, 0, 0)
    assert fac.inertia == ((inst.n, inst.m, 0) if form == "stabilized" else (inst.n, 0, 0))
    assert fac.n_perturbed == 0


def test_factor_reconstructs_matrix():
    inst = _tiny(2, 3, 7, "stabilized")
    A = O.instance_matrix(inst)
    fac = O.LDLT(A, O.block_signs("stabilized", inst.n, inst.m))
    L = fac.L().toarray()
    B = A.toarray()[np.ix_(fac.perm, fac.perm)]
    assert np.allclose(L @ np.diag(fac.D) @ L.T, B, rtol=0, atol=1e-12 * np.abs(B).max())


def test_cholesky_special_case_m0():
    """m = 0: the factorisation is the textbook Cholesky, C = L D^{1/2}."""
    inst = _tiny(3, 3, 11, "condensed")
    p = inst.pat
    A = O.kkt_condensed(p.n, 0, p.H_rowptr, p.H_colind, inst.H_val, np.zeros(1, np.int32),
                        np.zeros(0, np.int32), np.zeros(0), inst.Sigma, inst.delta, inst.rho)
    fac = O.LDLT(A, ordering="natural")
    Cc = np.linalg.cholesky(A.toarray())
    dC = np.diag(Cc)
    assert np.allclose(fac.D, dC ** 2, rtol=1e-12)
    assert np.allclose(fac.L().toarray(), Cc / dC[None, :], rtol=0, atol=1e-12)


def test_closed_form_dual_first_block_factorisation():
    """Section 3.2, Eq. ldlk2r: with the dual unknowns first, the first m
    pivots are -1/rho, L21 = -rho J^T, and the trailing factors are those of
    K = H + Sigma + delta I + rho J^T J (the condensed system)."""
    inst = _tiny(3, 4, 5, "stabilized", rho=1e3)
    n, m = inst.n, inst.m
    A = O.instance_matrix(inst)
    perm = np.concatenate([np.arange(n, n + m), np.arange(n)])
    fac = O.LDLT(A, O.block_signs("stabilized", n, m), perm=perm)
    assert np.all(fac.D[:m] == -1.0 / inst.rho)
    L = fac.L().toarray()
    p = inst.pat
    J = sp.csr_matrix((inst.J_val, p.J_colind, p.J_rowptr), shape=(m, n)).toarray()
    assert np.allclose(L[m:, :m], -inst.rho * J.T, rtol=1e-14, atol=0)
    assert np.allclose(L[:m, :m], np.eye(m))
    K = O.instance_matrix(synth.KKTInstance(pat=p, form="condensed", H_val=inst.H_val,
                                            J_val=inst.J_val, Sigma=inst.Sigma, delta=inst.delta,
                                            rho=inst.rho, b=inst.b[:n]))
    fk = O.LDLT(K, ordering="natural")
    assert np.allclose(fac.D[m:], fk.D, rtol=1e-9)
    assert np.allclose(L[m:, m:], fk.L().toarray(), rtol=0, atol=1e-9)


def test_cross_form_identity():
    """Section 3.3: the K2r solution [u; v] of [f; g] satisfies
    K u = f + rho J^T g and v = rho (J u - g)."""
    inst = _tiny(4, 5, 9, "stabilized", rho=1e4)
    n, m = inst.n, inst.m
    p = inst.pat
    x, _, eta, A = O.solve_instance(inst)
    assert eta < 1e-14
    u, v = x[:n, 0], x[n:, 0]
    f, g = inst.b[:n, 0], inst.b[n:, 0]
    J = sp.csr_matrix((inst.J_val, p.J_colind, p.J_rowptr), shape=(m, n))
    cond = synth.KKTInstance(pat=p, form="condensed", H_val=inst.H_val, J_val=inst.J_val,
                             Sigma=inst.Sigma, delta=inst.delta, rho=inst.rho,
                             b=(f + inst.rho * (J.T @ g)).reshape(n, 1))
    xk, _, _, _ = O.solve_instance(cond)
    scale = np.max(np.abs(u))
    assert np.max(np.abs(xk[:, 0] - u)) <= 1e-9 * scale
    assert np.max(np.abs(v - inst.rho * (J @ u - g))) <= 1e-8 * np.max(np.abs(v))


def test_golden_diag_H_identity_J():
    gd = read_golden(os.path.join(GOLDEN, "diag_H_identity_J.txt"))
    a = np.array(gd["a"])
    n = len(a)
    rho = gd["rho"][0]
    inst = custom_instance(np.diag(a), np.eye(n), np.zeros(n), 0.0, rho,
                           np.concatenate([gd["f"], gd["g"]]))
    x, fac, _, _ = O.solve_instance(inst)
    assert np.allclose(x[:n, 0], gd["u"], rtol=1e-15, atol=1e-15)
    assert np.allclose(x[n:, 0], gd["v"], rtol=1e-14, atol=1e-15)
    assert fac.inertia == tuple(int(t) for t in gd["inertia"])


def test_J_zero_is_block_diagonal():
    inst0 = _tiny(2, 2, 13, "stabilized")
    p = inst0.pat
    Hfull = O.kkt_condensed(p.n, 0, p.H_rowptr, p.H_colind, inst0.H_val, np.zeros(1, np.int32),
                            np.zeros(0, np.int32), np.zeros(0), np.zeros(p.n), 0.0, 1.0)
    m = 3
    inst = custom_instance(Hfull, sp.csr_matrix((m, p.n)), inst0.Sigma, inst0.delta, 7.0,
                           np.arange(p.n + m, dtype=float))
    x, fac, _, _ = O.solve_instance(inst)
    top = Hfull.toarray() + np.diag(inst0.Sigma + inst0.delta)
    assert np.allclose(x[:p.n, 0], np.linalg.solve(top, inst.b[:p.n, 0]), rtol=1e-12, atol=1e-12)
    assert np.allclose(x[p.n:, 0], -7.0 * inst.b[p.n:, 0], rtol=1e-15)


def test_golden_perturbed_pivot():
    gd = read_golden(os.path.join(GOLDEN, "perturbed_pivot_2x2.txt"))
    inst = custom_instance(np.array([[-1.0]]), np.array([[1.0]]), [1.0], 0.0, 1.0, [1.0, 0.0])
    A = O.instance_matrix(inst)
    assert np.array_equal(A.toarray(), [[0.0, 1.0], [1.0, -1.0]])
    sign = O.block_signs("stabilized", 1, 1)
    fac = O.LDLT(A, sign, ordering="natural", eps=gd["eps"][0], policy=0)
    assert fac.D[0] == gd["d0"][0]
    assert np.isclose(fac.D[1], gd["d1"][0], rtol=1e-15)
    assert np.isclose(fac.Lx[0], gd["l10"][0], rtol=1e-15)
    assert fac.inertia == tuple(int(t) for t in gd["inertia_perturb"])
    assert fac.n_perturbed == int(gd["n_perturbed"][0])
    stop = O.LDLT(A, sign, ordering="natural", eps=gd["eps"][0], policy=1)
    assert stop.inertia == tuple(int(t) for t in gd["inertia_stop"])
    assert stop.n_perturbed == 0
    # the perturbed factorisation is that of a nearby matrix: IR recovers x
    x, steps, eta = O.solve_ir(A, fac, inst.b[:, 0], max_steps=10, tol=1e-15)
    assert np.allclose(x, np.linalg.solve(A.toarray(), inst.b[:, 0]), rtol=1e-9)


def test_dual_perturbation_sign():
    """A dual zero pivot is replaced by -eps (sign of its block)."""
    # K2r with the dual index first and a zero dual block entry: rho -> inf
    inst = custom_instance(np.array([[2.0]]), np.array([[1.0]]), [0.0], 0.0, 1e300, [1.0, 1.0])
    A = O.instance_matrix(inst)
    fac = O.LDLT(A, O.block_signs("stabilized", 1, 1), perm=np.array([1, 0]))
    assert fac.D[0] == -1e-10 and fac.n_perturbed == 1
    assert fac.inertia == (1, 1, 0)


@pytest.mark.parametrize("form", ["stabilized", "condensed"])
def test_sqd_inertia_and_residual_20x25(form):
    inst = synth.stabilized_20x25()
    if form == "condensed":
        inst = synth.KKTInstance(pat=inst.pat, form="condensed", H_val=inst.H_val,
                                 J_val=inst.J_val, Sigma=inst.Sigma, delta=inst.delta,
                                 rho=inst.rho, b=inst.b[:inst.n])
    x, fac, eta, A = O.solve_instance(inst)
    assert fac.inertia == ((2000, 1000, 0) if form == "stabilized" else (2000, 0, 0))
    assert fac.n_perturbed == 0
    assert eta <= 1e-12


# ---------------------------------------------------------------- adjoint pins

def _loss_and_parts(inst, w):
    x, _, _, _ = O.solve_instance(inst, ir_steps=3)
    return float(np.sum(w * x))


@pytest.mark.parametrize("form", ["stabilized", "condensed"])
def test_adjoint_vs_central_differences(form):
    inst = _tiny(2, 3, 21, form, rho=50.0)
    rng = np.random.default_rng(0)
    w = rng.standard_normal(inst.b.shape)
    x, fac, _, A = O.solve_instance(inst)
    g = O.adjoint(inst, fac, A, x, w)

    def fd(get, setv, idx):
        v0 = get()[idx]
        h = 1e-6 * max(1.0, abs(v0))
        setv(idx, v0 + h)
        lp = _loss_and_parts(inst, w)
        setv(idx, v0 - h)
        lm = _loss_and_parts(inst, w)
        setv(idx, v0)
        return (lp - lm) / (2 * h)

    def setter(arr):
        def s(i, v):
            arr[i] = v
        return s

    for name, arr in (("g_H", inst.H_val), ("g_J", inst.J_val), ("g_Sigma", inst.Sigma),
                      ("g_b", inst.b.reshape(-1))):
        for idx in rng.choice(len(arr), size=min(6, len(arr)), replace=False):
            ref = fd(lambda: arr, setter(arr), idx)
            got = g[name].reshape(-1)[idx]
            assert abs(got - ref) <= 1e-6 * max(1.0, abs(ref)), (name, idx, got, ref)
    for name, attr in (("g_delta", "delta"), ("g_rho", "rho")):
        box = [getattr(inst, attr)]

        def sset(i, v, attr=attr):
            setattr(inst, attr, v)
        ref = fd(lambda: [getattr(inst, attr)], sset, 0)
        assert abs(g[name] - ref) <= 1e-6 * max(1.0, abs(ref)), (name, g[name], ref)
        del box


@pytest.mark.parametrize("form", ["stabilized", "condensed"])
def test_adjoint_vs_dense_autograd(form):
    """10x10 grid (n+m = 600 for K2r): gradients of w^T x against torch
    autograd through a dense FP64 torch.linalg.solve."""
    torch = pytest.importorskip("torch")
    inst = _tiny(10, 10, 31, form, rho=1e4)
    p = inst.pat
    n, m = p.n, p.m
    rng = np.random.default_rng(1)
    w = rng.standard_normal(inst.b.shape)
    x, fac, _, A = O.solve_instance(inst)
    g = O.adjoint(inst, fac, A, x, w)

    t = lambda a: torch.tensor(np.asarray(a, float), dtype=torch.float64, requires_grad=True)
    Hv, Jv, S, b = t(inst.H_val), t(inst.J_val), t(inst.Sigma), t(inst.b)
    rows = torch.tensor(np.repeat(np.arange(n), np.diff(p.H_rowptr)))
    cols = torch.tensor(p.H_colind.astype(np.int64))
    Jr = torch.tensor(np.repeat(np.arange(m), np.diff(p.J_rowptr)))
    Jc = torch.tensor(p.J_colind.astype(np.int64))
    Hd = torch.zeros(n, n, dtype=torch.float64).index_put((rows, cols), Hv, accumulate=True)
    off = rows != cols
    Hd = Hd.index_put((cols[off], rows[off]), Hv[off], accumulate=True)
    Hd = Hd + torch.diag(S + inst.delta)
    Jd = torch.zeros(m, n, dtype=torch.float64).index_put((Jr, Jc), Jv, accumulate=True)
    if form == "stabilized":
        K = torch.cat([torch.cat([Hd, Jd.T], 1),
                       torch.cat([Jd, -torch.eye(m, dtype=torch.float64) / inst.rho], 1)], 0)
    else:
        K = Hd + inst.rho * Jd.T @ Jd
    X = torch.linalg.solve(K, b)
    (X * torch.tensor(w)).sum().backward()
    for name, tt in (("g_H", Hv), ("g_J", Jv), ("g_Sigma", S), ("g_b", b)):
        ref = tt.grad.numpy().reshape(-1)
        got = np.asarray(g[name]).reshape(-1)
        assert np.max(np.abs(got - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref))), name


# ---------------------------------------------------------------- planted mistakes

def test_planted_mistake_dual_block_sign(monkeypatch):
    """A sign error in the (2,2) block of K2r breaks the cross-form identity
    (any rho) and the inertia pin (small rho)."""
    orig = O.kkt_stabilized

    def bad(n, m, *a):
        K = orig(n, m, *a).tolil()
        for i in range(n, n + m):
            K[i, i] = -K[i, i]
        return K.tocsc()
    monkeypatch.setattr(O.oracle, "kkt_stabilized", bad)
    inst = _tiny(2, 3, 3, "stabilized", rho=0.01)
    A = O.oracle.instance_matrix(inst)
    fac = O.LDLT(A, O.block_signs("stabilized", inst.n, inst.m))
    assert fac.inertia != (inst.n, inst.m, 0)
    inst = _tiny(2, 3, 3, "stabilized", rho=1e4)
    n, m, p = inst.n, inst.m, inst.pat
    A = O.oracle.instance_matrix(inst)
    u = O.LDLT(A, O.block_signs("stabilized", n, m)).solve(inst.b)[:n, 0]
    J = sp.csr_matrix((inst.J_val, p.J_colind, p.J_rowptr), shape=(m, n))
    K = O.kkt_condensed(n, m, p.H_rowptr, p.H_colind, inst.H_val, p.J_rowptr, p.J_colind,
                        inst.J_val, inst.Sigma, inst.delta, inst.rho)
    rhs = inst.b[:n, 0] + inst.rho * (J.T @ inst.b[n:, 0])
    assert not np.allclose(K @ u, rhs, rtol=1e-6, atol=1e-6)


def test_planted_mistake_dropped_sigma(monkeypatch):
    """Dropping Sigma from the (1,1) block breaks the golden closed form."""
    orig = O.kkt_stabilized

    def bad(n, m, Hp, Hi, Hv, Jp, Ji, Jv, Sigma, delta, rho):
        return orig(n, m, Hp, Hi, Hv, Jp, Ji, Jv, np.zeros_like(Sigma), delta, rho)
    monkeypatch.setattr(O.oracle, "kkt_stabilized", bad)
    gd = read_golden(os.path.join(GOLDEN, "diag_H_identity_J.txt"))
    n = 2
    inst = custom_instance(np.zeros((n, n)), np.eye(n), np.array(gd["a"]), 0.0, gd["rho"][0],
                           np.concatenate([gd["f"], gd["g"]]))
    A = O.oracle.instance_matrix(inst)
    x = O.LDLT(A, O.block_signs("stabilized", n, n)).solve(inst.b)
    assert not np.allclose(x[:n, 0], gd["u"], rtol=1e-6)


def test_planted_mistake_wrong_pivot(monkeypatch):
    """Corrupting one pivot of the factorisation breaks the dense pin."""
    inst = _tiny(2, 3, 17, "stabilized")
    A = O.instance_matrix(inst)
    fac = O.LDLT(A, O.block_signs("stabilized", inst.n, inst.m))
    fac.D[3] *= 1.001
    xd = np.linalg.solve(A.toarray(), inst.b)
    assert np.max(np.abs(fac.solve(inst.b) - xd)) > 1e-9 * np.max(np.abs(xd))


def test_planted_mistake_transposed_J_in_condensed(monkeypatch):
    """Using J J^T-like coupling (a transposed operand) in the condensed
    form breaks the cross-form identity."""
    inst = _tiny(2, 2, 19, "stabilized", rho=100.0)
    n, m, p = inst.n, inst.m, inst.pat
    J = sp.csr_matrix((inst.J_val, p.J_colind, p.J_rowptr), shape=(m, n))
    x, _, _, _ = O.solve_instance(inst)
    u = x[:n, 0]
    f, g = inst.b[:n, 0], inst.b[n:, 0]
    Kgood = O.kkt_condensed(n, m, p.H_rowptr, p.H_colind, inst.H_val, p.J_rowptr, p.J_colind,
                            inst.J_val, inst.Sigma, inst.delta, inst.rho)
    assert np.allclose(Kgood @ u, f + inst.rho * (J.T @ g), rtol=1e-9, atol=1e-9)
    Jt = J.toarray()
    bad = Kgood.toarray() - inst.rho * Jt.T @ Jt + inst.rho * np.kron(np.eye(2), Jt @ Jt.T)[:n, :n]
    assert not np.allclose(bad @ u, f + inst.rho * (J.T @ g), rtol=1e-6, atol=1e-6)


# ------------------------------------------------- inertia correction (Section 3.1)

def _scalar_instance(form):
    gd = read_golden(os.path.join(GOLDEN, "regularize_scalar.txt"))
    inst = custom_instance(np.array([[gd["h"][0]]]), np.array([[1.0]]), np.zeros(1), 0.0, gd["rho"][0],
                           np.ones(2 if form == "stabilized" else 1), form=form)
    return inst, gd


@pytest.mark.parametrize("form", ["stabilized", "condensed"])
def test_regularize_golden_scalar(form):
    inst, gd = _scalar_instance(form)
    fac, A, delta, tries, regular = O.regularize(inst, 0.0, gd["delta_first"][0], gd["growth"][0])
    assert regular and tries == int(gd["tries"][0]) and delta == gd["delta"][0]
    assert fac.inertia == tuple(int(v) for v in gd[f"inertia_{form}"])


def test_regularize_m0_is_the_shifted_spectrum():
    """m = 0: the loop stops at the first delta of the schedule above
    -lambda_min(H + Sigma) (textbook: H + Sigma + delta I is SPD iff
    delta > -lambda_min)."""
    lam = np.array([-2.5, 0.3, 1.0, 4.0, -0.7, 2.0])
    Q, _ = np.linalg.qr(np.random.default_rng(5).standard_normal((6, 6)))
    H = Q @ np.diag(lam) @ Q.T
    inst = custom_instance(H, np.zeros((0, 6)), np.zeros(6), 0.0, 1.0, np.ones(6), form="condensed")
    fac, A, delta, tries, regular = O.regularize(inst, 0.0, 1e-4, 10.0)
    sched = [0.0] + [1e-4 * 10.0 ** k for k in range(20)]
    want = next(i for i, d in enumerate(sched) if lam.min() + d > 0)
    assert regular and tries == want + 1 and np.isclose(delta, sched[want], rtol=1e-12)
    assert fac.inertia == (6, 0, 0)


@pytest.mark.parametrize("form", ["stabilized", "condensed"])
def test_regularize_matches_dense_eigenvalues(form):
    """On a tiny grid started at delta = 0 the loop's stopping delta is the
    first of the schedule at which the dense FP64 eigenvalues of the
    regularised matrix (rho-hat = rho + delta) have the regular inertia."""
    inst = _tiny(3, 3, 23, form, rho=0.5)
    p = inst.pat
    build = O.kkt_stabilized if form == "stabilized" else O.kkt_condensed
    want = (inst.n, inst.m if form == "stabilized" else 0, 0)
    sched = [0.0] + [1e-2 * 3.0 ** k for k in range(30)]
    stop = None
    for i, d in enumerate(sched):
        K = build(p.n, p.m, p.H_rowptr, p.H_colind, inst.H_val, p.J_rowptr, p.J_colind, inst.J_val,
                  inst.Sigma, d, inst.rho + d).toarray()
        ev = np.linalg.eigvalsh(K)
        assert np.min(np.abs(ev)) > 1e-8 * np.max(np.abs(ev))      # no decision near zero
        if ((ev > 0).sum(), (ev < 0).sum(), 0) == want:
            stop = i
            break
    assert stop is not None and stop > 0          # the test needs at least one correction
    fac, A, delta, tries, regular = O.regularize(inst, 0.0, 1e-2, 3.0, max_tries=40)
    assert regular and tries == stop + 1 and np.isclose(delta, sched[stop], rtol=1e-12)


def test_regularize_gives_up_after_max_tries():
    inst, gd = _scalar_instance("stabilized")
    fac, A, delta, tries, regular = O.regularize(inst, 0.0, gd["delta_first"][0], gd["growth"][0], max_tries=2)
    assert not regular and tries == 2 and delta == gd["delta_first"][0]


def test_planted_mistake_rho_hat_not_raised(monkeypatch):
    """Leaving rho-hat at rho while delta grows breaks the golden scalar pin."""
    orig = O.kkt_stabilized
    inst, gd = _scalar_instance("stabilized")

    def bad(n, m, Hp, Hi, Hv, Jp, Ji, Jv, Sigma, delta, rho):
        return orig(n, m, Hp, Hi, Hv, Jp, Ji, Jv, Sigma, delta, inst.rho)
    monkeypatch.setattr(O.oracle, "kkt_stabilized", bad)
    fac, A, delta, tries, regular = O.oracle.regularize(inst, 0.0, gd["delta_first"][0], gd["growth"][0])
    assert (delta, tries) != (gd["delta"][0], int(gd["tries"][0]))


# ------------------------------------------- condensed form with slacks (Eq. K1s)

def _k1s_case(seed=31, R=3, C=4, rho=50.0):
    inst = _tiny(R, C, seed, "condensed", rho=rho)
    rng = np.random.default_rng(seed)
    Ss = 10.0 ** rng.uniform(-2, 2, inst.m)
    Ss[rng.random(inst.m) < 0.4] = np.inf          # equality rows
    return inst, Ss


def _k1s_matrix(inst, Ss):
    p = inst.pat
    return O.kkt_condensed_slack(p.n, p.m, p.H_rowptr, p.H_colind, inst.H_val, p.J_rowptr, p.J_colind,
                                 inst.J_val, inst.Sigma, Ss, inst.delta, inst.rho)


def test_k1s_matches_the_unreduced_slack_system():
    """Solving Eq. K1s for Delta t and recovering Delta s gives the solution of
    the unreduced two-block system in (Delta t, Delta s) of Section 3.3 (Eq.
    K1'), assembled and solved densely here from its own blocks.  The
    right-hand side is the one the proof's elimination of Delta s produces,
    r_t + rho J_I^T (Sigma_s + rho I)^{-1} r_s (the statement of Eq. K1s
    prints it without the inverse, which this pin rejects)."""
    inst, Ss = _k1s_case()
    p, rho = inst.pat, inst.rho
    n, m = p.n, p.m
    Hd = O.kkt_condensed(n, 0, p.H_rowptr, p.H_colind, inst.H_val, np.zeros(1, np.int32), np.zeros(0, np.int32),
                         np.zeros(0), inst.Sigma, inst.delta, 1.0).toarray()
    J = sp.csr_matrix((inst.J_val, p.J_colind, p.J_rowptr), shape=(m, n)).toarray()
    I = np.flatnonzero(np.isfinite(Ss))
    JI = J[I]
    Kt = Hd + rho * J.T @ J                          # W_t + Sigma_t + delta I + rho (J_E^T J_E + J_I^T J_I)
    big = np.block([[Kt, -rho * JI.T], [-rho * JI, np.diag(Ss[I] + rho)]])
    rng = np.random.default_rng(4)
    rt, rsI = rng.standard_normal(n), rng.standard_normal(len(I))
    sol = np.linalg.solve(big, np.concatenate([rt, rsI]))
    A = _k1s_matrix(inst, Ss)
    fac = O.LDLT(A)
    rs = np.zeros(m)
    rs[I] = rsI
    rhs = O.k1s_rhs(m, p.J_rowptr, p.J_colind, inst.J_val, n, Ss, rho, rt, rs)[:, 0]
    assert not np.allclose(rhs, rt + rho * JI.T @ rsI)   # the printed form differs
    dt, _, eta = O.solve_ir(A, fac, rhs)
    assert eta <= 1e-12
    assert np.allclose(dt, sol[:n], rtol=1e-9, atol=1e-12)
    ds = O.k1s_slack_step(m, p.J_rowptr, p.J_colind, inst.J_val, n, Ss, rho, dt, rs)[:, 0]
    assert np.allclose(ds[I], sol[n:], rtol=1e-9, atol=1e-12)
    assert np.all(ds[np.isinf(Ss)] == 0.0)


def test_k1s_limits():
    """Sigma_s -> inf on every row gives Eq. K1 exactly (Omega = 1); Sigma_s = 0
    removes the inequality rows (Omega = 0)."""
    inst, _ = _k1s_case(seed=32)
    p = inst.pat
    K1 = O.kkt_condensed(p.n, p.m, p.H_rowptr, p.H_colind, inst.H_val, p.J_rowptr, p.J_colind, inst.J_val,
                         inst.Sigma, inst.delta, inst.rho)
    assert abs(_k1s_matrix(inst, np.full(p.m, np.inf)) - K1).max() == 0.0
    mask = np.arange(p.m) % 2 == 0
    Ss = np.where(mask, np.inf, 0.0)
    J = sp.csr_matrix((inst.J_val, p.J_colind, p.J_rowptr), shape=(p.m, p.n))
    JE = J[np.flatnonzero(mask)]
    want = O.kkt_condensed(p.n, 0, p.H_rowptr, p.H_colind, inst.H_val, np.zeros(1, np.int32),
                           np.zeros(0, np.int32), np.zeros(0), inst.Sigma, inst.delta, 1.0) + inst.rho * (JE.T @ JE)
    assert abs(_k1s_matrix(inst, Ss) - want).max() <= 1e-12 * abs(want).max()


def test_planted_mistake_inverted_omega(monkeypatch):
    """Omega = rho / (rho + Sigma_s) instead of Sigma_s / (rho + Sigma_s)
    breaks the unreduced-system pin."""
    orig = O.kkt_condensed_slack

    def bad(n, m, Hp, Hi, Hv, Jp, Ji, Jv, St, Ss, delta, rho):
        Ss = np.asarray(Ss, float)
        fin = np.isfinite(Ss)
        alt = Ss.copy()
        alt[fin] = rho * rho / np.maximum(Ss[fin], 1e-300)   # Omega' = rho / (rho + Sigma_s)
        return orig(n, m, Hp, Hi, Hv, Jp, Ji, Jv, St, alt, delta, rho)
    monkeypatch.setattr(O.oracle, "kkt_condensed_slack", bad)
    monkeypatch.setattr(O, "kkt_condensed_slack", bad)
    with pytest.raises(AssertionError):
        test_k1s_matches_the_unreduced_slack_system()


# ------------------------------------------------ Newton step (Section 3.1-3.3)

def _k3_dense(inst, pt, mu):
    """Eq. K3 assembled from its blocks (finite bounds only carry a z row and
    column; an infinite bound has no multiplier) and solved densely.
    Returns dx, dr, dy, dz_lower, dz_upper (zeros where the bound is infinite)."""
    p = inst.pat
    n, m, rho = p.n, p.m, inst.rho
    H = O.kkt_condensed(n, 0, p.H_rowptr, p.H_colind, inst.H_val, np.zeros(1, np.int32), np.zeros(0, np.int32),
                        np.zeros(0), np.zeros(n), 0.0, 1.0).toarray()
    J = sp.csr_matrix((inst.J_val, p.J_colind, p.J_rowptr), shape=(m, n)).toarray()
    x, lo, up, zl, zu = pt["x"], pt["lower"], pt["upper"], pt["z_lower"], pt["z_upper"]
    BL, BU = np.flatnonzero(np.isfinite(lo)), np.flatnonzero(np.isfinite(up))
    nl, nu = len(BL), len(BU)
    N = n + 2 * m + nl + nu
    K = np.zeros((N, N))
    ix, ir, iy = slice(0, n), slice(n, n + m), slice(n + m, n + 2 * m)
    il, iu = n + 2 * m + np.arange(nl), n + 2 * m + nl + np.arange(nu)
    K[ix, ix] = H
    K[ix, iy] = -J.T
    K[BL, il] = -1.0
    K[BU, iu] = 1.0
    K[ir, ir] = rho * np.eye(m)
    K[ir, iy] = -np.eye(m)
    K[iy, ix] = J
    K[iy, ir] = np.eye(m)
    K[il, BL] = zl[BL]
    K[il, il] = (x - lo)[BL]
    K[iu, BU] = -zu[BU]
    K[iu, iu] = (up - x)[BU]
    rhs = -np.concatenate([pt["grad_phi"] - J.T @ pt["y"] - zl + zu, pt["y_k"] + rho * pt["r"] - pt["y"],
                           pt["c"] + pt["r"], zl[BL] * (x - lo)[BL] - mu, zu[BU] * (up - x)[BU] - mu])
    sol = np.linalg.solve(K, rhs)
    dzl, dzu = np.zeros(n), np.zeros(n)
    dzl[BL], dzu[BU] = sol[il], sol[iu]
    return sol[ix], sol[ir], sol[iy], dzl, dzu


def _newton_case(form, seed=41):
    from tests.helpers import newton_point
    inst = _tiny(2, 3, seed, form, rho=20.0)
    pt, sigma = newton_point(inst, seed)
    return inst, pt, sigma


@pytest.mark.parametrize("form", ["stabilized", "condensed"])
def test_newton_step_matches_the_full_newton_system(form):
    """Solving the factored system (Eq. K2r or K1, with Sigma from the point,
    delta = 0) with the oracle's right-hand side and recovering the other
    components reproduces the dense solution of Eq. K3."""
    inst, pt, sigma = _newton_case(form)
    p, mu = inst.pat, 0.05
    build = O.kkt_stabilized if form == "stabilized" else O.kkt_condensed
    A = build(p.n, p.m, p.H_rowptr, p.H_colind, inst.H_val, p.J_rowptr, p.J_colind, inst.J_val, sigma, 0.0,
              inst.rho)
    b = O.newton_rhs(form, p.n, p.m, p.J_rowptr, p.J_colind, inst.J_val, pt, mu, inst.rho)
    X, _, eta = O.solve_ir(A, O.LDLT(A, O.block_signs(form, p.n, p.m)), b)
    assert eta <= 1e-12
    rec = O.newton_recover(form, p.n, p.m, p.J_rowptr, p.J_colind, inst.J_val, pt, mu, inst.rho, X)
    dx, dr, dy, dzl, dzu = _k3_dense(inst, pt, mu)
    scale = max(1.0, np.max(np.abs(np.concatenate([dx, dr, dy, dzl, dzu]))))
    for got, want in ((rec["dx"], dx), (rec["dr"], dr), (rec["dy"], dy), (rec["dz_lower"], dzl),
                      (rec["dz_upper"], dzu)):
        assert np.max(np.abs(got - want)) <= 1e-9 * scale


def test_planted_mistake_dropped_barrier_term(monkeypatch):
    """Dropping the barrier gradient from the right-hand side breaks the
    full-Newton-system pin."""
    orig = O.newton_rhs

    def bad(form, n, m, Jp, Ji, Jv, pt, mu, rho):
        return orig(form, n, m, Jp, Ji, Jv, pt, 0.0, rho)
    monkeypatch.setattr(O, "newton_rhs", bad)
    with pytest.raises(AssertionError):
        test_newton_step_matches_the_full_newton_system("stabilized")


# ------------------------------------------------ helpers that set the parity bar

def test_backward_error_hand_computed():
    """eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf), worked by hand:
    A = [[2, 1], [1, 3]], x = [1, 1], b = [3, 5]: r = [0, 1], ||A||_inf = 4,
    ||x||_inf = 1, ||b||_inf = 5, so eta = 1/9; a second column with the exact
    solution has eta = 0 and the largest column is reported."""
    A = sp.csr_matrix(np.array([[2.0, 1.0], [1.0, 3.0]]))
    assert O.backward_error(A, np.array([1.0, 1.0]), np.array([3.0, 5.0])) == pytest.approx(1.0 / 9.0, rel=1e-15)
    X = np.array([[1.0, 0.4], [1.0, 0.8]])          # column 2 solves A x = [1.6, 2.8] exactly
    B = np.array([[3.0, 1.6], [5.0, 2.8]])
    assert O.backward_error(A, X, B) == pytest.approx(1.0 / 9.0, rel=1e-15)
    assert O.backward_error(A, X[:, 1], B[:, 1]) <= 1e-16
    # invariant under a common scaling of A and b (x unchanged)
    assert O.backward_error(7.0 * A, np.array([1.0, 1.0]), 7.0 * np.array([3.0, 5.0])) == pytest.approx(1.0 / 9.0)


def test_cond1_estimate_against_the_exact_condition_number():
    """kappa_1 of a small SPD and an SQD matrix against ||A||_1 ||A^-1||_1
    from a dense inverse (the estimate is a lower bound, exact on these
    sizes), and exactly max|d| / min|d| for a diagonal matrix."""
    rng = np.random.default_rng(3)
    for form in ("stabilized", "condensed"):
        inst = _tiny(2, 2, 5, form, rho=10.0)
        A = O.instance_matrix(inst)
        fac = O.LDLT(A, O.block_signs(form, inst.n, inst.m))
        Ad = A.toarray()
        exact = np.linalg.norm(Ad, 1) * np.linalg.norm(np.linalg.inv(Ad), 1)
        est = O.cond1_estimate(A, fac)
        assert exact / 3.0 <= est <= exact * (1 + 1e-10)
    d = rng.uniform(0.1, 10.0, 12) * rng.choice([-1.0, 1.0], 12)
    D = sp.diags(d, format="csc")
    est = O.cond1_estimate(D, O.LDLT(D, np.where(d > 0, 1, -1).astype(np.int32)))
    assert est == pytest.approx(np.max(np.abs(d)) / np.min(np.abs(d)), rel=1e-12)


def _true_min_power(Hs_at):
    """Smallest delta in {0} U {10^k} with H + Sigma + delta I positive definite,
    from the eigenvalues (Hs_at(delta) gives the dense matrix)."""
    lam = np.linalg.eigvalsh(Hs_at(0.0)).min()
    if lam > 0:
        return 0.0
    k = int(np.floor(np.log10(-lam)))
    while np.linalg.eigvalsh(Hs_at(10.0 ** k)).min() <= 0:
        k += 1
    return 10.0 ** k


def test_certified_delta_against_true_smallest_power():
    """The generator's delta (a sufficient certificate, no factorisation)
    against the true smallest power of ten from the eigenvalues, on 40 small
    grids: never below it, at most one power above it.  The count of
    instances where it is one power above is printed (-s)."""
    rng = np.random.default_rng(11)
    above = 0
    for t in range(40):
        R, C = int(rng.integers(5, 11)), int(rng.integers(5, 11))
        inst = synth.random_instance(R, C, seed=1000 + t, form="condensed", rho=1.0)
        p = inst.pat

        def Hs_at(d):
            return O.kkt_condensed(p.n, 0, p.H_rowptr, p.H_colind, inst.H_val, np.zeros(1, np.int32),
                                   np.zeros(0, np.int32), np.zeros(0), inst.Sigma, d, 1.0).toarray()
        true = _true_min_power(Hs_at)
        assert inst.delta >= true
        assert true == 0.0 or inst.delta <= 10.0 * true
        above += inst.delta > true
    print(f"certified delta above the true smallest power of ten in {above} of 40 instances")
