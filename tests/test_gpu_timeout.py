"""Failure detection of the bounded inter-CTA waits, without faulting or
hanging anything.

Every wait of one CTA on another inside the kernels (the chained triangular
sweeps, the macro panel's row CTAs waiting for the diagonal block, the
tensor-core pipeline) gives up after options.wait_cycles clock cycles, sets
the call's error flag and lets the kernel finish; the host reports
NCL_ERR_TIMEOUT.  ncl_kkt_selftest_wait_timeout launches a real sweep or
panel kernel arranged so that one awaited flag is never published, with a
short limit: the launch must return, report the timeout, and leave the
handle usable (the same solution after the sweep test; a refactor after
the panel test, whose row CTAs went on without the diagonal block).
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_05885_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT = 9
STATE = 5


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda:0")


@pytest.mark.parametrize("prec,eta_tol", [("fp32_ir", 1e-10), ("fp64", 1e-12)])
def test_wait_limit_runs_out_and_handle_recovers(prec, eta_tol):
    from paper_2510_05885_gb300 import ncl_kkt as nk
    inst = synth.random_instance(40, 40, seed=140, form="stabilized", rho=1e4)
    p = inst.pat
    K = nk.KKT(0, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec=prec)
    A = O.instance_matrix(inst)
    args = (_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), inst.delta, inst.rho)
    K.factor(*args)
    X0, s0 = K.solve(_t(inst.b))
    x0 = X0.cpu().numpy()
    assert s0.status == 0 and O.backward_error(A, x0, inst.b) <= eta_tol

    # a chained sweep whose first block-row never publishes: about 50 us of waiting
    assert nk.ncl_kkt_selftest_wait_timeout(K._h, 0, 100000) == TIMEOUT
    X1, s1 = K.solve(_t(inst.b))                # the factors are untouched
    assert s1.status == 0
    assert np.array_equal(X1.cpu().numpy(), x0)

    # macro-panel row CTAs whose diagonal block never comes
    assert nk.ncl_kkt_selftest_wait_timeout(K._h, 1, 100000) == TIMEOUT
    with pytest.raises(nk.NclError) as e:
        K.solve(_t(inst.b))
    assert e.value.status == STATE
    finfo = K.factor(*args)
    assert finfo.inertia == (inst.n, inst.m, 0)
    X2, s2 = K.solve(_t(inst.b))
    assert s2.status == 0
    assert np.array_equal(X2.cpu().numpy(), x0)  # same factors, same sweeps: bitwise
    K.close()


def test_short_wait_limit_option_is_honoured_when_nothing_waits_long():
    """A handle whose wait_cycles is short but still far above what a real
    wait takes on this small system factors and solves normally."""
    from paper_2510_05885_gb300 import ncl_kkt as nk
    inst = synth.random_instance(20, 20, seed=141, form="stabilized", rho=1e4)
    p = inst.pat
    K = nk.KKT(0, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec="fp32_ir",
               wait_cycles=200000000)
    K.factor(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), inst.delta, inst.rho)
    X, s = K.solve(_t(inst.b))
    assert s.status == 0
    assert O.backward_error(O.instance_matrix(inst), X.cpu().numpy(), inst.b) <= 1e-10
    K.close()


def test_selftest_arguments():
    from paper_2510_05885_gb300 import ncl_kkt as nk
    inst = synth.random_instance(3, 3, seed=142, form="stabilized", rho=1e4)
    p = inst.pat
    K = nk.KKT(0, p.n, p.m, p.H_rowptr, p.H_colind, p.J_rowptr, p.J_colind, prec="fp64")
    with pytest.raises(nk.NclError) as e:
        nk.ncl_kkt_selftest_wait_timeout(K._h, 0, 1000)       # before a factor
    assert e.value.status == STATE
    K.factor(_t(inst.H_val), _t(inst.J_val), _t(inst.Sigma), inst.delta, inst.rho)
    with pytest.raises(nk.NclError) as e:
        nk.ncl_kkt_selftest_wait_timeout(K._h, 0, 1000)       # no supernode of two block-rows here
    assert e.value.status == 1
    with pytest.raises(nk.NclError):
        nk.ncl_kkt_selftest_wait_timeout(K._h, 2, 1000)
    with pytest.raises(nk.NclError):
        nk.ncl_kkt_selftest_wait_timeout(K._h, 0, 0)
    K.close()
