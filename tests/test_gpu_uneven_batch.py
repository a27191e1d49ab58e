"""GPU parity of a batch of uneven instances: sixteen stabilized grids of
5..20 buses a side (patterns and sizes all different), one block-diagonal
handle, the one-graph factor + solve entry point, two right-hand sides;
each instance against its own oracle solve (the tolerances of
test_gpu_parity)."""
import numpy as np
import pytest

from paper_2510_05885_gb300 import synth
from tests.test_gpu_parity import DEV, _t, check_against_oracle, nk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def uneven_instances():
    rng = np.random.default_rng(21)
    return [synth.random_instance(5 + t, int(rng.integers(5, 21)), seed=300 + t, form="stabilized", rho=1e4,
                                  nrhs=2) for t in range(16)]


@pytest.mark.parametrize("prec,eta_tol", [("fp64", 1e-12), ("fp32_ir", 1e-10)])
def test_batch_16_uneven_sides(prec, eta_tol):
    batch = uneven_instances()
    assert len({i.dim for i in batch}) > 8
    pats = [(i.n, i.m, i.pat.H_rowptr, i.pat.H_colind, i.pat.J_rowptr, i.pat.J_colind) for i in batch]
    K = nk().KKT.batch(0, pats, prec=prec)
    Hv = _t(np.concatenate([i.H_val for i in batch]))
    Jv = _t(np.concatenate([i.J_val for i in batch]))
    S = _t(np.concatenate([i.Sigma for i in batch]))
    B = np.concatenate([i.b for i in batch], axis=0)
    Bc = _t(B.T.copy())
    Xc = torch.empty_like(Bc)
    infos, sinfo = nk().ncl_kkt_batch_factor_solve(K._h, Hv, Jv, S, [i.delta for i in batch],
                                                   [i.rho for i in batch], 2, Bc, K.dim, Xc, K.dim)
    torch.cuda.synchronize()
    assert sinfo.status == 0
    X = Xc.cpu().numpy().T
    off = 0
    for inst, fi in zip(batch, infos):
        assert fi.inertia == (inst.n, inst.m, 0)
        check_against_oracle(inst, prec, X[off:off + inst.dim], fi, sinfo, eta_tol)
        off += inst.dim
    assert off == K.dim
