"""The tcgen05 split-TF32 update kernel in isolation, against an FP64 torch
reference of the same product: C -= L_a diag(d) L_b^T on the lower part."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K,row_a,row_b", [
    (128, 128, 32, 0, 0),        # one tile, one K stage
    (64, 64, 8, 3, 3),           # ragged everything, smaller than a tile
    (300, 250, 100, 5, 57),      # ragged M, N, K; several tiles; N < M
    (513, 513, 700, 0, 0),       # many K stages (pipeline wraps), ragged tail
    (1000, 129, 33, 0, 871),     # tall, two column tiles
])
def test_tensor_update_matches_fp64(M, N, K, row_a, row_b):
    from paper_2510_05885_gb300 import ncl_kkt as nk
    g = torch.Generator(device="cpu").manual_seed(M * 7 + K)
    rows = max(row_a + M, row_b + N) + 3
    ld = (K + 3) // 4 * 4 + 4
    L = torch.randn(rows, ld, generator=g, dtype=torch.float32)
    d = torch.randn(K, generator=g, dtype=torch.float32)
    C = torch.randn(M, N + 5, generator=g, dtype=torch.float32)
    A = L[row_a:row_a + M, :K].double()
    B = L[row_b:row_b + N, :K].double()
    upd = (A * d.double()) @ B.T
    scale = (A.abs() * d.double().abs()) @ B.abs().T
    mask = torch.zeros(M, N + 5, dtype=torch.bool)
    mask[:, :N] = torch.tril(torch.ones(M, N, dtype=torch.bool))
    ref = C.double().clone()
    ref[:, :N] -= torch.where(mask[:, :N], upd, torch.zeros_like(upd))
    Cd = C.cuda()
    nk.ncl_kkt_selftest_tensor_update(L.cuda(), d.cuda(), K, row_a, row_b, M, N, Cd)
    out = Cd.cpu().double()
    err = (out - ref).abs()
    tol = 2e-6 * torch.cat([scale, torch.zeros(M, 5, dtype=torch.float64)], 1) + 1e-6 * C.double().abs() + 1e-6
    assert torch.all(err[mask] <= tol[mask]), float((err[mask] / tol[mask]).max())
    # entries above the diagonal and beyond column N are left untouched
    assert torch.equal(out[~mask], C.double()[~mask])
