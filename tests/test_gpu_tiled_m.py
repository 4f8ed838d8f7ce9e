"""GPU tests of the tiled M: with wide increments (d > 8, FP32) each warp computes a strip's
M_ij = <dx_i, dy_j> / 4^lambda for all columns at once, with every operand row loaded once for 32
cells, instead of each cell reading two increment rows.  The inner products run in the same order
as the per-cell form, so every result must agree bit for bit with SK_FLAG_NO_TILED_M; the oracle
pins both on sampled pairs.  (The approximation scheme computes M on the tensor cores by default
for 8 < d <= 32; these tests turn that off to compare the two FMA-pipe forms.)
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2502_08470_gb300 import workloads as W

pytestmark = pytest.mark.gpu

sk = pytest.importorskip("paper_2502_08470_gb300.sigkernel")


@pytest.fixture(scope="module", autouse=True)
def _cuda_available():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _paths(seed, lengths, d):
    return [W.brownian(1, n, d, seed=seed + i)[0] for i, n in enumerate(lengths)]


@pytest.mark.parametrize("d", [20, 37])
@pytest.mark.parametrize("scheme,N,lam", [("approx", 6, 0), ("approx", 5, 1), ("interp", 7, 0)])
@pytest.mark.parametrize("pipeline", [False, True])
def test_tiled_m_is_bitwise_the_per_cell_m(d, scheme, N, lam, pipeline):
    Xs = _paths(201, [130, 40, 257, 9], d)
    Ys = _paths(301, [100, 33, 260], d)
    X = sk.Paths.from_list([torch.tensor(x) for x in Xs])
    Y = sk.Paths.from_list([torch.tensor(y) for y in Ys])
    kw = dict(scheme=scheme, degree=N, dyadic=lam, compute="f32", strip_pipeline=pipeline, tensor_cores=False)
    G = sk.sigkernel_gram(X, Y, **kw)
    G0 = sk.sigkernel_gram(X, Y, tiled_m=False, **kw)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    assert torch.equal(G, G0)
    ref = oracle.pairs([Xs[2], Xs[0]], [Ys[2], Ys[0]], [0, 1], [0, 1], scheme, N, lam)
    got = G.cpu().numpy()[[2, 0], [2, 0]]
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-4


def test_tiled_m_with_the_forward_tape():
    X = torch.tensor(W.brownian(3, 70, 24, seed=401), device="cuda")
    Y = torch.tensor(W.brownian(2, 90, 24, seed=402), device="cuda")
    G, tape = sk.sigkernel_forward_tape(X, Y, degree=6, compute="f32", tensor_cores=False)
    G0 = sk.sigkernel_gram(X, Y, degree=6, compute="f32", tiled_m=False, tensor_cores=False)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    assert torch.equal(G, G0)
