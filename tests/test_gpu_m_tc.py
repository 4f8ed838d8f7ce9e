"""GPU tests of the forward's M on the tensor cores: for the FP32 approximation scheme with
4 < d <= 32 a tcgen05 GEMM writes every cell's M_ij = <dx_i, dy_j> / 4^lambda (three BF16 parts of
each increment, six part products, FP32 accumulation) in the sweep's warp-step layout, per chunk
of pairs, and the one-warp-per-pair sweep reads it.

M then differs from the FMA-pipe inner product by about 2^-22 of sum_k |dx_ik dy_jk| per cell, the
order of FP32 rounding.  A perturbation of the cells' M moves k(x, y) in proportion to the kernel's
own scale sqrt(k(x, x) k(y, y)) (the bound of k(x, y) for a positive definite kernel), not to
|k(x, y)|, which can sit near zero for these oscillating kernels (Brownian paths, d >= 12), so the
errors are measured against that scale: at most 2e-5 of it from the FMA-pipe forward
(SK_FLAG_NO_TC) and 1e-4 of it from the oracle (the mixed-precision forms' bound).  Shapes
span several 128 x 128 tiles with ragged tails, both operand widths (d <= 16 and 16 < d <= 32), a
dyadic refinement, empty and one-increment paths, and batches past the 8 GB budget of
precomputed M (several chunks).
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


def _diag(P, n, **kw):
    """k(p, p) of the first n paths of P, on the FMA pipe."""
    idx = np.arange(n)
    return sk.sigkernel_pairs(P, P, idx, idx, tensor_cores=False, **kw).cpu().numpy()


def _nerr(a, b, kx, ky):
    """max |a - b| / sqrt(k(x, x) k(y, y)) over the entries (kx, ky broadcast against a)."""
    return np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.sqrt(np.abs(kx * ky)))


@pytest.mark.parametrize("d", [5, 8, 12, 20, 32])
@pytest.mark.parametrize("N,lam", [(6, 0), (4, 1)])
def test_gram_matches_the_fma_pipe_and_the_oracle(d, N, lam):
    Xs = _paths(501, [300, 40, 129, 1, 2, 257], d)
    Ys = _paths(601, [131, 33, 260, 128], d)
    X = sk.Paths.from_list([torch.tensor(x) for x in Xs])
    Y = sk.Paths.from_list([torch.tensor(y) for y in Ys])
    kw = dict(degree=N, dyadic=lam, compute="f32")
    G = sk.sigkernel_gram(X, Y, **kw)
    G0 = sk.sigkernel_gram(X, Y, tensor_cores=False, **kw)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    g, g0 = G.cpu().numpy(), G0.cpu().numpy()
    kx, ky = _diag(X, len(Xs), **kw), _diag(Y, len(Ys), **kw)
    assert np.all(g[3] == 1.0)             # a one-point path: no cells, k = 1
    assert _nerr(g, g0, kx[:, None], ky[None, :]) < 2e-5
    ia, ib = [0, 2, 4, 5], [2, 0, 1, 3]
    ref = oracle.pairs([Xs[i] for i in ia], [Ys[j] for j in ib], list(range(4)), list(range(4)), "approx", N, lam)
    assert _nerr(g[ia, ib], ref, kx[ia], ky[ib]) < 1e-4


@pytest.mark.parametrize("d", [4, 33])
def test_outside_the_operand_widths_the_fma_pipe_runs(d):
    X = torch.tensor(W.brownian(5, 100, d, seed=701), device="cuda")
    Y = torch.tensor(W.brownian(4, 90, d, seed=702), device="cuda")
    G = sk.sigkernel_gram(X, Y, degree=6, compute="f32")
    G0 = sk.sigkernel_gram(X, Y, degree=6, compute="f32", tensor_cores=False)
    torch.cuda.synchronize()
    assert torch.equal(G, G0)


def test_symmetric_gram_and_pairs_in_several_chunks():
    # 129 paths of 513 points: the symmetric Gram has 8385 items of 1 MB of M each, more than the
    # 8 GB budget holds, so the forward runs in chunks (Gram items by item_base; the pair list by
    # offset pair indices and outputs).
    n, pts, d = 129, 513, 32
    Xn = W.brownian(n, pts, d, seed=801)
    X = torch.tensor(Xn, device="cuda")
    kw = dict(degree=6, compute="f32")
    G = sk.sigkernel_gram(X, **kw)
    G0 = sk.sigkernel_gram(X, tensor_cores=False, **kw)
    rng = np.random.default_rng(802)
    m = 8300
    pa = rng.integers(0, n, m)
    pb = rng.integers(0, n, m)
    K = sk.sigkernel_pairs(X, X, pa, pb, **kw)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    g, g0 = G.cpu().numpy(), G0.cpu().numpy()
    kd = np.diag(g0)
    assert np.array_equal(g, g.T)
    assert _nerr(g, g0, kd[:, None], kd[None, :]) < 2e-5
    assert _nerr(K.cpu().numpy(), g0[pa, pb], kd[pa], kd[pb]) < 2e-5
    # both sides of the chunk boundaries are sampled against the oracle
    idx = [0, 7295, 7296, m - 1]
    ref = oracle.pairs([Xn[pa[k]] for k in idx], [Xn[pb[k]] for k in idx], list(range(4)), list(range(4)), "approx", 6, 0)
    assert _nerr(K.cpu().numpy()[idx], ref, kd[pa[idx]], kd[pb[idx]]) < 1e-4


def test_tape_forward_and_gradients():
    Xs = _paths(901, [200, 70, 129], 24)
    Ys = _paths(951, [90, 140], 24)
    X = sk.Paths.from_list([torch.tensor(x) for x in Xs])
    Y = sk.Paths.from_list([torch.tensor(y) for y in Ys])
    G, tape = sk.sigkernel_forward_tape(X, Y, degree=6, compute="f32")
    G0, tape0 = sk.sigkernel_forward_tape(X, Y, degree=6, compute="f32", tensor_cores=False)
    gout = torch.tensor(np.random.default_rng(3).standard_normal((3, 2)), device="cuda")
    gx, gy = sk.sigkernel_backward_tape(tape, gout, X, Y, degree=6, compute="f32")
    gx0, gy0 = sk.sigkernel_backward_tape(tape0, gout, X, Y, degree=6, compute="f32")
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    kx, ky = _diag(X, 3, degree=6, compute="f32"), _diag(Y, 2, degree=6, compute="f32")
    assert _nerr(G.cpu().numpy(), G0.cpu().numpy(), kx[:, None], ky[None, :]) < 2e-5
    scale = gx0.abs().max().item()
    assert (gx - gx0).abs().max().item() < 1e-4 * scale
    assert (gy - gy0).abs().max().item() < 1e-4 * gy0.abs().max().item()
