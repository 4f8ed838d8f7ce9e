"""GPU parity of the tensor-core contraction (tcgen05, BF16 high and low parts, three products,
FP32 accumulation) that turns the tape adjoint's dk/dM into increment gradients for 8 < d <= 32
in FP32: against the FMA-pipe contraction on the same tape (SK_FLAG_NO_TC), and against the
oracle's complex-step gradients.

A BF16 x 3 product x y = (hx + lx)(hy + ly) - lx ly, with hx = bf16(x) and lx = bf16(x - hx),
carries at most about 3 * 2^-16 (4.6e-5) relative error: the rounding of lx and ly and the dropped
lx ly, each up to 2^-16 (BF16 keeps 8 significant bits; tests/test_tc_splits.py checks the bound
on CPU, where random pairs reach 2.6e-5).  The contraction sums such products in FP32, whose
independent rounding errors partly cancel, so the two contractions are held to 5e-5 of the
gradient's scale, and both meet the FP32 bar of 1e-4 against the oracle.  The paths leave
ragged 128-cell tiles (zero padding inside the tile grid), the dyadic case refines the rows and
columns the operand tiles map back to coarse increments, and the symmetric Gram shares one set of
operand tiles between X and Y.
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


def _cuda(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def _scaled_err(g, ref):
    return float(np.max(np.abs(g - ref)) / max(np.max(np.abs(ref)), 1e-300))


def _both(X, Y, Wt, **kw):
    sym = Y is None
    _, tape = sk.sigkernel_forward_tape(_cuda(X), None if sym else _cuda(Y), compute="f32", **kw)
    tc = sk.sigkernel_backward_tape(tape, _cuda(Wt), _cuda(X), None if sym else _cuda(Y), compute="f32", **kw)
    fma = sk.sigkernel_backward_tape(tape, _cuda(Wt), _cuda(X), None if sym else _cuda(Y), compute="f32",
                                     tensor_cores=False, **kw)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    return [g.cpu().numpy() for g in tc], [g.cpu().numpy() for g in fma]


@pytest.mark.parametrize("d", [12, 16, 24, 32])
@pytest.mark.parametrize("scheme,N,lam", [("approx", 6, 0), ("approx", 4, 1), ("interp", 5, 0)])
def test_tc_contraction_matches_the_fma_contraction(d, scheme, N, lam):
    X = W.brownian(3, 140, d, seed=500 + d)   # 139 rows: a full and a ragged 128-row block
    Y = W.brownian(2, 90, d, seed=510 + d)
    Wt = np.random.default_rng(520 + d).normal(size=(3, 2))
    tc, fma = _both(X, Y, Wt, scheme=scheme, degree=N, dyadic=lam)
    for a, b in zip(tc, fma):
        assert np.all(np.isfinite(a))
        assert _scaled_err(a, b) < 5e-5


@pytest.mark.parametrize("d", [16, 32])
def test_tc_contraction_matches_the_oracle(d):
    X = W.brownian(2, 60, d, seed=530 + d)
    Y = W.brownian(2, 45, d, seed=540 + d, drift=0.3)
    Wt = np.array([[0.8, -1.1], [0.4, 1.7]])
    tc, _ = _both(X, Y, Wt, scheme="approx", degree=6)
    rX, rY = np.zeros_like(X), np.zeros_like(Y)
    for a in range(2):
        for b in range(2):
            gx, gy = oracle.grad(X[a], Y[b], "approx", 6)
            rX[a] += Wt[a, b] * gx
            rY[b] += Wt[a, b] * gy
    assert _scaled_err(tc[0].reshape(X.shape), rX) < 1e-4
    assert _scaled_err(tc[1].reshape(Y.shape), rY) < 1e-4


def test_tc_contraction_symmetric_gram_and_pairs():
    X = W.brownian(4, 257, 20, seed=550)
    Wt = np.random.default_rng(551).normal(size=(4, 4))
    tc, fma = _both(X, None, Wt, scheme="approx", degree=6)
    assert _scaled_err(tc[0], fma[0]) < 5e-5
    # pair list with repeats: the same rows accumulate from several items
    pa, pb = [0, 1, 1, 3, 0], [2, 2, 0, 3, 0]
    wts = _cuda([0.5, -1.0, 2.0, 0.25, 1.5])
    Xt = _cuda(X)
    _, tape = sk.sigkernel_forward_tape(Xt, Xt, pair_a=pa, pair_b=pb, compute="f32")
    g1 = sk.sigkernel_backward_tape(tape, wts, Xt, Xt, pair_a=pa, pair_b=pb, compute="f32")[0].cpu().numpy()
    g2 = sk.sigkernel_backward_tape(tape, wts, Xt, Xt, pair_a=pa, pair_b=pb, compute="f32",
                                    tensor_cores=False)[0].cpu().numpy()
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    assert _scaled_err(g1, g2) < 5e-5


def test_mmd2_gradient_with_and_without_tensor_cores():
    A = torch.tensor(W.brownian(24, 129, 32, seed=560), device="cuda")
    B = torch.tensor(W.brownian(20, 129, 32, seed=561, drift=0.5, vol=1.2), device="cuda")
    m1, means, gA1, gB1 = sk.sigkernel_mmd2(A, B, compute="f32", grads=True)
    m2, _, gA2, gB2 = sk.sigkernel_mmd2(A, B, compute="f32", grads=True, tensor_cores=False)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    # the forward's M also comes from the tensor cores (at most about 2^-23 relative per product): the
    # value agrees to FP32 rounding on the scale of the kernel means
    assert abs(m1.item() - m2.item()) < 2e-5 * means.abs().sum().item()
    assert _scaled_err(gA1.cpu().numpy(), gA2.cpu().numpy()) < 5e-5
    assert _scaled_err(gB1.cpu().numpy(), gB2.cpu().numpy()) < 5e-5
