"""GPU parity of the adjoint of the finite-difference schemes (Definition "dyadic scheme", eq.
(secondexplicitscheme), Remark "higherfd"): the reverse wavefront over the forward's per-column
tape (sk_bwd_fd.cuh), through sigkernel_backward (chunked tapes) and the tape calls, against the
oracle's complex-step gradients of the same discrete scheme.

Tolerances as for the polynomial adjoints: 1e-9 of the gradient's scale in FP64, 1e-4 in FP32.
Two-strip paths with ragged tails, dyadic orders 0..4 (a lane then carries 1..16 node rows), the
symmetric Gram, pair lists, the tensor-core contraction (d > 8 in FP32) and MMD^2.
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


def _oracle_grads(X, Y, pa, pb, wts, scheme, lam):
    rX, rY = np.zeros_like(X), np.zeros_like(Y)
    for w, a, b in zip(wts, pa, pb):
        gx, gy = oracle.grad(X[a], Y[b], scheme, 2, lam)
        rX[a] += w * gx
        rY[b] += w * gy
    return rX, rY


@pytest.mark.parametrize("scheme", ["fd1", "fd2", "fd_implicit"])
@pytest.mark.parametrize("lam", [0, 1, 2, 3])
def test_fd_backward_f64_matches_complex_step(scheme, lam):
    X = W.brownian(2, 40, 3, seed=700 + lam)   # 39 coarse rows: two strips, ragged tail
    Y = W.brownian(2, 23, 3, seed=710 + lam)
    pa, pb = [0, 1, 1], [1, 0, 1]
    wts = np.array([0.7, -1.3, 2.0])
    gX, gY = sk.sigkernel_backward(_cuda(wts), _cuda(X), _cuda(Y), pair_a=pa, pair_b=pb, scheme=scheme, dyadic=lam,
                                   compute="f64")
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    rX, rY = _oracle_grads(X, Y, pa, pb, wts, scheme, lam)
    assert _scaled_err(gX.cpu().numpy().reshape(X.shape), rX) < 1e-9
    assert _scaled_err(gY.cpu().numpy().reshape(Y.shape), rY) < 1e-9


@pytest.mark.parametrize("scheme,lam", [("fd1", 0), ("fd2", 2), ("fd_implicit", 1), ("fd1", 4)])
def test_fd_backward_f32_matches_complex_step(scheme, lam):
    X = W.brownian(2, 37, 4, seed=720 + lam)
    Y = W.brownian(2, 35, 4, seed=730 + lam)
    pa, pb = [0, 1], [1, 0]
    wts = np.array([1.0, -0.5])
    gX, gY = sk.sigkernel_backward(_cuda(wts), _cuda(X), _cuda(Y), pair_a=pa, pair_b=pb, scheme=scheme, dyadic=lam,
                                   compute="f32")
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    rX, rY = _oracle_grads(X, Y, pa, pb, wts, scheme, lam)
    assert _scaled_err(gX.cpu().numpy().reshape(X.shape), rX) < 1e-4
    assert _scaled_err(gY.cpu().numpy().reshape(Y.shape), rY) < 1e-4


@pytest.mark.parametrize("compute,tol", [("f64", 1e-9), ("f32", 1e-4)])
def test_fd_gram_backward_symmetric_and_tensor_core_contraction(compute, tol):
    X = W.brownian(3, 30, 12, seed=740)     # d = 12: the tensor-core contraction in FP32
    Wt = np.random.default_rng(741).normal(size=(3, 3))
    gX, _ = sk.sigkernel_backward(_cuda(Wt), _cuda(X), None, scheme="fd2", dyadic=1, compute=compute)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    rX = np.zeros_like(X)
    for a in range(3):
        for b in range(3):
            gx, gy = oracle.grad(X[a], X[b], "fd2", 2, 1)
            rX[a] += Wt[a, b] * gx
            rX[b] += Wt[a, b] * gy
    assert _scaled_err(gX.cpu().numpy().reshape(X.shape), rX) < tol


def test_fd_tape_calls_and_mmd2_gradient():
    X = W.brownian(2, 45, 2, seed=750)
    Y = W.brownian(3, 33, 2, seed=751)
    Wt = np.random.default_rng(752).normal(size=(2, 3))
    Xt, Yt = _cuda(X), _cuda(Y)
    G, tape = sk.sigkernel_forward_tape(Xt, Yt, scheme="fd1", dyadic=2, compute="f64")
    ref = oracle.gram(list(X), list(Y), "fd1", 2, 2)
    assert np.max(np.abs(G.cpu().numpy() - ref) / np.abs(ref)) < 1e-11
    gX, gY = sk.sigkernel_backward_tape(tape, _cuda(Wt), Xt, Yt, scheme="fd1", dyadic=2, compute="f64")
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    rX, rY = _oracle_grads(X, Y, [a for a in range(2) for b in range(3)], [b for a in range(2) for b in range(3)],
                           Wt.ravel(), "fd1", 2)
    assert _scaled_err(gX.cpu().numpy().reshape(X.shape), rX) < 1e-9
    assert _scaled_err(gY.cpu().numpy().reshape(Y.shape), rY) < 1e-9
    # MMD^2 of the FD scheme: gradient against the oracle's complex-step derivative on entries
    A = W.brownian(3, 17, 2, seed=753)
    B = W.brownian(3, 17, 2, seed=754, drift=0.4)
    _, _, gA, gB = sk.sigkernel_mmd2(_cuda(A), _cuda(B), scheme="fd2", dyadic=1, compute="f64", grads=True)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    gA = gA.cpu().numpy().reshape(A.shape)
    for (path, p, c) in [(0, 3, 0), (2, 16, 1), (1, 0, 1)]:
        ref = oracle.mmd2_grad_entry(A, B, 0, path, p, c, "fd2", 2, 1)
        assert abs(gA[path, p, c] - ref) <= 1e-9 * max(1.0, abs(ref))
