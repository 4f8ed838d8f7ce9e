"""GPU tests of the chunked tape adjoints of sigkernel_backward and sigkernel_mmd2: the results
must be ordered on the caller's stream (read right after the call on that stream, with no
device-wide synchronisation in between), the whole call must capture into a CUDA graph and replay
on new inputs, and the MMD^2 gradient solved in several chunks per Gram block must match the
backward of each block.

These runs also guard the shared-memory rings of the tape adjoint and the FMA contraction: a ring
slot that the warp has read is fenced (fence.proxy.async) before a bulk copy refills it.  Without
the fence the refill could overtake a pending load of the slot when other kernels kept the
load/store units busy (seen as intermittent FP32 gradient errors up to 1e-3 of scale while a
forward kernel ran beside the adjoint).
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


def _scaled(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("scheme,lam", [("approx", 0), ("fd1", 1)])
def test_backward_on_a_side_stream_is_ordered_for_the_caller(scheme, lam):
    """The call on a non-default torch stream: its gradients are complete for the next kernel on
    that stream."""
    X = torch.tensor(W.brownian(6, 80, 3, seed=71), device="cuda")
    Y = torch.tensor(W.brownian(5, 70, 3, seed=72), device="cuda")
    g = torch.tensor(np.random.default_rng(73).standard_normal((6, 5)), device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        gx, gy = sk.sigkernel_backward(g, X, Y, scheme=scheme, degree=6, dyadic=lam, compute="f64")
        # consumed on the caller's stream right away, without a device-wide synchronisation
        tot_x, tot_y = gx.sum(), gy.sum()
    s.synchronize()
    assert sk.device_status() == 0
    Xn, Yn = X.cpu().numpy(), Y.cpu().numpy()
    ref = np.zeros(Xn.shape)
    gn = g.cpu().numpy()
    for a in range(6):
        for b in range(5):
            gxa, _ = oracle.grad(Xn[a], Yn[b], scheme, 6 if scheme == "approx" else 2, lam)
            ref[a] += gn[a, b] * gxa
    assert _scaled(gx.cpu().numpy(), ref.reshape(-1, 3)) < 1e-9  # gradients come in the rows layout
    assert abs(tot_x.item() - gx.sum().item()) <= 1e-12 * gx.abs().sum().item()
    assert abs(tot_y.item() - gy.sum().item()) <= 1e-12 * gy.abs().sum().item()


def test_backward_captures_into_a_cuda_graph():
    X = torch.tensor(W.brownian(8, 65, 4, seed=81), device="cuda")
    Y = torch.tensor(W.brownian(8, 65, 4, seed=82), device="cuda")
    g = torch.tensor(np.random.default_rng(83).standard_normal((8, 8)), device="cuda")
    gx0, _ = sk.sigkernel_backward(g, X, Y, compute="f32")  # an eager call before the capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            gx, gy = sk.sigkernel_backward(g, X, Y, compute="f32")
    torch.cuda.synchronize()
    for seed in (84, 85):
        X.copy_(torch.tensor(W.brownian(8, 65, 4, seed=seed), device="cuda"))
        gx.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        ref, _ = sk.sigkernel_backward(g, X, Y, compute="f32")
        torch.cuda.synchronize()
        assert sk.device_status() == 0
        assert _scaled(gx.cpu().numpy(), ref.cpu().numpy()) < 1e-12


def test_mmd2_gradient_across_many_chunks_matches_the_backward_of_each_block():
    # 120 + 120 paths of 513 points (14.7 MB of tape per pair at N = 6): 64 GiB of tape hold 4663
    # pairs, rounded down to the adjoint's 3648 resident warps, so K_AA and K_BB (7260 pairs) run in
    # 2 chunks each and K_AB (14400) in 4
    n = 120
    A = torch.tensor(W.brownian(n, 513, 3, seed=91), device="cuda")
    B = torch.tensor(W.brownian(n, 513, 3, seed=92, drift=0.5, vol=1.2), device="cuda")
    m, means, gA, gB = sk.sigkernel_mmd2(A, B, compute="f32", grads=True)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    w = 1.0 / (n * n)
    full = lambda v: torch.full((n, n), v, device="cuda", dtype=torch.float64)
    gaa, _ = sk.sigkernel_backward(full(w), A, None, compute="f32")
    gbb, _ = sk.sigkernel_backward(full(w), B, None, compute="f32")
    gab, gba = sk.sigkernel_backward(full(-2 * w), A, B, compute="f32")
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    # The FP32 contraction sums columns with shared-memory atomics, whose order varies from run to
    # run, and the MMD gradient is a difference of the blocks' gradients (the two samples are
    # alike), so the error is measured against the size of the parts, not of their sum.
    for g, p1, p2 in ((gA, gaa, gab), (gB, gbb, gba)):
        scale = (p1.abs() + p2.abs()).max().item()
        assert (g - (p1 + p2)).abs().max().item() < 1e-5 * scale
