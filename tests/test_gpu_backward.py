"""GPU adjoint parity: the reverse wavefront (through the C ABI) against the oracle's complex-step
derivatives of the same discrete scheme, plus central differences and MMD^2.

Tolerances: FP64 adjoints agree with the complex-step derivative to rounding (relative 1e-9 of the
gradient's scale); FP32 adjoints are held to the mixed-precision bar (relative error <= 1e-4 of
the gradient's scale).
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


def _oracle_gram_grad(X, Y, Wt, N, lam, sym, scheme="approx"):
    """d/dX, d/dY of sum_ab Wt[a,b] k(X_a, Y_b) from the oracle's complex-step gradients."""
    gX = np.zeros_like(X)
    gY = np.zeros_like(Y)
    for a in range(X.shape[0]):
        for b in range(Y.shape[0]):
            if Wt[a, b] == 0.0:
                continue
            gx, gy = oracle.grad(X[a], Y[b], scheme, N, lam)
            gX[a] += Wt[a, b] * gx
            gY[b] += Wt[a, b] * gy
    if sym:
        return gX + gY, None
    return gX, gY


@pytest.mark.parametrize("checkpoint", [False, True])
@pytest.mark.parametrize("N,lam", [(2, 0), (4, 0), (6, 0), (6, 1), (9, 0)])
def test_pairs_backward_f64_matches_complex_step(N, lam, checkpoint):
    """sigkernel_backward from chunked forward tapes (default) and the checkpointing adjoint."""
    X = W.brownian(2, 40, 3, seed=51)   # 39 rows: two strips with a ragged tail
    Y = W.brownian(2, 35, 3, seed=52)
    pa, pb = [0, 1, 1], [1, 0, 1]
    wts = np.array([0.7, -1.3, 2.0])
    gX, gY = sk.sigkernel_backward(_cuda(wts), _cuda(X), _cuda(Y), pair_a=pa, pair_b=pb, degree=N, dyadic=lam,
                                   compute="f64", checkpoint=checkpoint)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    rX = np.zeros_like(X)
    rY = np.zeros_like(Y)
    for w, a, b in zip(wts, pa, pb):
        gx, gy = oracle.grad(X[a], Y[b], "approx", N, lam)
        rX[a] += w * gx
        rY[b] += w * gy
    assert _scaled_err(gX.cpu().numpy().reshape(X.shape), rX) < 1e-9
    assert _scaled_err(gY.cpu().numpy().reshape(Y.shape), rY) < 1e-9


@pytest.mark.parametrize("checkpoint", [False, True])
def test_pairs_backward_f32_matches_complex_step(checkpoint):
    X = W.brownian(2, 70, 4, seed=53)
    Y = W.brownian(2, 66, 4, seed=54)
    pa, pb = [0, 1], [1, 0]
    wts = np.array([1.0, 0.5])
    gX, gY = sk.sigkernel_backward(_cuda(wts), _cuda(X), _cuda(Y), pair_a=pa, pair_b=pb, degree=6, compute="f32",
                                   checkpoint=checkpoint)
    torch.cuda.synchronize()
    rX = np.zeros_like(X)
    rY = np.zeros_like(Y)
    for w, a, b in zip(wts, pa, pb):
        gx, gy = oracle.grad(X[a], Y[b], "approx", 6)
        rX[a] += w * gx
        rY[b] += w * gy
    assert _scaled_err(gX.cpu().numpy().reshape(X.shape), rX) < 1e-4
    assert _scaled_err(gY.cpu().numpy().reshape(Y.shape), rY) < 1e-4


@pytest.mark.parametrize("checkpoint", [False, True])
@pytest.mark.parametrize("sym", [False, True])
@pytest.mark.parametrize("compute", ["f64", "f32"])
def test_gram_backward_matches_oracle(sym, compute, checkpoint):
    X = W.brownian(3, 33, 2, seed=55)
    Y = X if sym else W.brownian(4, 29, 2, seed=56)
    rng = np.random.default_rng(57)
    Wt = rng.normal(size=(X.shape[0], Y.shape[0]))
    gX, gY = sk.sigkernel_backward(_cuda(Wt), _cuda(X), None if sym else _cuda(Y), degree=5, compute=compute,
                                   checkpoint=checkpoint)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    rX, rY = _oracle_gram_grad(X, Y, Wt, 5, 0, sym)
    tol = 1e-9 if compute == "f64" else 1e-4
    assert _scaled_err(gX.cpu().numpy().reshape(X.shape), rX) < tol
    if not sym:
        assert _scaled_err(gY.cpu().numpy().reshape(Y.shape), rY) < tol


def test_backward_ragged_and_trivial_paths():
    lengths = [1, 2, 5, 33, 34, 70]
    Xs = [W.brownian(1, L, 3, seed=60 + i)[0] for i, L in enumerate(lengths)]
    PX = sk.Paths.from_list([torch.tensor(x) for x in Xs])
    pa = [0, 1, 2, 3, 4, 5, 5, 3]
    pb = [5, 4, 3, 2, 1, 0, 3, 5]
    wts = np.linspace(-1.0, 1.5, len(pa))
    gX, _ = sk.sigkernel_backward(_cuda(wts), PX, PX, pair_a=pa, pair_b=pb, degree=6, compute="f64")
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    ref = [np.zeros_like(x) for x in Xs]
    for w, a, b in zip(wts, pa, pb):
        gx, gy = oracle.grad(Xs[a], Xs[b], "approx", 6)
        ref[a] += w * gx
        ref[b] += w * gy
    got = gX.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(lengths)])
    scale = max(np.max(np.abs(r)) for r in ref)
    for i in range(len(Xs)):
        assert np.max(np.abs(got[off[i]:off[i + 1]] - ref[i])) < 1e-9 * scale
    assert np.all(got[0:1] == 0.0)  # a single-point path has k = 1 and no gradient


def test_backward_f32_rescaled_huge_kernels():
    X = 14.0 * W.brownian(2, 49, 2, seed=58)
    Y = 14.0 * W.brownian(2, 49, 2, seed=59)
    k = oracle.kernel(X[1], Y[0], "approx", 8, 1)
    assert abs(k) > 1e39  # |k| ~ 3e51: beyond FP32 without the exponents
    gX, gY = sk.sigkernel_backward(_cuda([1.0]), _cuda(X), _cuda(Y), pair_a=[1], pair_b=[0], degree=8, dyadic=1,
                                   compute="f32")
    torch.cuda.synchronize()
    gx, gy = oracle.grad(X[1], Y[0], "approx", 8, 1)
    got = gX.cpu().numpy().reshape(X.shape)[1]
    assert np.all(np.isfinite(got))
    assert _scaled_err(got, gx) < 1e-3


def test_gradient_matches_central_differences_on_sampled_coordinates():
    X = W.brownian(1, 30, 3, seed=61)
    Y = W.brownian(1, 27, 3, seed=62)
    gX, gY = sk.sigkernel_backward(_cuda([1.0]), _cuda(X), _cuda(Y), pair_a=[0], pair_b=[0], degree=6,
                                   compute="f64")
    gx = gX.cpu().numpy().reshape(X.shape)[0]
    rng = np.random.default_rng(63)
    h = 1e-4
    for _ in range(16):
        p, c = rng.integers(0, 30), rng.integers(0, 3)
        xp, xm = X[0].copy(), X[0].copy()
        xp[p, c] += h
        xm[p, c] -= h
        fd = (oracle.kernel(xp, Y[0], "approx", 6) - oracle.kernel(xm, Y[0], "approx", 6)) / (2 * h)
        assert abs(gx[p, c] - fd) < 1e-6 * max(1.0, abs(fd))


# ------------------------------------------------------------------------------------------
# MMD^2 and its gradient
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("unbiased", [False, True])
def test_mmd2_matches_oracle(unbiased):
    A = W.brownian(4, 20, 2, seed=64)
    B = W.brownian(3, 20, 2, seed=65, drift=0.5, vol=1.2)
    m, means, gA, gB = sk.sigkernel_mmd2(_cuda(A), _cuda(B), degree=6, compute="f64", unbiased=unbiased, grads=True)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    ref = oracle.mmd2(A, B, "approx", 6, unbiased=unbiased)
    assert abs(m.item() - ref) < 1e-11 * max(1.0, abs(ref))
    gA = gA.cpu().numpy().reshape(A.shape)
    gB = gB.cpu().numpy().reshape(B.shape)
    rng = np.random.default_rng(66)
    for _ in range(6):
        side = int(rng.integers(0, 2))
        S = A if side == 0 else B
        path, p, c = rng.integers(0, S.shape[0]), rng.integers(0, 20), rng.integers(0, 2)
        ref_g = oracle.mmd2_grad_entry(A, B, side, path, p, c, "approx", 6, unbiased=unbiased)
        got = (gA if side == 0 else gB)[path, p, c]
        assert abs(got - ref_g) < 1e-9 * max(1.0, np.max(np.abs(gA)))


@pytest.mark.parametrize("compute,tol", [("f64", 1e-9), ("f32", 1e-4)])
def test_mmd2_interpolation_gradient_matches_oracle(compute, tol):
    """MMD^2 gradients of the interpolation scheme (N = 6) from the chunked tape adjoint, against
    the oracle's complex-step derivative."""
    A = W.brownian(4, 20, 2, seed=67)
    B = W.brownian(3, 20, 2, seed=68, drift=0.5, vol=1.2)
    m, means, gA, gB = sk.sigkernel_mmd2(_cuda(A), _cuda(B), scheme="interp", degree=6, compute=compute, grads=True)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    ref = oracle.mmd2(A, B, "interp", 6)
    assert abs(m.item() - ref) < tol * max(1.0, abs(ref))
    gA = gA.cpu().numpy().reshape(A.shape)
    gB = gB.cpu().numpy().reshape(B.shape)
    scale = max(np.max(np.abs(gA)), np.max(np.abs(gB)))
    rng = np.random.default_rng(69)
    for _ in range(6):
        side = int(rng.integers(0, 2))
        S = A if side == 0 else B
        path, p, c = rng.integers(0, S.shape[0]), rng.integers(0, 20), rng.integers(0, 2)
        ref_g = oracle.mmd2_grad_entry(A, B, side, path, p, c, "interp", 6)
        got = (gA if side == 0 else gB)[path, p, c]
        assert abs(got - ref_g) < tol * scale, (side, path, p, c, got, ref_g)


def test_mmd2_workload_gradient_central_differences_f32():
    """Two batches (Brownian vs Brownian with drift 0.5 and volatility 1.2), FP32 adjoint; 16 random
    coordinates checked against central differences (h = 1e-4) of the FP64 oracle."""
    A = W.brownian(6, 33, 4, seed=7)
    B = W.brownian(6, 33, 4, seed=8, drift=0.5, vol=1.2)
    m, _, gA, gB = sk.sigkernel_mmd2(_cuda(A), _cuda(B), degree=6, compute="f32", grads=True)
    torch.cuda.synchronize()
    gA = gA.cpu().numpy().reshape(A.shape)
    gB = gB.cpu().numpy().reshape(B.shape)
    rng = np.random.default_rng(67)
    h = 1e-4
    scale = max(np.max(np.abs(gA)), np.max(np.abs(gB)))
    for _ in range(16):
        side = int(rng.integers(0, 2))
        S = A if side == 0 else B
        path, p, c = rng.integers(0, 6), rng.integers(0, 33), rng.integers(0, 4)
        Sp, Sm = S.copy(), S.copy()
        Sp[path, p, c] += h
        Sm[path, p, c] -= h
        if side == 0:
            fd = (oracle.mmd2(Sp, B, "approx", 6) - oracle.mmd2(Sm, B, "approx", 6)) / (2 * h)
        else:
            fd = (oracle.mmd2(A, Sp, "approx", 6) - oracle.mmd2(A, Sm, "approx", 6)) / (2 * h)
        got = (gA if side == 0 else gB)[path, p, c]
        assert abs(got - fd) < 1e-4 * scale


def test_autograd_gram_and_mmd():
    X = _cuda(W.brownian(3, 25, 2, seed=68)).requires_grad_(True)
    Y = _cuda(W.brownian(2, 21, 2, seed=69)).requires_grad_(True)
    kern = sk.SigKernel("approx", 6, 0, "f64")
    G = kern.gram(X, Y)
    wts = torch.randn(3, 2, dtype=torch.float64, device="cuda")
    (G * wts).sum().backward()
    gX, gY = sk.sigkernel_backward(wts, X.detach(), Y.detach(), degree=6, compute="f64")
    assert torch.allclose(X.grad.reshape(-1, 2), gX, rtol=1e-12, atol=1e-14)
    assert torch.allclose(Y.grad.reshape(-1, 2), gY, rtol=1e-12, atol=1e-14)
    A = _cuda(W.brownian(3, 15, 2, seed=70)).requires_grad_(True)
    B = _cuda(W.brownian(3, 15, 2, seed=71, drift=0.5)).requires_grad_(True)
    m = kern.mmd2(A, B)
    m.backward()
    assert A.grad is not None and torch.isfinite(A.grad).all()
    Ad, Bd = A.detach().cpu().numpy(), B.detach().cpu().numpy()
    ref = oracle.mmd2_grad_entry(Ad, Bd, 0, 1, 4, 1, "approx", 6)
    assert abs(A.grad[1, 4, 1].item() - ref) < 1e-9 * max(1.0, A.grad.abs().max().item())


@pytest.mark.parametrize("tape", [None, True, False])
def test_gradcheck_small(tape):
    """gradcheck runs backward several times on one graph: the wrapper keeps its tape for that."""
    X = _cuda(W.brownian(2, 6, 2, seed=72)).requires_grad_(True)
    Y = _cuda(W.brownian(2, 5, 2, seed=73)).requires_grad_(True)
    kern = sk.SigKernel("approx", 5, 0, "f64", tape=tape)
    assert torch.autograd.gradcheck(lambda x, y: kern.gram(x, y), (X, Y), eps=1e-6, atol=1e-8, rtol=1e-6)


# ------------------------------------------------------------------------------------------
# Adjoint from a forward tape: same gradients as the checkpointing adjoint and the oracle
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("compute,tol", [("f64", 1e-9), ("f32", 1e-4)])
@pytest.mark.parametrize("sym", [False, True])
def test_tape_backward_matches_oracle(compute, tol, sym):
    X = W.brownian(3, 41, 3, seed=74)
    Y = X if sym else W.brownian(4, 37, 3, seed=75)
    rng = np.random.default_rng(76)
    Wt = rng.normal(size=(X.shape[0], Y.shape[0]))
    Xt = _cuda(X)
    Yt = None if sym else _cuda(Y)
    G, tape = sk.sigkernel_forward_tape(Xt, Yt, degree=6, compute=compute)
    G2 = sk.sigkernel_gram(Xt, Yt, degree=6, compute=compute)
    torch.cuda.synchronize()
    assert torch.equal(G, G2)  # recording the tape does not change the forward
    gX, gY = sk.sigkernel_backward_tape(tape, _cuda(Wt), Xt, Yt, degree=6, compute=compute)
    cX, cY = sk.sigkernel_backward(_cuda(Wt), Xt, Yt, degree=6, compute=compute)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    # same arithmetic per cell; the dk/dM contraction sums in another order (FP32: ~1e-7)
    assert _scaled_err(gX.cpu().numpy(), cX.cpu().numpy()) < (1e-12 if compute == "f64" else 1e-5)
    rX, rY = _oracle_gram_grad(X, Y, Wt, 6, 0, sym)
    assert _scaled_err(gX.cpu().numpy().reshape(X.shape), rX) < tol
    if not sym:
        assert _scaled_err(gY.cpu().numpy().reshape(Y.shape), rY) < tol


def test_tape_backward_pairs_dyadic_and_rescaled():
    X = 14.0 * W.brownian(2, 49, 2, seed=58)
    Y = 14.0 * W.brownian(2, 49, 2, seed=59)
    pa, pb = [1, 0], [0, 1]
    out, tape = sk.sigkernel_forward_tape(_cuda(X), _cuda(Y), pair_a=pa, pair_b=pb, degree=8, dyadic=1,
                                          compute="f32")
    gX, gY = sk.sigkernel_backward_tape(tape, _cuda([1.0, 0.0]), _cuda(X), _cuda(Y), pair_a=pa, pair_b=pb,
                                        degree=8, dyadic=1, compute="f32")
    torch.cuda.synchronize()
    gx, gy = oracle.grad(X[1], Y[0], "approx", 8, 1)
    got = gX.cpu().numpy().reshape(X.shape)[1]
    assert np.all(np.isfinite(got))
    assert _scaled_err(got, gx) < 1e-3


@pytest.mark.parametrize("compute,tol", [("f64", 1e-9), ("f32", 1e-4)])
def test_tape_backward_wide_d_matches_oracle(compute, tol):
    """d = 37 (40 padded): the contraction takes coordinates 32 at a time, the second pass partial."""
    X = W.brownian(2, 17, 37, seed=78)
    Y = W.brownian(2, 15, 37, seed=79)
    Wt = np.array([[0.7, -1.3], [0.4, 2.1]])
    G, tape = sk.sigkernel_forward_tape(_cuda(X), _cuda(Y), degree=5, compute=compute)
    gX, gY = sk.sigkernel_backward_tape(tape, _cuda(Wt), _cuda(X), _cuda(Y), degree=5, compute=compute)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    rX, rY = _oracle_gram_grad(X, Y, Wt, 5, 0, False)
    assert _scaled_err(gX.cpu().numpy().reshape(X.shape), rX) < tol
    assert _scaled_err(gY.cpu().numpy().reshape(Y.shape), rY) < tol


@pytest.mark.parametrize("compute,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_tape_backward_long_paths_match_checkpoint_adjoint(compute, tol):
    """1300-point paths: the contraction's per-increment sums exceed its shared-memory
    accumulators and go straight to the FP64 gradients.  The checkpointing adjoint (pinned against
    the oracle elsewhere) is the reference at this size."""
    X = W.brownian(1, 1300, 2, seed=80)
    Y = W.brownian(2, 1250, 2, seed=81)
    pa, pb = [0, 0], [1, 0]
    wts = _cuda([0.6, -1.1])
    out, tape = sk.sigkernel_forward_tape(_cuda(X), _cuda(Y), pair_a=pa, pair_b=pb, degree=6, compute=compute)
    gX, gY = sk.sigkernel_backward_tape(tape, wts, _cuda(X), _cuda(Y), pair_a=pa, pair_b=pb, degree=6,
                                        compute=compute)
    cX, cY = sk.sigkernel_backward(wts, _cuda(X), _cuda(Y), pair_a=pa, pair_b=pb, degree=6, compute=compute,
                                   checkpoint=True)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    assert np.all(np.isfinite(gX.cpu().numpy()))
    assert _scaled_err(gX.cpu().numpy(), cX.cpu().numpy()) < tol
    assert _scaled_err(gY.cpu().numpy(), cY.cpu().numpy()) < tol


@pytest.mark.parametrize("compute,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_tape_backward_column_windows_match_checkpoint_adjoint(compute, tol):
    """d = 12 (16 coordinates per contraction pass) and 300-point paths at lambda = 1 (598 refined
    columns): the contraction sweeps its column accumulator over 2 (FP32) or 3 (FP64) windows
    whose edges split coarse increments' sub-columns.  The checkpointing adjoint is the reference."""
    X = W.brownian(2, 300, 12, seed=82)
    Y = W.brownian(2, 300, 12, seed=83)
    Wt = _cuda([[0.9, -0.4], [1.3, 0.2]])
    G, tape = sk.sigkernel_forward_tape(_cuda(X), _cuda(Y), degree=5, dyadic=1, compute=compute)
    gX, gY = sk.sigkernel_backward_tape(tape, Wt, _cuda(X), _cuda(Y), degree=5, dyadic=1, compute=compute)
    cX, cY = sk.sigkernel_backward(Wt, _cuda(X), _cuda(Y), degree=5, dyadic=1, compute=compute, checkpoint=True)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    assert _scaled_err(gX.cpu().numpy(), cX.cpu().numpy()) < tol
    assert _scaled_err(gY.cpu().numpy(), cY.cpu().numpy()) < tol


# ------------------------------------------------------------------------------------------
# Adjoint of the interpolation scheme (tape path): projection transpose, the corner term and the
# endpoint seed on the unprojected series
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("compute,tol", [("f64", 1e-9), ("f32", 1e-4)])
@pytest.mark.parametrize("N", [3, 6])
def test_tape_backward_interp_matches_oracle(compute, tol, N):
    X = W.brownian(2, 33, 2, seed=81)   # 32 rows: the top row is lane 31 of a full strip
    Y = W.brownian(2, 25, 2, seed=82)
    Wt = np.array([[0.9, -0.4], [1.7, 0.3]])
    G, tape = sk.sigkernel_forward_tape(_cuda(X), _cuda(Y), scheme="interp", degree=N, compute=compute)
    G0 = sk.sigkernel_gram(_cuda(X), _cuda(Y), scheme="interp", degree=N, compute=compute)
    gX, gY = sk.sigkernel_backward_tape(tape, _cuda(Wt), _cuda(X), _cuda(Y), scheme="interp", degree=N,
                                        compute=compute)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    assert torch.equal(G, G0)
    rX, rY = _oracle_gram_grad(X, Y, Wt, N, 0, False, scheme="interp")
    assert _scaled_err(gX.cpu().numpy().reshape(X.shape), rX) < tol
    assert _scaled_err(gY.cpu().numpy().reshape(Y.shape), rY) < tol


def test_tape_backward_interp_symmetric_dyadic_rescaled():
    X = 10.0 * W.brownian(3, 30, 2, seed=83)   # |k| far outside FP32 without the exponents
    G, tape = sk.sigkernel_forward_tape(_cuda(X), None, scheme="interp", degree=5, dyadic=1, compute="f32")
    Wt = np.random.default_rng(84).normal(size=(3, 3))
    gX, _ = sk.sigkernel_backward_tape(tape, _cuda(Wt), _cuda(X), None, scheme="interp", degree=5, dyadic=1,
                                       compute="f32")
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    got = gX.cpu().numpy().reshape(X.shape)
    assert np.all(np.isfinite(got))
    rX, _ = _oracle_gram_grad(X, X, Wt, 5, 1, True, scheme="interp")
    assert _scaled_err(got, rX) < 1e-3


def test_autograd_with_tape():
    X = _cuda(W.brownian(4, 30, 2, seed=77)).requires_grad_(True)
    kern = sk.SigKernel("approx", 6, 0, "f64", tape=True)
    G = kern.gram(X)
    wts = torch.randn(4, 4, dtype=torch.float64, device="cuda")
    (G * wts).sum().backward()
    gX, _ = sk.sigkernel_backward(wts, X.detach(), None, degree=6, compute="f64")
    assert torch.allclose(X.grad.reshape(-1, 2), gX, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("compute,tol", [("f64", 1e-9), ("f32", 1e-4)])
@pytest.mark.parametrize("sym", [False, True])
def test_backward_interpolation_runs_chunked_tapes(compute, tol, sym):
    """sigkernel_backward for the interpolation scheme (no checkpointing adjoint): forward tapes
    recorded in chunks, each followed by the tape adjoint.  Against the oracle's complex-step
    gradients, and against the explicit tape calls (the same kernels; only the order of the FP64
    atomic sums may differ)."""
    X = W.brownian(3, 35, 2, seed=91)
    Y = X if sym else W.brownian(2, 30, 2, seed=92)
    Wt = np.array([[0.7, -1.2, 0.4], [0.3, 1.1, -0.6], [-0.8, 0.5, 0.9]])[:, :Y.shape[0]]
    if sym:
        Wt = 0.5 * (Wt + Wt.T)
    Xt = _cuda(X)
    Yt = None if sym else _cuda(Y)
    gX, gY = sk.sigkernel_backward(_cuda(Wt), Xt, Yt, scheme="interp", degree=5, compute=compute)
    G, tape = sk.sigkernel_forward_tape(Xt, Yt, scheme="interp", degree=5, compute=compute)
    tX, tY = sk.sigkernel_backward_tape(tape, _cuda(Wt), Xt, Yt, scheme="interp", degree=5, compute=compute)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    same_tol = 1e-12 if compute == "f64" else 1e-5  # FP32 column sums meet in shared-memory atomics
    scale = float(tX.abs().max())
    assert float((gX - tX).abs().max()) <= same_tol * scale
    rX, rY = _oracle_gram_grad(X, Y, Wt, 5, 0, sym, scheme="interp")
    assert _scaled_err(gX.cpu().numpy().reshape(X.shape), rX) < tol
    if not sym:
        assert float((gY - tY).abs().max()) <= same_tol * float(tY.abs().max())
        assert _scaled_err(gY.cpu().numpy().reshape(Y.shape), rY) < tol
