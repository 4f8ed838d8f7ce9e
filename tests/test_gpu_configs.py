"""GPU parity at the full sizes of the workload configurations beyond the 128x128 Gram, on sampled
outputs the FP64 oracle can compute one by one.

* Oscillatory: 64 pairs of 1025-point paths on [0, 1], d = 4, coordinate j = sin(w_j t + phi_j)
  plus N(0, 1e-3) noise; polynomial interpolation of order 8 (FP32 and FP64) and the FD scheme
  up to dyadic refinement 6, each against the oracle of the same scheme.
* Uneven batch: 4096 pairs, lengths log-uniform in [64, 4096], d = 16, BF16 points, FP32 cells;
  the oracle gets the same BF16-rounded points in FP64.
* MMD^2: 256 + 256 paths of 513 points, d = 32 (Brownian against Brownian with drift 0.5 and
  volatility 1.2), FP32, gradients from forward tapes in chunks of pairs (and, for paths too long
  for a chunk to fill the GPU, from the checkpointing adjoint).  The value is checked against the three
  Grams, Gram entries against the oracle, and the gradient on 16 random coordinates against
  central differences (h = 1e-4) of the FP64 GPU forward.  Perturbing one path changes only its
  own row and column of the Grams, so each difference needs only those pairs.
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


def _rel(a, b):
    return abs(a - b) / abs(b)


@pytest.fixture(scope="module")
def oscillatory():
    X = W.oscillatory(64, 1025, 4, seed=5)
    Y = W.oscillatory(64, 1025, 4, seed=6)
    return X, Y, torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")


@pytest.mark.parametrize("compute,tol", [("f32", 1e-4), ("f64", 1e-10)])
def test_oscillatory_interpolation_order8(oscillatory, compute, tol):
    X, Y, Xt, Yt = oscillatory
    idx = np.arange(64)
    out = sk.sigkernel_pairs(Xt, Yt, idx, idx, scheme="interp", degree=8, compute=compute)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    ref = oracle.pairs([X[17]], [Y[17]], [0], [0], "interp", 8, 0)[0]
    assert _rel(got[17], ref) < tol


@pytest.mark.parametrize("scheme,lam,tol", [("fd1", 2, 1e-4), ("fd2", 4, 1e-4), ("fd1", 6, 1e-3)])
def test_oscillatory_fd_refinement(oscillatory, scheme, lam, tol):
    X, Y, Xt, Yt = oscillatory
    idx = np.arange(64)
    out = sk.sigkernel_pairs(Xt, Yt, idx, idx, scheme=scheme, dyadic=lam, compute="f32")
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    ref = oracle.pairs([X[3]], [Y[3]], [0], [0], scheme, 2, lam)[0]
    assert _rel(got[3], ref) < tol


def test_uneven_batch_bf16():
    Xs = W.uneven(4096, 64, 4096, 16, seed=6)
    Ys = W.uneven(4096, 64, 4096, 16, seed=7)
    PX = sk.Paths.from_list(Xs, dtype=torch.bfloat16)
    PY = sk.Paths.from_list(Ys, dtype=torch.bfloat16)
    idx = torch.arange(4096, dtype=torch.int64, device="cuda")
    out = sk.sigkernel_pairs(PX, PY, idx, idx, compute="f32")
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    lens = np.array([len(x) * len(y) for x, y in zip(Xs, Ys)])
    rng = np.random.default_rng(8)
    sample = list(rng.choice(np.where(lens < 600 * 600)[0], 3, replace=False)) + [int(np.argmax(lens))]
    for k in sample:
        x = W.round_bf16(Xs[k])
        y = W.round_bf16(Ys[k])
        ref = oracle.pairs([x], [y], [0], [0], "approx", 6, 0)[0]
        assert _rel(got[k], ref) < 1e-4, k


@pytest.fixture(scope="module")
def mmd_batches():
    A = W.brownian(256, 513, 32, seed=7)
    B = W.brownian(256, 513, 32, seed=8, drift=0.5, vol=1.2)
    return A, B


def test_mmd2_value_and_gram_entries(mmd_batches):
    A, B = mmd_batches
    At, Bt = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    m, parts = sk.sigkernel_mmd2(At, Bt, degree=6, compute="f32")
    Kaa = sk.sigkernel_gram(At, None, degree=6, compute="f32")
    Kbb = sk.sigkernel_gram(Bt, None, degree=6, compute="f32")
    Kab = sk.sigkernel_gram(At, Bt, degree=6, compute="f32")
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    means = [Kaa.mean().item(), Kbb.mean().item(), Kab.mean().item()]
    assert np.allclose(parts.cpu().numpy(), means, rtol=1e-12)
    assert _rel(m.item(), means[0] + means[1] - 2 * means[2]) < 1e-10
    ref = oracle.pairs([A[3], B[7]], [A[11], B[200]], [0, 1, 0], [0, 1, 1], "approx", 6, 0)
    got = [Kaa[3, 11].item(), Kbb[7, 200].item(), Kab[3, 200].item()]
    assert max(_rel(g, r) for g, r in zip(got, ref)) < 1e-4


def test_mmd2_gradient_central_differences(mmd_batches):
    A, B = mmd_batches
    n, m_ = A.shape[0], B.shape[0]
    At, Bt = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    _, _, gA, gB = sk.sigkernel_mmd2(At, Bt, degree=6, compute="f32", grads=True)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    gA = gA.cpu().numpy().reshape(A.shape)
    gB = gB.cpu().numpy().reshape(B.shape)
    scale = max(np.abs(gA).max(), np.abs(gB).max())

    def path_terms(S, T_same, T_other, i, path):
        """MMD^2 terms that depend on path i of side S (the rest is constant): its row and
        column of the same-side Gram and its row of the cross Gram, FP64 on the GPU."""
        Ssame = T_same.copy()
        Ssame[i] = path
        same = sk.sigkernel_pairs(torch.tensor(Ssame, device="cuda"), torch.tensor(path[None], device="cuda"),
                                  np.arange(len(Ssame)), np.zeros(len(Ssame), dtype=np.int64), compute="f64")
        cross = sk.sigkernel_pairs(torch.tensor(path[None], device="cuda"), torch.tensor(T_other, device="cuda"),
                                   np.zeros(len(T_other), dtype=np.int64), np.arange(len(T_other)), compute="f64")
        same = same.cpu().numpy()
        cross = cross.cpu().numpy()
        ns, no = len(T_same), len(T_other)
        # K(S_i, S_i) once, K(S_i, S_j) and K(S_j, S_i) for j != i, over ns^2; cross over ns no
        return (2 * same.sum() - same[i]) / ns ** 2 - 2 * cross.sum() / (ns * no)

    rng = np.random.default_rng(9)
    h = 1e-4
    for _ in range(16):
        side = int(rng.integers(0, 2))
        S, O, g = (A, B, gA) if side == 0 else (B, A, gB)
        i, p, c = int(rng.integers(0, S.shape[0])), int(rng.integers(0, 513)), int(rng.integers(0, 32))
        xp, xm = S[i].copy(), S[i].copy()
        xp[p, c] += h
        xm[p, c] -= h
        fd = (path_terms(S, S, O, i, xp) - path_terms(S, S, O, i, xm)) / (2 * h)
        assert abs(g[i, p, c] - fd) < 1e-3 * scale, (side, i, p, c, g[i, p, c], fd)


def test_mmd2_long_paths_take_the_checkpointing_adjoint():
    """40 + 40 paths of 1025 points: one pair's tape is ~67 MB, so a 64 GiB chunk holds fewer pairs
    than half the adjoint's resident warps and each Gram block takes the checkpointing adjoint.
    Gradient entries against central differences of the FP64 GPU forward."""
    A = W.brownian(40, 1025, 2, seed=11)
    B = W.brownian(40, 1025, 2, seed=12, drift=0.5, vol=1.2)
    At, Bt = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    _, _, gA, gB = sk.sigkernel_mmd2(At, Bt, degree=6, compute="f32", grads=True)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    gA = gA.cpu().numpy().reshape(A.shape)
    gB = gB.cpu().numpy().reshape(B.shape)
    scale = max(np.abs(gA).max(), np.abs(gB).max())

    def path_terms(S, O, i, path):
        Ssame = S.copy()
        Ssame[i] = path
        same = sk.sigkernel_pairs(torch.tensor(Ssame, device="cuda"), torch.tensor(path[None], device="cuda"),
                                  np.arange(len(S)), np.zeros(len(S), dtype=np.int64), compute="f64").cpu().numpy()
        cross = sk.sigkernel_pairs(torch.tensor(path[None], device="cuda"), torch.tensor(O, device="cuda"),
                                   np.zeros(len(O), dtype=np.int64), np.arange(len(O)), compute="f64").cpu().numpy()
        return (2 * same.sum() - same[i]) / len(S) ** 2 - 2 * cross.sum() / (len(S) * len(O))

    rng = np.random.default_rng(13)
    h = 1e-4
    for _ in range(6):
        side = int(rng.integers(0, 2))
        S, O, g = (A, B, gA) if side == 0 else (B, A, gB)
        i, p, c = int(rng.integers(0, 40)), int(rng.integers(0, 1025)), int(rng.integers(0, 2))
        xp, xm = S[i].copy(), S[i].copy()
        xp[p, c] += h
        xm[p, c] -= h
        fd = (path_terms(S, O, i, xp) - path_terms(S, O, i, xm)) / (2 * h)
        assert abs(g[i, p, c] - fd) < 1e-3 * scale, (side, i, p, c, g[i, p, c], fd)
