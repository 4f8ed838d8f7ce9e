"""Randomised GPU parity: seeded random configurations (scheme, order, dyadic refinement, d, ragged
lengths, pair lists with repeats, FP32 and FP64) against the oracle, plus forward and tape-adjoint
agreement for the polynomial schemes.

Each configuration is small enough for the oracle to finish in well under a second; together they
cross the strip boundaries (32 rows), the vector widths of the increment rows (d padded to 4 or
2), the tiled-M threshold (d >= 12) and the lengths that leave single-point paths.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2502_08470_gb300 import workloads as W

pytestmark = pytest.mark.gpu

sk = pytest.importorskip("paper_2502_08470_gb300.sigkernel")

SCHEMES = ["fd1", "fd2", "fd_implicit", "approx", "interp"]


@pytest.fixture(scope="module", autouse=True)
def _cuda_available():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _config(seed):
    rng = np.random.default_rng(seed)
    scheme = SCHEMES[int(rng.integers(0, len(SCHEMES)))]
    N = int(rng.integers(2, 13 if scheme == "interp" else 17))
    lam = int(rng.integers(0, 3))
    d = int(rng.integers(1, 21))
    compute = "f64" if rng.random() < 0.5 else "f32"
    lx = [int(v) for v in rng.integers(1, 70, size=int(rng.integers(1, 5)))]
    ly = [int(v) for v in rng.integers(1, 70, size=int(rng.integers(1, 5)))]
    npairs = int(rng.integers(1, 9))
    pa = rng.integers(0, len(lx), size=npairs)
    pb = rng.integers(0, len(ly), size=npairs)
    scale = float(rng.uniform(0.3, 1.5))
    return scheme, N, lam, d, compute, lx, ly, pa, pb, scale


@pytest.mark.parametrize("seed", range(24))
def test_random_configuration_matches_oracle(seed):
    scheme, N, lam, d, compute, lx, ly, pa, pb, scale = _config(1000 + seed)
    Xs = [scale * W.brownian(1, n, d, seed=2000 + 10 * seed + i)[0] for i, n in enumerate(lx)]
    Ys = [scale * W.brownian(1, n, d, seed=3000 + 10 * seed + i)[0] for i, n in enumerate(ly)]
    # keep every sub-cell's m = <dx, dy> / 4^lambda within 1/2: the schemes stay well conditioned
    # (the implicit one is singular at m = 4) and FP32 can be held to a fixed bar
    mmax = max((np.abs(np.diff(Xs[a], axis=0) @ np.diff(Ys[b], axis=0).T).max(initial=0.0)
                for a, b in zip(pa, pb)), default=0.0) / 4 ** lam
    if mmax > 0.5:
        f = np.sqrt(0.5 / mmax)
        Xs, Ys = [f * x for x in Xs], [f * y for y in Ys]
    PX = sk.Paths.from_list([torch.tensor(x) for x in Xs])
    PY = sk.Paths.from_list([torch.tensor(y) for y in Ys])
    got = sk.sigkernel_pairs(PX, PY, pa, pb, scheme=scheme, degree=N, dyadic=lam, compute=compute)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    ref = oracle.pairs(Xs, Ys, pa, pb, scheme, N, lam)
    # relative to |k| + 1 (k = 1 + ..., and a kernel value can cross zero)
    tol = 1e-10 if compute == "f64" else 2e-4
    err = np.abs(got.cpu().numpy() - ref) / (np.abs(ref) + 1.0)
    assert np.max(err) < tol, (scheme, N, lam, d, compute, lx, ly, err)


@pytest.mark.parametrize("seed", range(8))
def test_random_configuration_tape_gradient_matches_oracle(seed):
    rng = np.random.default_rng(5000 + seed)
    scheme = "approx" if seed % 2 == 0 else "interp"
    N = int(rng.integers(2, 9))
    lam = int(rng.integers(0, 2))
    d = int(rng.integers(1, 14))
    compute = "f64" if seed % 4 < 2 else "f32"
    x = W.brownian(1, int(rng.integers(3, 40)), d, seed=6000 + seed)[0]
    y = W.brownian(1, int(rng.integers(3, 40)), d, seed=7000 + seed)[0]
    X, Y = torch.tensor(x[None], device="cuda"), torch.tensor(y[None], device="cuda")
    idx = [0]
    kw = dict(pair_a=idx, pair_b=idx, scheme=scheme, degree=N, dyadic=lam, compute=compute)
    out, tape = sk.sigkernel_forward_tape(X, Y, **kw)
    gX, gY = sk.sigkernel_backward_tape(tape, torch.ones(1, dtype=torch.float64, device="cuda"), X, Y, **kw)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    rx, ry = oracle.grad(x, y, scheme, N, lam)
    scale = max(np.max(np.abs(rx)), np.max(np.abs(ry)))
    tol = 1e-9 if compute == "f64" else 2e-4
    assert np.max(np.abs(gX.cpu().numpy().reshape(x.shape) - rx)) < tol * scale
    assert np.max(np.abs(gY.cpu().numpy().reshape(y.shape) - ry)) < tol * scale
