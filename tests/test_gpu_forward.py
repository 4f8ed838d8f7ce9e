"""GPU forward parity: the CUDA wavefront (through the C ABI) against the FP64 CPU oracle.

Sizes span several 32-row strips with ragged tails; the full-size workloads are checked on sampled
entries.  Tolerances: FP64 cell updates agree with the oracle to rounding (the two sides sum in
different orders and coordinates); FP32 cell updates are held to the mixed-precision MAPE bar
(<= 1e-4) and usually land near 1e-6.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2502_08470_gb300 import workloads as W

pytestmark = pytest.mark.gpu

sk = pytest.importorskip("paper_2502_08470_gb300.sigkernel")


def _cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda")


def _gram_gpu(X, Y=None, **kw):
    G = sk.sigkernel_gram(_cuda(X), None if Y is None else _cuda(Y), **kw)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    return G.cpu().numpy()


def _rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def _mape(a, b):
    return float(np.mean(_rel(a, b)))


@pytest.fixture(scope="module", autouse=True)
def _cuda_available():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


# ------------------------------------------------------------------------------------------
# Polynomial approximation, FP64 plain wavefront
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("N", [2, 4, 6, 9, 16])
@pytest.mark.parametrize("lam", [0, 1])
def test_approx_f64_gram_matches_oracle(N, lam):
    X = W.brownian(5, 41, 3, seed=31)   # 40 rows: two strips, ragged tail of 8
    Y = W.brownian(4, 70, 3, seed=32)   # 69 columns
    G = _gram_gpu(X, Y, scheme="approx", degree=N, dyadic=lam, compute="f64")
    R = oracle.gram(list(X), list(Y), "approx", N, lam)
    assert np.max(_rel(G, R)) < 1e-11


@pytest.mark.parametrize("N", [2, 4, 6, 8])
def test_interp_f64_gram_matches_oracle(N):
    X = W.brownian(3, 37, 2, seed=33)
    Y = W.brownian(4, 34, 2, seed=34)
    G = _gram_gpu(X, Y, scheme="interp", degree=N, compute="f64")
    R = oracle.gram(list(X), list(Y), "interp", N)
    assert np.max(_rel(G, R)) < 1e-10


@pytest.mark.parametrize("scheme", ["fd1", "fd2", "fd_implicit"])
@pytest.mark.parametrize("lam", [0, 1, 2, 3, 5])
def test_fd_f64_gram_matches_oracle(scheme, lam):
    L = 20 if lam < 5 else 6
    X = W.brownian(3, L + 3, 2, seed=35)
    Y = W.brownian(3, L, 2, seed=36)
    G = _gram_gpu(X, Y, scheme=scheme, dyadic=lam, compute="f64")
    R = oracle.gram(list(X), list(Y), scheme, 0, lam)
    assert np.max(_rel(G, R)) < 1e-11


# ------------------------------------------------------------------------------------------
# FP32 cell updates with per-lane exponents
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("scheme,N,lam", [("approx", 6, 0), ("approx", 4, 2), ("interp", 6, 0),
                                          ("fd1", 0, 2), ("fd2", 0, 1), ("fd_implicit", 0, 0),
                                          ("fd_implicit", 0, 3)])
def test_f32_gram_mape(scheme, N, lam):
    X = W.brownian(6, 75, 4, seed=37)
    Y = W.brownian(5, 66, 4, seed=38)
    G = _gram_gpu(X, Y, scheme=scheme, degree=max(N, 2), dyadic=lam, compute="f32")
    R = oracle.gram(list(X), list(Y), scheme, max(N, 2), lam)
    assert _mape(G, R) < 1e-5
    assert np.max(_rel(G, R)) < 1e-4


def test_f32_rescaling_keeps_huge_kernels_finite():
    # Scaled Brownian paths: k up to ~1e50, beyond FP32's range without the exponents.
    X = 12.0 * W.brownian(3, 65, 2, seed=39)
    Y = 12.0 * W.brownian(3, 65, 2, seed=40)
    R = oracle.gram(list(X), list(Y), "approx", 10, 2)
    assert np.max(np.abs(R)) > 1e39
    G = _gram_gpu(X, Y, scheme="approx", degree=10, dyadic=2, compute="f32")
    assert np.all(np.isfinite(G))
    assert np.max(_rel(G, R)) < 1e-3


# ------------------------------------------------------------------------------------------
# Symmetric Gram, pair lists, ragged lengths, dtypes, increments input
# ------------------------------------------------------------------------------------------
def test_symmetric_gram_equals_full_gram():
    X = W.brownian(9, 50, 3, seed=41)
    Gs = _gram_gpu(X, None, scheme="approx", degree=6, compute="f64")
    Gf = _gram_gpu(X, X.copy(), scheme="approx", degree=6, compute="f64")
    np.testing.assert_array_equal(Gs, Gs.T)
    assert np.max(_rel(Gs, Gf)) < 1e-13
    ev = np.linalg.eigvalsh(Gs)
    assert ev.min() >= -1e-12 * ev.max()


@pytest.mark.parametrize("compute", ["f64", "f32"])
def test_ragged_pairs_match_oracle(compute):
    rng = np.random.default_rng(42)
    lengths_x = [1, 2, 3, 33, 64, 65, 97, 31, 32]
    lengths_y = [2, 1, 40, 5, 66, 33]
    Xs = [W.brownian(1, L, 3, seed=100 + i)[0] for i, L in enumerate(lengths_x)]
    Ys = [W.brownian(1, L, 3, seed=200 + i)[0] for i, L in enumerate(lengths_y)]
    pa = rng.integers(0, len(Xs), size=40)
    pb = rng.integers(0, len(Ys), size=40)
    PX = sk.Paths.from_list([torch.tensor(x) for x in Xs])
    PY = sk.Paths.from_list([torch.tensor(y) for y in Ys])
    for scheme, N in (("approx", 5), ("interp", 4), ("fd2", 0), ("fd_implicit", 0)):
        out = sk.sigkernel_pairs(PX, PY, pa, pb, scheme=scheme, degree=max(N, 2), compute=compute)
        torch.cuda.synchronize()
        assert sk.device_status() == 0
        ref = oracle.pairs(Xs, Ys, pa, pb, scheme, max(N, 2))
        tol = 1e-11 if compute == "f64" else 1e-4
        assert np.max(_rel(out.cpu().numpy(), ref)) < tol, scheme
        # single-point paths have the trivial signature
        trivial = (np.array(lengths_x)[pa] == 1) | (np.array(lengths_y)[pb] == 1)
        assert np.all(out.cpu().numpy()[trivial] == 1.0)


def test_unsorted_queue_gives_identical_results():
    Xs = [W.brownian(1, L, 2, seed=300 + L)[0] for L in (10, 90, 45, 130)]
    PX = sk.Paths.from_list([torch.tensor(x) for x in Xs])
    pa = [0, 1, 2, 3, 3, 1]
    pb = [3, 2, 1, 0, 3, 1]
    a = sk.sigkernel_pairs(PX, PX, pa, pb, scheme="approx", degree=6, sort=True)
    b = sk.sigkernel_pairs(PX, PX, pa, pb, scheme="approx", degree=6, sort=False)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_reduced_precision_inputs(dtype):
    X = W.brownian(4, 60, 8, seed=43)
    Y = W.brownian(3, 50, 8, seed=44)
    rounder = W.round_f32 if dtype == torch.float32 else W.round_bf16
    Xr, Yr = rounder(X), rounder(Y)
    G = sk.sigkernel_gram(_cuda(Xr, dtype), _cuda(Yr, dtype), scheme="approx", degree=6, compute="f64")
    torch.cuda.synchronize()
    R = oracle.gram(list(Xr), list(Yr), "approx", 6)
    tol = 1e-6 if dtype == torch.float32 else 1e-4  # increments of rounded points, formed in f32
    assert np.max(_rel(G.cpu().numpy(), R)) < tol


def test_increments_input_mode():
    X = W.brownian(3, 30, 3, seed=45)
    Y = W.brownian(2, 44, 3, seed=46)
    incX = [np.diff(x, axis=0) for x in X]
    incY = [np.diff(y, axis=0) for y in Y]
    PX = sk.Paths.from_list([torch.tensor(v) for v in incX], increments=True)
    PY = sk.Paths.from_list([torch.tensor(v) for v in incY], increments=True)
    G = sk.sigkernel_gram(PX, PY, scheme="approx", degree=6)
    torch.cuda.synchronize()
    R = oracle.gram(list(X), list(Y), "approx", 6)
    assert np.max(_rel(G.cpu().numpy(), R)) < 1e-11


# ------------------------------------------------------------------------------------------
# Closed form: linear paths -> 0F1(;1;<u,v>) (Remark "mbf"); the single-pair workload
# ------------------------------------------------------------------------------------------
def test_linear_pairs_closed_form():
    from math import factorial
    X = W.linear(64, 33, 2, seed=2)
    Y = W.linear(64, 33, 2, seed=3)
    U = W.linear_directions(64, 2, seed=2)
    V = W.linear_directions(64, 2, seed=3)
    z = np.einsum("kd,kd->k", U, V)
    want = np.array([sum(zz ** n / factorial(n) ** 2 for n in range(60)) for zz in z])
    PX = sk.Paths.from_dense(_cuda(X))
    PY = sk.Paths.from_dense(_cuda(Y))
    idx = np.arange(64)
    got = sk.sigkernel_pairs(PX, PY, idx, idx, scheme="approx", degree=14, compute="f64").cpu().numpy()
    assert np.max(_rel(got, want)) < 1e-12


def test_single_pair_workload_approx4_and_fd2():
    X = W.brownian(2, 33, 2, seed=1)
    for scheme, N, lam in (("approx", 4, 0), ("fd1", 0, 2), ("fd2", 0, 2)):
        got = sk.sigkernel_pairs(_cuda(X[:1]), _cuda(X[1:]), [0], [0], scheme=scheme, degree=max(N, 2),
                                 dyadic=lam, compute="f64").cpu().numpy()
        ref = oracle.kernel(X[0], X[1], scheme, max(N, 2), lam)
        assert abs(got[0] - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("compute", ["f64", "f32"])
def test_fd_implicit_singular_cell_reports_nonfinite(compute):
    """Remark "higherfd" read with the trapezoid weight 1/4: a cell with m = <dx, dy> = 4 makes
    the implicit cell equation singular (1 - m/4 = 0); the call records SK_ERR_NONFINITE and the
    other pairs of the batch are unaffected."""
    x = np.array([[[0.0, 0.0], [2.0, 0.0]]])
    y = np.array([[[0.0, 0.0], [2.0, 1.0]], [[0.0, 0.0], [0.5, 0.3]]])
    out = sk.sigkernel_pairs(_cuda(x), _cuda(y), [0, 0], [0, 1], scheme="fd_implicit", compute=compute)
    torch.cuda.synchronize()
    assert sk.device_status() == -6
    got = out.cpu().numpy()
    assert not np.isfinite(got[0])
    m = 2.0 * 0.5
    assert got[1] == pytest.approx((1 + 0.75 * m) / (1 - 0.25 * m), rel=1e-6)


# ------------------------------------------------------------------------------------------
# Full-size Gram workload (128 x 128 paths, 257 points, d = 8), sampled entries
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("compute,tol", [("f32", 1e-4), ("f64", 1e-11)])
def test_full_size_gram_sampled(compute, tol):
    X = W.brownian(128, 257, 8, seed=3)
    Y = W.brownian(128, 257, 8, seed=4)
    G = _gram_gpu(X, Y, scheme="approx", degree=6, compute=compute)
    rng = np.random.default_rng(5)
    pa = rng.integers(0, 128, size=12)
    pb = rng.integers(0, 128, size=12)
    ref = oracle.pairs(list(X), list(Y), pa, pb, "approx", 6)
    assert np.max(_rel(G[pa, pb], ref)) < tol
    assert np.all(np.isfinite(G))


# ------------------------------------------------------------------------------------------
# Error paths (host-side checks, and a device-side length check that only records a code)
# ------------------------------------------------------------------------------------------
def test_invalid_arguments_are_rejected():
    X = _cuda(W.brownian(2, 10, 2, seed=47))
    with pytest.raises(sk.SigKernelError) as e:
        sk.sigkernel_gram(X, X.clone(), scheme="approx", degree=1)
    assert e.value.code == -1
    with pytest.raises(sk.SigKernelError):
        sk.sigkernel_gram(X, X.clone(), scheme="approx", degree=6, dyadic=9)
    with pytest.raises(sk.SigKernelError) as e:
        sk.sigkernel_gram(X, X.clone(), scheme="interp", degree=13)
    assert e.value.code == -1


def test_bad_length_sets_device_error_and_nan():
    X = _cuda(W.brownian(3, 12, 2, seed=48))
    P = sk.Paths.from_dense(X)
    P.max_len = 5  # every path is longer than the declared bound
    out = sk.sigkernel_pairs(P, P, [0, 1], [1, 2], scheme="approx", degree=4)
    torch.cuda.synchronize()
    assert sk.device_status() == -7
    assert torch.isnan(out).all()
    assert sk.device_status() == 0  # the word was cleared
