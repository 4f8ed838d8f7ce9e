"""GPU tests of the strip pipeline: long pairs swept by a block of warps, one 32-row strip per warp,
with the strip hand-off ordered by progress counters in shared memory.

Each cell runs the same arithmetic on the same inputs in the pipelined and the one-warp sweep,
so the two must agree bit for bit; the oracle pins both on sampled pairs.  The batches mix
pairs of one strip (one warp each, inside the same launch) with pairs of up to ten strips, and
the path lengths leave ragged last strips and tiles.
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


def _ragged(seed, lengths, d):
    return [W.brownian(1, n, d, seed=seed + i)[0] for i, n in enumerate(lengths)]


LX = [300, 20, 97, 257, 33, 161]   # 1 to 10 strips of 32 rows
LY = [129, 300, 40, 7, 64]


def _paths(seed, lengths, d=3):
    return sk.Paths.from_list([torch.tensor(x) for x in _ragged(seed, lengths, d)])


CASES = [
    ("approx", 6, 0, "f32", 1e-4),
    ("approx", 6, 0, "f64", 1e-11),
    ("approx", 4, 1, "f32", 1e-4),
    ("interp", 8, 0, "f32", 1e-4),
    ("interp", 5, 0, "f64", 1e-11),
    ("fd1", 0, 2, "f32", 1e-4),
    ("fd2", 0, 3, "f64", 1e-11),
    ("fd_implicit", 0, 2, "f32", 1e-4),
    ("fd_implicit", 0, 1, "f64", 1e-11),
]


@pytest.mark.parametrize("scheme,N,lam,compute,tol", CASES)
def test_pipelined_gram_is_bitwise_the_one_warp_gram(scheme, N, lam, compute, tol):
    X = _paths(31, LX)
    Y = _paths(61, LY)
    kw = dict(scheme=scheme, degree=max(N, 2), dyadic=lam, compute=compute)
    G1 = sk.sigkernel_gram(X, Y, strip_pipeline=False, **kw)
    G2 = sk.sigkernel_gram(X, Y, strip_pipeline=True, **kw)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    assert torch.equal(G1, G2)
    # sampled pairs against the oracle, including the 10-strip one
    Xs, Ys = _ragged(31, LX, 3), _ragged(61, LY, 3)
    pa, pb = [0, 3, 5, 2], [1, 0, 4, 2]
    ref = oracle.pairs([Xs[a] for a in pa], [Ys[b] for b in pb], list(range(4)), list(range(4)), scheme,
                       max(N, 2), lam)
    got = G2.cpu().numpy()[pa, pb]
    assert np.max(np.abs(got - ref) / np.abs(ref)) < tol


@pytest.mark.parametrize("compute", ["f32", "f64"])
def test_pipelined_symmetric_gram(compute):
    X = _paths(91, [200, 31, 130, 64, 300])
    G1 = sk.sigkernel_gram(X, None, compute=compute, strip_pipeline=False)
    G2 = sk.sigkernel_gram(X, None, compute=compute, strip_pipeline=True)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    assert torch.equal(G1, G2)
    assert torch.equal(G2, G2.T)


def test_pipelined_pairs_list_with_repeats():
    X = _paths(101, [400, 50])
    Y = _paths(131, [380, 90, 33])
    pa, pb = [0, 0, 1, 0, 0], [0, 1, 2, 0, 2]
    o1 = sk.sigkernel_pairs(X, Y, pa, pb, compute="f32", strip_pipeline=False)
    o2 = sk.sigkernel_pairs(X, Y, pa, pb, compute="f32", strip_pipeline=True)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    assert torch.equal(o1, o2)
    assert o2[0].item() == o2[3].item()


def test_long_pairs_take_the_pipeline_by_default():
    """Few pairs of 1025-point paths (32 strips each): the library pipelines them on its own
    (the launch has 16-warp blocks) and the results equal the one-warp sweep (itself pinned to the
    oracle in the forward tests)."""
    rng = np.random.default_rng(5)
    X = W.oscillatory(4, 1025, 4, seed=5)
    Y = W.oscillatory(4, 1025, 4, seed=6)
    Xt, Yt = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    pa = rng.integers(0, 4, 6)
    pb = rng.integers(0, 4, 6)
    auto = sk.sigkernel_pairs(Xt, Yt, pa, pb, scheme="interp", degree=8, compute="f32", time_kernel=True)
    torch.cuda.synchronize()
    t_auto = sk.last_kernel_ms()
    one = sk.sigkernel_pairs(Xt, Yt, pa, pb, scheme="interp", degree=8, compute="f32", strip_pipeline=False,
                             time_kernel=True)
    torch.cuda.synchronize()
    t_one = sk.last_kernel_ms()
    assert sk.device_status() == 0
    assert torch.equal(auto, one)
    assert t_auto < t_one  # 16 warps per pair instead of 1


@pytest.mark.parametrize("scheme,N,compute", [("approx", 6, "f32"), ("approx", 6, "f64"), ("interp", 8, "f32")])
def test_grid_pipeline_spreads_few_long_pairs_over_blocks(scheme, N, compute):
    """Four pairs with up to 128 strips: each pair's ring of warps spans several co-resident
    blocks (progress words in global memory).  Results equal the one-warp sweep bit for bit, the
    shortest pair is pinned to the oracle, and the spread sweep is faster."""
    Xs = [W.brownian(1, n, 3, seed=141 + i)[0] for i, n in enumerate((4097, 1500, 700))]
    Ys = [W.brownian(1, n, 3, seed=151 + i)[0] for i, n in enumerate((3000, 64))]
    PX = sk.Paths.from_list([torch.tensor(x) for x in Xs])
    PY = sk.Paths.from_list([torch.tensor(y) for y in Ys])
    pa, pb = [0, 1, 2, 0], [0, 1, 0, 1]
    kw = dict(scheme=scheme, degree=N, compute=compute)
    auto = sk.sigkernel_pairs(PX, PY, pa, pb, time_kernel=True, **kw)
    torch.cuda.synchronize()
    t_auto = sk.last_kernel_ms()
    one = sk.sigkernel_pairs(PX, PY, pa, pb, strip_pipeline=False, time_kernel=True, **kw)
    torch.cuda.synchronize()
    t_one = sk.last_kernel_ms()
    assert sk.device_status() == 0
    assert torch.equal(auto, one)
    ref = oracle.pairs([Xs[1]], [Ys[1]], [0], [0], scheme, N, 0)[0]
    tol = 1e-4 if compute == "f32" else 1e-11
    assert abs(auto[1].item() - ref) <= tol * abs(ref)
    assert t_auto < t_one / 4


def test_grid_pipeline_captures_into_a_cuda_graph():
    """One pair of 4097-point paths (a ring of eight 16-warp blocks, launched co-resident) replayed
    from a CUDA graph on new inputs written into the same buffers."""
    X = torch.tensor(W.brownian(1, 4097, 3, seed=161), device="cuda")
    Y = torch.tensor(W.brownian(1, 4097, 3, seed=162), device="cuda")
    idx = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    sk.sigkernel_pairs(X, Y, idx, idx, compute="f32", out=out)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            sk.sigkernel_pairs(X, Y, idx, idx, compute="f32", out=out)
    torch.cuda.synchronize()
    X.copy_(torch.tensor(W.brownian(1, 4097, 3, seed=163), device="cuda"))
    out.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    ref = sk.sigkernel_pairs(X, Y, idx, idx, compute="f32", strip_pipeline=False)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    assert torch.equal(out, ref)
