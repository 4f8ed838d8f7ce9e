"""GPU tests of the launch-shape autotuner and of CUDA-graph capture of the forward calls.

Every launch shape runs the same per-cell arithmetic, so a tuned call must return bit for bit
what the default shape returns (with M on the FMA pipe: the tensor-core M of the one-warp-per-pair
shape rounds differently, so these calls pass tensor_cores=False).  A call given its workspace
allocates and synchronises nothing, so it can be captured in a CUDA graph and replayed on new
input values written into the same buffers.
"""
import numpy as np
import pytest
import torch

from paper_2502_08470_gb300 import workloads as W

pytestmark = pytest.mark.gpu

sk = pytest.importorskip("paper_2502_08470_gb300.sigkernel")


@pytest.fixture(scope="module", autouse=True)
def _cuda_available():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _uneven_batch(n, seed, dtype=torch.bfloat16):
    X = sk.Paths.from_list(W.uneven(n, 64, 2048, 16, seed=seed), dtype=dtype)
    Y = sk.Paths.from_list(W.uneven(n, 64, 2048, 16, seed=seed + 1), dtype=dtype)
    return X, Y


def test_autotune_uneven_batch_chooses_the_pipeline_and_keeps_results():
    sk.autotune_clear()
    X, Y = _uneven_batch(192, 40)
    idx = torch.arange(192, dtype=torch.int64, device="cuda")
    ref = sk.sigkernel_pairs(X, Y, idx, idx, compute="f32", strip_pipeline=False, tensor_cores=False)
    shape, ms = sk.autotune(X, Y, idx, idx, compute="f32", trials=2)
    assert ms > 0
    # 192 pairs of up to 2047 x 2047 cells cannot fill the GPU one warp per pair
    assert shape["strip_pipeline"] is True
    tuned = sk.sigkernel_pairs(X, Y, idx, idx, compute="f32", tensor_cores=False)  # the remembered shape
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    assert torch.equal(tuned, ref)
    sk.autotune_clear()


def test_autotune_gram_returns_an_explicit_shape():
    sk.autotune_clear()
    X = torch.tensor(W.brownian(24, 65, 4, seed=41), device="cuda")
    shape, ms = sk.autotune(X, None, compute="f64", trials=1)
    assert shape["strip_pipeline"] or shape["warps_per_block"] in (1, 2, 4)
    G = sk.sigkernel_gram(X, None, compute="f64")
    G0 = sk.sigkernel_gram(X, None, compute="f64", strip_pipeline=False)
    torch.cuda.synchronize()
    assert torch.equal(G, G0)
    sk.autotune_clear()


def test_gram_call_captures_into_a_cuda_graph():
    X = torch.tensor(W.brownian(32, 129, 8, seed=42), device="cuda")
    Y = torch.tensor(W.brownian(32, 129, 8, seed=43), device="cuda")
    ws = sk.gram_workspace(X, Y, compute="f32")
    G = torch.empty(32, 32, dtype=torch.float64, device="cuda")
    sk.sigkernel_gram(X, Y, compute="f32", workspace=ws, out=G)  # eager run before capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            sk.sigkernel_gram(X, Y, compute="f32", workspace=ws, out=G)
    torch.cuda.synchronize()
    for seed in (44, 45):
        X.copy_(torch.tensor(W.brownian(32, 129, 8, seed=seed), device="cuda"))
        G.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        ref = sk.sigkernel_gram(X, Y, compute="f32")
        torch.cuda.synchronize()
        assert sk.device_status() == 0
        assert torch.equal(G, ref)


def test_autotuned_uneven_batch_captures_into_a_cuda_graph():
    """The uneven-batch workload as one autotuned persistent launch replayed from a CUDA graph."""
    sk.autotune_clear()
    X, Y = _uneven_batch(128, 50)
    idx = torch.arange(128, dtype=torch.int64, device="cuda")
    shape, _ = sk.autotune(X, Y, idx, idx, compute="f32", trials=1)
    out = torch.empty(128, dtype=torch.float64, device="cuda")
    sk.sigkernel_pairs(X, Y, idx, idx, compute="f32", out=out, tensor_cores=False)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            sk.sigkernel_pairs(X, Y, idx, idx, compute="f32", out=out, tensor_cores=False)
    torch.cuda.synchronize()
    rng = np.random.default_rng(51)
    X.rows.mul_(torch.tensor(rng.uniform(0.5, 1.5, size=(1, 16)), dtype=X.rows.dtype, device="cuda"))
    out.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    ref = sk.sigkernel_pairs(X, Y, idx, idx, compute="f32", strip_pipeline=not shape["strip_pipeline"],
                             tensor_cores=False)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    assert torch.equal(out, ref)
    sk.autotune_clear()
