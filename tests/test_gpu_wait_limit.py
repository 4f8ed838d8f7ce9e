"""GPU test of the bounded waits of the strip pipeline: a hand-off wait that runs out records
SK_ERR_DEVICE_TIMEOUT in the device error word and the kernel still returns, leaving the context
usable, so the next call is exact.

The waits poll a progress word that another warp of the same launch publishes (plain memory
polls, no barrier); sigkernel_set_wait_limit shortens them to one poll, which cannot cover the 31
steps a pipelined strip lags the strip below it, so the first wait of the second strip runs out.
Nothing is faulted: the limit only decides when a bounded wait gives up.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2502_08470_gb300 import workloads as W

pytestmark = pytest.mark.gpu
sk = pytest.importorskip("paper_2502_08470_gb300.sigkernel")

SK_ERR_DEVICE_TIMEOUT = -5


@pytest.fixture(scope="module", autouse=True)
def _cuda_available():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("scheme,N,lam,compute,tol", [("approx", 6, 0, "f32", 1e-4), ("fd1", 2, 1, "f64", 1e-11)])
def test_exhausted_hand_off_wait_reports_a_timeout_and_the_next_call_is_exact(scheme, N, lam, compute, tol):
    X = W.brownian(2, 300, 3, seed=301)  # 299 rows: 10 strips
    Y = W.brownian(2, 129, 3, seed=302)
    Xt, Yt = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    kw = dict(scheme=scheme, degree=N, dyadic=lam, compute=compute, strip_pipeline=True)
    assert sk.device_status() == 0
    sk.set_wait_limit(1)
    try:
        sk.sigkernel_gram(Xt, Yt, **kw)
        torch.cuda.synchronize()
        assert sk.device_status() == SK_ERR_DEVICE_TIMEOUT
    finally:
        sk.set_wait_limit(0)
    G = sk.sigkernel_gram(Xt, Yt, **kw)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    ref = oracle.gram(list(X), list(Y), scheme, N, lam)
    assert np.max(np.abs(G.cpu().numpy() - ref) / np.abs(ref)) < tol


def test_exhausted_wait_of_a_ring_spanning_blocks():
    """One pair of 4097-point paths (128 strips): its ring of 16-warp blocks spans co-resident
    blocks and the progress words live in global memory."""
    X = W.brownian(1, 4097, 2, seed=303)
    Y = W.brownian(1, 1025, 2, seed=304)
    Xt, Yt = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    i0 = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert sk.device_status() == 0
    sk.set_wait_limit(1)
    try:
        sk.sigkernel_pairs(Xt, Yt, i0, i0, compute="f32")
        torch.cuda.synchronize()
        assert sk.device_status() == SK_ERR_DEVICE_TIMEOUT
    finally:
        sk.set_wait_limit(0)
    out = sk.sigkernel_pairs(Xt, Yt, i0, i0, compute="f32")
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    ref = oracle.kernel(X[0], Y[0], "approx", 6)
    assert abs(out.item() - ref) / abs(ref) < 1e-4
