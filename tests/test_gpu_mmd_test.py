"""GPU parity of the two-sample permutation test on MMD^2 (sigkernel_mmd2_test) against the oracle's
test over the pooled Gram.

The pooled samples span two 32-path label words with a ragged tail, and the relabelling counts
leave a ragged last block of the statistics kernel.  Statistics are differences of Gram means, so
they are compared with an absolute tolerance scaled by the mean |K|; the p-value is checked against
its definition on the GPU's own statistics, and against the oracle's p-value wherever no
statistic lies within the tolerance of the observed one.
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


def _check_against_oracle(A, B, labels, got, scheme, N, lam, unbiased, tol):
    obs, p, stats = (t.cpu().numpy() if t.dim() else t.item() for t in got)
    r_obs, r_p, r_stats = oracle.mmd2_permutation_test(A, B, labels, scheme, N, lam, unbiased=unbiased)
    Z = list(A) + list(B)
    scale = np.abs(oracle.gram(Z[:4], Z[-4:], scheme, N, lam)).mean()
    assert abs(obs - r_obs) <= tol * scale
    assert np.max(np.abs(stats - r_stats)) <= tol * scale
    # the p-value is its definition on the GPU's statistics ...
    assert p == (1 + np.count_nonzero(stats >= obs)) / (1 + len(stats))
    # ... and the oracle's wherever no statistic is within the tolerance of the observed one
    if np.all(np.abs(r_stats - r_obs) > 2 * tol * scale):
        assert p == r_p


@pytest.mark.parametrize("unbiased", [False, True])
@pytest.mark.parametrize("compute,tol", [("f64", 1e-11), ("f32", 1e-5)])
def test_permutation_test_matches_oracle(unbiased, compute, tol):
    A = W.brownian(17, 21, 3, seed=81)
    B = W.brownian(23, 21, 3, seed=82, drift=0.3)  # 40 pooled paths: two label words, tail of 8
    labels = W.split_labels(37, 17, 23, seed=83)   # 38 statistics: last block holds 6 of 8
    got = sk.sigkernel_mmd2_test(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"),
                                 labels=torch.tensor(labels, device="cuda"), degree=5, compute=compute,
                                 unbiased=unbiased)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    _check_against_oracle(A, B, labels, got, "approx", 5, 0, unbiased, tol)


@pytest.mark.parametrize("scheme,N,lam", [("interp", 6, 0), ("fd_implicit", 2, 2)])
def test_permutation_test_ragged_paths_other_schemes(scheme, N, lam):
    As = [W.brownian(1, L, 2, seed=90 + L)[0] for L in (5, 33, 12, 40, 2, 19, 27)]
    Bs = [W.brownian(1, L, 2, seed=190 + L, drift=0.5)[0] for L in (30, 8, 21, 3, 36)]
    PA = sk.Paths.from_list([torch.tensor(x) for x in As])
    PB = sk.Paths.from_list([torch.tensor(x) for x in Bs])
    labels = W.split_labels(9, 7, 5, seed=91)
    got = sk.sigkernel_mmd2_test(PA, PB, labels=torch.tensor(labels, device="cuda"), scheme=scheme, degree=N,
                                 dyadic=lam, compute="f64")
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    _check_against_oracle(As, Bs, labels, got, scheme, N, lam, False, 1e-11)


def test_no_relabellings_gives_the_mmd2_of_the_split():
    A = torch.tensor(W.brownian(6, 15, 2, seed=84), device="cuda")
    B = torch.tensor(W.brownian(9, 15, 2, seed=85), device="cuda")
    obs, p, stats = sk.sigkernel_mmd2_test(A, B, permutations=0, degree=6)
    m, _ = sk.sigkernel_mmd2(A, B, degree=6)
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    assert stats.numel() == 0 and p.item() == 1.0
    assert obs.item() == pytest.approx(m.item(), rel=1e-12)


def test_a_bad_relabelling_is_reported_and_isolated():
    A = W.brownian(5, 9, 2, seed=86)
    B = W.brownian(4, 9, 2, seed=87)
    labels = W.split_labels(11, 5, 4, seed=88)
    labels[3, np.flatnonzero(labels[3])[0]] = 0  # marks 4 paths instead of 5
    out = sk.sigkernel_mmd2_test(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"),
                                 labels=torch.tensor(labels, device="cuda"), degree=4)
    torch.cuda.synchronize()
    assert sk.device_status() == -8
    stats = out[2].cpu().numpy()
    assert np.isnan(stats[3]) and np.all(np.isfinite(np.delete(stats, 3)))
    assert np.isnan(out[1].item())  # no p-value over the remaining relabellings
    good = np.delete(labels, 3, axis=0)
    _, _, r_stats = oracle.mmd2_permutation_test(A, B, good, "approx", 4)
    assert np.max(np.abs(np.delete(stats, 3) - r_stats)) < 1e-11


def test_full_size_mmd_workload_permutation_test():
    """256 + 256 paths of 513 points, d = 32, FP32 cells, 1000 relabellings: the observed statistic
    equals sigkernel_mmd2 (same Gram entries, another reduction) and three relabellings equal
    sigkernel_mmd2 of the relabelled sets (whose Grams solve some pairs with x and y exchanged, so
    entries agree to FP32 rounding).  Drift 0.5 and volatility 1.2 separate the samples."""
    A = W.brownian(256, 513, 32, seed=7)
    B = W.brownian(256, 513, 32, seed=8, drift=0.5, vol=1.2)
    At, Bt = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    labels = torch.tensor(W.split_labels(1000, 256, 256, seed=89), device="cuda")
    obs, p, stats = sk.sigkernel_mmd2_test(At, Bt, labels=labels, compute="f32")
    m, parts = sk.sigkernel_mmd2(At, Bt, compute="f32")
    torch.cuda.synchronize()
    assert sk.device_status() == 0
    assert obs.item() == pytest.approx(m.item(), rel=1e-10)
    assert p.item() == 1 / 1001
    Z = torch.cat([At, Bt])
    lab = labels.cpu().numpy()
    for k in (0, 499, 999):
        first = torch.tensor(lab[k] != 0, device="cuda")
        mk, _ = sk.sigkernel_mmd2(Z[first], Z[~first], compute="f32")
        assert abs(stats[k].item() - mk.item()) <= 1e-5 * parts.abs().max().item()
