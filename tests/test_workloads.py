"""CPU checks that the seeded generators draw the input recipes they document: shapes, starting
points, increment means and variances, value ranges, the log-uniform length mix of the ragged
batch, exact BF16 rounding and the relabellings of the permutation test.  Statistical checks use
tolerances of about five standard errors."""
import numpy as np
import pytest
import torch

from paper_2502_08470_gb300 import workloads as W


def test_brownian_increments_have_the_stated_law():
    n, L, d = 64, 257, 8
    X = W.brownian(n, L, d, seed=3)
    assert X.shape == (n, L, d) and np.all(X[:, 0] == 0.0)
    inc = np.diff(X, axis=1).ravel()
    var = 1.0 / (L - 1)
    assert abs(inc.mean()) < 5 * np.sqrt(var / inc.size)
    assert abs(inc.var() / var - 1.0) < 5 * np.sqrt(2.0 / inc.size)
    # drift and volatility: increments N(drift/(L-1), vol^2/(L-1))
    Y = W.brownian(n, L, d, seed=4, drift=0.5, vol=1.2)
    jnc = np.diff(Y, axis=1).ravel()
    var = 1.44 / (L - 1)
    assert abs(jnc.mean() - 0.5 / (L - 1)) < 5 * np.sqrt(var / jnc.size)
    assert abs(jnc.var() / var - 1.0) < 5 * np.sqrt(2.0 / jnc.size)


def test_generators_are_seeded():
    assert np.array_equal(W.brownian(3, 9, 2, seed=7), W.brownian(3, 9, 2, seed=7))
    assert not np.array_equal(W.brownian(3, 9, 2, seed=7), W.brownian(3, 9, 2, seed=8))
    assert np.array_equal(W.oscillatory(2, 33, 4, seed=5), W.oscillatory(2, 33, 4, seed=5))
    a, b = W.uneven(5, 64, 4096, 16, seed=9), W.uneven(5, 64, 4096, 16, seed=9)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_linear_paths_are_straight_lines_through_the_origin():
    X = W.linear(4, 17, 3, seed=2)
    u = W.linear_directions(4, 3, seed=2)
    s = np.arange(17) / 16
    assert np.allclose(X, s[None, :, None] * u[:, None, :], rtol=0, atol=1e-15)
    inc = np.diff(X, axis=1)
    assert np.allclose(inc, inc[:, :1], rtol=0, atol=1e-15)  # equal increments


def test_oscillatory_paths():
    X = W.oscillatory(64, 1025, 4, seed=6)
    noise = np.sqrt(1e-3)
    assert X.shape == (64, 1025, 4)
    assert np.all(np.abs(X) < 1 + 6 * noise)
    # w >= 10 on t in [0, 1] sweeps at least 10 rad of phase: 10 / pi > 3 half-periods, so every
    # coordinate changes sign at least 3 times
    crossings = np.count_nonzero(np.diff(np.sign(X), axis=1), axis=1)
    assert crossings.min() >= 3


def test_sin_and_cos_paths():
    n, L = 200, 50
    x, y = W.sinpath(n, L, seed=1), W.cospath(n, L, seed=2)
    assert x.shape == y.shape == (n, L, 2)
    assert np.all(np.abs(x) <= 1) and np.all(np.abs(y) <= 1)
    # E sin(U) = 0, E cos(V) = exp(-1/2) for standard normal U, V
    se = 1.0 / np.sqrt(x.size)
    assert abs(x.mean()) < 5 * se
    assert abs(y.mean() - np.exp(-0.5)) < 5 * se


def test_uneven_batch_is_log_uniform():
    Lmin, Lmax = 64, 4096
    lens = W.uneven_lengths(4096, Lmin, Lmax, seed=11)
    assert lens.min() >= Lmin and lens.max() <= Lmax
    # log-uniform: half the lengths below the geometric mean of the bounds, a quarter below the
    # point a quarter of the way from ln Lmin to ln Lmax
    se = 0.5 / np.sqrt(lens.size)
    assert abs(np.mean(lens < np.sqrt(Lmin * Lmax)) - 0.5) < 5 * se
    assert abs(np.mean(lens < (Lmin ** 3 * Lmax) ** 0.25) - 0.25) < 5 * se
    paths = W.uneven(64, Lmin, Lmax, 16, seed=12)
    assert [p.shape[0] for p in paths] == list(W.uneven_lengths(64, Lmin, Lmax, seed=12))
    z = np.concatenate([np.diff(p, axis=0).ravel() * np.sqrt(p.shape[0]) for p in paths])
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)  # increments N(0, 1/L)


def test_bf16_rounding_matches_torch_and_is_exact():
    rng = np.random.default_rng(13)
    a = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000),
                        [0.0, -0.0, 1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8)]])
    r = W.round_bf16(a)
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(r, ref)
    # ties go to the even mantissa
    assert r[-3] == 1.0 and r[-2] == 1 + 2.0 ** -6 and r[-1] == -1.0
    bits = r.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)
    assert np.array_equal(W.round_f32(a), a.astype(np.float32).astype(np.float64))


def test_split_labels_are_uniform_relabellings():
    nperm, na, nb = 4000, 17, 23
    lab = W.split_labels(nperm, na, nb, seed=83)
    assert lab.shape == (nperm, na + nb) and lab.dtype == np.uint8
    assert np.all(lab.sum(axis=1) == na)
    # each pooled path is in the first sample with probability na / (na + nb)
    p = na / (na + nb)
    se = np.sqrt(p * (1 - p) / nperm)
    assert np.max(np.abs(lab.mean(axis=0) - p)) < 5 * se
    assert len({row.tobytes() for row in lab}) == nperm  # C(40, 17) ~ 8.9e10: repeats are unlikely


@pytest.mark.parametrize("na,nb", [(1, 1), (5, 0), (0, 3)])
def test_split_labels_degenerate_sizes(na, nb):
    lab = W.split_labels(3, na, nb, seed=0)
    assert lab.shape == (3, na + nb) and np.all(lab.sum(axis=1) == na)
