"""Seeded synthetic path generators shaped like the paper's workloads.

This module holds no signature-kernel arithmetic: it only draws random paths (numpy
``default_rng``) so that the CUDA path and the CPU oracle can be fed identical inputs.  Every
generator returns float64 numpy arrays of points; paths start at the origin and are cumulative
sums of their increments (piecewise-linear paths, Section 2).

Workloads
  * ``brownian``     Brownian motion on [0, 1]: L points, increments N(0, vol^2/(L-1)) + drift/(L-1)
                     (the paper's 2-d standard Brownian batches, Section 4, and the Gram / MMD sets).
  * ``linear``       x_k = (k/(L-1)) u with u ~ N(0, I_d): straight lines, for which the exact kernel
                     is 0F1(;1;<u,v>) (Remark "mbf").
  * ``oscillatory``  coordinate j = sin(w_j t + phi_j) + eps, w_j ~ U(10, 200), phi_j ~ U(0, 2 pi),
                     eps ~ N(0, 1e-3) (variance), t uniform on [0, 1].
  * ``sinpath``      x_i = sin(U_i), U_i ~ N(0, I_2) i.i.d. (eq. (sinpath), Appendix B); ``cospath``
                     the matching y_i = cos(V_i).
  * ``uneven``       ragged batch: lengths floor(exp(U(ln Lmin, ln Lmax))), increments N(0, 1/L).
  * ``split_labels`` random relabellings of a pooled sample of na + nb paths (uniform random
                     permutations of the labels 1 x na, 0 x nb), the draws of a permutation test.
"""
from __future__ import annotations

import numpy as np


def brownian(n: int, L: int, d: int, seed: int, drift: float = 0.0, vol: float = 1.0) -> np.ndarray:
    """[n, L, d] Brownian paths on [0, 1] sampled at L equally spaced times, starting at 0."""
    rng = np.random.default_rng(seed)
    steps = L - 1
    out = np.zeros((n, L, d))
    if steps > 0:
        inc = rng.standard_normal((n, steps, d)) * (vol / np.sqrt(steps)) + drift / steps
        out[:, 1:, :] = np.cumsum(inc, axis=1)
    return out


def linear(n: int, L: int, d: int, seed: int) -> np.ndarray:
    """[n, L, d] straight paths x_k = (k / (L-1)) u, u ~ N(0, I_d)."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n, 1, d))
    s = (np.arange(L, dtype=np.float64) / (L - 1)).reshape(1, L, 1)
    return s * u


def linear_directions(n: int, d: int, seed: int) -> np.ndarray:
    """The directions u used by ``linear`` with the same seed (for closed-form checks)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 1, d))[:, 0, :]


def oscillatory(n: int, L: int, d: int, seed: int, wmin: float = 10.0, wmax: float = 200.0,
                noise_var: float = 1e-3) -> np.ndarray:
    """[n, L, d] highly oscillatory paths on t in [0, 1]."""
    rng = np.random.default_rng(seed)
    t = np.linspace(0.0, 1.0, L).reshape(1, L, 1)
    w = rng.uniform(wmin, wmax, size=(n, 1, d))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=(n, 1, d))
    eps = rng.standard_normal((n, L, d)) * np.sqrt(noise_var)
    return np.sin(w * t + phi) + eps


def sinpath(n: int, L: int, seed: int, d: int = 2) -> np.ndarray:
    """[n, L, d] points x_i = sin(U_i), U_i ~ N(0, I_d) i.i.d. (eq. (sinpath))."""
    rng = np.random.default_rng(seed)
    return np.sin(rng.standard_normal((n, L, d)))


def cospath(n: int, L: int, seed: int, d: int = 2) -> np.ndarray:
    """[n, L, d] points y_i = cos(V_i), V_i ~ N(0, I_d) i.i.d. (eq. (sinpath))."""
    rng = np.random.default_rng(seed)
    return np.cos(rng.standard_normal((n, L, d)))


def uneven_lengths(n: int, Lmin: int, Lmax: int, seed: int) -> np.ndarray:
    """n lengths floor(exp(U(ln Lmin, ln Lmax))) (log-uniform), clipped to [Lmin, Lmax]."""
    rng = np.random.default_rng(seed)
    L = np.floor(np.exp(rng.uniform(np.log(Lmin), np.log(Lmax), size=n))).astype(np.int64)
    return np.clip(L, Lmin, Lmax)


def uneven(n: int, Lmin: int, Lmax: int, d: int, seed: int) -> list[np.ndarray]:
    """n ragged Brownian paths: length L_k log-uniform in [Lmin, Lmax], increments N(0, 1/L_k)."""
    lengths = uneven_lengths(n, Lmin, Lmax, seed)
    rng = np.random.default_rng(seed + 1_000_003)
    out = []
    for L in lengths:
        inc = rng.standard_normal((int(L) - 1, d)) / np.sqrt(float(L))
        p = np.zeros((int(L), d))
        p[1:] = np.cumsum(inc, axis=0)
        out.append(p)
    return out


def round_bf16(a: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 (round-to-nearest-even) and return float64.

    Pure data conversion, so that a BF16 input seen by the GPU and the float64 input seen by the
    oracle are the same numbers."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def round_f32(a: np.ndarray) -> np.ndarray:
    """Round float64 values to float32 and return float64 (same purpose as ``round_bf16``)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def split_labels(nperm: int, na: int, nb: int, seed: int) -> np.ndarray:
    """[nperm, na + nb] uint8: row p marks with 1 the na pooled paths that relabelling p assigns to
    the first sample (a uniformly random permutation of na ones and nb zeros)."""
    rng = np.random.default_rng(seed)
    base = np.concatenate([np.ones(na, dtype=np.uint8), np.zeros(nb, dtype=np.uint8)])
    out = np.empty((nperm, na + nb), dtype=np.uint8)
    for p in range(nperm):
        out[p] = base[rng.permutation(na + nb)]
    return out
