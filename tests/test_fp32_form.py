"""CPU model of the kernels' mixed-precision cell form: FP32 cells with a power-of-two exponent
per lane, against the FP64 oracle and closed forms.

The model restates what the FP32 wavefront kernels do:
* The approximation map runs in FP32 on factorial-scaled edge coefficients, with
  e_m = M^m / m! formed in FP64 and rounded.
* Each lane's two output edges share one exponent. When the leading coefficient of either edge
  leaves [2^-64, 2^64], both edges are rescaled by 2^-+64 and the exponent moves by 64
  (rescale_edges).
* A cell's two input edges are first brought to the larger of their exponents, and a side more
  than 126 binary orders below is flushed to zero (align_inputs).
* The endpoint is summed in FP64 and scaled by 2^exponent.

What it shows:
* On Brownian pairs the FP32 form stays within 1e-6 of the oracle, on the kernel's own scale
  sqrt(k(x, x) k(y, y)).
* For a linear pair with <u, v> = 2500 the kernel is about 1.07e42, beyond FP32's 3.4e38. The
  exponents keep the FP32 form within 2e-5 of the FP64 scheme; without them the cells overflow.
* For <u, v> = -2500 the approximation scheme of order 6 itself is lost: the FP64 oracle gives
  about -4.6e23 where 0F1(;1;-2500) = J0(100) = 0.0200. Theorem "prop:globalte" bounds the
  scheme's error only in absolute terms, through a factor that grows with sup |<x', y'>|. The
  FP32 form follows the oracle there, so the loss is the scheme's and not FP32's. The
  interpolation scheme (Section 3.3) keeps such oscillatory kernels: within 1e-7 of 0F1 at
  N = 8.
* The interpolation scheme's FP32 floor on oscillatory paths (about 1e-5 to 1e-4 on the GPU)
  comes from FP32 cells as such. The same form in FP32, with J = 6 extra terms and the
  compiled projection, lands 4e-7 to 7e-5 from the oracle. In FP64 with J = 10 it lands within
  1e-11.
"""
import os
import re
from math import factorial

import numpy as np
import pytest
from scipy.special import hyp0f1

import oracle
from paper_2502_08470_gb300 import workloads as W

F = np.float32


def fp32_form(x, y, N, exponents=True):
    hank = np.array([[factorial(n) / factorial(n + k) for k in range(N + 1)] for n in range(N + 1)]).astype(F)
    M = (np.diff(x, axis=0).astype(F) @ np.diff(y, axis=0).astype(F).T).astype(F)
    rows, cols = M.shape
    unit = np.zeros(N + 1, F)
    unit[0] = 1
    inv = np.array([1.0 / factorial(n) for n in range(N + 1)])
    b_col = [(unit.copy(), 0) for _ in range(cols)]   # edge entering each column from the row below
    for i in range(rows):
        a, ea = unit.copy(), 0                        # edge carried along the row
        for j in range(cols):
            b, eb = b_col[j]
            if exponents and ea != eb:                # align_inputs
                if ea > eb:
                    b = b * F(2.0 ** (eb - ea)) if eb - ea >= -126 else np.zeros_like(b)
                else:
                    a = a * F(2.0 ** (ea - eb)) if ea - eb >= -126 else np.zeros_like(a)
                    ea = eb
            m = float(M[i, j])
            e = np.array([m ** k / factorial(k) for k in range(N + 1)]).astype(F)
            ct, cr = np.zeros(N + 1, F), np.zeros(N + 1, F)
            for n in range(N + 1):
                ct[n] = np.dot(a[:n + 1], e[n::-1]) + e[n] * np.dot(b[1:], hank[n, 1:])
                cr[n] = np.dot(b[:n + 1], e[n::-1]) + e[n] * np.dot(a[1:], hank[n, 1:])
            if i == rows - 1 and j == cols - 1:
                return 0.5 * (ct.astype(np.float64) @ inv + cr.astype(np.float64) @ inv) * 2.0 ** ea
            a, bo = ct, cr
            if exponents:                             # rescale_edges
                mag = max(abs(a[0]), abs(bo[0]))
                if mag > 2.0 ** 64:
                    a, bo, ea = a * F(2.0 ** -64), bo * F(2.0 ** -64), ea + 64
                elif mag < 2.0 ** -64:
                    full = max(np.abs(a).max(), np.abs(bo).max())
                    if 0 < full < 2.0 ** -64:
                        a, bo, ea = a * F(2.0 ** 64), bo * F(2.0 ** 64), ea - 64
            b_col[j] = (bo, ea)
    return 1.0


def _linear_pair(z, points=65, seed=1):
    """x = s u, y = t v on [0, 1] with <u, v> = z (u, v in R^3): k = 0F1(;1;z)."""
    rng = np.random.default_rng(seed)
    u, v = rng.standard_normal(3), rng.standard_normal(3)
    v = v * (z / (u @ v))
    s = (np.arange(points) / (points - 1))[:, None]
    return s * u, s * v


@pytest.mark.parametrize("seed", range(3))
def test_fp32_form_follows_the_oracle_on_brownian_pairs(seed):
    X = W.brownian(1, 41, 3, seed=300 + seed)[0]
    Y = W.brownian(1, 37, 3, seed=400 + seed, drift=0.5)[0]
    want = oracle.kernel(X, Y, "approx", 6)
    scale = np.sqrt(oracle.kernel(X, X, "approx", 6) * oracle.kernel(Y, Y, "approx", 6))
    assert abs(fp32_form(X, Y, 6) - want) < 1e-6 * scale


def test_exponents_carry_fp32_cells_past_the_fp32_range():
    x, y = _linear_pair(2500.0)
    scheme = oracle.kernel(x, y, "approx", 6)
    assert 1e41 < scheme < 1e43 and scheme == pytest.approx(hyp0f1(1, 2500.0), rel=1e-3)
    assert fp32_form(x, y, 6) == pytest.approx(scheme, rel=2e-5)
    with np.errstate(over="ignore", invalid="ignore"):
        assert not np.isfinite(fp32_form(x, y, 6, exponents=False))


def test_oscillatory_kernel_lost_by_the_approximation_scheme_not_by_fp32():
    x, y = _linear_pair(-2500.0)
    exact = hyp0f1(1, -2500.0)                       # J0(100)
    assert exact == pytest.approx(0.019985850304, rel=1e-9)
    scheme = oracle.kernel(x, y, "approx", 6)
    assert abs(scheme - exact) > 1e20                # the order-6 scheme on this grid
    assert fp32_form(x, y, 6) == pytest.approx(scheme, rel=2e-5)
    assert oracle.kernel(x, y, "interp", 8) == pytest.approx(exact, rel=1e-7)


TABLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2502_08470_gb300", "csrc",
                     "sk_projection_table.h")


def _projection(N, J):
    """The generated projection of series terms N+1..N+J onto the degree-N Chebyshev interpolant,
    as the kernels compile it in."""
    P = np.zeros((N + 1, J))
    for key, val in re.findall(r"case (\d+): return ([-+0-9.eE]+);", open(TABLE).read()):
        key = int(key)
        if key // 1024 == N and key % 32 < J:
            P[(key % 1024) // 32, key % 32] = float(val)
    return P


def interp_form(x, y, N, J, dtype):
    """The interpolation cell as the kernels compute it (the approximation map extended to N + J
    terms, the right edge taking a_0 as its corner term, then the constant projection), in the
    given floating type.  It carries no exponents: the kernel values of the paths below stay
    within FP32's range."""
    NE = N + J
    P = _projection(N, J).astype(dtype)
    hank = np.array([[factorial(n) / factorial(n + k) for k in range(N + 1)] for n in range(NE + 1)]).astype(dtype)
    M = (np.diff(x, axis=0) @ np.diff(y, axis=0).T).astype(dtype)
    rows, cols = M.shape
    unit = np.zeros(N + 1, dtype)
    unit[0] = 1
    inv = np.array([1.0 / factorial(n) for n in range(NE + 1)])
    b_col = [unit.copy() for _ in range(cols)]
    for i in range(rows):
        a = unit.copy()
        for j in range(cols):
            b = b_col[j]
            m = float(M[i, j])
            e = np.array([m ** k / factorial(k) for k in range(NE + 1)]).astype(dtype)
            bc = b.copy()
            bc[0] = a[0]
            ct, cr = np.zeros(NE + 1, dtype), np.zeros(NE + 1, dtype)
            for n in range(NE + 1):
                kk = min(n, N)
                ct[n] = np.dot(a[:kk + 1], e[n::-1][:kk + 1]) + e[n] * np.dot(b[1:], hank[n, 1:])
                cr[n] = np.dot(bc[:kk + 1], e[n::-1][:kk + 1]) + e[n] * np.dot(a[1:], hank[n, 1:])
            if i == rows - 1 and j == cols - 1:
                return 0.5 * (ct.astype(np.float64) @ inv + cr.astype(np.float64) @ inv)
            a = ct[:N + 1] + P @ ct[N + 1:]
            b_col[j] = cr[:N + 1] + P @ cr[N + 1:]
    return 1.0


@pytest.mark.parametrize("seed", range(3))
def test_interpolation_fp32_floor_on_oscillatory_paths_is_the_fp32_cells(seed):
    X = W.oscillatory(1, 65, 4, seed=900 + seed)[0]
    Y = W.oscillatory(1, 65, 4, seed=950 + seed)[0]
    want = oracle.kernel(X, Y, "interp", 8)
    assert interp_form(X, Y, 8, 10, np.float64) == pytest.approx(want, rel=1e-11)
    assert interp_form(X, Y, 8, 6, np.float32) == pytest.approx(want, rel=2e-4)


def test_the_projection_cannot_amplify_rounding():
    """Every entry of the compiled projection (N = 2..12, J = 6 and 10) is at most 1/2 in
    magnitude, so applying it in FP32 adds rounding of the order of the projected terms
    themselves; no ill-conditioned polynomial fit enters the interpolation cells."""
    for J in (6, 10):
        for N in range(2, 13):
            P = _projection(N, J)
            assert np.count_nonzero(P) > 0
            assert np.abs(P).max() <= 0.5
