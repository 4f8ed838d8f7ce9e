"""CPU check of the cell form the CUDA kernels compute, against the oracle's literal schemes.

The kernels hold each edge as factorial-scaled coefficients a_n = n! p_n ds^n, b_n = n! q_n dt^n,
for which the explicit update after Definition "def:polyapproxscheme" becomes
    a'_n = sum_{k<=n} a_k e_{n-k} + e_n sum_{k>=1} b_k n!/(n+k)!,   e_m = M^m / m!,
    b'_n = sum_{k<=n} b_k e_{n-k} + e_n sum_{k>=1} a_k n!/(n+k)!,
a map of M = <dx_i, dy_j> alone; the endpoint is 1/2 sum_n (a_n + b_n)/n!.  The interpolation
scheme (Definition "def:polyinterpscheme") is the same series kept to N + J terms (the right edge
taking a_0 for its corner term, eq. (interpformula) as printed), followed by the constant
projection onto the interpolant at the Chebyshev extrema, read here from the generated table
that the kernels compile in; its endpoint sums the unprojected series.

A numpy restatement of that form, cell by cell in row-major order on the dyadically refined grid
(sub-cell M = M_ij / 4^lambda), must reproduce the oracle, which works in physical coordinates
with powers of ds, dt, a Vandermonde solve per edge and 0F1 summed to convergence.
"""
import os
import re
from math import factorial

import numpy as np
import pytest

import oracle
from paper_2502_08470_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLE = os.path.join(ROOT, "paper_2502_08470_gb300", "csrc", "sk_projection_table.h")


def _projection(N, J):
    P = np.zeros((N + 1, J))
    for key, val in re.findall(r"case (\d+): return ([-+0-9.eE]+);", open(TABLE).read()):
        key = int(key)
        if key // 1024 == N and key % 32 < J:
            P[(key % 1024) // 32, key % 32] = float(val)
    return P


def normalised_form(x, y, N, lam, interp=False, J=10):
    NE = N + J if interp else N
    P = _projection(N, J) if interp else None
    hank = np.array([[factorial(n) / factorial(n + k) for k in range(N + 1)] for n in range(NE + 1)])
    dx = np.repeat(np.diff(x, axis=0), 2 ** lam, axis=0) / 2 ** lam
    dy = np.repeat(np.diff(y, axis=0), 2 ** lam, axis=0) / 2 ** lam
    M = dx @ dy.T
    rows, cols = M.shape
    unit = np.eye(N + 1)[0]
    b_col = [unit.copy() for _ in range(cols)]  # left edges entering the current row
    for i in range(rows):
        a = unit.copy()                          # bottom edge of cell (i, 0)
        for j in range(cols):
            b = b_col[j]
            e = np.array([M[i, j] ** m / factorial(m) for m in range(NE + 1)])
            ct, cr = np.zeros(NE + 1), np.zeros(NE + 1)
            bc = b.copy()
            if interp:
                bc[0] = a[0]                     # the printed corner term g_0 on the right edge
            for n in range(NE + 1):
                ct[n] = sum(a[k] * e[n - k] for k in range(min(n, N) + 1)) + e[n] * (b[1:] @ hank[n, 1:])
                cr[n] = sum(bc[k] * e[n - k] for k in range(min(n, N) + 1)) + e[n] * (a[1:] @ hank[n, 1:])
            if i == rows - 1 and j == cols - 1:
                inv = np.array([1.0 / factorial(n) for n in range(NE + 1)])
                return 0.5 * (ct @ inv + cr @ inv)
            if interp:
                a, b_col[j] = ct[:N + 1] + P @ ct[N + 1:], cr[:N + 1] + P @ cr[N + 1:]
            else:
                a, b_col[j] = ct, cr
    return 1.0


@pytest.mark.parametrize("N,lam", [(2, 0), (4, 1), (6, 0), (9, 2)])
def test_approximation_form_equals_the_oracle(N, lam):
    X = W.brownian(2, 6, 3, seed=60 + N)
    Y = W.brownian(2, 5, 3, seed=70 + N, drift=0.4)
    for a in range(2):
        want = oracle.kernel(X[a], Y[a], "approx", N, lam)
        assert normalised_form(X[a], Y[a], N, lam) == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("N,lam", [(2, 0), (3, 1), (6, 0), (8, 1)])
def test_interpolation_as_extension_plus_projection_equals_the_oracle(N, lam):
    """J = 10 extra series terms (the FP64 kernels' count); the sub-cell |M| of these paths
    reaches 1.6."""
    X = W.brownian(2, 6, 3, seed=80 + N)
    Y = W.brownian(2, 5, 3, seed=90 + N, drift=0.4)
    for a in range(2):
        want = oracle.kernel(X[a], Y[a], "interp", N, lam)
        assert normalised_form(X[a], Y[a], N, lam, interp=True, J=10) == pytest.approx(want, rel=1e-12)


def test_series_lengths_of_the_kernels():
    """The interpolation kernels keep J = 6 extra series terms in FP32 and J = 10 in FP64.  On
    paths whose largest cell |M| is about 4.5, J = 6 stays within 1e-9 of the oracle (FP32 rounds
    at 6e-8) and J = 10 within 1e-13; at |M| <= 0.5 even J = 4 reaches FP64 rounding."""
    X = W.brownian(1, 9, 2, seed=91)[0]
    Y = W.brownian(1, 8, 2, seed=92)[0]
    assert np.abs(np.diff(X, axis=0) @ np.diff(Y, axis=0).T).max() < 0.5
    want = oracle.kernel(X, Y, "interp", 6)
    assert normalised_form(X, Y, 6, 0, interp=True, J=4) == pytest.approx(want, rel=1e-13)
    X, Y = 3 * X, 3 * Y
    assert 4 < np.abs(np.diff(X, axis=0) @ np.diff(Y, axis=0).T).max() < 5
    want = oracle.kernel(X, Y, "interp", 6)
    assert normalised_form(X, Y, 6, 0, interp=True, J=6) == pytest.approx(want, rel=1e-9)
    assert normalised_form(X, Y, 6, 0, interp=True, J=10) == pytest.approx(want, rel=1e-13)
    assert normalised_form(X, Y, 6, 0, interp=True, J=4) != pytest.approx(want, rel=1e-8)  # too short
