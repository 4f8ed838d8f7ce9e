"""CPU checks of the compile-time interpolation projection used by the CUDA wavefront
(csrc/sk_projection_table.h): it is what its generator produces, and it equals an independent
float64 Vandermonde solve at the Chebyshev extrema (Definition "interpooperator")."""
import math
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2502_08470_gb300", "csrc")


def _table():
    txt = open(os.path.join(CSRC, "sk_projection_table.h")).read()
    T = {N: np.zeros((N + 1, 12)) for N in range(2, 13)}
    for key, val in re.findall(r"case (\d+): return ([-+0-9.eE]+);", txt):
        key = int(key)
        N, n, jj = key // 1024, (key % 1024) // 32, key % 32
        T[N][n, jj] = float(val)
    return T


def test_header_is_generator_output():
    out = subprocess.run([sys.executable, os.path.join(CSRC, "gen_projection_table.py")], capture_output=True,
                         text=True, check=True).stdout
    assert out == open(os.path.join(CSRC, "sk_projection_table.h")).read()


@pytest.mark.parametrize("N", [2, 3, 5, 8, 12])
def test_projection_matches_float64_vandermonde(N):
    P = _table()[N]
    u = 0.5 * (1.0 + np.cos(np.pi * np.arange(N + 1) / N))
    V = np.vander(u, N + 1, increasing=True)
    W = np.stack([u ** (N + 1 + jj) for jj in range(12)], axis=1)
    R = np.linalg.solve(V, W)
    ref = np.array([[R[n, jj] * math.factorial(n) / math.factorial(N + 1 + jj) for jj in range(12)]
                    for n in range(N + 1)])
    assert np.max(np.abs(P - ref)) < 1e-9 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("N", [4, 8, 12])
def test_projection_interpolates_exponential(N):
    # f(u) = exp(l u) has factorial-scaled series c_j = l^j.  The projected coefficients
    # a = c_{0..N} + P c_{N+1..N+12} define a degree-N polynomial that must take the values of f at
    # the N+1 Chebyshev extrema (the interpolation property of Omega^N), up to the series tail.
    lam = 0.7
    P = _table()[N]
    c = np.array([lam ** j for j in range(N + 13)])
    a = c[:N + 1] + P @ c[N + 1:N + 13]
    u = 0.5 * (1.0 + np.cos(np.pi * np.arange(N + 1) / N))
    vals = np.array([sum(a[n] * ur ** n / math.factorial(n) for n in range(N + 1)) for ur in u])
    assert np.max(np.abs(vals - np.exp(lam * u))) < 1e-14
