"""CPU check of the adjoint the CUDA kernels compute, against the oracle's complex-step gradients.

The paper defines no gradient; the kernels differentiate the discrete scheme exactly (reverse
mode).  In the factorial-scaled form each cell maps its entering edges (a along the row, b along
the column) to the series
    ct_n = sum_{k<=n} a_k e_{n-k} + e_n sum_{k>=1} b_k n!/(n+k)!,
    cr_n = sum_{k<=n} b~_k e_{n-k} + e_n sum_{k>=1} a_k n!/(n+k)!,   e_m = M^m/m!, de_m/dM = e_{m-1},
with b~ = b for the approximation scheme and b~_0 = a_0 (the printed corner term) for the
interpolation scheme, whose outgoing edges are then projected (c_{0..N} + P c_{N+1..N+J}).
The adjoint runs the cells in reverse: the transposed map sends the outgoing-edge adjoints to the
entering edges, the interpolation scheme first applies P^T, the corner cell is seeded from the
endpoint 1/2 sum_n (ct_n + cr_n)/n! (on the unprojected series for interpolation), and
dk/dM = sum_n (ctbar_n dct_n/dM + crbar_n dcr_n/dM).  The chain rule through
M = <dx_i, dy_j> / 4^lambda gives the point gradients.  A numpy restatement of these steps must
match the oracle, which differentiates its own physical-coordinate scheme by the complex step.
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


def value_and_grad(x, y, N, lam, interp=False, J=10):
    NE = N + J if interp else N
    P = _projection(N, J) if interp else np.zeros((N + 1, 0))
    h = np.array([[factorial(n) / factorial(n + k) if k >= 1 else 0.0 for k in range(N + 1)]
                  for n in range(NE + 1)])
    R = 2 ** lam
    dx = np.repeat(np.diff(x, axis=0), R, axis=0) / R
    dy = np.repeat(np.diff(y, axis=0), R, axis=0) / R
    M = dx @ dy.T
    rows, cols = M.shape
    unit = np.eye(N + 1)[0]

    def series(a, b, m):
        e = np.array([m ** k / factorial(k) for k in range(NE + 1)])
        bt = b.copy()
        if interp:
            bt[0] = a[0]
        ct = np.array([sum(a[k] * e[n - k] for k in range(min(n, N) + 1)) + e[n] * (h[n] @ b) for n in range(NE + 1)])
        cr = np.array([sum(bt[k] * e[n - k] for k in range(min(n, N) + 1)) + e[n] * (h[n] @ a) for n in range(NE + 1)])
        return e, ct, cr

    project = lambda c: c[:N + 1] + P @ c[N + 1:]  # noqa: E731
    # forward, keeping every cell's entering edges
    A, B = {}, {}
    b_col = [unit.copy() for _ in range(cols)]
    for i in range(rows):
        a = unit.copy()
        for j in range(cols):
            A[i, j], B[i, j] = a, b_col[j]
            _, ct, cr = series(a, b_col[j], M[i, j])
            if i == rows - 1 and j == cols - 1:
                inv = np.array([1.0 / factorial(n) for n in range(NE + 1)])
                kval = 0.5 * (ct @ inv + cr @ inv)
            a, b_col[j] = project(ct), project(cr)
    # reverse
    Mbar = np.zeros_like(M)
    abar_next = {}  # adjoint of the edge leaving cell (i, j) along the row / along the column
    bbar_next = {}
    for i in range(rows - 1, -1, -1):
        for j in range(cols - 1, -1, -1):
            a, b = A[i, j], B[i, j]
            e, _, _ = series(a, b, M[i, j])
            de = np.concatenate([[0.0], e[:-1]])
            if i == rows - 1 and j == cols - 1:
                ctb = crb = np.array([0.5 / factorial(n) for n in range(NE + 1)])
            else:
                ga = abar_next.get((i, j), np.zeros(N + 1))
                gb = bbar_next.get((i, j), np.zeros(N + 1))
                ctb = np.concatenate([ga, P.T @ ga])
                crb = np.concatenate([gb, P.T @ gb])
            abar, bbar = np.zeros(N + 1), np.zeros(N + 1)
            bt = b.copy()
            if interp:
                bt[0] = a[0]
            mb = 0.0
            for n in range(NE + 1):
                for k in range(min(n, N) + 1):
                    abar[k] += ctb[n] * e[n - k]
                    if interp and k == 0:
                        abar[0] += crb[n] * e[n]
                    else:
                        bbar[k] += crb[n] * e[n - k]
                abar += crb[n] * e[n] * h[n]
                bbar += ctb[n] * e[n] * h[n]
                mb += ctb[n] * (sum(a[k] * de[n - k] for k in range(min(n, N) + 1)) + de[n] * (h[n] @ b))
                mb += crb[n] * (sum(bt[k] * de[n - k] for k in range(min(n, N) + 1)) + de[n] * (h[n] @ a))
            Mbar[i, j] = mb
            if j > 0:
                abar_next[i, j - 1] = abar  # a entered from the cell to the left
            if i > 0:
                bbar_next[i - 1, j] = bbar  # b entered from the cell below
    gdx = (Mbar @ dy).reshape(-1, R, x.shape[1]).sum(axis=1) / R
    gdy = (Mbar.T @ dx).reshape(-1, R, y.shape[1]).sum(axis=1) / R

    def to_points(gd):
        g = np.zeros((gd.shape[0] + 1, gd.shape[1]))
        g[1:] += gd
        g[:-1] -= gd
        return g
    return kval, to_points(gdx), to_points(gdy)


@pytest.mark.parametrize("scheme", ["approx", "interp"])
@pytest.mark.parametrize("N,lam", [(2, 0), (4, 1), (6, 0)])
def test_reverse_mode_of_the_cell_form_gives_the_oracle_gradient(scheme, N, lam):
    x = W.brownian(1, 6, 3, seed=110 + N)[0]
    y = W.brownian(1, 5, 3, seed=120 + N, drift=0.4)[0]
    k, gx, gy = value_and_grad(x, y, N, lam, interp=scheme == "interp")
    assert k == pytest.approx(oracle.kernel(x, y, scheme, N, lam), rel=1e-12)
    rx, ry = oracle.grad(x, y, scheme, N, lam)
    scale = max(np.abs(rx).max(), np.abs(ry).max())
    assert np.abs(gx - rx).max() <= 1e-11 * scale
    assert np.abs(gy - ry).max() <= 1e-11 * scale


def approx_grad_from_output_derivatives(x, y, N, lam):
    """The approximation scheme's adjoint as the tape kernels run it: the forward records, per
    cell, only the derivatives of its outputs with respect to M,
        d ct_n / dM = T_{n-1} + e_{n-1} ha_n,   d cr_n / dM = S_{n-1} + e_{n-1} hb_n   (n >= 1),
    with the Toeplitz sums T_n = sum_{k<=n} a_k e_{n-k}, S_n = sum_{k<=n} b_k e_{n-k} and the
    couplings ha_n = sum_{k>=1} b_k n!/(n+k)!, hb_n = sum_{k>=1} a_k n!/(n+k)!; the reverse sweep
    then needs only M and those derivatives: dk/dM = sum_n (ctbar_n dct_n/dM + crbar_n dcr_n/dM)."""
    h = np.array([[factorial(n) / factorial(n + k) if k >= 1 else 0.0 for k in range(N + 1)]
                  for n in range(N + 1)])
    R = 2 ** lam
    dx = np.repeat(np.diff(x, axis=0), R, axis=0) / R
    dy = np.repeat(np.diff(y, axis=0), R, axis=0) / R
    M = dx @ dy.T
    rows, cols = M.shape
    unit = np.eye(N + 1)[0]
    DA, DB = {}, {}
    b_col = [unit.copy() for _ in range(cols)]
    for i in range(rows):
        a = unit.copy()
        for j in range(cols):
            b = b_col[j]
            e = np.array([M[i, j] ** k / factorial(k) for k in range(N + 1)])
            T = np.array([sum(a[k] * e[n - k] for k in range(n + 1)) for n in range(N + 1)])
            S = np.array([sum(b[k] * e[n - k] for k in range(n + 1)) for n in range(N + 1)])
            ha, hb = h @ b, h @ a
            DA[i, j] = np.array([T[n - 1] + e[n - 1] * ha[n] for n in range(1, N + 1)])
            DB[i, j] = np.array([S[n - 1] + e[n - 1] * hb[n] for n in range(1, N + 1)])
            ct, cr = T + e * ha, S + e * hb
            if i == rows - 1 and j == cols - 1:
                inv = np.array([1.0 / factorial(n) for n in range(N + 1)])
                kval = 0.5 * (ct @ inv + cr @ inv)
            a, b_col[j] = ct, cr
    Mbar = np.zeros_like(M)
    abar_next, bbar_next = {}, {}
    for i in range(rows - 1, -1, -1):
        for j in range(cols - 1, -1, -1):
            e = np.array([M[i, j] ** k / factorial(k) for k in range(N + 1)])
            if i == rows - 1 and j == cols - 1:
                ga = gb = np.array([0.5 / factorial(n) for n in range(N + 1)])
            else:
                ga = abar_next.get((i, j), np.zeros(N + 1))
                gb = bbar_next.get((i, j), np.zeros(N + 1))
            abar = np.array([sum(ga[n] * e[n - k] for n in range(k, N + 1)) for k in range(N + 1)]) + h.T @ (gb * e)
            bbar = np.array([sum(gb[n] * e[n - k] for n in range(k, N + 1)) for k in range(N + 1)]) + h.T @ (ga * e)
            Mbar[i, j] = ga[1:] @ DA[i, j] + gb[1:] @ DB[i, j]
            if j > 0:
                abar_next[i, j - 1] = abar
            if i > 0:
                bbar_next[i - 1, j] = bbar
    gdx = (Mbar @ dy).reshape(-1, R, x.shape[1]).sum(axis=1) / R
    gdy = (Mbar.T @ dx).reshape(-1, R, y.shape[1]).sum(axis=1) / R

    def to_points(gd):
        g = np.zeros((gd.shape[0] + 1, gd.shape[1]))
        g[1:] += gd
        g[:-1] -= gd
        return g
    return kval, to_points(gdx), to_points(gdy)


@pytest.mark.parametrize("N,lam", [(2, 0), (3, 1), (6, 0)])
def test_adjoint_from_output_derivatives_gives_the_oracle_gradient(N, lam):
    x = W.brownian(1, 6, 3, seed=130 + N)[0]
    y = W.brownian(1, 5, 3, seed=140 + N, drift=-0.3)[0]
    k, gx, gy = approx_grad_from_output_derivatives(x, y, N, lam)
    assert k == pytest.approx(oracle.kernel(x, y, "approx", N, lam), rel=1e-12)
    rx, ry = oracle.grad(x, y, "approx", N, lam)
    scale = max(np.abs(rx).max(), np.abs(ry).max())
    assert np.abs(gx - rx).max() <= 1e-11 * scale
    assert np.abs(gy - ry).max() <= 1e-11 * scale
