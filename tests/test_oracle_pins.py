"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms, library Bessel
functions, brute-force truncated signatures, convergence orders, symmetries and invariants.
"""
from math import factorial

import numpy as np
import pytest
import scipy.special as sps

import oracle
from paper_2502_08470_gb300 import workloads as W

SCHEMES = ["fd1", "fd2", "approx", "interp", "fd_implicit"]


def _seg(v0, v1):
    return np.array([v0, v1], dtype=np.float64)


def _i0_series(z, terms=60):
    """0F1(;1;z) = sum z^n/(n!)^2 (Remark "mbf")."""
    return sum(z ** n / factorial(n) ** 2 for n in range(terms))


# --------------------------------------------------------------------------------------------
# Polynomial approximation: single-cell and two-cell closed forms (Remark after
# Definition "def:polyapproxscheme", with p = q = e_0; first-cell formula of Prop. multistepestimate)
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("N", [2, 3, 4, 6, 9, 12])
@pytest.mark.parametrize("M", [0.37, -0.81, 1.7, -2.3])
def test_approx_single_cell_truncated_series(N, M):
    # one segment each; <dx, dy> = M.  The scheme returns sum_{n<=N} M^n/(n!)^2 exactly.
    x = _seg([0.0, 0.0], [1.0, 0.0])
    y = _seg([0.0, 0.0], [M, 0.5])
    want = sum(M ** n / factorial(n) ** 2 for n in range(N + 1))
    got = oracle.kernel(x, y, "approx", N)
    assert got == pytest.approx(want, rel=1e-14, abs=1e-15)
    # the same with non-unit, non-uniform partitions (only C * ds * dt enters)
    got2 = oracle.kernel(x, y, "approx", N, s=[0.3, 0.35], t=[-2.0, 5.0])
    assert got2 == pytest.approx(want, rel=1e-13, abs=1e-14)


@pytest.mark.parametrize("N", [2, 3, 5, 8])
def test_approx_one_by_two_closed_form(N):
    """x: one segment, y: two segments; M1, M2 the two cell constants.

    Working the scheme's update by hand on these two cells (top edge of cell (0,1) is the
    binomial convolution, right edge picks up the q-to-p coupling term of the Remark) gives
      k_hat = 1/2 [ sum_{m<=N} (M1+M2)^m/(m!)^2 + sum_{n<=N} sum_{k<=N} M1^k M2^n/(k! n! (n+k)!) ].
    """
    rng = np.random.default_rng(11 + N)
    dx = rng.normal(size=3)
    dy1, dy2 = rng.normal(size=3), rng.normal(size=3)
    x = np.stack([np.zeros(3), dx])
    y = np.stack([np.zeros(3), dy1, dy1 + dy2])
    M1, M2 = dx @ dy1, dx @ dy2
    top = sum((M1 + M2) ** m / factorial(m) ** 2 for m in range(N + 1))
    right = sum(M1 ** k * M2 ** n / (factorial(k) * factorial(n) * factorial(n + k))
                for n in range(N + 1) for k in range(N + 1))
    want = 0.5 * (top + right)
    assert oracle.kernel(x, y, "approx", N) == pytest.approx(want, rel=1e-13)
    # swapping the roles of x and y mirrors the grid (symmetry of the update)
    assert oracle.kernel(y, x, "approx", N) == pytest.approx(want, rel=1e-13)


def _first_row_recursion(dx, dys, s, t, N):
    """The approximation scheme on a grid of one row of cells, from the recursions printed in the
    proof of Prop. "multistepestimate". Along the first row, the top edge's coefficients (powers of
    s - s_0) obey p^{0,j+1}_n = sum_k p^{0j}_k (C_0j dt_j)^{n-k} k! / ((n-k)! n!). The right edge
    gets q^{1,j}_n = sum_k p^{0j}_k C_0j^n ds^{n+k} k! / ((n+k)! n!), with C_0j = <dx, dy_j> /
    (ds dt_j). Kept to n <= N, these are the scheme's own coefficients: p^{0,j+1}_n depends on
    p^{0j}_k for k <= n only. The endpoint averages the last cell's top and right edges."""
    ds = s[1] - s[0]
    p = np.zeros(N + 1)
    p[0] = 1.0                                   # k(s, t_0) = 1
    for j, dy in enumerate(dys):
        dt = t[j + 1] - t[j]
        C = float(dx @ dy) / (ds * dt)
        q = np.array([sum(p[k] * C ** n * ds ** (n + k) * factorial(k) / (factorial(n + k) * factorial(n))
                          for k in range(N + 1)) for n in range(N + 1)])
        p = np.array([sum(p[k] * (C * dt) ** (n - k) * factorial(k) / (factorial(n - k) * factorial(n))
                          for k in range(n + 1)) for n in range(N + 1)])
    return 0.5 * (sum(p[n] * ds ** n for n in range(N + 1)) + sum(q[n] * dt ** n for n in range(N + 1)))


@pytest.mark.parametrize("N", [2, 4, 6, 9])
@pytest.mark.parametrize("K", [1, 3, 8])
def test_approx_one_row_follows_the_printed_first_row_recursion(N, K):
    """One x segment against K y segments, on non-uniform partitions: the oracle's general
    grid sweep against the paper's first-row recursion (and the mirrored grid against it too)."""
    rng = np.random.default_rng(100 * N + K)
    dx = 1.3 * rng.normal(size=3)
    dys = rng.normal(size=(K, 3)) / np.sqrt(K)
    x = np.stack([np.zeros(3), dx])
    y = np.vstack([np.zeros(3), np.cumsum(dys, axis=0)])
    s = [0.2, 0.2 + rng.uniform(0.5, 2.0)]
    t = list(np.concatenate([[-1.0], -1.0 + np.cumsum(rng.uniform(0.3, 1.5, K))]))
    want = _first_row_recursion(dx, dys, s, t, N)
    assert oracle.kernel(x, y, "approx", N, s=s, t=t) == pytest.approx(want, rel=1e-13)
    assert oracle.kernel(y, x, "approx", N, s=t, t=s) == pytest.approx(want, rel=1e-13)


# --------------------------------------------------------------------------------------------
# Polynomial interpolation: the single-cell solution is 0F1(1; M) = I_0(2 sqrt M)  (Prop.
# "propinterp" and the Remark after it); checked against scipy's Bessel functions.
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("N", [2, 4, 7])
@pytest.mark.parametrize("M", [0.05, 0.9, 3.0, -0.4, -1.4458, -4.0])
def test_interp_single_cell_bessel(N, M):
    x = _seg([0.0, 0.0], [1.0, 0.0])
    y = _seg([0.0, 0.0], [M, -0.3])
    if M >= 0:
        want = sps.iv(0, 2.0 * np.sqrt(M))
    else:
        want = sps.j0(2.0 * np.sqrt(-M))
    got = oracle.kernel(x, y, "interp", N)
    assert got == pytest.approx(want, rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("N", [2, 3, 5])
def test_interp_two_by_two_grid_from_library_routines(N):
    """The interpolation scheme on a 2 x 2 grid assembled from library routines: each incoming
    edge is interpolated at the N + 1 Chebyshev extrema of its interval (Def. "interpooperator")
    by numpy.polyfit, and each cell's solution is eq. (interpformula) of Prop. "propinterp" with
    scipy's 0F1, its first term weighted by the bottom interpolant's constant g_0 (reading 3).
    Pins the node set, the corner term and the order of the 0F1 parameters where the single-cell
    pin cannot: there both edges are constant."""
    x = np.array([[0.0, 0.0], [0.7, -0.4], [1.1, 0.5]])
    y = np.array([[0.0, 0.0], [-0.5, 0.9], [0.4, 1.3]])
    s = t = np.array([0.0, 0.5, 1.0])

    def omega(f, a, b):  # monomial coefficients in (r - a) of the interpolant at the extrema
        nodes = 0.5 * (a + b) + 0.5 * (b - a) * np.cos(np.pi * np.arange(N + 1) / N)
        return np.polyfit(nodes - a, [f(r) for r in nodes], N)[::-1]

    def solve(i, j, g, h):  # closure of cell (i, j): k on [s_i, s_i+1] x [t_j, t_j+1]
        C = (x[i + 1] - x[i]) @ (y[j + 1] - y[j]) / ((s[i + 1] - s[i]) * (t[j + 1] - t[j]))

        def k(a, b):
            u, v = a - s[i], b - t[j]
            z = C * u * v
            return g[0] * sps.hyp0f1(1, z) + sum((g[n] * u ** n + h[n] * v ** n) * sps.hyp0f1(n + 1, z)
                                                 for n in range(1, N + 1))
        return k

    one = lambda r: 1.0  # noqa: E731  (the boundary k(s_0, .) = k(., t_0) = 1)
    k00 = solve(0, 0, omega(one, s[0], s[1]), omega(one, t[0], t[1]))
    k01 = solve(0, 1, omega(lambda r: k00(r, t[1]), s[0], s[1]), omega(one, t[1], t[2]))
    k10 = solve(1, 0, omega(one, s[1], s[2]), omega(lambda r: k00(s[1], r), t[0], t[1]))
    k11 = solve(1, 1, omega(lambda r: k10(r, t[1]), s[1], s[2]), omega(lambda r: k01(s[1], r), t[1], t[2]))
    want = k11(s[2], t[2])
    assert oracle.kernel(x, y, "interp", N) == pytest.approx(want, rel=1e-12)


# --------------------------------------------------------------------------------------------
# Linear paths x = s u, y = t v: exact kernel 0F1(;1;<u,v>)  (Remark "mbf")
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("L", [5, 17, 33])
def test_linear_paths_converge_to_0f1(L):
    X = W.linear(6, L, 2, seed=2)
    U = W.linear_directions(6, 2, seed=2)
    for a in range(3):
        x, y = X[2 * a], X[2 * a + 1]
        z = U[2 * a] @ U[2 * a + 1]
        want = _i0_series(z)
        assert oracle.kernel(x, y, "approx", 14) == pytest.approx(want, rel=1e-13)
        assert oracle.kernel(x, y, "interp", 9) == pytest.approx(want, rel=1e-12)
        # FD is only O(4^-lambda) accurate (Section 2)
        assert oracle.kernel(x, y, "fd2", 0, lam=3) == pytest.approx(want, rel=1e-4)


# --------------------------------------------------------------------------------------------
# Brute-force truncated signature kernel (Definition 1.1, Chen's identity) — the paper's own
# accuracy benchmark at level 21 (Section 4).  First pin the brute force itself.
# --------------------------------------------------------------------------------------------
def test_signature_level1_level2_closed_forms():
    rng = np.random.default_rng(5)
    x = np.cumsum(rng.normal(size=(5, 3)), axis=0)
    inc = np.diff(x, axis=0)
    # level 1: total increment
    np.testing.assert_allclose(oracle.signature_level(x, 1), x[-1] - x[0], rtol=1e-14, atol=1e-14)
    # level 2 of a piecewise-linear path: sum_{i<j} d_i (x) d_j + 1/2 sum_i d_i (x) d_i
    S2 = np.zeros((3, 3))
    for i in range(len(inc)):
        for j in range(i + 1, len(inc)):
            S2 += np.outer(inc[i], inc[j])
        S2 += 0.5 * np.outer(inc[i], inc[i])
    np.testing.assert_allclose(oracle.signature_level(x, 2), S2.ravel(), rtol=1e-13, atol=1e-13)


def test_signature_one_dimensional_and_tree_like():
    # d = 1: S_n(x) = (x_T - x_0)^n / n!, so the kernel is sum (DX DY)^n/(n!)^2
    x = np.array([[0.0], [0.4], [-0.2], [0.9]])
    y = np.array([[1.0], [0.3], [1.5]])
    DX, DY = 0.9, 0.5
    want = sum((DX * DY) ** n / factorial(n) ** 2 for n in range(13))
    assert oracle.sig_trunc(x, y, 12) == pytest.approx(want, rel=1e-14)
    # a path followed by its reversal has trivial signature (Chen; the signature characterises
    # paths up to tree-like equivalence, Section 1)
    rng = np.random.default_rng(3)
    p = np.cumsum(rng.normal(size=(4, 2)), axis=0)
    tree = np.concatenate([p, p[-2::-1]], axis=0)
    for n in (1, 2, 3, 4):
        np.testing.assert_allclose(oracle.signature_level(tree, n), 0.0, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_schemes_match_brute_force_signature_kernel(seed):
    X = W.brownian(2, 7, 2, seed=100 + seed)
    Y = W.brownian(2, 6, 2, seed=200 + seed)
    for a in range(2):
        x, y = X[a], Y[a]
        truth = oracle.sig_trunc(x, y, 18)
        assert oracle.kernel(x, y, "approx", 14) == pytest.approx(truth, rel=1e-13)
        assert oracle.kernel(x, y, "interp", 10) == pytest.approx(truth, rel=1e-13)
        assert oracle.kernel(x, y, "fd2", lam=4) == pytest.approx(truth, rel=1e-4)
        assert oracle.kernel(x, y, "fd1", lam=4) == pytest.approx(truth, rel=1e-2)


def test_three_dimensional_brute_force():
    X = W.brownian(1, 5, 3, seed=41)
    Y = W.brownian(1, 6, 3, seed=42)
    truth = oracle.sig_trunc(X[0], Y[0], 12)
    assert oracle.kernel(X[0], Y[0], "approx", 14) == pytest.approx(truth, rel=1e-12)
    assert oracle.kernel(X[0], Y[0], "interp", 10) == pytest.approx(truth, rel=1e-12)


# --------------------------------------------------------------------------------------------
# Finite differences: closed forms on one cell, and the 2^{-2 lambda} convergence rate
# (Definition "dyadic scheme"; Theorem 3.5 of Salvi et al. as quoted in Section 2)
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("m", [0.3, -0.7, 1.9])
def test_fd_single_cell_closed_forms(m):
    x = _seg([0.0], [1.0])
    y = _seg([0.0], [m])
    # lambda = 0: one update from three unit corners
    assert oracle.kernel(x, y, "fd1") == pytest.approx(1.0 + m, rel=1e-15)
    assert oracle.kernel(x, y, "fd2") == pytest.approx(1.0 + m + m * m / 4.0, rel=1e-15)


@pytest.mark.parametrize("m", [0.3, -0.7, 1.9, -3.1])
def test_fd_implicit_single_cell_closed_form(m):
    """Remark "higherfd", four-corner trapezoid rule: from three unit corners the cell equation
    k11 = 1 + (m/4)(3 + k11) has the solution (1 + 3m/4)/(1 - m/4) = 1 + m + m^2/4 + m^3/16 + ...,
    which agrees with the exact sum m^n/(n!)^2 up to the m^3 term."""
    x = _seg([0.0], [1.0])
    y = _seg([0.0], [m])
    assert oracle.kernel(x, y, "fd_implicit") == pytest.approx((1.0 + 0.75 * m) / (1.0 - 0.25 * m), rel=1e-15)


@pytest.mark.parametrize("lam", [0, 1])
def test_fd_implicit_solves_the_global_linear_system(lam):
    """The marching update against one dense solve of every cell equation at once: unknowns
    k(i, j) for i, j >= 1, boundary k(0, .) = k(., 0) = 1, and for each (refined) cell
    k11 - k10 - k01 + k00 - (m/4)(k00 + k10 + k01 + k11) = 0 with m = <dx_i, dy_j>.  The paths
    differ in length and direction, so a transposed or shifted increment index changes the
    answer.  For lambda = 1 the refined grid is built here by inserting midpoints."""
    X = W.brownian(1, 4, 3, seed=71)[0]
    Y = W.brownian(1, 6, 3, seed=72)[0] * 1.7
    x, y = X, Y
    for _ in range(lam):
        x = np.concatenate([np.stack([x[:-1], 0.5 * (x[:-1] + x[1:])], 1).reshape(-1, 3), x[-1:]])
        y = np.concatenate([np.stack([y[:-1], 0.5 * (y[:-1] + y[1:])], 1).reshape(-1, 3), y[-1:]])
    dx, dy = np.diff(x, axis=0), np.diff(y, axis=0)
    nI, nJ = len(dx), len(dy)
    idx = lambda i, j: (i - 1) * nJ + (j - 1)
    A = np.zeros((nI * nJ, nI * nJ))
    b = np.zeros(nI * nJ)
    for i in range(nI):
        for j in range(nJ):
            m = dx[i] @ dy[j]
            row = idx(i + 1, j + 1)
            for (a, c), coef in (((i + 1, j + 1), 1 - m / 4), ((i + 1, j), -1 - m / 4),
                                 ((i, j + 1), -1 - m / 4), ((i, j), 1 - m / 4)):
                if a == 0 or c == 0:
                    b[row] -= coef  # boundary value 1 moved to the right-hand side
                else:
                    A[row, idx(a, c)] += coef
    k = np.linalg.solve(A, b)
    assert oracle.kernel(X, Y, "fd_implicit", lam=lam) == pytest.approx(k[-1], rel=1e-12)


def test_fd_implicit_beats_the_two_corner_rule():
    """The four-corner quadrature has a smaller error constant than the first-order explicit
    update at equal refinement (same 4^-lambda rate); with the Remark's printed factor 1/2 the
    implicit scheme would not converge at all."""
    X = W.linear(2, 9, 2, seed=7)
    U = W.linear_directions(2, 2, seed=7)
    want = _i0_series(U[0] @ U[1])
    for lam in (2, 3, 4):
        e1 = abs(oracle.kernel(X[0], X[1], "fd1", lam=lam) - want)
        ei = abs(oracle.kernel(X[0], X[1], "fd_implicit", lam=lam) - want)
        assert ei < e1 / 10


@pytest.mark.parametrize("scheme", ["fd1", "fd2", "fd_implicit"])
def test_fd_convergence_rate(scheme):
    X = W.linear(2, 9, 2, seed=7)
    U = W.linear_directions(2, 2, seed=7)
    want = _i0_series(U[0] @ U[1])
    errs = [abs(oracle.kernel(X[0], X[1], scheme, lam=lam) - want) for lam in range(1, 6)]
    ratios = [errs[k] / errs[k + 1] for k in range(len(errs) - 1)]
    for r in ratios[1:]:
        assert 3.5 < r < 4.5, ratios


# --------------------------------------------------------------------------------------------
# Symmetry, invariants and positive semi-definiteness
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("scheme", SCHEMES)
def test_symmetry_in_x_and_y(scheme):
    X = W.brownian(2, 9, 3, seed=9)
    Y = W.brownian(1, 12, 3, seed=10)
    for x in X:
        a = oracle.kernel(x, Y[0], scheme, 5, lam=1)
        b = oracle.kernel(Y[0], x, scheme, 5, lam=1)
        assert a == pytest.approx(b, rel=1e-13)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_invariants(scheme):
    X = W.brownian(2, 10, 2, seed=12)
    x, y = X[0], X[1]
    k = oracle.kernel(x, y, scheme, 6)
    # constant path: M = 0 everywhere, k = 1 exactly
    assert oracle.kernel(np.ones((7, 2)) * 0.3, y, scheme, 6) == 1.0
    # translation invariance
    assert oracle.kernel(x + 3.0, y - 1.0, scheme, 6) == pytest.approx(k, rel=1e-13)
    # k(c x, y) = k(x, c y)
    assert oracle.kernel(2.5 * x, y, scheme, 6) == pytest.approx(oracle.kernel(x, 2.5 * y, scheme, 6),
                                                                 rel=1e-13)
    # a path with a single point has trivial signature
    assert oracle.kernel(x[:1], y, scheme, 6) == 1.0


@pytest.mark.parametrize("scheme", ["approx", "interp"])
def test_time_partition_invariance(scheme):
    rng = np.random.default_rng(13)
    X = W.brownian(2, 9, 2, seed=13)
    k0 = oracle.kernel(X[0], X[1], scheme, 6)
    s = np.concatenate([[0.0], np.cumsum(rng.uniform(0.2, 2.0, size=8))])
    t = np.concatenate([[-1.0], -1.0 + np.cumsum(rng.uniform(0.05, 0.5, size=8))])
    k1 = oracle.kernel(X[0], X[1], scheme, 6, s=s, t=t)
    assert k1 == pytest.approx(k0, rel=1e-12)


def test_tree_like_path_gives_one():
    rng = np.random.default_rng(14)
    p = np.cumsum(rng.normal(size=(5, 2)) * 0.4, axis=0)
    tree = np.concatenate([p, p[-2::-1]], axis=0)
    y = W.brownian(1, 8, 2, seed=15)[0]
    assert oracle.kernel(tree, y, "approx", 16) == pytest.approx(1.0, abs=1e-12)
    assert oracle.kernel(tree, y, "interp", 12) == pytest.approx(1.0, abs=1e-12)


def test_gram_is_positive_semidefinite():
    X = W.brownian(10, 9, 2, seed=16)
    G = oracle.gram(list(X), list(X), "approx", 12)
    np.testing.assert_allclose(G, G.T, rtol=1e-13)
    ev = np.linalg.eigvalsh(0.5 * (G + G.T))
    assert ev.min() >= -1e-12 * ev.max()


# --------------------------------------------------------------------------------------------
# Global truncation error bound (Theorem "prop:globalte"); the bound is loose, it must hold.
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("N", [2, 3, 4, 6])
def test_global_truncation_error_bound(N):
    X = W.brownian(2, 6, 2, seed=17)
    x, y = X[0], X[1]
    truth = oracle.kernel(x, y, "approx", 18)
    approx = oracle.kernel(x, y, "approx", N)
    lx, ly = x.shape[0] - 1, y.shape[0] - 1
    dxs, dys = np.diff(x, axis=0), np.diff(y, axis=0)
    delta = max(1.0 / lx, 1.0 / ly)
    K = np.abs(dxs @ dys.T).max() * lx * ly  # sup |C_ij| with uniform partitions
    n = lx + ly - 1
    f = np.prod([sps.iv(0, 2.0 * np.sqrt(m * K) * delta) for m in range(n + 1)])
    xi = (K * delta ** 2) ** (N + 1) / factorial(N + 1) ** 2
    bound = f * xi * (n ** (N + 2) / (N + 2) + n ** (N + 1))
    assert abs(truth - approx) <= bound


@pytest.mark.parametrize("N", [2, 3, 4])
def test_hybrid_scheme_converges_at_the_rate_of_the_bound(N):
    """The hybrid method of Section 3.2 (the approximation scheme on the dyadically refined grid)
    against the brute-force signature kernel.  Refining once halves Delta, keeps C and doubles
    l_x + l_y, so the bound of Theorem "prop:globalte" scales by 4^-(N+1) 2^(N+2) = 2^-N: the
    measured error ratio per refinement settles at 2^N (within [0.9, 1.5] x 2^N at lambda >= 2).
    A refinement that mis-scaled the sub-cells (a dropped 2^-lambda on one side, say) would not
    converge to the truth at all."""
    X = W.brownian(2, 7, 2, seed=100)
    Y = W.brownian(2, 6, 2, seed=200)
    x, y = X[0], Y[0]
    truth = oracle.sig_trunc(x, y, 18)
    err = [abs(oracle.kernel(x, y, "approx", N, lam) - truth) / abs(truth) for lam in range(5)]
    assert all(err[lam + 1] < err[lam] for lam in range(4))
    for lam in (2, 3):
        assert 0.9 * 2 ** N <= err[lam] / err[lam + 1] <= 1.5 * 2 ** N, (lam, err)
    # the interpolation scheme on the same refined grids converges to the same truth
    ierr = [abs(oracle.kernel(x, y, "interp", 2, lam) - truth) / abs(truth) for lam in range(5)]
    assert ierr[4] < 1e-3 * ierr[0] and ierr[4] < 1e-9


# --------------------------------------------------------------------------------------------
# Complex-step gradients: central differences, and the single-cell closed form
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("scheme", SCHEMES)
def test_complex_step_matches_central_differences(scheme):
    X = W.brownian(2, 6, 2, seed=18)
    x, y = X[0], X[1]
    gx, gy = oracle.grad(x, y, scheme, 5, lam=1)
    h = 1e-5
    for side, p, c in [(0, 0, 0), (0, 3, 1), (0, 5, 0), (1, 2, 1), (1, 0, 1)]:
        a = (x if side == 0 else y).copy()
        ap, am = a.copy(), a.copy()
        ap[p, c] += h
        am[p, c] -= h
        if side == 0:
            fd = (oracle.kernel(ap, y, scheme, 5, lam=1) - oracle.kernel(am, y, scheme, 5, lam=1)) / (2 * h)
            g = gx[p, c]
        else:
            fd = (oracle.kernel(x, ap, scheme, 5, lam=1) - oracle.kernel(x, am, scheme, 5, lam=1)) / (2 * h)
            g = gy[p, c]
        assert g == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_gradient_single_cell_closed_form():
    N = 7
    x = np.array([[0.1, 0.2], [0.5, -0.3]])
    y = np.array([[0.0, 0.0], [0.9, 0.4]])
    dxv, dyv = x[1] - x[0], y[1] - y[0]
    M = dxv @ dyv
    dk = sum(n * M ** (n - 1) / factorial(n) ** 2 for n in range(1, N + 1))
    gx, gy = oracle.grad(x, y, "approx", N)
    np.testing.assert_allclose(gx[1], dk * dyv, rtol=1e-13)
    np.testing.assert_allclose(gx[0], -dk * dyv, rtol=1e-13)
    np.testing.assert_allclose(gy[1], dk * dxv, rtol=1e-13)


# --------------------------------------------------------------------------------------------
# MMD^2 (Sections 1 and 4 name it; the estimator is the standard one)
# --------------------------------------------------------------------------------------------
def test_mmd2_estimators_and_gradient():
    A = W.brownian(3, 5, 2, seed=19)
    B = W.brownian(4, 5, 2, seed=20, drift=0.5, vol=1.2)
    Kaa = oracle.gram(list(A), list(A), "approx", 6)
    Kbb = oracle.gram(list(B), list(B), "approx", 6)
    Kab = oracle.gram(list(A), list(B), "approx", 6)
    biased = Kaa.mean() + Kbb.mean() - 2 * Kab.mean()
    assert oracle.mmd2(A, B, "approx", 6) == pytest.approx(biased, rel=1e-13)
    unb = ((Kaa.sum() - np.trace(Kaa)) / 6 + (Kbb.sum() - np.trace(Kbb)) / 12 - 2 * Kab.mean())
    assert oracle.mmd2(A, B, "approx", 6, unbiased=True) == pytest.approx(unb, rel=1e-12)
    # identical sets: biased MMD^2 = 0
    assert abs(oracle.mmd2(A, A, "approx", 6)) < 1e-14
    h = 1e-5
    for side, path, p, c in [(0, 1, 2, 0), (1, 3, 4, 1)]:
        g = oracle.mmd2_grad_entry(A, B, side, path, p, c, "approx", 6)
        Ap, Am, Bp, Bm = A.copy(), A.copy(), B.copy(), B.copy()
        if side == 0:
            Ap[path, p, c] += h
            Am[path, p, c] -= h
        else:
            Bp[path, p, c] += h
            Bm[path, p, c] -= h
        fd = (oracle.mmd2(Ap, Bp, "approx", 6) - oracle.mmd2(Am, Bm, "approx", 6)) / (2 * h)
        assert g == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_pairs_threads_agree_with_single_calls():
    X = list(W.brownian(5, 8, 2, seed=21))
    Y = [W.brownian(1, L, 2, seed=22 + L)[0] for L in (4, 9, 13)]
    pa = [0, 4, 2, 1]
    pb = [2, 0, 1, 2]
    out = oracle.pairs(X, Y, pa, pb, "approx", 6, threads=3)
    for k in range(4):
        assert out[k] == oracle.kernel(X[pa[k]], Y[pb[k]], "approx", 6)


# --------------------------------------------------------------------------------------------
# Two-sample permutation test on MMD^2 (Sections 1 and 4 name hypothesis testing; the standard
# permutation test): statistics against the separately pinned MMD^2 code on relabelled sets
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("unbiased", [False, True])
def test_permutation_statistics_are_mmd2_of_the_relabelled_sets(unbiased):
    A = W.brownian(5, 6, 2, seed=61)
    B = W.brownian(4, 6, 2, seed=62, drift=0.4)
    Z = np.concatenate([A, B])
    labels = W.split_labels(6, 5, 4, seed=63)
    obs, p, stats = oracle.mmd2_permutation_test(A, B, labels, "approx", 5, unbiased=unbiased)
    assert obs == pytest.approx(oracle.mmd2(A, B, "approx", 5, unbiased=unbiased), rel=1e-12)
    for row, s in zip(labels, stats):
        first = row != 0
        want = oracle.mmd2(Z[first], Z[~first], "approx", 5, unbiased=unbiased)
        assert s == pytest.approx(want, rel=1e-11, abs=1e-13)
    assert p == (1 + np.count_nonzero(stats >= obs)) / 7


def test_permutation_test_invariances_and_extremes():
    A = W.brownian(6, 5, 2, seed=64)
    B = W.brownian(6, 5, 2, seed=65, drift=3.0)
    n = 12
    ident = (np.arange(n) < 6).astype(np.uint8)
    swapped = 1 - ident  # the two samples exchanged: the biased MMD^2 is symmetric in them
    within = ident.copy()
    labels = np.stack([ident, swapped, within] + list(W.split_labels(20, 6, 6, seed=66)))
    obs, p, stats = oracle.mmd2_permutation_test(A, B, labels, "approx", 4)
    assert stats[0] == obs and stats[2] == obs
    assert stats[1] == pytest.approx(obs, rel=1e-12)
    # a drift of 3 separates the samples: every proper relabelling scores below the split itself
    proper = [k for k in range(3, len(labels)) if not (np.array_equal(labels[k], ident)
                                                       or np.array_equal(labels[k], swapped))]
    assert np.all(stats[proper] < obs)
    ties = np.count_nonzero(stats >= obs)
    assert ties >= 2 and p == (1 + ties) / (1 + len(labels))


def test_permutation_p_values_are_valid_under_the_null():
    """Under H0 (both samples from one law) the permutation p-value is uniform on {1/40, ..., 1}
    (39 relabellings): P(p <= a) <= a and E p = 0.5125.  100 independent tests at a = 0.1 expect
    10 rejections (17 or more has probability about 0.02)."""
    ps = []
    for t in range(100):
        A = W.brownian(6, 5, 2, seed=1000 + 2 * t)
        B = W.brownian(6, 5, 2, seed=1001 + 2 * t)
        _, p, _ = oracle.mmd2_permutation_test(A, B, W.split_labels(39, 6, 6, seed=3000 + t), "approx", 4)
        assert 1 / 40 <= p <= 1
        ps.append(p)
    ps = np.array(ps)
    assert np.count_nonzero(ps <= 0.1) <= 16
    assert 0.42 < ps.mean() < 0.6


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("lam", [0, 1])
def test_repeated_point_leaves_every_scheme_unchanged(scheme, lam):
    """A repeated point adds a zero increment: its cells have M = 0, where the Goursat solution is
    the bilinear k(s, v) + k(u, t) - k(u, v) of its edges, which every scheme carries exactly
    (polynomial edges keep their degree; the FD update is exact).  The output is unchanged up to
    rounding, with the repeat at the start or inside either path, and for the interpolation and
    FD schemes also at the end.  The approximation scheme's top and right edges carry corner
    values that differ by its truncation error (the Remark after Definition
    "def:polyapproxscheme" takes p_0 on one and q_0 on the other), and its endpoint averages the
    two, so a zero row appended at the end moves the average by half that difference."""
    X = W.brownian(1, 9, 3, seed=101)[0]
    Y = W.brownian(1, 7, 3, seed=102)[0]
    k0 = oracle.kernel(X, Y, scheme, 5, lam=lam)
    for where in ((0, 4) if scheme == "approx" else (0, 4, 8)):
        Xr = np.insert(X, where, X[where], axis=0)
        assert oracle.kernel(Xr, Y, scheme, 5, lam=lam) == pytest.approx(k0, rel=1e-12), where
    Yr = np.insert(Y, 3, Y[3], axis=0)
    assert oracle.kernel(X, Yr, scheme, 5, lam=lam) == pytest.approx(k0, rel=1e-12)


def test_appended_zero_row_moves_the_approximation_endpoint_by_the_corner_mismatch():
    """The exception above, quantified: with an appended zero row the approximation scheme's
    output becomes a(1) + b(1) - (a(0) + b(0)) / 2, where a and b are the edges entering the final
    (zero) cell, so it moves by half their corner mismatch.  That mismatch is truncation error and
    shrinks fast with the order."""
    X = W.brownian(1, 9, 3, seed=101)[0]
    Y = W.brownian(1, 7, 3, seed=102)[0]
    Xr = np.insert(X, 8, X[8], axis=0)
    gaps = [abs(oracle.kernel(Xr, Y, "approx", N) - oracle.kernel(X, Y, "approx", N)) for N in (3, 5, 7, 9)]
    assert gaps[0] > 1e-6
    assert all(gaps[k + 1] < gaps[k] / 10 for k in range(3)), gaps
