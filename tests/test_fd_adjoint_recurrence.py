"""CPU check of the reverse-mode recurrence of the finite-difference schemes (Definition "dyadic
scheme", eq. (secondexplicitscheme), Remark "higherfd").

Every FD sub-cell update has the form k11 = alpha(m) (k10 + k01) - beta(m) k00 with
  FD1:       alpha = 1 + m/2,                beta = 1
  FD2:       alpha = 1 + m/2 + m^2/12,       beta = 1 - m^2/12
  implicit:  alpha = (1 + m/4) / (1 - m/4),  beta = 1
so the adjoint of the node values obeys the same three-point recurrence run backwards:
  kbar(I, J) = alpha(m_{I-1,J}) kbar(I, J+1) + alpha(m_{I,J-1}) kbar(I+1, J) - beta(m_{I,J}) kbar(I+1, J+1),
and dk/dm of a sub-cell is kbar(I+1, J+1) (alpha'(m) (k10 + k01) - beta'(m) k00).  A GPU adjoint of
the FD schemes is that wavefront in reverse over the forward's node values.  Here a numpy
restatement of the forward and of this recurrence is checked against the oracle's values and
its complex-step gradients (which differentiate the forward code itself).
"""
import numpy as np
import pytest

import oracle
from paper_2502_08470_gb300 import workloads as W

COEF = {
    "fd1": (lambda m: 1 + m / 2, lambda m: np.ones_like(m), lambda m: np.full_like(m, 0.5), lambda m: np.zeros_like(m)),
    "fd2": (lambda m: 1 + m / 2 + m * m / 12, lambda m: 1 - m * m / 12, lambda m: 0.5 + m / 6, lambda m: -m / 6),
    "fd_implicit": (lambda m: (1 + m / 4) / (1 - m / 4), lambda m: np.ones_like(m),
                    lambda m: 0.5 / (1 - m / 4) ** 2, lambda m: np.zeros_like(m)),
}


def _refined_increments(x, lam):
    dx = np.diff(x, axis=0) / 2 ** lam
    return np.repeat(dx, 2 ** lam, axis=0)


def fd_value_and_grad(x, y, scheme, lam):
    alpha, beta, dalpha, dbeta = COEF[scheme]
    dxr, dyr = _refined_increments(x, lam), _refined_increments(y, lam)
    m = dxr @ dyr.T                                   # sub-cell increments' inner products
    nI, nJ = m.shape
    a, b = alpha(m), beta(m)
    K = np.ones((nI + 1, nJ + 1))
    for u in range(nI):
        for w in range(nJ):
            K[u + 1, w + 1] = a[u, w] * (K[u + 1, w] + K[u, w + 1]) - b[u, w] * K[u, w]
    Kb = np.zeros_like(K)
    Kb[nI, nJ] = 1.0
    mb = np.zeros_like(m)
    for u in range(nI - 1, -1, -1):
        for w in range(nJ - 1, -1, -1):
            g = Kb[u + 1, w + 1]
            Kb[u + 1, w] += a[u, w] * g
            Kb[u, w + 1] += a[u, w] * g
            Kb[u, w] -= b[u, w] * g
            mb[u, w] = g * (dalpha(m[u, w]) * (K[u + 1, w] + K[u, w + 1]) - dbeta(m[u, w]) * K[u, w])
    # chain rule through m = <dxr_u, dyr_w>, dxr_u = dx_{u >> lam} / 2^lam, x_p -> dx_{p-1}, dx_p
    gdxr, gdyr = mb @ dyr, mb.T @ dxr
    gdx = gdxr.reshape(-1, 2 ** lam, x.shape[1]).sum(axis=1) / 2 ** lam
    gdy = gdyr.reshape(-1, 2 ** lam, y.shape[1]).sum(axis=1) / 2 ** lam

    def to_points(gd):
        g = np.zeros((gd.shape[0] + 1, gd.shape[1]))
        g[1:] += gd
        g[:-1] -= gd
        return g
    return K[nI, nJ], to_points(gdx), to_points(gdy)


@pytest.mark.parametrize("scheme", ["fd1", "fd2", "fd_implicit"])
@pytest.mark.parametrize("lam", [0, 1, 2])
def test_reverse_recurrence_gives_the_oracle_gradient(scheme, lam):
    x = W.brownian(1, 9, 3, seed=40 + lam)[0]
    y = W.brownian(1, 7, 3, seed=50 + lam, drift=0.3)[0]
    k, gx, gy = fd_value_and_grad(x, y, scheme, lam)
    ref = oracle.kernel(x, y, scheme, 2, lam)
    assert abs(k - ref) <= 1e-13 * abs(ref)
    rx, ry = oracle.grad(x, y, scheme, 2, lam)
    scale = max(np.abs(rx).max(), np.abs(ry).max())
    assert np.abs(gx - rx).max() <= 1e-12 * scale
    assert np.abs(gy - ry).max() <= 1e-12 * scale


def test_recurrence_with_a_large_implicit_step():
    """Sub-cells with m between 1.9 and 3.45, near the implicit scheme's pole at m = 4, where
    alpha reaches 13.5 and alpha' 26."""
    x = 1.3 * np.array([[0.0, 0.0], [1.2, 0.9], [1.5, 2.3]])
    y = 1.3 * np.array([[0.0, 0.0], [1.1, 0.8], [1.0, 2.2]])
    k, gx, gy = fd_value_and_grad(x, y, "fd_implicit", 0)
    assert abs(k - oracle.kernel(x, y, "fd_implicit", 2, 0)) <= 1e-13 * abs(k)
    rx, ry = oracle.grad(x, y, "fd_implicit", 2, 0)
    scale = max(np.abs(rx).max(), np.abs(ry).max())
    assert np.abs(gx - rx).max() <= 1e-12 * scale and np.abs(gy - ry).max() <= 1e-12 * scale
