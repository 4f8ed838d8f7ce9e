"""Accuracy report of the schemes on the GPU: mean absolute percentage error (MAPE) against a
converged solution, over the orders and refinements of the paper's accuracy study (Section 4 and
Appendix "Additional Experiments", Figures "errorvslevel" and "errorvslevelsin", Tables 1-3).

Workloads: 8 x 8 batches of 2-d paths of a given length,
  * ``sin``: x_i = sin(U_i) against y_i = cos(V_i), U_i, V_i ~ N(0, I_2) i.i.d. (eq. (sinpath));
  * ``brownian``: unit-rate Brownian motion sampled at dt = 0.01 (step variance 0.01 per
    coordinate), the reading of the tables' "standard Brownian motion".

Orders: the approximation scheme runs N = 2..16 (the library's range; the paper's sweep goes to
17, where every batch here is already at its rounding floor), the interpolation scheme N = 2..12.

Truth: the interpolation scheme of order 12 in FP64 at dyadic order ``truth_lambda`` (default 3),
checked against the approximation scheme of order 16 at the same refinement (their largest
relative disagreement is reported as ``truth_check``).  The paper uses the level-21 truncated
signature kernel, whose truncation error grows with the length of the sin/cos paths: against the
interpolation scheme of order 12 at lambda = 2, one pair differs by 4e-15 (relative) at 10
points, 1.6e-10 at 30 and 1.6e-6 at 50.

Run ``python -m paper_2502_08470_gb300.accuracy`` for a JSON report.
"""
from __future__ import annotations

import json

import numpy as np
import torch

from . import sigkernel as sk
from . import workloads as W


def _brownian_dt(n: int, L: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    out = np.zeros((n, L, 2))
    out[:, 1:] = np.cumsum(rng.standard_normal((n, L - 1, 2)) * 0.1, axis=1)
    return out


def batch(kind: str, L: int, seed: int = 0):
    """The 8 x 8 workload of one kind and length as two [8, L, 2] float64 arrays."""
    if kind == "sin":
        return W.sinpath(8, L, seed=seed), W.cospath(8, L, seed=seed + 1)
    if kind == "brownian":
        return _brownian_dt(8, L, seed), _brownian_dt(8, L, seed + 1)
    raise ValueError(kind)


def _gram(X, Y, **kw) -> np.ndarray:
    G = sk.sigkernel_gram(X, Y, **kw)
    torch.cuda.synchronize()
    status = sk.device_status()
    if status != 0:
        raise sk.SigKernelError(status, "device error word set by an accuracy run")
    return G.cpu().numpy()


def mape_pct(G: np.ndarray, truth: np.ndarray) -> float:
    return 100.0 * float(np.mean(np.abs(G - truth) / np.abs(truth)))


def report(kind: str = "sin", lengths=(10, 50, 100, 200), compute: str = "f64", truth_lambda: int = 3,
           approx_orders=range(2, 17), interp_orders=range(2, 13), fd_lambdas=range(0, 7), seed: int = 0) -> dict:
    """MAPE (percent) per scheme and order / refinement for each length: ``approx`` and ``interp``
    by order N at lambda = 0, ``approx8_hybrid`` by lambda at N = 8, ``fd1`` / ``fd2`` /
    ``fd_implicit`` by lambda."""
    out = {"workload": f"8 x 8 pairs of 2-d {kind} paths", "compute": compute, "truth": f"interp N=12, "
           f"lambda={truth_lambda}, FP64", "lengths": {}}
    for L in lengths:
        Xn, Yn = batch(kind, L, seed)
        X, Y = torch.tensor(Xn, device="cuda"), torch.tensor(Yn, device="cuda")
        truth = _gram(X, Y, scheme="interp", degree=12, dyadic=truth_lambda, compute="f64")
        check = _gram(X, Y, scheme="approx", degree=16, dyadic=truth_lambda, compute="f64")
        row = {"truth_check": float(np.max(np.abs(check - truth) / np.abs(truth)))}
        row["approx"] = {N: mape_pct(_gram(X, Y, scheme="approx", degree=N, compute=compute), truth)
                         for N in approx_orders}
        row["interp"] = {N: mape_pct(_gram(X, Y, scheme="interp", degree=N, compute=compute), truth)
                         for N in interp_orders}
        # the hybrid method of Section 3.2: the approximation scheme of order 8 on refined grids
        row["approx8_hybrid"] = {lam: mape_pct(_gram(X, Y, scheme="approx", degree=8, dyadic=lam, compute=compute),
                                               truth) for lam in (0, 1, 2, 3)}
        for fd in ("fd1", "fd2", "fd_implicit"):
            row[fd] = {lam: mape_pct(_gram(X, Y, scheme=fd, dyadic=lam, compute=compute), truth) for lam in fd_lambdas}
        out["lengths"][L] = row
    return out


if __name__ == "__main__":
    print(json.dumps({k: report(k) for k in ("sin", "brownian")}, indent=1))
