"""FP64 CPU oracle for the signature-kernel schemes (TEST INFRASTRUCTURE ONLY).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It is a plain restatement of the paper's definitions in C
(``sigkernel_oracle.c`` + ``oracle_schemes.h``), compiled with gcc on first use and called
through ctypes.  It shares no code with the CUDA library and never imports it.

Schemes (ids follow the C library's enum for convenience of the tests only):
  0 "fd1"     first-order explicit finite differences on P_lambda   (Definition "dyadic scheme")
  1 "fd2"     second-order explicit finite differences              (eq. secondexplicitscheme)
  2 "approx"  polynomial approximation scheme of order N            (Def. polyapproxscheme)
  3 "interp"  polynomial interpolation scheme of order N            (Def. polyinterpscheme)
  4 "fd_implicit"  implicit finite differences, four-corner trapezoid rule (Remark higherfd)

Beyond the schemes: MMD^2 and its gradient (C), and the two-sample permutation test on MMD^2
(``mmd2_permutation_test``, numpy over the oracle's Gram).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "sigkernel_oracle.c"), os.path.join(_HERE, "oracle_schemes.h")]
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

SCHEMES = {"fd1": 0, "fd2": 1, "approx": 2, "interp": 3, "fd_implicit": 4}


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (idempotent unless the sources changed)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = force or not os.path.exists(_SO) or any(
        os.path.getmtime(s) > os.path.getmtime(_SO) for s in _SRC)
    if stale:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC[0], "-lm", "-lpthread"]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        P = ctypes.c_void_p
        lib.sko_scheme.restype = d
        lib.sko_scheme.argtypes = [i32, P, i64, P, i64, i32, i32, i32, P, P]
        lib.sko_pairs.restype = i32
        lib.sko_pairs.argtypes = [i32, P, P, P, P, i32, P, P, i64, i32, i32, i32, P]
        lib.sko_grad_entry.restype = d
        lib.sko_grad_entry.argtypes = [i32, P, i64, P, i64, i32, i32, i32, i32, i64, i32]
        lib.sko_grad_pair.restype = None
        lib.sko_grad_pair.argtypes = [i32, P, i64, P, i64, i32, i32, i32, P, P, i32]
        lib.sko_sig_trunc.restype = d
        lib.sko_sig_trunc.argtypes = [P, i64, P, i64, i32, i32]
        lib.sko_signature_level.restype = None
        lib.sko_signature_level.argtypes = [P, i64, i32, i32, P]
        lib.sko_mmd2.restype = d
        lib.sko_mmd2.argtypes = [i32, P, i64, P, i64, i64, i32, i32, i32, i32]
        lib.sko_mmd2_grad_entry.restype = d
        lib.sko_mmd2_grad_entry.argtypes = [i32, P, i64, P, i64, i64, i32, i32, i32, i32, i32, i64, i64, i32]
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _sid(scheme) -> int:
    return SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)


def kernel(x, y, scheme="approx", N=6, lam=0, s=None, t=None) -> float:
    """Scheme output k_hat(x, y) for one pair of piecewise-linear paths x [Lx, d], y [Ly, d].

    ``s`` / ``t`` are optional time partitions (default uniform on [0, 1])."""
    x, y = _f64(x), _f64(y)
    assert x.ndim == 2 and y.ndim == 2 and x.shape[1] == y.shape[1]
    sg = _f64(s) if s is not None else None
    tg = _f64(t) if t is not None else None
    return _load().sko_scheme(_sid(scheme), _ptr(x), x.shape[0], _ptr(y), y.shape[0], x.shape[1], N, lam,
                              _ptr(sg) if sg is not None else None, _ptr(tg) if tg is not None else None)


def _concat(paths):
    paths = [_f64(p) for p in paths]
    off = np.zeros(len(paths) + 1, dtype=np.int64)
    off[1:] = np.cumsum([p.shape[0] for p in paths])
    return np.ascontiguousarray(np.concatenate(paths, axis=0)), off


def pairs(X, Y, pa, pb, scheme="approx", N=6, lam=0, threads=0) -> np.ndarray:
    """k_hat for the pairs (X[pa[k]], Y[pb[k]]); X, Y are sequences of [L_i, d] arrays."""
    Xc, xo = _concat(X)
    Yc, yo = _concat(Y)
    pa = np.ascontiguousarray(np.asarray(pa, dtype=np.int64))
    pb = np.ascontiguousarray(np.asarray(pb, dtype=np.int64))
    out = np.empty(pa.shape[0], dtype=np.float64)
    d = Xc.shape[1]
    _load().sko_pairs(_sid(scheme), _ptr(Xc), _ptr(xo), _ptr(Yc), _ptr(yo), d, _ptr(pa), _ptr(pb),
                      pa.shape[0], N, lam, threads, _ptr(out))
    return out


def gram(X, Y, scheme="approx", N=6, lam=0, threads=0) -> np.ndarray:
    """Gram matrix G[a, b] = k_hat(X[a], Y[b])."""
    nx, ny = len(X), len(Y)
    pa, pb = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    return pairs(X, Y, pa.ravel(), pb.ravel(), scheme, N, lam, threads).reshape(nx, ny)


def grad_entry(x, y, side, p, c, scheme="approx", N=6, lam=0) -> float:
    """d k_hat / d x[p, c] (side 0) or d k_hat / d y[p, c] (side 1), complex step."""
    x, y = _f64(x), _f64(y)
    return _load().sko_grad_entry(_sid(scheme), _ptr(x), x.shape[0], _ptr(y), y.shape[0], x.shape[1], N,
                                  lam, side, p, c)


def grad(x, y, scheme="approx", N=6, lam=0, threads=0):
    """Full gradients (dk/dx [Lx, d], dk/dy [Ly, d]) of one pair, complex step, coordinates split
    over ``threads`` threads (0 = all cores)."""
    x, y = _f64(x), _f64(y)
    gx = np.empty_like(x)
    gy = np.empty_like(y)
    _load().sko_grad_pair(_sid(scheme), _ptr(x), x.shape[0], _ptr(y), y.shape[0], x.shape[1], N, lam,
                          _ptr(gx), _ptr(gy), threads)
    return gx, gy


def sig_trunc(x, y, level) -> float:
    """sum_{n<=level} <S_n(x), S_n(y)> by brute-force truncated signatures."""
    x, y = _f64(x), _f64(y)
    return _load().sko_sig_trunc(_ptr(x), x.shape[0], _ptr(y), y.shape[0], x.shape[1], level)


def signature_level(x, level) -> np.ndarray:
    """Level-n tensor of the signature of one path, flattened in base-d index order."""
    x = _f64(x)
    d = x.shape[1]
    out = np.empty(d ** level, dtype=np.float64)
    _load().sko_signature_level(_ptr(x), x.shape[0], d, level, _ptr(out))
    return out


def mmd2(A, B, scheme="approx", N=6, lam=0, unbiased=False) -> float:
    """MMD^2 between equal-length path batches A [na, L, d] and B [nb, L, d]."""
    A, B = _f64(A), _f64(B)
    na, L, d = A.shape
    return _load().sko_mmd2(_sid(scheme), _ptr(A), na, _ptr(B), B.shape[0], L, d, N, lam, int(unbiased))


def mmd2_grad_entry(A, B, side, path, p, c, scheme="approx", N=6, lam=0, unbiased=False) -> float:
    """d MMD^2 / d A[path, p, c] (side 0) or B[path, p, c] (side 1), complex step."""
    A, B = _f64(A), _f64(B)
    na, L, d = A.shape
    return _load().sko_mmd2_grad_entry(_sid(scheme), _ptr(A), na, _ptr(B), B.shape[0], L, d, N, lam,
                                       int(unbiased), side, path, p, c)


def mmd2_permutation_test(A, B, labels, scheme="approx", N=6, lam=0, unbiased=False):
    """Two-sample permutation test on MMD^2 (the paper names statistical hypothesis testing as a
    use of the kernel, Sections 1 and 4, without defining it; this is the standard test).

    The pooled sample Z = (A_0..A_{na-1}, B_0..B_{nb-1}) has Gram matrix K = gram(Z, Z).  A
    relabelling marks na paths of Z as the first sample; its statistic is MMD^2 of the two marked
    subsets, from the means of the blocks of K: biased  mean K_11 + mean K_00 - 2 mean K_10;
    unbiased  the same with the diagonals of K_11 and K_00 left out of their sums and means over
    na (na - 1) and nb (nb - 1).  The observed statistic is that of the given split (the first
    na paths of Z).  p-value = (1 + #{p : stat_p >= observed}) / (1 + nperm).

    labels: [nperm, na + nb], nonzero = first sample; every row must mark exactly na paths.
    Returns (observed, p_value, stats[nperm])."""
    A, B = list(A), list(B)
    na, nb = len(A), len(B)
    n = na + nb
    K = gram(A + B, A + B, scheme, N, lam)
    labels = np.asarray(labels)
    assert labels.ndim == 2 and labels.shape[1] == n

    def stat(first):
        a, b = np.flatnonzero(first), np.flatnonzero(~first)
        assert len(a) == na
        Kaa, Kbb, Kab = K[np.ix_(a, a)], K[np.ix_(b, b)], K[np.ix_(a, b)]
        if unbiased:
            saa = (Kaa.sum() - np.trace(Kaa)) / (na * (na - 1))
            sbb = (Kbb.sum() - np.trace(Kbb)) / (nb * (nb - 1))
        else:
            saa, sbb = Kaa.mean(), Kbb.mean()
        return saa + sbb - 2.0 * Kab.mean()

    observed = stat(np.arange(n) < na)
    stats = np.array([stat(row != 0) for row in labels])
    p_value = (1 + np.count_nonzero(stats >= observed)) / (1 + len(stats))
    return observed, p_value, stats
