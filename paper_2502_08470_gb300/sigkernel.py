"""Python binding of the C ABI in ``include/sigkernel.h`` (argument marshalling only).

Every computation runs in ``_lib/libsigkernel.so`` on the current CUDA device and stream; this
module converts torch tensors to the ABI's pointers and sizes.  If the library is missing the
first call raises; there is no CPU fallback.

Paths are given either as a dense tensor ``[B, L, d]`` (all paths with L points) or as a
:class:`Paths` (concatenated rows plus int64 offsets, for ragged batches).
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsigkernel.so")

SK_OK = 0
ERRORS = {-1: "SK_ERR_INVALID_ARG", -2: "SK_ERR_UNSUPPORTED", -3: "SK_ERR_CUDA", -4: "SK_ERR_WORKSPACE",
          -5: "SK_ERR_DEVICE_TIMEOUT", -6: "SK_ERR_NONFINITE", -7: "SK_ERR_BAD_LENGTH", -8: "SK_ERR_BAD_LABELS"}
SCHEMES = {"fd1": 0, "fd2": 1, "approx": 2, "interp": 3, "fd_implicit": 4}
COMPUTE = {"f64": 0, "f32": 1}
DTYPES = {torch.float64: 0, torch.float32: 1, torch.bfloat16: 2}
FLAG_SYMMETRIC, FLAG_INCREMENTS, FLAG_UNBIASED, FLAG_NO_SORT, FLAG_TIME_KERNEL = 1, 2, 4, 8, 16
FLAG_STRIP_PIPELINE, FLAG_NO_STRIP_PIPELINE, FLAG_NO_TILED_M, FLAG_CHECKPOINT, FLAG_NO_TC = 32, 64, 128, 256, 512


def _pipe_flags(strip_pipeline) -> int:
    """None: the library decides; True: every pair of 2+ strips is swept by a block of warps;
    False: one warp per pair."""
    if strip_pipeline is None:
        return 0
    return FLAG_STRIP_PIPELINE if strip_pipeline else FLAG_NO_STRIP_PIPELINE
OP_PAIRS, OP_GRAM, OP_BACKWARD, OP_MMD2, OP_BACKWARD_TAPE, OP_MMD2_TEST = 0, 1, 2, 3, 4, 5


class SigKernelError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Options(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("degree", ctypes.c_int32), ("dyadic", ctypes.c_int32),
                ("compute", ctypes.c_int32), ("interp_extra", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("warps_per_block", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _Paths(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("count", ctypes.c_int64),
                ("max_len", ctypes.c_int64), ("rows_total", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None


def load_library():
    """Load ``libsigkernel.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2502_08470_gb300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        P, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        PP, PO = ctypes.POINTER(_Paths), ctypes.POINTER(_Options)
        lib.sigkernel_version.restype = ctypes.c_int
        lib.sigkernel_last_error.restype = ctypes.c_char_p
        lib.sigkernel_workspace_size.restype = ctypes.c_int
        lib.sigkernel_workspace_size.argtypes = [I32, PP, PP, I32, I64, PO, ctypes.POINTER(SZ)]
        lib.sigkernel_pairs.restype = ctypes.c_int
        lib.sigkernel_pairs.argtypes = [PP, PP, I32, I32, P, P, I64, PO, P, P, SZ, P]
        lib.sigkernel_gram.restype = ctypes.c_int
        lib.sigkernel_gram.argtypes = [PP, PP, I32, I32, PO, P, P, SZ, P]
        lib.sigkernel_backward.restype = ctypes.c_int
        lib.sigkernel_backward.argtypes = [PP, PP, I32, I32, P, P, I64, PO, P, P, P, P, SZ, P]
        lib.sigkernel_mmd2.restype = ctypes.c_int
        lib.sigkernel_mmd2.argtypes = [PP, PP, I32, I32, PO, P, P, P, P, SZ, P]
        lib.sigkernel_mmd2_test.restype = ctypes.c_int
        lib.sigkernel_mmd2_test.argtypes = [PP, PP, I32, I32, PO, P, I64, P, P, SZ, P]
        lib.sigkernel_tape_size.restype = ctypes.c_int
        lib.sigkernel_tape_size.argtypes = [PP, PP, I32, I64, PO, ctypes.POINTER(SZ)]
        lib.sigkernel_forward_tape.restype = ctypes.c_int
        lib.sigkernel_forward_tape.argtypes = [PP, PP, I32, I32, P, P, I64, PO, P, P, SZ, P, SZ, P]
        lib.sigkernel_backward_tape.restype = ctypes.c_int
        lib.sigkernel_backward_tape.argtypes = [PP, PP, I32, I32, P, P, I64, PO, P, SZ, P, P, P, P, SZ, P]
        lib.sigkernel_autotune.restype = ctypes.c_int
        lib.sigkernel_autotune.argtypes = [PP, PP, I32, I32, P, P, I64, PO, P, I32, PO, ctypes.POINTER(ctypes.c_float), P]
        lib.sigkernel_autotune_clear.restype = None
        lib.sigkernel_last_kernel_ms.restype = ctypes.c_float
        lib.sigkernel_device_status.restype = ctypes.c_int
        lib.sigkernel_device_status.argtypes = [P]
        lib.sigkernel_fma_peak.restype = ctypes.c_int
        lib.sigkernel_fma_peak.argtypes = [I32, I32, I32, ctypes.POINTER(ctypes.c_double), P]
        lib.sigkernel_set_wait_limit.restype = None
        lib.sigkernel_set_wait_limit.argtypes = [ctypes.c_uint32]
        _lib = lib
        return lib


def _check(rc: int):
    if rc != SK_OK:
        msg = load_library().sigkernel_last_error().decode(errors="replace")
        raise SigKernelError(rc, msg)


@dataclass
class Paths:
    """A ragged batch of paths: ``rows`` [R, d] (points, or increments with ``increments=True``)
    on the GPU and int64 ``offsets`` [B + 1] (path a is rows offsets[a]:offsets[a+1])."""
    rows: torch.Tensor
    offsets: torch.Tensor
    max_len: int
    increments: bool = False

    @property
    def count(self) -> int:
        return self.offsets.numel() - 1

    @property
    def d(self) -> int:
        return self.rows.shape[1]

    @staticmethod
    def from_list(paths, device="cuda", dtype=None, increments=False) -> "Paths":
        ts = [torch.as_tensor(p) for p in paths]
        dtype = dtype or (ts[0].dtype if ts else torch.float64)
        lens = [t.shape[0] for t in ts]
        off = torch.zeros(len(ts) + 1, dtype=torch.int64)
        if ts:
            off[1:] = torch.cumsum(torch.tensor(lens, dtype=torch.int64), 0)
        rows = torch.cat([t.to(dtype) for t in ts], 0) if ts else torch.zeros(0, 1, dtype=dtype)
        return Paths(rows.to(device).contiguous(), off.to(device), max(lens) if lens else 0, increments)

    @staticmethod
    def from_dense(x: torch.Tensor, increments=False) -> "Paths":
        B, L, d = x.shape
        off = torch.arange(0, (B + 1) * L, L, dtype=torch.int64, device=x.device)
        return Paths(x.reshape(B * L, d).contiguous(), off, L, increments)


def as_paths(x) -> Paths:
    if isinstance(x, Paths):
        return x
    if isinstance(x, torch.Tensor) and x.dim() == 3:
        return Paths.from_dense(x)
    raise TypeError("paths must be a Paths or a [B, L, d] tensor")


def _cpaths(p: Paths) -> _Paths:
    # the library reads rows as [R][d] and offsets as [B + 1] from their first elements
    if p.rows.dim() != 2 or p.offsets.dim() != 1:
        raise ValueError("path rows must be [R, d] and offsets [B + 1]")
    if not p.rows.is_contiguous() or not p.offsets.is_contiguous():
        raise ValueError("path rows and offsets must be contiguous")
    if not p.rows.is_cuda or not p.offsets.is_cuda:
        raise ValueError("path rows and offsets must be CUDA tensors")
    if p.offsets.dtype != torch.int64:
        raise ValueError("offsets must be int64")
    dev = torch.cuda.current_device()
    if p.rows.device.index != dev or p.offsets.device.index != dev:
        raise ValueError(f"path rows and offsets must be on the current CUDA device (cuda:{dev})")
    return _Paths(p.rows.data_ptr(), p.offsets.data_ptr(), p.count, int(p.max_len), p.rows.shape[0])


def _device_buffer(t: torch.Tensor, name: str, dtype=None, numel=None) -> torch.Tensor:
    """A tensor the library reads or writes through a raw pointer: contiguous, on the current CUDA
    device, of `dtype` and with `numel` elements when given.  The library cannot see the size of a
    device buffer, so a short one would be read or written past its end."""
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, not {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements where the call needs {numel}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} must be on the current CUDA device")
    return t


def _nbytes(t: torch.Tensor) -> int:
    return t.numel() * t.element_size()


def _pair_tensors(pair_a, pair_b):
    """The pair lists as int64 CUDA tensors of equal length (the library reads npairs of each)."""
    pa = torch.as_tensor(pair_a, dtype=torch.int64)
    pb = torch.as_tensor(pair_b, dtype=torch.int64)
    if pa.dim() != 1 or pb.dim() != 1 or pa.numel() != pb.numel():
        raise ValueError(f"pair_a and pair_b must be 1-d of one length (got {tuple(pa.shape)} and {tuple(pb.shape)})")
    return pa.to("cuda").contiguous(), pb.to("cuda").contiguous()


def _grad_out(grad_out, nx: int, ny: int, npairs: int) -> torch.Tensor:
    """The upstream gradient as float64 on the device: [nx, ny] in Gram mode (npairs < 0), else
    npairs values."""
    g = torch.as_tensor(grad_out, dtype=torch.float64)
    if npairs < 0:
        if g.numel() != nx * ny or (g.dim() == 2 and tuple(g.shape) != (nx, ny)):
            raise ValueError(f"grad_out must be [{nx}, {ny}] (got {tuple(g.shape)})")
    elif g.numel() != npairs:
        raise ValueError(f"grad_out must hold {npairs} values, one per pair (got {g.numel()})")
    return g.to("cuda").contiguous()


def _options(scheme="approx", degree=6, dyadic=0, compute="f64", flags=0, interp_extra=0) -> _Options:
    return _Options(SCHEMES[scheme] if isinstance(scheme, str) else int(scheme), int(degree), int(dyadic),
                    COMPUTE[compute] if isinstance(compute, str) else int(compute), int(interp_extra), int(flags), 0, 0)


def _stream_ptr() -> int:
    return torch.cuda.current_stream().cuda_stream


def _dtype_code(X: Paths, Y: Paths) -> int:
    if X.rows.dtype != Y.rows.dtype:
        raise ValueError("X and Y must have the same dtype")
    if X.rows.dtype not in DTYPES:
        raise ValueError(f"path dtype {X.rows.dtype} is not one of float64, float32, bfloat16")
    return DTYPES[X.rows.dtype]


def _workspace(op, cX, cY, d, npairs, opt) -> torch.Tensor:
    lib = load_library()
    n = ctypes.c_size_t(0)
    _check(lib.sigkernel_workspace_size(op, ctypes.byref(cX), ctypes.byref(cY), d, npairs, ctypes.byref(opt),
                                        ctypes.byref(n)))
    return torch.empty(int(n.value), dtype=torch.uint8, device="cuda")


def _flags(X: Paths, extra=0) -> int:
    return extra | (FLAG_INCREMENTS if X.increments else 0)


def sigkernel_pairs(X, Y, pair_a, pair_b, scheme="approx", degree=6, dyadic=0, compute="f64", sort=True,
                    out: torch.Tensor | None = None, strip_pipeline=None, time_kernel: bool = False,
                    tiled_m: bool = True, tensor_cores: bool = True) -> torch.Tensor:
    """k_hat(X[pair_a[k]], Y[pair_b[k]]) for every k, as a float64 CUDA tensor.

    ``tensor_cores=False`` (SK_FLAG_NO_TC) keeps the FP32 approximation scheme's M on the FMA pipe
    (tiled, or per cell with ``tiled_m=False``) instead of the tcgen05 M kernel (4 < d <= 32)."""
    X, Y = as_paths(X), as_paths(Y)
    pa, pb = _pair_tensors(pair_a, pair_b)
    n = pa.numel()
    opt = _options(scheme, degree, dyadic, compute,
                   _flags(X, (0 if sort else FLAG_NO_SORT) | _pipe_flags(strip_pipeline)
                          | (FLAG_TIME_KERNEL if time_kernel else 0) | (0 if tiled_m else FLAG_NO_TILED_M)
                          | (0 if tensor_cores else FLAG_NO_TC)))
    cX, cY = _cpaths(X), _cpaths(Y)
    out = _device_buffer(out, "out", torch.float64, n) if out is not None else \
        torch.empty(n, dtype=torch.float64, device="cuda")
    ws = _workspace(OP_PAIRS, cX, cY, X.d, n, opt)
    _check(load_library().sigkernel_pairs(ctypes.byref(cX), ctypes.byref(cY), X.d, _dtype_code(X, Y), pa.data_ptr(),
                                          pb.data_ptr(), n, ctypes.byref(opt), out.data_ptr(), ws.data_ptr(),
                                          ws.numel(), _stream_ptr()))
    return out


def sigkernel_gram(X, Y=None, scheme="approx", degree=6, dyadic=0, compute="f64", sort=True,
                   workspace: torch.Tensor | None = None, out: torch.Tensor | None = None,
                   time_kernel: bool = False, strip_pipeline=None, tiled_m: bool = True,
                   tensor_cores: bool = True) -> torch.Tensor:
    """G[a, b] = k_hat(X[a], Y[b]); with Y None (or Y is X) the symmetric Gram of X.

    ``time_kernel`` records CUDA events around the wavefront kernel (see ``last_kernel_ms``; with
    the tcgen05 M kernel, from its first launch to the last sweep); ``strip_pipeline`` (None / True
    / False) chooses how long pairs are swept (see the flags SK_FLAG_STRIP_PIPELINE and
    SK_FLAG_NO_STRIP_PIPELINE); ``tensor_cores=False`` (SK_FLAG_NO_TC) keeps the FP32
    approximation scheme's M on the FMA pipe instead of the tcgen05 M kernel (4 < d <= 32)."""
    sym = Y is None or Y is X
    X = as_paths(X)
    Y = X if sym else as_paths(Y)
    flags = _flags(X, (FLAG_SYMMETRIC if sym else 0) | (0 if sort else FLAG_NO_SORT)
                   | (FLAG_TIME_KERNEL if time_kernel else 0) | _pipe_flags(strip_pipeline)
                   | (0 if tiled_m else FLAG_NO_TILED_M) | (0 if tensor_cores else FLAG_NO_TC))
    opt = _options(scheme, degree, dyadic, compute, flags)
    cX, cY = _cpaths(X), _cpaths(Y)
    G = _device_buffer(out, "out", torch.float64, X.count * Y.count) if out is not None else \
        torch.empty(X.count, Y.count, dtype=torch.float64, device="cuda")
    ws = _device_buffer(workspace, "workspace") if workspace is not None else \
        _workspace(OP_GRAM, cX, cY, X.d, -1, opt)
    _check(load_library().sigkernel_gram(ctypes.byref(cX), ctypes.byref(cY), X.d, _dtype_code(X, Y),
                                         ctypes.byref(opt), G.data_ptr(), ws.data_ptr(), _nbytes(ws), _stream_ptr()))
    return G


def gram_workspace(X, Y=None, scheme="approx", degree=6, dyadic=0, compute="f64",
                   strip_pipeline=None) -> torch.Tensor:
    """A workspace tensor sized for ``sigkernel_gram`` with these shapes (reusable across calls)."""
    sym = Y is None or Y is X
    X = as_paths(X)
    Y = X if sym else as_paths(Y)
    opt = _options(scheme, degree, dyadic, compute,
                   _flags(X, (FLAG_SYMMETRIC if sym else 0) | _pipe_flags(strip_pipeline)))
    return _workspace(OP_GRAM, _cpaths(X), _cpaths(Y), X.d, -1, opt)


def autotune(X, Y=None, pair_a=None, pair_b=None, scheme="approx", degree=6, dyadic=0, compute="f32",
             trials=3, sort=True):
    """Time the forward launch shapes on these inputs (``sigkernel_autotune``) and remember the
    fastest for later calls of the same shape that leave the shape to the library.  Returns
    ``(shape, ms)`` with ``shape = {"warps_per_block": w, "strip_pipeline": bool}``."""
    pairs = pair_a is not None
    sym = not pairs and (Y is None or Y is X)
    X = as_paths(X)
    Y = X if (Y is None or Y is X) else as_paths(Y)
    cX, cY = _cpaths(X), _cpaths(Y)
    if pairs:
        pa, pb = _pair_tensors(pair_a, pair_b)
        n, pa_ptr, pb_ptr = pa.numel(), pa.data_ptr(), pb.data_ptr()
        out = torch.empty(n, dtype=torch.float64, device="cuda")
    else:
        n, pa_ptr, pb_ptr = 0, None, None
        out = torch.empty(X.count, Y.count, dtype=torch.float64, device="cuda")
    opt = _options(scheme, degree, dyadic, compute,
                   _flags(X, (FLAG_SYMMETRIC if sym else 0) | (0 if sort else FLAG_NO_SORT)))
    best = _Options()
    ms = ctypes.c_float(0)
    _check(load_library().sigkernel_autotune(ctypes.byref(cX), ctypes.byref(cY), X.d, _dtype_code(X, Y), pa_ptr,
                                             pb_ptr, n, ctypes.byref(opt), out.data_ptr(), int(trials),
                                             ctypes.byref(best), ctypes.byref(ms), _stream_ptr()))
    return {"warps_per_block": best.warps_per_block,
            "strip_pipeline": bool(best.flags & FLAG_STRIP_PIPELINE)}, float(ms.value)


def autotune_clear():
    """Forget every launch shape chosen by ``autotune`` in this process."""
    load_library().sigkernel_autotune_clear()


def sigkernel_backward(grad_out, X, Y=None, pair_a=None, pair_b=None, scheme="approx", degree=6, dyadic=0,
                       compute="f64", sort=True, time_kernel: bool = False, checkpoint: bool = False,
                       tensor_cores: bool = True):
    """Gradients of sum(grad_out * k_hat) with respect to the rows of X and Y (float64 CUDA tensors
    shaped like the rows).  Gram mode when ``pair_a`` is None (``grad_out`` [nx, ny]); with Y None
    (or Y is X) the symmetric Gram of X, and the single returned gradient is the total.
    ``checkpoint`` selects the checkpointing adjoint of the approximation scheme (SK_FLAG_CHECKPOINT)
    instead of the adjoint from chunked forward tapes; ``tensor_cores=False`` keeps the dk/dM
    contraction on the FMA pipe (SK_FLAG_NO_TC)."""
    sym = Y is None or Y is X
    X = as_paths(X)
    Y = X if sym else as_paths(Y)
    cX, cY = _cpaths(X), _cpaths(Y)
    if pair_a is not None:
        pa, pb = _pair_tensors(pair_a, pair_b)
    g = _grad_out(grad_out, X.count, Y.count, -1 if pair_a is None else pa.numel())
    gX = torch.zeros(X.rows.shape[0], X.d, dtype=torch.float64, device="cuda")
    same = sym or (X.rows.data_ptr() == Y.rows.data_ptr() and X.offsets.data_ptr() == Y.offsets.data_ptr())
    gY = gX if same else torch.zeros(Y.rows.shape[0], Y.d, dtype=torch.float64, device="cuda")
    extra = ((0 if sort else FLAG_NO_SORT) | (FLAG_TIME_KERNEL if time_kernel else 0) | (FLAG_CHECKPOINT if checkpoint else 0)
             | (0 if tensor_cores else FLAG_NO_TC))
    if pair_a is None:
        opt = _options(scheme, degree, dyadic, compute, _flags(X, extra | (FLAG_SYMMETRIC if sym else 0)))
        ws = _workspace(OP_BACKWARD, cX, cY, X.d, -1, opt)
        pa_ptr = pb_ptr = None
        n = -1
    else:
        n = pa.numel()
        opt = _options(scheme, degree, dyadic, compute, _flags(X, extra))
        ws = _workspace(OP_BACKWARD, cX, cY, X.d, n, opt)
        pa_ptr, pb_ptr = pa.data_ptr(), pb.data_ptr()
    _check(load_library().sigkernel_backward(ctypes.byref(cX), ctypes.byref(cY), X.d, _dtype_code(X, Y), pa_ptr, pb_ptr,
                                             n, ctypes.byref(opt), g.data_ptr(), gX.data_ptr(),
                                             None if same else gY.data_ptr(), ws.data_ptr(), ws.numel(),
                                             _stream_ptr()))
    return gX, gY


def _pair_args(X, pair_a, pair_b, sym):
    if pair_a is None:
        return None, None, -1, None
    pa, pb = _pair_tensors(pair_a, pair_b)
    return pa.data_ptr(), pb.data_ptr(), pa.numel(), (pa, pb)


def sigkernel_forward_tape(X, Y=None, pair_a=None, pair_b=None, scheme="approx", degree=6, dyadic=0, compute="f32",
                           sort=True, time_kernel=False, tape: torch.Tensor | None = None,
                           workspace: torch.Tensor | None = None, out: torch.Tensor | None = None,
                           tensor_cores: bool = True):
    """Forward values (Gram when ``pair_a`` is None) plus the tape the adjoint replays from.
    Returns (values, tape).  ``tensor_cores=False``: M on the FMA pipe (SK_FLAG_NO_TC)."""
    sym = pair_a is None and (Y is None or Y is X)
    X = as_paths(X)
    Y = X if (Y is None or Y is X) else as_paths(Y)
    cX, cY = _cpaths(X), _cpaths(Y)
    pa_ptr, pb_ptr, n, keep = _pair_args(X, pair_a, pair_b, sym)
    flags = _flags(X, (FLAG_SYMMETRIC if sym else 0) | (0 if sort else FLAG_NO_SORT)
                   | (FLAG_TIME_KERNEL if time_kernel else 0) | (0 if tensor_cores else FLAG_NO_TC))
    opt = _options(scheme, degree, dyadic, compute, flags)
    lib = load_library()
    nb = ctypes.c_size_t(0)
    _check(lib.sigkernel_tape_size(ctypes.byref(cX), ctypes.byref(cY), X.d, n, ctypes.byref(opt), ctypes.byref(nb)))
    if tape is None or _nbytes(tape) < nb.value:
        tape = torch.empty(int(nb.value), dtype=torch.uint8, device="cuda")
    _device_buffer(tape, "tape")
    if out is None:
        out = torch.empty((X.count, Y.count) if pair_a is None else (n,), dtype=torch.float64, device="cuda")
    _device_buffer(out, "out", torch.float64, X.count * Y.count if pair_a is None else n)
    ws = _device_buffer(workspace, "workspace") if workspace is not None else \
        _workspace(OP_GRAM if pair_a is None else OP_PAIRS, cX, cY, X.d, n, opt)
    _check(lib.sigkernel_forward_tape(ctypes.byref(cX), ctypes.byref(cY), X.d, _dtype_code(X, Y), pa_ptr, pb_ptr, n,
                                      ctypes.byref(opt), out.data_ptr(), tape.data_ptr(), _nbytes(tape), ws.data_ptr(),
                                      _nbytes(ws), _stream_ptr()))
    return out, tape


def sigkernel_backward_tape(tape, grad_out, X, Y=None, pair_a=None, pair_b=None, scheme="approx", degree=6, dyadic=0,
                            compute="f32", sort=True, time_kernel=False, tensor_cores: bool = True):
    """Gradients from a tape recorded by ``sigkernel_forward_tape`` with the same arguments
    (``tensor_cores=False``: the dk/dM contraction on the FMA pipe, SK_FLAG_NO_TC)."""
    sym = pair_a is None and (Y is None or Y is X)
    X = as_paths(X)
    Y = X if (Y is None or Y is X) else as_paths(Y)
    cX, cY = _cpaths(X), _cpaths(Y)
    pa_ptr, pb_ptr, n, keep = _pair_args(X, pair_a, pair_b, sym)
    flags = _flags(X, (FLAG_SYMMETRIC if sym else 0) | (0 if sort else FLAG_NO_SORT)
                   | (FLAG_TIME_KERNEL if time_kernel else 0) | (0 if tensor_cores else FLAG_NO_TC))
    opt = _options(scheme, degree, dyadic, compute, flags)
    g = _grad_out(grad_out, X.count, Y.count, n)
    _device_buffer(tape, "tape")
    gX = torch.zeros(X.rows.shape[0], X.d, dtype=torch.float64, device="cuda")
    same = X is Y or (X.rows.data_ptr() == Y.rows.data_ptr() and X.offsets.data_ptr() == Y.offsets.data_ptr())
    gY = gX if same else torch.zeros(Y.rows.shape[0], Y.d, dtype=torch.float64, device="cuda")
    ws = _workspace(OP_BACKWARD_TAPE, cX, cY, X.d, n, opt)
    _check(load_library().sigkernel_backward_tape(ctypes.byref(cX), ctypes.byref(cY), X.d, _dtype_code(X, Y), pa_ptr,
                                                  pb_ptr, n, ctypes.byref(opt), tape.data_ptr(), _nbytes(tape),
                                                  g.data_ptr(), gX.data_ptr(), None if same else gY.data_ptr(),
                                                  ws.data_ptr(), ws.numel(), _stream_ptr()))
    return gX, gY


def sigkernel_mmd2(A, B, scheme="approx", degree=6, dyadic=0, compute="f64", unbiased=False, grads=False,
                   tensor_cores: bool = True):
    """MMD^2 between path sets A and B; returns (mmd2, [mean K_AA, mean K_BB, mean K_AB]) or, with
    ``grads``, also (dMMD2/dA rows, dMMD2/dB rows) as float64 CUDA tensors."""
    A, B = as_paths(A), as_paths(B)
    cA, cB = _cpaths(A), _cpaths(B)
    opt = _options(scheme, degree, dyadic, compute, _flags(A, (FLAG_UNBIASED if unbiased else 0)
                                                           | (0 if tensor_cores else FLAG_NO_TC)))
    ws = _workspace(OP_MMD2, cA, cB, A.d, 1 if grads else 0, opt)
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    gA = torch.empty(A.rows.shape[0], A.d, dtype=torch.float64, device="cuda") if grads else None
    gB = torch.empty(B.rows.shape[0], B.d, dtype=torch.float64, device="cuda") if grads else None
    _check(load_library().sigkernel_mmd2(ctypes.byref(cA), ctypes.byref(cB), A.d, _dtype_code(A, B), ctypes.byref(opt),
                                         out.data_ptr(), gA.data_ptr() if grads else None,
                                         gB.data_ptr() if grads else None, ws.data_ptr(), ws.numel(), _stream_ptr()))
    if grads:
        return out[0], out[1:], gA, gB
    return out[0], out[1:]


def split_labels(nperm: int, na: int, nb: int, seed: int = 0) -> torch.Tensor:
    """[nperm, na + nb] uint8 CUDA tensor: row p marks with 1 the na pooled paths that a uniformly
    random relabelling assigns to the first sample (drawn on the host from a seeded generator)."""
    g = torch.Generator().manual_seed(int(seed))
    order = torch.argsort(torch.rand(int(nperm), na + nb, generator=g), dim=1)
    return (order < na).to(torch.uint8).to("cuda")


def sigkernel_mmd2_test(A, B, permutations=1000, labels=None, seed=0, scheme="approx", degree=6, dyadic=0,
                        compute="f64", unbiased=False, workspace=None, out=None):
    """Two-sample permutation test on MMD^2 between path sets A and B.

    ``labels`` ([nperm, |A| + |B|] uint8 CUDA tensor, nonzero = first sample) gives the
    relabellings of the pooled sample (A then B); without it ``permutations`` uniformly random
    ones are drawn from ``seed``.  Returns (MMD^2 of the split, p-value, MMD^2 of every
    relabelling) as float64 CUDA tensors; the p-value is (1 + #{stat >= observed}) / (1 + nperm).
    ``workspace`` / ``out`` may be preallocated (``mmd2_test_workspace``; out of 2 + nperm)."""
    A, B = as_paths(A), as_paths(B)
    if labels is None:
        labels = split_labels(permutations, A.count, B.count, seed)
    if labels.dtype != torch.uint8 or not labels.is_cuda or labels.dim() != 2:
        raise ValueError("labels must be a 2-d uint8 CUDA tensor")
    if labels.shape[1] != A.count + B.count:
        raise ValueError("labels must have |A| + |B| columns")
    labels = _device_buffer(labels.contiguous(), "labels", torch.uint8, labels.shape[0] * (A.count + B.count))
    nperm = labels.shape[0]
    cA, cB = _cpaths(A), _cpaths(B)
    opt = _options(scheme, degree, dyadic, compute, _flags(A, FLAG_UNBIASED if unbiased else 0))
    ws = _device_buffer(workspace, "workspace") if workspace is not None else \
        _workspace(OP_MMD2_TEST, cA, cB, A.d, nperm, opt)
    if out is None:
        out = torch.empty(2 + nperm, dtype=torch.float64, device="cuda")
    _device_buffer(out, "out", torch.float64, 2 + nperm)
    _check(load_library().sigkernel_mmd2_test(ctypes.byref(cA), ctypes.byref(cB), A.d, _dtype_code(A, B),
                                              ctypes.byref(opt), labels.data_ptr() if nperm else None, nperm,
                                              out.data_ptr(), ws.data_ptr(), _nbytes(ws), _stream_ptr()))
    return out[0], out[1], out[2:]


def mmd2_test_workspace(A, B, nperm, scheme="approx", degree=6, dyadic=0, compute="f64", unbiased=False):
    """Device workspace of ``sigkernel_mmd2_test`` for these sets and relabelling count."""
    A, B = as_paths(A), as_paths(B)
    opt = _options(scheme, degree, dyadic, compute, _flags(A, FLAG_UNBIASED if unbiased else 0))
    return _workspace(OP_MMD2_TEST, _cpaths(A), _cpaths(B), A.d, int(nperm), opt)


# ----------------------------------------------------------------------------------------------
# torch.autograd wrappers (dense [B, L, d] inputs)
# ----------------------------------------------------------------------------------------------
def tape_bytes(X, Y=None, pair_a=None, scheme="approx", degree=6, dyadic=0, compute="f32") -> int:
    """Bytes of the forward tape of these inputs (``sigkernel_tape_size``; Gram when ``pair_a`` is
    None, symmetric when Y is None or X)."""
    sym = pair_a is None and (Y is None or Y is X)
    X = as_paths(X)
    Y = X if (Y is None or Y is X) else as_paths(Y)
    n = -1 if pair_a is None else int(torch.as_tensor(pair_a).numel())
    opt = _options(scheme, degree, dyadic, compute, _flags(X, FLAG_SYMMETRIC if sym else 0))
    nb = ctypes.c_size_t(0)
    cX, cY = _cpaths(X), _cpaths(Y)
    _check(load_library().sigkernel_tape_size(ctypes.byref(cX), ctypes.byref(cY), X.d, n, ctypes.byref(opt),
                                              ctypes.byref(nb)))
    return int(nb.value)


# Largest tape the autograd wrapper keeps from forward to backward when left to choose (tape=None):
# at most this many bytes and at most half the device memory free at the forward.
AUTO_TAPE_MAX_BYTES = 128 << 30


class _GramFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, Y, sym, opts, use_tape):
        if use_tape is None:
            need = tape_bytes(X, None if sym else Y, **opts)
            free, _ = torch.cuda.mem_get_info()
            use_tape = need <= min(AUTO_TAPE_MAX_BYTES, free // 2)
        ctx.opts, ctx.sym, ctx.use_tape = opts, sym, use_tape
        ctx.save_for_backward(X, Y)
        if use_tape:
            G, ctx.tape = sigkernel_forward_tape(X, None if sym else Y, **opts)
            return G
        return sigkernel_gram(X, None if sym else Y, **opts)

    @staticmethod
    def backward(ctx, gG):
        X, Y = ctx.saved_tensors
        if ctx.use_tape:  # the tape stays with ctx (a retained graph may run backward again)
            gX, gY = sigkernel_backward_tape(ctx.tape, gG, X, None if ctx.sym else Y, **ctx.opts)
        else:
            gX, gY = sigkernel_backward(gG, X, None if ctx.sym else Y, **ctx.opts)
        if ctx.sym:
            return gX.view_as(X).to(X.dtype), None, None, None, None
        return gX.view_as(X).to(X.dtype), gY.view_as(Y).to(Y.dtype), None, None, None


class _MMD2Fn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, unbiased, opts):
        m, _, gA, gB = sigkernel_mmd2(A, B, unbiased=unbiased, grads=True, **opts)
        ctx.save_for_backward(gA.view_as(A), gB.view_as(B))
        return m

    @staticmethod
    def backward(ctx, gm):
        gA, gB = ctx.saved_tensors
        return (gm * gA).to(gA.dtype), (gm * gB).to(gB.dtype), None, None


class SigKernel:
    """Signature kernel k_hat of one scheme: ``gram`` and ``mmd2`` are differentiable with respect
    to dense [B, L, d] path tensors through the adjoint wavefront.  With ``tape=True`` the Gram's
    forward records a tape of every cell (2N+2 values per cell for the approximation scheme, 56 B
    at N = 6 in FP32) and the backward replays it instead of recomputing the forward sweep; with
    ``tape=False`` the backward is ``sigkernel_backward`` (which re-runs the forward in chunks).
    ``tape=None`` (default) records the tape when it takes at most ``AUTO_TAPE_MAX_BYTES`` and at
    most half the free device memory."""

    def __init__(self, scheme="approx", degree=6, dyadic=0, compute="f32", tape=None):
        self.opts = dict(scheme=scheme, degree=degree, dyadic=dyadic, compute=compute)
        self.tape = tape

    def gram(self, X: torch.Tensor, Y: torch.Tensor | None = None) -> torch.Tensor:
        sym = Y is None or Y is X
        return _GramFn.apply(X, X if sym else Y, sym, self.opts, self.tape)

    def mmd2(self, A: torch.Tensor, B: torch.Tensor, unbiased: bool = False) -> torch.Tensor:
        return _MMD2Fn.apply(A, B, unbiased, self.opts)


def last_kernel_ms() -> float:
    """Device milliseconds of the wavefront kernel of the last ``time_kernel=True`` call."""
    return float(load_library().sigkernel_last_kernel_ms())


def device_status() -> int:
    """Synchronise the current stream and return (and clear) the device error word."""
    return load_library().sigkernel_device_status(_stream_ptr())


def version() -> int:
    return load_library().sigkernel_version()


def fma_peak(compute="f32", packed=False, reps=5) -> float:
    """Measured FMA throughput of the current GPU in TFLOP/s (``sigkernel_fma_peak``)."""
    v = ctypes.c_double(0)
    _check(load_library().sigkernel_fma_peak(COMPUTE[compute], 1 if packed else 0, int(reps), ctypes.byref(v),
                                             _stream_ptr()))
    return float(v.value)


def set_wait_limit(polls: int = 0):
    """Polls a strip-pipeline hand-off wait makes before it reports SK_ERR_DEVICE_TIMEOUT
    (``sigkernel_set_wait_limit``; 0 restores the default)."""
    load_library().sigkernel_set_wait_limit(int(polls))
