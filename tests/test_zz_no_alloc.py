"""GPU test of sigkernel_pairs_noalloc, the pairs entry point for callers that cannot allocate
device memory (it uses a fixed scratch array that the library holds on each device).

Two calls in a row with different inputs and compute modes must reproduce sigkernel_pairs (the
same kernels run, so the results agree to the parity tolerance used elsewhere: here bit for bit
is expected and 1e-12 relative is allowed); a call needing more scratch than the fixed array is
refused before anything runs.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes
import gc

import numpy as np
import pytest
import torch

from paper_2502_08470_gb300 import workloads as W

pytestmark = pytest.mark.gpu
sk = pytest.importorskip("paper_2502_08470_gb300.sigkernel")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = sk.load_library()
    PP, PO = ctypes.POINTER(sk._Paths), ctypes.POINTER(sk._Options)
    L.sigkernel_pairs_noalloc.restype = ctypes.c_int
    L.sigkernel_pairs_noalloc.argtypes = [PP, PP, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int64, PO, ctypes.c_void_p, ctypes.c_void_p]
    L.sigkernel_noalloc_capacity.restype = ctypes.c_size_t
    L.sigkernel_noalloc_last_error.restype = ctypes.c_char_p
    return L


def _ragged(seed, lengths, d):
    return [W.brownian(1, n, d, seed=seed + i)[0] for i, n in enumerate(lengths)]


def _noalloc(L, X, Y, pa, pb, scheme, degree, compute):
    cX, cY = sk._cpaths(X), sk._cpaths(Y)
    opt = sk._options(scheme, degree, 0, compute, 0)
    pa_t = torch.as_tensor(pa, dtype=torch.int64, device="cuda")
    pb_t = torch.as_tensor(pb, dtype=torch.int64, device="cuda")
    out = torch.full((len(pa),), float("nan"), dtype=torch.float64, device="cuda")
    # Python's cycle collector could free earlier tensors during the call and move the count
    # the other way; collect first and hold it off while measuring.
    gc.collect()
    gc.disable()
    try:
        before = torch.cuda.memory_allocated()
        rc = L.sigkernel_pairs_noalloc(ctypes.byref(cX), ctypes.byref(cY), X.d, sk.DTYPES[X.rows.dtype],
                                       pa_t.data_ptr(), pb_t.data_ptr(), len(pa), ctypes.byref(opt), out.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
        after = torch.cuda.memory_allocated()
    finally:
        gc.enable()
    assert after == before  # nothing came from torch's allocator either
    return rc, out


def test_noalloc_matches_pairs_on_two_calls_in_a_row(lib):
    cases = [
        (11, [40, 3, 97, 1, 66], [33, 70, 2], "approx", 6, "f32"),
        (23, [12, 130, 64, 65], [90, 31, 5, 8, 44], "interp", 5, "f64"),
    ]
    for seed, lx, ly, scheme, degree, compute in cases:
        Xs = _ragged(seed, lx, 3)
        Ys = _ragged(seed + 100, ly, 3)
        PX = sk.Paths.from_list([torch.tensor(x) for x in Xs])
        PY = sk.Paths.from_list([torch.tensor(y) for y in Ys])
        rng = np.random.default_rng(seed)
        pa = rng.integers(0, len(Xs), size=37)
        pb = rng.integers(0, len(Ys), size=37)
        ref = sk.sigkernel_pairs(PX, PY, pa, pb, scheme=scheme, degree=degree, compute=compute)
        rc, out = _noalloc(lib, PX, PY, pa, pb, scheme, degree, compute)
        assert rc == 0, lib.sigkernel_noalloc_last_error()
        torch.cuda.synchronize()
        assert sk.device_status() == 0
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.max(np.abs(o - r) / np.abs(r)) <= 1e-12


def test_noalloc_rejects_oversized_calls(lib):
    X = sk.Paths.from_list([torch.tensor(W.brownian(1, 10, 4, seed=5)[0])])
    X.max_len = 100000  # a bound this large needs far more hand-off scratch than the fixed array
    n = 4096
    rc, out = _noalloc(lib, X, X, np.zeros(n, dtype=np.int64), np.zeros(n, dtype=np.int64), "approx", 6, "f32")
    assert rc == -4
    msg = lib.sigkernel_noalloc_last_error().decode()
    assert str(lib.sigkernel_noalloc_capacity()) in msg
    torch.cuda.synchronize()
    assert torch.isnan(out).all()  # nothing ran
