"""GPU test of sigkernel_pairs_noalloc, the pairs entry point for callers that cannot allocate
device memory (it uses a fixed scratch array that the library holds on each device).

Two calls in a row with different inputs and compute modes must reproduce sigkernel_pairs (the
same kernels run, so the results agree to the parity tolerance used elsewhere: here bit for bit
is expected and 1e-12 relative is allowed); a call needing more scratch than the fixed array is
refused before anything runs.  "Allocates nothing" is checked on both allocators a call could
reach: torch's caching allocator, and the device's default stream-ordered memory pool, which
serves the library's own cudaMallocAsync (its high watermark must not rise during the call; a
sigkernel_pairs call without a workspace, which allocates from that pool, shows that the check
sees an allocation).  This file is collected last so that a run stopping at the first failure
has already run every other test.
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


CU_MEMPOOL_ATTR_USED_MEM_CURRENT, CU_MEMPOOL_ATTR_USED_MEM_HIGH = 7, 8  # CUmemPool_attribute (cuda.h)


class _DefaultPool:
    """The current device's default memory pool, read through the driver API."""

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def _get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def start(self):
        """Synchronise, reset the high watermark; returns the bytes in use."""
        torch.cuda.synchronize()
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, ctypes.byref(zero)) == 0
        return self._get(CU_MEMPOOL_ATTR_USED_MEM_CURRENT)

    def high(self):
        torch.cuda.synchronize()
        return self._get(CU_MEMPOOL_ATTR_USED_MEM_HIGH)


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
    pool = _DefaultPool()
    try:
        before = torch.cuda.memory_allocated()
        in_use = pool.start()
        rc = L.sigkernel_pairs_noalloc(ctypes.byref(cX), ctypes.byref(cY), X.d, sk.DTYPES[X.rows.dtype],
                                       pa_t.data_ptr(), pb_t.data_ptr(), len(pa), ctypes.byref(opt), out.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
        high = pool.high()
        after = torch.cuda.memory_allocated()
    finally:
        gc.enable()
    assert after == before  # nothing came from torch's allocator
    assert high <= in_use   # nor from the device's default pool (the library's own cudaMallocAsync)
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


def test_the_pool_check_sees_a_self_allocating_call(lib):
    """Positive control of the default-pool check: sigkernel_pairs with no workspace allocates its
    own from that pool (cudaMallocAsync), and the high watermark shows it."""
    X = sk.Paths.from_list([torch.tensor(x) for x in _ragged(7, [50, 60], 3)])
    cX = sk._cpaths(X)
    opt = sk._options("approx", 6, 0, "f32", 0)
    pa = torch.zeros(2, dtype=torch.int64, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    pool = _DefaultPool()
    in_use = pool.start()
    rc = sk.load_library().sigkernel_pairs(ctypes.byref(cX), ctypes.byref(cX), X.d, sk.DTYPES[X.rows.dtype],
                                           pa.data_ptr(), pa.data_ptr(), 2, ctypes.byref(opt), out.data_ptr(), None,
                                           0, torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    assert pool.high() > in_use
