"""CPU checks of the Python binding's host-side marshalling (no library call, no GPU): ragged and
dense path sets become the ABI's rows + int64 offsets + max_len, options become sk_options with
the header's codes, and host tensors are refused before any pointer reaches the library."""
import pytest
import torch

from paper_2502_08470_gb300 import sigkernel as sk


def test_ragged_paths_become_rows_and_offsets():
    lens = [5, 1, 12, 3]
    paths = [torch.arange(L * 2, dtype=torch.float32).reshape(L, 2) + 100 * i for i, L in enumerate(lens)]
    P = sk.Paths.from_list(paths, device="cpu")
    assert P.count == 4 and P.d == 2 and P.max_len == 12
    assert P.offsets.dtype == torch.int64 and P.offsets.tolist() == [0, 5, 6, 18, 21]
    assert P.rows.dtype == torch.float32 and P.rows.shape == (21, 2) and P.rows.is_contiguous()
    for i, p in enumerate(paths):
        assert torch.equal(P.rows[P.offsets[i]:P.offsets[i + 1]], p)
    # an explicit dtype converts every path; an empty list gives no paths
    assert sk.Paths.from_list(paths, device="cpu", dtype=torch.float64).rows.dtype == torch.float64
    E = sk.Paths.from_list([], device="cpu")
    assert E.count == 0 and E.offsets.tolist() == [0] and E.max_len == 0


def test_dense_paths_and_as_paths():
    x = torch.randn(3, 7, 4, dtype=torch.float64)
    P = sk.as_paths(x)
    assert P.count == 3 and P.d == 4 and P.max_len == 7
    assert P.offsets.tolist() == [0, 7, 14, 21]
    assert torch.equal(P.rows.view(3, 7, 4), x)
    assert sk.as_paths(P) is P
    with pytest.raises(TypeError):
        sk.as_paths(torch.randn(7, 4))
    inc = sk.Paths.from_dense(x, increments=True)
    assert sk._flags(inc, sk.FLAG_SYMMETRIC) == sk.FLAG_SYMMETRIC | sk.FLAG_INCREMENTS
    assert sk._flags(P, sk.FLAG_NO_SORT) == sk.FLAG_NO_SORT


def test_options_carry_the_header_codes():
    o = sk._options("interp", 8, 2, "f32", flags=sk.FLAG_SYMMETRIC)
    assert (o.scheme, o.degree, o.dyadic, o.compute, o.interp_extra, o.flags, o.warps_per_block, o.reserved) == (
        sk.SCHEMES["interp"], 8, 2, sk.COMPUTE["f32"], 0, sk.FLAG_SYMMETRIC, 0, 0)
    assert sk._options(4, 2).scheme == sk.SCHEMES["fd_implicit"]  # integer codes pass through
    with pytest.raises(KeyError):
        sk._options("fd3")
    assert sk._pipe_flags(None) == 0
    assert sk._pipe_flags(True) == sk.FLAG_STRIP_PIPELINE
    assert sk._pipe_flags(False) == sk.FLAG_NO_STRIP_PIPELINE


def test_host_tensors_and_mixed_dtypes_are_refused():
    P = sk.Paths.from_list([torch.zeros(3, 2)], device="cpu")
    with pytest.raises(ValueError, match="CUDA"):
        sk._cpaths(P)
    A = sk.Paths.from_list([torch.zeros(3, 2, dtype=torch.float32)], device="cpu")
    B = sk.Paths.from_list([torch.zeros(3, 2, dtype=torch.float64)], device="cpu")
    with pytest.raises(ValueError, match="same dtype"):
        sk._dtype_code(A, B)
    assert sk._dtype_code(A, A) == sk.DTYPES[torch.float32]
    with pytest.raises(ValueError, match="float16"):
        sk._dtype_code(*(2 * [sk.Paths.from_list([torch.zeros(3, 2, dtype=torch.float16)], device="cpu")]))


def test_strided_or_misshapen_paths_are_refused():
    """The library reads rows [R][d] and offsets [B + 1] as dense arrays: a transposed or sliced
    view, or a tensor of the wrong rank, is refused before any pointer is taken."""
    rows = torch.zeros(2, 5, dtype=torch.float64)
    off = torch.tensor([0, 3, 5], dtype=torch.int64)
    with pytest.raises(ValueError, match="contiguous"):
        sk._cpaths(sk.Paths(rows.t(), off, 3))
    with pytest.raises(ValueError, match="contiguous"):
        sk._cpaths(sk.Paths(torch.zeros(5, 4)[:, ::2], off, 3))
    with pytest.raises(ValueError, match="contiguous"):
        sk._cpaths(sk.Paths(torch.zeros(5, 2), torch.arange(6, dtype=torch.int64)[::2], 3))
    with pytest.raises(ValueError, match=r"\[R, d\]"):
        sk._cpaths(sk.Paths(torch.zeros(5), off, 3))
    with pytest.raises(ValueError, match=r"\[R, d\]"):
        sk._cpaths(sk.Paths(torch.zeros(5, 2), off.reshape(1, 3), 3))
    # dense host tensors pass these checks and stop at the device check
    with pytest.raises(ValueError, match="CUDA"):
        sk._cpaths(sk.Paths(torch.zeros(5, 2), off, 3))


def test_buffers_passed_as_pointers_are_checked_before_use():
    """Outputs, workspaces, tapes, upstream gradients and pair lists reach the library as raw
    pointers whose sizes it cannot see: a wrong dtype, a wrong element count, a strided view, a
    short pair list or a mis-shaped upstream gradient is refused on the host."""
    out = torch.zeros(6, dtype=torch.float64)
    with pytest.raises(ValueError, match="float64"):
        sk._device_buffer(out.float(), "out", torch.float64, 6)
    with pytest.raises(ValueError, match="5 elements"):
        sk._device_buffer(out[:5], "out", torch.float64, 6)
    with pytest.raises(ValueError, match="contiguous"):
        sk._device_buffer(torch.zeros(12, dtype=torch.float64)[::2], "out", torch.float64, 6)
    with pytest.raises(ValueError, match="CUDA"):
        sk._device_buffer(out, "out", torch.float64, 6)
    assert sk._nbytes(torch.zeros(3, dtype=torch.float64)) == 24
    with pytest.raises(ValueError, match="one length"):
        sk._pair_tensors([0, 1, 2], [0, 1])
    with pytest.raises(ValueError, match="one length"):
        sk._pair_tensors([[0, 1]], [[0, 1]])
    with pytest.raises(ValueError, match=r"\[3, 2\]"):
        sk._grad_out(torch.zeros(2, 3), 3, 2, -1)       # transposed Gram weights
    with pytest.raises(ValueError, match=r"\[3, 2\]"):
        sk._grad_out(torch.zeros(5), 3, 2, -1)
    with pytest.raises(ValueError, match="one per pair"):
        sk._grad_out([1.0, 2.0], 3, 2, 3)


def test_a_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libsigkernel.so every call raises: there is no CPU or library fallback."""
    monkeypatch.setattr(sk, "_lib", None)
    monkeypatch.setattr(sk, "LIB_PATH", str(tmp_path / "libsigkernel.so"))
    with pytest.raises(RuntimeError, match="missing"):
        sk.load_library()
    with pytest.raises(RuntimeError, match="missing"):
        sk.version()
