"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every entry point
declared in include/sigkernel.h; host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sigkernel.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2502_08470_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sigkernel_\w+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("sigkernel_pairs", "sigkernel_gram", "sigkernel_backward", "sigkernel_mmd2", "sigkernel_mmd2_test",
                     "sigkernel_workspace_size", "sigkernel_device_status", "sigkernel_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_binding():
    from paper_2502_08470_gb300 import sigkernel as sk
    assert ctypes.sizeof(sk._Options) == 32
    assert ctypes.sizeof(sk._Paths) == 40


def test_version_and_host_side_validation(lib):
    from paper_2502_08470_gb300 import sigkernel as sk
    lib.sigkernel_version.restype = ctypes.c_int
    assert lib.sigkernel_version() >= 100
    lib.sigkernel_workspace_size.restype = ctypes.c_int
    lib.sigkernel_last_error.restype = ctypes.c_char_p
    X = sk._Paths(0, 0, 0, 0, 0)
    n = ctypes.c_size_t(1)
    bad = sk._options("approx", 1)  # order N = 1 is below the Definition's N >= 2
    rc = lib.sigkernel_workspace_size(1, ctypes.byref(X), ctypes.byref(X), 2, ctypes.c_int64(-1), ctypes.byref(bad),
                                      ctypes.byref(n))
    assert rc == -1 and n.value == 0
    assert b"order" in lib.sigkernel_last_error()
    bad = sk._options("approx", 6, dyadic=12)
    assert lib.sigkernel_workspace_size(1, ctypes.byref(X), ctypes.byref(X), 2, ctypes.c_int64(-1),
                                        ctypes.byref(bad), ctypes.byref(n)) == -1
    bad = sk._options("approx", 6)
    assert lib.sigkernel_workspace_size(1, ctypes.byref(X), ctypes.byref(X), 0, ctypes.c_int64(-1),
                                        ctypes.byref(bad), ctypes.byref(n)) == -1
    assert b"d = 0" in lib.sigkernel_last_error()
    bad = sk._options("approx", 6, flags=sk.FLAG_STRIP_PIPELINE | sk.FLAG_NO_STRIP_PIPELINE)
    assert lib.sigkernel_workspace_size(1, ctypes.byref(X), ctypes.byref(X), 2, ctypes.c_int64(-1),
                                        ctypes.byref(bad), ctypes.byref(n)) == -1
    assert b"together" in lib.sigkernel_last_error()
    bad = sk._options("approx", 6, flags=1 << 20)
    assert lib.sigkernel_workspace_size(1, ctypes.byref(X), ctypes.byref(X), 2, ctypes.c_int64(-1),
                                        ctypes.byref(bad), ctypes.byref(n)) == -1
    assert b"unknown flag" in lib.sigkernel_last_error()
    bad = sk._options(max(sk.SCHEMES.values()) + 1, 6)
    assert lib.sigkernel_workspace_size(1, ctypes.byref(X), ctypes.byref(X), 2, ctypes.c_int64(-1),
                                        ctypes.byref(bad), ctypes.byref(n)) == -1
    assert b"unknown scheme" in lib.sigkernel_last_error()
    ok = sk._options("approx", 6)
    assert lib.sigkernel_workspace_size(sk.OP_MMD2_TEST, ctypes.byref(X), ctypes.byref(X), 2, ctypes.c_int64(-1),
                                        ctypes.byref(ok), ctypes.byref(n)) == -1
    assert b"nperm" in lib.sigkernel_last_error()
    # a call with invalid options returns before touching any device
    lib.sigkernel_gram.restype = ctypes.c_int
    bad = sk._options("interp", 20)
    rc = lib.sigkernel_gram(ctypes.byref(X), ctypes.byref(X), 2, 0, ctypes.byref(bad), None, None,
                            ctypes.c_size_t(0), None)
    assert rc == -1


def test_path_lengths_beyond_the_refined_bound_are_refused(lib):
    """(max_len << dyadic) above the bound is refused before any device call, also for a max_len
    so large that the shift itself would overflow."""
    from paper_2502_08470_gb300 import sigkernel as sk
    lib.sigkernel_workspace_size.restype = ctypes.c_int
    lib.sigkernel_last_error.restype = ctypes.c_char_p
    n = ctypes.c_size_t(1)
    ok = sk._Paths(0, 0, 0, 10, 0)
    for max_len, lam in ((131073, 0), (65537, 1), (513, 8), (1 << 62, 8), ((1 << 63) - 1, 1)):
        big = sk._Paths(0, 0, 0, max_len, 0)
        opt = sk._options("approx", 6, dyadic=lam)
        for X, Y in ((big, ok), (ok, big)):
            rc = lib.sigkernel_workspace_size(sk.OP_PAIRS, ctypes.byref(X), ctypes.byref(Y), 2, ctypes.c_int64(1),
                                              ctypes.byref(opt), ctypes.byref(n))
            assert rc == -2 and n.value == 0
            assert b"max_len" in lib.sigkernel_last_error()


def test_misaligned_device_pointers_are_refused(lib):
    """Rows misaligned for their element type, offsets, outputs, gradients or pair lists off 8
    bytes, and a tape off 256 bytes, are refused before any device work."""
    from paper_2502_08470_gb300 import sigkernel as sk
    lib.sigkernel_last_error.restype = ctypes.c_char_p
    for f in ("sigkernel_gram", "sigkernel_pairs", "sigkernel_backward", "sigkernel_backward_tape"):
        getattr(lib, f).restype = ctypes.c_int
    ok = sk._Paths(0x10000, 0x20000, 1, 10, 10)
    opt = sk._options("approx", 6)
    vp = ctypes.c_void_p
    cases = [
        (sk._Paths(0x10004, 0x20000, 1, 10, 10), ok, sk.DTYPES[torch.float64], vp(0x30000), b"X->rows is not 8"),
        (ok, sk._Paths(0x10002, 0x20000, 1, 10, 10), sk.DTYPES[torch.float32], vp(0x30000), b"Y->rows is not 4"),
        (sk._Paths(0x10001, 0x20000, 1, 10, 10), ok, sk.DTYPES[torch.bfloat16], vp(0x30000), b"X->rows is not 2"),
        (sk._Paths(0x10000, 0x20004, 1, 10, 10), ok, sk.DTYPES[torch.float64], vp(0x30000), b"X->offsets"),
        (ok, ok, sk.DTYPES[torch.float64], vp(0x30004), b"G is not 8"),
    ]
    for X, Y, dt, G, msg in cases:
        rc = lib.sigkernel_gram(ctypes.byref(X), ctypes.byref(Y), 2, dt, ctypes.byref(opt), G, None,
                                ctypes.c_size_t(0), None)
        assert rc == -1 and msg in lib.sigkernel_last_error(), (msg, lib.sigkernel_last_error())
    f64 = sk.DTYPES[torch.float64]
    rc = lib.sigkernel_pairs(ctypes.byref(ok), ctypes.byref(ok), 2, f64, vp(0x40000), vp(0x40004), ctypes.c_int64(1),
                             ctypes.byref(opt), vp(0x30000), None, ctypes.c_size_t(0), None)
    assert rc == -1 and b"pair_b is not 8" in lib.sigkernel_last_error()
    rc = lib.sigkernel_backward(ctypes.byref(ok), ctypes.byref(ok), 2, f64, None, None, ctypes.c_int64(-1),
                                ctypes.byref(opt), vp(0x30000), vp(0x50002), None, None, ctypes.c_size_t(0), None)
    assert rc == -1 and b"grad_X is not 8" in lib.sigkernel_last_error()
    rc = lib.sigkernel_backward_tape(ctypes.byref(ok), ctypes.byref(ok), 2, f64, None, None, ctypes.c_int64(-1),
                                     ctypes.byref(opt), vp(0x60010), ctypes.c_size_t(1 << 20), vp(0x30000),
                                     vp(0x50000), None, None, ctypes.c_size_t(0), None)
    assert rc == -1 and b"256-byte" in lib.sigkernel_last_error()


def _header_constants():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return {k: int(v) for k, v in re.findall(r"\b(SK_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}


def _header_struct_fields(name):
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", text).group(1)
    return re.findall(r"(\w+)\s*;", body)


def test_binding_constants_match_the_header():
    """Every code, scheme, mode, flag and op the binding passes has the header's value."""
    from paper_2502_08470_gb300 import sigkernel as sk
    h = _header_constants()
    assert {code: name for code, name in sk.ERRORS.items()} == {v: k for k, v in h.items() if k.startswith("SK_ERR_")}
    schemes = {"fd1": "SK_FD1", "fd2": "SK_FD2", "approx": "SK_POLY_APPROX", "interp": "SK_POLY_INTERP",
               "fd_implicit": "SK_FD_IMPLICIT"}
    assert {k: h[v] for k, v in schemes.items()} == sk.SCHEMES
    assert sk.COMPUTE == {"f64": h["SK_COMPUTE_F64"], "f32": h["SK_COMPUTE_F32"]}
    assert sorted(sk.DTYPES.values()) == sorted(h[k] for k in ("SK_F64", "SK_F32", "SK_BF16"))
    flags = {k[len("SK_FLAG_"):]: v for k, v in h.items() if k.startswith("SK_FLAG_")}
    assert flags == {k[len("FLAG_"):]: getattr(sk, k) for k in dir(sk) if k.startswith("FLAG_")}
    ops = {k[len("SK_OP_"):]: v for k, v in h.items() if k.startswith("SK_OP_")}
    assert ops == {k[len("OP_"):]: getattr(sk, k) for k in dir(sk) if k.startswith("OP_")}


def test_binding_structs_follow_the_header_field_order():
    from paper_2502_08470_gb300 import sigkernel as sk
    assert [f for f, _ in sk._Options._fields_] == _header_struct_fields("sk_options")
    assert [f for f, _ in sk._Paths._fields_] == _header_struct_fields("sk_paths")


def test_a_plain_c_caller_compiles_links_and_gets_argument_errors(lib, tmp_path):
    """The header is C99 and the library links into a C program: the program reads the version
    and gets SK_ERR_INVALID_ARG with a message for a bad order, with no device involved."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2502_08470_gb300 import build
    libdir = os.path.dirname(build.LIB)
    src = tmp_path / "caller.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "sigkernel.h"
int main(void) {
    sk_paths X;
    sk_options o;
    size_t bytes = 1;
    int rc;
    memset(&X, 0, sizeof X);
    memset(&o, 0, sizeof o);
    if (sigkernel_version() < 100) return 2;
    o.scheme = SK_POLY_APPROX;
    o.degree = 1;                      /* the schemes take N >= 2 */
    o.compute = SK_COMPUTE_F64;
    rc = sigkernel_workspace_size(SK_OP_PAIRS, &X, &X, 2, 1, &o, &bytes);
    if (rc != SK_ERR_INVALID_ARG || bytes != 0) return 3;
    if (strstr(sigkernel_last_error(), "order") == NULL) return 4;
    puts("ok");
    return 0;
}
""")
    exe = tmp_path / "caller"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-L", libdir, "-lsigkernel", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
