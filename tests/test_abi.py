"""The C-ABI library loads and exports every symbol include/*.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        for m in re.finditer(r"JSVD_API\s+[^;(]*?\b(jsvd_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2202_08361_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_symbols()
    for required in ("jsvd_evd2x2_batched", "jsvd_version", "jsvd_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    lib.jsvd_version.restype = ctypes.c_int
    assert lib.jsvd_version() >= 100
    lib.jsvd_strerror.restype = ctypes.c_char_p
    lib.jsvd_strerror.argtypes = [ctypes.c_int]
    assert lib.jsvd_strerror(0) == b"success"
    assert b"invalid" in lib.jsvd_strerror(-3)


def test_argument_errors_need_no_gpu(lib):
    """Argument checks return -i before anything touches the device."""
    from paper_2202_08361_gb300 import _native
    L = _native.lib()
    s = _native.EvdStreams()
    assert L.jsvd_evd2x2_batched(7, ctypes.byref(s), 10, None) == -1
    assert L.jsvd_evd2x2_batched(0, None, 10, None) == -2
    assert L.jsvd_evd2x2_batched(0, ctypes.byref(s), 10, None) == -2
    assert L.jsvd_evd2x2_batched(0, ctypes.byref(s), 0, None) == 0  # n = 0: no-op
    s.a11 = s.a22 = s.a21_re = s.cos_phi = s.ea_tan_re = 8
    assert L.jsvd_evd2x2_batched(0, ctypes.byref(s), -1, None) == -3
    assert L.jsvd_evd2x2_batched(1, ctypes.byref(s), 10, None) == -2  # complex needs a21_im
    assert L.jsvd_evd2x2_batched(0, ctypes.byref(s), 0, None) == 0  # n = 0: no-op
    # the host-buffer EVD checks its arguments before touching the device
    sz = ctypes.c_size_t(0)
    assert L.jsvd_evd2x2_host_workspace_size(ctypes.byref(sz)) == 0 and sz.value > 0
    h = _native.EvdStreams()
    assert L.jsvd_evd2x2_batched_host(7, ctypes.byref(h), 10, None, 0, None) == -1
    assert L.jsvd_evd2x2_batched_host(0, None, 10, None, 0, None) == -2
    assert L.jsvd_evd2x2_batched_host(0, ctypes.byref(h), 10, None, 0, None) == -2
    assert L.jsvd_evd2x2_batched_host(0, ctypes.byref(h), 0, None, 0, None) == 0
    h.a11 = h.a22 = h.a21_re = h.cos_phi = h.ea_tan_re = 8
    assert L.jsvd_evd2x2_batched_host(0, ctypes.byref(h), -1, None, 0, None) == -3
    assert L.jsvd_evd2x2_batched_host(0, ctypes.byref(h), 10, None, 0, None) == -4
    assert L.jsvd_evd2x2_batched_host(0, ctypes.byref(h), 10, 256, 0, None) == _native.JSVD_E_WORKSPACE
    assert L.jsvd_tune_set(99, 0, 0) == -1
    assert L.jsvd_tune_set(1, 100, 8) == -2
    assert L.jsvd_tune_set(1, 256, 0) == -3
    assert L.jsvd_tune_set(4, 8, 0) == -2           # placements are 0..7
    assert L.jsvd_tune_set(4, -2, 0) == -2
    assert L.jsvd_tune_set(4, 1, 3) == -3           # fields: 0, 1 or 2
    assert L.jsvd_tune_set(4, 1, 2) == 0
    assert L.jsvd_tune_set(4, -1, 0) == 0           # back to the defaults
    assert L.jsvd_tune_set(_native.JSVD_TUNE_EVD_HOST, 2, 0) == -2
    assert L.jsvd_tune_set(_native.JSVD_TUNE_EVD_HOST, 1, 0) == 0
    assert L.jsvd_tune_set(_native.JSVD_TUNE_EVD_HOST, 0, 0) == 0
    assert L.jsvd_tune_set(_native.JSVD_TUNE_EVD32_DIV, 8, 0) == -2   # placements 0..7
    assert L.jsvd_tune_set(_native.JSVD_TUNE_EVD32_DIV, 1, 3) == -3   # fields 0..2
    assert L.jsvd_tune_set(_native.JSVD_TUNE_EVD32_DIV, -1, 0) == 0
    assert L.jsvd_tune_set(_native.JSVD_TUNE_SVD_STEP, 6, 0) == -2
    assert L.jsvd_tune_set(_native.JSVD_TUNE_SVD_SKIP, 2, 0) == -2
    assert L.jsvd_tune_set(_native.JSVD_TUNE_SVD_SKIP, 1, 0) == 0
    assert L.jsvd_tune_set(_native.JSVD_TUNE_SVD_STEP, 0, 0) == 0
    # the complex 3M product: argument checks come before any CUDA call
    d = ctypes.c_void_p(16)  # never dereferenced: every call below fails its checks
    z = L.jsvd_zgemm
    assert z(2, 0, 4, 4, 4, 1.0, d, d, 4, d, d, 4, 0.0, d, d, 4, None) == -1
    assert z(0, 2, 4, 4, 4, 1.0, d, d, 4, d, d, 4, 0.0, d, d, 4, None) == -2
    assert z(0, 1, 4, 4, 4, 1.0, d, d, 4, d, d, 4, 0.0, d, d, 4, None) == -2  # herm needs A^H
    assert z(1, 1, 4, 5, 4, 1.0, d, d, 4, d, d, 4, 0.0, d, d, 4, None) == -4  # herm needs N = M
    assert z(0, 0, -1, 4, 4, 1.0, d, d, 4, d, d, 4, 0.0, d, d, 4, None) == -3
    assert z(0, 0, 4, 4, 4, 1.0, None, d, 4, d, d, 4, 0.0, d, d, 4, None) == -7
    assert z(0, 0, 4, 4, 4, 1.0, d, None, 4, d, d, 4, 0.0, d, d, 4, None) == -8
    assert z(0, 0, 8, 4, 4, 1.0, d, d, 4, d, d, 4, 0.0, d, d, 8, None) == -9   # lda < M
    assert z(0, 0, 4, 4, 4, 1.0, d, d, 4, d, None, 4, 0.0, d, d, 4, None) == -11
    e = ctypes.c_void_p(32)
    assert z(1, 1, 4, 4, 4, 1.0, d, d, 4, e, d, 4, 0.0, d, d, 4, None) == -10  # herm: B = A
    assert z(1, 1, 4, 4, 4, 1.0, d, d, 4, d, d, 4, 0.5, d, d, 4, None) == -13  # herm: beta = 0
    assert z(0, 0, 4, 4, 4, 1.0, d, d, 4, d, d, 4, 0.0, d, None, 4, None) == -15
    assert z(0, 0, 4, 4, 4, 1.0, d, d, 4, d, d, 4, 0.0, d, d, 3, None) == -16


def test_plain_c_user_compiles_and_runs(tmp_path):
    """include/jsvd.h is a C header: a C99 program compiled with -pedantic
    -Werror links libjsvd.so and gets the documented answers from the
    host-side entry points (no GPU needed)."""
    import subprocess
    from paper_2202_08361_gb300 import build
    lib = build.build()
    exe = str(tmp_path / "c_abi_user")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I" + os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "native", "c_abi_user.c"), "-o", exe,
                    lib, "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    out = dict(line.split(" ", 1) for line in
               subprocess.run([exe], check=True, capture_output=True, text=True).stdout.splitlines())
    rc, size = out["svd_ws"].split()
    assert rc == "0" and int(size) > 4096 * 2048 * 16
    assert out["svd_ws_bad_n"] == "-4"
    assert out["svd_ws_bad_opts"] == "-2"
    assert out["host_ws"].split()[0] == "0" and int(out["host_ws"].split()[1]) > 0
    assert out["evd_missing_stream"] == "-2"
    assert out["evd_empty"] == "0"
    assert out["tune_bad"] == "-2" and out["tune_ok"] == "0"
    assert "workspace" in out["message"]

