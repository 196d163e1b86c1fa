"""ctypes binding of libjsvd.so (include/jsvd.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library.  There is no CPU fallback; if the library has not
been built the first call raises.
"""
import ctypes
import os

from . import build as _build

JSVD_OK = 0
JSVD_E_CUDA = -100
JSVD_E_NONFINITE = -101
JSVD_E_TIMEOUT = -102
JSVD_E_WORKSPACE = -103
JSVD_E_UNSUPPORTED = -104
JSVD_NOT_CONVERGED = 1

JSVD_REAL = 0
JSVD_COMPLEX = 1

JSVD_TUNE_EVD_LAUNCH = 1
JSVD_TUNE_SVD_GRID = 2
JSVD_TUNE_BATCH_WARPS = 3
JSVD_TUNE_EVD_ARITH = 4
JSVD_TUNE_BATCH_SMEM = 5
JSVD_TUNE_EVD32_DIV = 6
JSVD_TUNE_EVD_HOST = 7
JSVD_TUNE_SVD_STEP = 8
JSVD_TUNE_SVD_SKIP = 9

JSVD_FP64 = 0
JSVD_MIXED_FP32_FP64 = 1


class JsvdError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        msg = "%s failed: %d (%s)" % (what, code, strerror(code))
        if code == JSVD_E_CUDA:
            msg += ": " + last_cuda_error()
        super().__init__(msg)


class EvdStreams(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in
                ("a11", "a22", "a21_re", "a21_im", "cos_phi", "ea_tan_re", "ea_tan_im",
                 "lambda1", "lambda2", "zeta_p")]


class EvdStreamsF32(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("a11", "a22", "a21_re", "a21_im", "cos_phi",
                                                "ea_tan_re", "ea_tan_im", "lambda1", "lambda2",
                                                "zeta_p")]


class Opts(ctypes.Structure):
    _fields_ = [("max_sweeps", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("rescale_exp", ctypes.c_int32), ("permute", ctypes.c_int32),
                ("compensated", ctypes.c_int32)]


# jsvd_info as laid out in device memory: int32 status, int32 sweeps,
# int64 rotations, int32 rescales, int32 sweeps_fp32, int32 gs_steps,
# int32 reserved (32 bytes)
INFO_BYTES = 32

# size of the static scratch of jsvd_svd_noalloc (JSVD_NOALLOC_SCRATCH_BYTES)
NOALLOC_SCRATCH_BYTES = 16 << 20


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


def lib():
    """The loaded library (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(
                "libjsvd.so is not built: run `python -c \"import __graft_entry__ as g; "
                "g.build()\"` (or python -m paper_2202_08361_gb300.build); there is no "
                "CPU fallback")
        L = ctypes.CDLL(_build.LIB)
        L.jsvd_version.restype = ctypes.c_int
        L.jsvd_strerror.argtypes = [ctypes.c_int]
        L.jsvd_strerror.restype = ctypes.c_char_p
        L.jsvd_last_cuda_error.restype = ctypes.c_char_p
        L.jsvd_tune_set.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.jsvd_tune_set.restype = ctypes.c_int
        L.jsvd_evd2x2_batched.argtypes = [ctypes.c_int, ctypes.POINTER(EvdStreams), _i64, _vp]
        L.jsvd_evd2x2_batched.restype = ctypes.c_int
        L.jsvd_evd2x2_batched_f32.argtypes = [ctypes.c_int, ctypes.POINTER(EvdStreamsF32), _i64,
                                              _vp]
        L.jsvd_evd2x2_batched_f32.restype = ctypes.c_int
        L.jsvd_colnorm_ef.argtypes = [ctypes.c_int, _i64, _i64, _vp, _i64, _vp, _vp, _vp]
        L.jsvd_colnorm_ef.restype = ctypes.c_int
        L.jsvd_evd2x2_host_workspace_size.argtypes = [ctypes.POINTER(ctypes.c_size_t)]
        L.jsvd_evd2x2_host_workspace_size.restype = ctypes.c_int
        L.jsvd_evd2x2_batched_host.argtypes = [ctypes.c_int, ctypes.POINTER(EvdStreams), _i64, _vp,
                                               ctypes.c_size_t, _vp]
        L.jsvd_evd2x2_batched_host.restype = ctypes.c_int
        _sz = ctypes.c_size_t
        L.jsvd_svd_workspace_size.argtypes = [ctypes.c_int, ctypes.POINTER(Opts), _i64, _i64,
                                              ctypes.POINTER(_sz)]
        L.jsvd_svd_workspace_size.restype = ctypes.c_int
        _d = ctypes.c_void_p
        L.jsvd_svd.argtypes = [ctypes.c_int, ctypes.POINTER(Opts), _i64, _i64, _vp, _i64, _vp, _i64,
                               _d, _d, _d, _vp, _i64, _vp, _sz, _vp, _vp]
        L.jsvd_svd.restype = ctypes.c_int
        L.jsvd_svd_f32_workspace_size.argtypes = [ctypes.c_int, ctypes.POINTER(Opts), _i64, _i64,
                                                  ctypes.POINTER(_sz)]
        L.jsvd_svd_f32_workspace_size.restype = ctypes.c_int
        L.jsvd_svd_f32.argtypes = [ctypes.c_int, ctypes.POINTER(Opts), _i64, _i64, _vp, _i64, _vp,
                                   _i64, _vp, _vp, _i64, _vp, _sz, _vp, _vp]
        L.jsvd_svd_f32.restype = ctypes.c_int
        L.jsvd_svd_noalloc.argtypes = [ctypes.c_int, ctypes.POINTER(Opts), _i64, _i64, _vp, _i64,
                                       _vp, _i64, _d, _d, _d, _vp, _i64, _vp, _vp]
        L.jsvd_svd_noalloc.restype = ctypes.c_int
        L.jsvd_dgemm.argtypes = [ctypes.c_int, _i64, _i64, _i64, ctypes.c_double, _vp, _i64, _vp,
                                 _i64, ctypes.c_double, _vp, _i64, _vp]
        L.jsvd_dgemm.restype = ctypes.c_int
        L.jsvd_zgemm.argtypes = [ctypes.c_int, ctypes.c_int, _i64, _i64, _i64, ctypes.c_double,
                                 _vp, _vp, _i64, _vp, _vp, _i64, ctypes.c_double, _vp, _vp, _i64,
                                 _vp]
        L.jsvd_zgemm.restype = ctypes.c_int
        _pi64 = ctypes.POINTER(ctypes.c_int64)
        _pvp = ctypes.POINTER(ctypes.c_void_p)
        L.jsvd_svd_batched_workspace_size.argtypes = [ctypes.c_int, ctypes.POINTER(Opts), _i64,
                                                      _pi64, _pi64, ctypes.POINTER(_sz)]
        L.jsvd_svd_batched_workspace_size.restype = ctypes.c_int
        L.jsvd_svd_batched_prepare.argtypes = [ctypes.c_int, ctypes.POINTER(Opts), _i64, _pi64,
                                               _pi64, _pvp, _pi64, _pvp, _pi64, _pvp, _pvp, _pvp,
                                               _pvp, _pi64, _vp, _sz, _vp]
        L.jsvd_svd_batched_prepare.restype = ctypes.c_int
        L.jsvd_svd_batched_launch.argtypes = [ctypes.c_int, ctypes.POINTER(Opts), _i64, _vp, _vp,
                                              _vp]
        L.jsvd_svd_batched_launch.restype = ctypes.c_int
        L.jsvd_svd_adjoint_batched.argtypes = [_i64, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                               _vp]
        L.jsvd_svd_adjoint_batched.restype = ctypes.c_int
        L.jsvd_sign_gauge_batched.argtypes = [_i64, _i64, _i64, _vp, _vp, _vp]
        L.jsvd_sign_gauge_batched.restype = ctypes.c_int
        L.jsvd_selftest_fp64.argtypes = [_i64, ctypes.c_uint64, _vp, _vp]
        L.jsvd_selftest_fp64.restype = ctypes.c_int
        L.jsvd_selftest_fp32div.argtypes = [_i64, ctypes.c_uint64, _vp, _vp]
        L.jsvd_selftest_fp32div.restype = ctypes.c_int
        L.jsvd_selftest_barrier.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64, _vp,
                                            _vp]
        L.jsvd_selftest_barrier.restype = ctypes.c_int
        L.jsvd_probe_fp64_rate.argtypes = [ctypes.c_int, _i64, ctypes.c_int, ctypes.c_int, _vp,
                                           _vp]
        L.jsvd_probe_fp64_rate.restype = ctypes.c_int
        L.jsvd_ordering.argtypes = [ctypes.c_int32, _vp, _vp]
        L.jsvd_ordering.restype = ctypes.c_int
        _lib = L
    return _lib


def strerror(code):
    return lib().jsvd_strerror(int(code)).decode()


def last_cuda_error():
    return lib().jsvd_last_cuda_error().decode()


def check(rc, what):
    if rc != JSVD_OK:
        raise JsvdError(rc, what)
    return rc
