"""GB300-native Jacobi SVD hot path (arXiv 2202.08361).

Python face of libjsvd.so (include/jsvd.h).  Functions carry the C-ABI
names without the `jsvd_` prefix and take torch CUDA tensors; torch is only
used for device memory and streams.
"""
import ctypes

from . import _native
from ._native import (JSVD_COMPLEX, JSVD_E_CUDA, JSVD_E_NONFINITE, JSVD_E_TIMEOUT,
                      JSVD_E_UNSUPPORTED, JSVD_E_WORKSPACE, JSVD_NOT_CONVERGED, JSVD_OK,
                      JSVD_REAL, JSVD_TUNE_EVD_LAUNCH, JsvdError)

__all__ = ["evd2x2_batched", "version", "tune_set", "JsvdError", "JSVD_REAL", "JSVD_COMPLEX"]


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _vec(t, name, n=None, dtype=None):
    torch = _torch()
    dtype = dtype or torch.float64
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s" % (name, dtype))
    if t.dim() != 1 or not t.is_contiguous():
        raise ValueError("%s must be a contiguous 1-D tensor" % name)
    if n is not None and t.numel() != n:
        raise ValueError("%s must have %d elements" % (name, n))
    return t.data_ptr()


def version():
    return _native.lib().jsvd_version()


def tune_set(knob, value, value2=0):
    return _native.check(_native.lib().jsvd_tune_set(int(knob), int(value), int(value2)),
                         "jsvd_tune_set")


def evd2x2_batched(a11, a22, a21_re, a21_im=None, *, out=None, want_lambda=True,
                   want_zeta_p=True, stream=None):
    """Batched 2x2 Hermitian EVD (jsvd_evd2x2_batched).

    Real if a21_im is None.  Returns a dict of CUDA tensors: cos_phi,
    ea_tan_re (REAL: sign(a21) tan(phi)), ea_tan_im (COMPLEX only), lambda1,
    lambda2, zeta_p (int32 (zeta' << 1) | p).  `out` may supply them.
    """
    torch = _torch()
    cplx = a21_im is not None
    n = a11.numel()
    s = _native.EvdStreams()
    s.a11 = _vec(a11, "a11", n)
    s.a22 = _vec(a22, "a22", n)
    s.a21_re = _vec(a21_re, "a21_re", n)
    s.a21_im = _vec(a21_im, "a21_im", n) if cplx else None
    if out is None:
        dev = a11.device
        e = lambda dt=torch.float64: torch.empty(n, dtype=dt, device=dev)
        out = {"cos_phi": e(), "ea_tan_re": e()}
        if cplx:
            out["ea_tan_im"] = e()
        if want_lambda:
            out["lambda1"] = e()
            out["lambda2"] = e()
        if want_zeta_p:
            out["zeta_p"] = e(torch.int32)
    s.cos_phi = _vec(out["cos_phi"], "cos_phi", n)
    s.ea_tan_re = _vec(out["ea_tan_re"], "ea_tan_re", n)
    s.ea_tan_im = _vec(out["ea_tan_im"], "ea_tan_im", n) if cplx else None
    s.lambda1 = _vec(out["lambda1"], "lambda1", n) if "lambda1" in out else None
    s.lambda2 = _vec(out["lambda2"], "lambda2", n) if "lambda2" in out else None
    s.zeta_p = _vec(out["zeta_p"], "zeta_p", n, torch.int32) if "zeta_p" in out else None
    rc = _native.lib().jsvd_evd2x2_batched(JSVD_COMPLEX if cplx else JSVD_REAL,
                                           ctypes.byref(s), n, _stream_handle(stream))
    _native.check(rc, "jsvd_evd2x2_batched")
    return out
