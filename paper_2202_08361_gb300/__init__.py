"""GB300-native Jacobi SVD hot path (arXiv 2202.08361).

Python face of libjsvd.so (include/jsvd.h).  Functions carry the C-ABI
names without the `jsvd_` prefix and take torch CUDA tensors; torch is only
used for device memory and streams.
"""
import ctypes

from . import _native
from ._native import (JSVD_COMPLEX, JSVD_E_CUDA, JSVD_E_NONFINITE, JSVD_E_TIMEOUT,
                      JSVD_E_UNSUPPORTED, JSVD_E_WORKSPACE, JSVD_FP64, JSVD_MIXED_FP32_FP64,
                      JSVD_NOT_CONVERGED, JSVD_OK, JSVD_REAL, JSVD_TUNE_BATCH_SMEM,
                      JSVD_TUNE_EVD32_DIV, JSVD_TUNE_EVD_HOST, JSVD_TUNE_SVD_STEP,
                      JSVD_TUNE_SVD_SKIP,
                      JSVD_TUNE_BATCH_WARPS, JSVD_TUNE_EVD_ARITH, JSVD_TUNE_EVD_LAUNCH,
                      JSVD_TUNE_SVD_GRID, JsvdError)

__all__ = ["evd2x2_batched", "evd2x2_batched_host", "evd2x2_host_workspace_size", "svd",
           "svd_workspace_size", "colnorm_ef", "ordering", "decode_info", "dgemm", "zgemm", "BatchedSVD", "pack_matrices", "svd_batched", "svd_adjoint_batched",
           "sign_gauge_batched", "svd_diff", "version", "tune_set", "JsvdError", "JSVD_REAL",
           "JSVD_COMPLEX"]


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _vec(t, name, n=None, dtype=None, host=False):
    torch = _torch()
    dtype = dtype or torch.float64
    if not isinstance(t, torch.Tensor) or t.is_cuda == host:
        raise TypeError("%s must be a %s tensor" % (name, "CPU" if host else "CUDA"))
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
    """Batched 2x2 Hermitian EVD (jsvd_evd2x2_batched, or
    jsvd_evd2x2_batched_f32 for float32 streams).

    Real if a21_im is None.  Returns a dict of CUDA tensors: cos_phi,
    ea_tan_re (REAL: sign(a21) tan(phi)), ea_tan_im (COMPLEX only), lambda1,
    lambda2, zeta_p (int32 (zeta' << 1) | p).  `out` may supply them.
    """
    torch = _torch()
    cplx = a21_im is not None
    n = a11.numel()
    f32 = isinstance(a11, torch.Tensor) and a11.dtype == torch.float32
    dt = torch.float32 if f32 else torch.float64
    s = _native.EvdStreamsF32() if f32 else _native.EvdStreams()
    s.a11 = _vec(a11, "a11", n, dt)
    s.a22 = _vec(a22, "a22", n, dt)
    s.a21_re = _vec(a21_re, "a21_re", n, dt)
    s.a21_im = _vec(a21_im, "a21_im", n, dt) if cplx else None
    if out is None:
        dev = a11.device
        e = lambda t=dt: torch.empty(n, dtype=t, device=dev)
        out = {"cos_phi": e(), "ea_tan_re": e()}
        if cplx:
            out["ea_tan_im"] = e()
        if want_lambda:
            out["lambda1"] = e()
            out["lambda2"] = e()
        if want_zeta_p:
            out["zeta_p"] = e(torch.int32)
    s.cos_phi = _vec(out["cos_phi"], "cos_phi", n, dt)
    s.ea_tan_re = _vec(out["ea_tan_re"], "ea_tan_re", n, dt)
    s.ea_tan_im = _vec(out["ea_tan_im"], "ea_tan_im", n, dt) if cplx else None
    s.lambda1 = _vec(out["lambda1"], "lambda1", n, dt) if "lambda1" in out else None
    s.lambda2 = _vec(out["lambda2"], "lambda2", n, dt) if "lambda2" in out else None
    s.zeta_p = _vec(out["zeta_p"], "zeta_p", n, torch.int32) if "zeta_p" in out else None
    field = JSVD_COMPLEX if cplx else JSVD_REAL
    L = _native.lib()
    if f32:
        rc = L.jsvd_evd2x2_batched_f32(field, ctypes.byref(s), n, _stream_handle(stream))
    else:
        rc = L.jsvd_evd2x2_batched(field, ctypes.byref(s), n, _stream_handle(stream))
    _native.check(rc, "jsvd_evd2x2_batched_f32" if f32 else "jsvd_evd2x2_batched")
    return out


def evd2x2_host_workspace_size():
    sz = ctypes.c_size_t(0)
    _native.check(_native.lib().jsvd_evd2x2_host_workspace_size(ctypes.byref(sz)),
                  "jsvd_evd2x2_host_workspace_size")
    return sz.value


def evd2x2_batched_host(a11, a22, a21_re, a21_im=None, *, out=None, want_lambda=True,
                        want_zeta_p=True, work=None, device=None, stream=None):
    """Batched 2x2 Hermitian EVD of HOST streams (jsvd_evd2x2_batched_host):
    CPU tensors in and out, computed on the current CUDA device.  With every
    tensor pinned the kernel reads and writes them in place over the host
    link; otherwise they are staged in pipelined chunks.  Keep the tensors
    alive until `stream` has passed the call.
    Returns the output dict (CPU tensors; `out` may supply them, pinned
    ones are best).  Asynchronous on `stream`: synchronise before reading
    the outputs.  `work` is a device workspace (uint8, at least
    evd2x2_host_workspace_size() bytes), allocated if None."""
    torch = _torch()
    cplx = a21_im is not None
    n = a11.numel()
    s = _native.EvdStreams()
    s.a11 = _vec(a11, "a11", n, host=True)
    s.a22 = _vec(a22, "a22", n, host=True)
    s.a21_re = _vec(a21_re, "a21_re", n, host=True)
    s.a21_im = _vec(a21_im, "a21_im", n, host=True) if cplx else None
    if out is None:
        e = lambda dt=torch.float64: torch.empty(n, dtype=dt).pin_memory()
        out = {"cos_phi": e(), "ea_tan_re": e()}
        if cplx:
            out["ea_tan_im"] = e()
        if want_lambda:
            out["lambda1"] = e()
            out["lambda2"] = e()
        if want_zeta_p:
            out["zeta_p"] = e(torch.int32)
    s.cos_phi = _vec(out["cos_phi"], "cos_phi", n, host=True)
    s.ea_tan_re = _vec(out["ea_tan_re"], "ea_tan_re", n, host=True)
    s.ea_tan_im = _vec(out["ea_tan_im"], "ea_tan_im", n, host=True) if cplx else None
    s.lambda1 = _vec(out["lambda1"], "lambda1", n, host=True) if "lambda1" in out else None
    s.lambda2 = _vec(out["lambda2"], "lambda2", n, host=True) if "lambda2" in out else None
    s.zeta_p = (_vec(out["zeta_p"], "zeta_p", n, torch.int32, host=True) if "zeta_p" in out
                else None)
    need = evd2x2_host_workspace_size()
    if work is None:
        work = torch.empty(need, dtype=torch.uint8,
                           device=device if device is not None else torch.cuda.current_device())
    if not work.is_cuda or work.dtype != torch.uint8 or work.numel() < need:
        raise ValueError("work must be a CUDA uint8 tensor of at least %d bytes" % need)
    rc = _native.lib().jsvd_evd2x2_batched_host(JSVD_COMPLEX if cplx else JSVD_REAL,
                                                ctypes.byref(s), n, ctypes.c_void_p(work.data_ptr()),
                                                work.numel(), _stream_handle(stream))
    _native.check(rc, "jsvd_evd2x2_batched_host")
    return out


def colnorm_ef(A, stream=None):
    """Wide-exponent Frobenius norms of the columns of a CUDA matrix
    (jsvd_colnorm_ef, Alg. rnF): (e, f) float64 tensors with
    ||a_j|| = 2^e_j f_j, e_j = -inf for a zero column."""
    torch = _torch()
    if not isinstance(A, torch.Tensor) or not A.is_cuda or A.dim() != 2:
        raise TypeError("A must be a 2-D CUDA tensor")
    cplx = A.dtype == torch.complex128
    if not cplx and A.dtype != torch.float64:
        raise TypeError("A must be float64 or complex128")
    m, n = A.shape
    Ac, lda = colmajor(A)
    e = torch.empty(n, dtype=torch.float64, device=A.device)
    f = torch.empty(n, dtype=torch.float64, device=A.device)
    rc = _native.lib().jsvd_colnorm_ef(JSVD_COMPLEX if cplx else JSVD_REAL, m, n,
                                       ctypes.c_void_p(Ac.data_ptr()), lda,
                                       ctypes.c_void_p(e.data_ptr()),
                                       ctypes.c_void_p(f.data_ptr()), _stream_handle(stream))
    _native.check(rc, "jsvd_colnorm_ef")
    return e, f


# ---------------------------------------------------------------------------
# SVD

def _opts(max_sweeps=0, mode=JSVD_FP64, rescale_exp=0, permute=False, compensated=False):
    o = _native.Opts()
    o.compensated = 1 if compensated else 0
    o.max_sweeps = int(max_sweeps)
    o.mode = int(mode)
    o.rescale_exp = int(rescale_exp)
    o.permute = 1 if permute else 0
    return o


def _opts_ref(o):
    return ctypes.byref(o)


def _mode(mode):
    if mode in (JSVD_FP64, "fp64"):
        return JSVD_FP64
    if mode in (JSVD_MIXED_FP32_FP64, "mixed"):
        return JSVD_MIXED_FP32_FP64
    raise ValueError("mode must be 'fp64' or 'mixed'")


def colmajor(t):
    """A column-major view of a 2-D tensor (copying only if needed) and its
    leading dimension."""
    m, n = t.shape
    if t.stride(0) == 1 and t.stride(1) >= max(m, 1):
        return t, t.stride(1)
    c = t.t().contiguous().t()
    return c, max(m, 1)


def colmajor_empty(m, n, dtype, device):
    torch = _torch()
    return torch.empty((n, m), dtype=dtype, device=device).t()


def svd_workspace_size(m, n, complex_=False, mode="fp64"):
    sz = ctypes.c_size_t(0)
    o = _opts(mode=_mode(mode))
    rc = _native.lib().jsvd_svd_workspace_size(JSVD_COMPLEX if complex_ else JSVD_REAL,
                                               ctypes.byref(o), int(m), int(n), ctypes.byref(sz))
    _native.check(rc, "jsvd_svd_workspace_size")
    return sz.value


def decode_info(info):
    """jsvd_info tensor(s) (uint8, 32 bytes each, on any device) -> dict or
    list of dicts.  Synchronises with the device if info lives there."""
    import struct
    raw = bytes(info.detach().cpu().numpy().tobytes())
    out = []
    for k in range(len(raw) // _native.INFO_BYTES):
        st, sw, rot, resc, s32, gs, _ = struct.unpack_from("<iiqiiii", raw, k * _native.INFO_BYTES)
        out.append(dict(status=st, sweeps=sw, rotations=rot, rescales=resc, sweeps_fp32=s32,
                        gs_steps=gs))
    return out[0] if len(out) == 1 else out


def svd(A, *, max_sweeps=0, mode="fp64", rescale_exp=0, permute=False, compensated=False,
        work=None, out=None, stream=None):
    """One-sided Jacobi SVD of a CUDA tensor A (m x n, m >= n; float64 or
    complex128: jsvd_svd; float32 or complex64: jsvd_svd_f32, which returns
    U, sigma, V in single precision and no sigma_e / sigma_f).  Returns dict(U, sigma, sigma_e, sigma_f, V,
    info); U and V are column-major views, info a 32-byte device tensor
    (decode_info).  compensated forms the pivot pairs' dot-products by the
    compensated summation (Alg. zdpscl' / ddpscl')."""
    torch = _torch()
    if not isinstance(A, torch.Tensor) or not A.is_cuda or A.dim() != 2:
        raise TypeError("A must be a 2-D CUDA tensor")
    if A.dtype in (torch.float32, torch.complex64):
        return _svd_f32(A, max_sweeps=max_sweeps, permute=permute, work=work, out=out,
                        stream=stream)
    cplx = A.dtype == torch.complex128
    if not cplx and A.dtype != torch.float64:
        raise TypeError("A must be float64, complex128, float32 or complex64")
    m, n = A.shape
    Ac, lda = colmajor(A)
    dev = A.device
    if out is None:
        out = {"U": colmajor_empty(m, n, A.dtype, dev), "V": colmajor_empty(n, n, A.dtype, dev),
               "sigma": torch.empty(n, dtype=torch.float64, device=dev),
               "sigma_e": torch.empty(n, dtype=torch.float64, device=dev),
               "sigma_f": torch.empty(n, dtype=torch.float64, device=dev),
               "info": torch.zeros(_native.INFO_BYTES, dtype=torch.uint8, device=dev)}
    U, ldu = colmajor(out["U"])
    V, ldv = colmajor(out["V"])
    o = _opts(max_sweeps, _mode(mode), rescale_exp, permute, compensated)
    need = svd_workspace_size(m, n, cplx, mode)
    if work is None:
        work = torch.empty(need, dtype=torch.uint8, device=dev)
    ptr = lambda k: out[k].data_ptr() if out.get(k) is not None else None
    rc = _native.lib().jsvd_svd(JSVD_COMPLEX if cplx else JSVD_REAL, ctypes.byref(o), m, n,
                                Ac.data_ptr(), lda, U.data_ptr(), ldu, ptr("sigma"),
                                ptr("sigma_e"), ptr("sigma_f"), V.data_ptr(), ldv,
                                work.data_ptr(), work.numel(), ptr("info"),
                                _stream_handle(stream))
    _native.check(rc, "jsvd_svd")
    out["U"], out["V"] = U, V
    return out


def _svd_f32(A, *, max_sweeps=0, permute=False, work=None, out=None, stream=None):
    """The single precision SVD (jsvd_svd_f32): U, V float32/complex64,
    sigma float32, info."""
    torch = _torch()
    cplx = A.dtype == torch.complex64
    m, n = A.shape
    Ac, lda = colmajor(A)
    dev = A.device
    if out is None:
        out = {"U": colmajor_empty(m, n, A.dtype, dev), "V": colmajor_empty(n, n, A.dtype, dev),
               "sigma": torch.empty(n, dtype=torch.float32, device=dev),
               "info": torch.zeros(_native.INFO_BYTES, dtype=torch.uint8, device=dev)}
    U, ldu = colmajor(out["U"])
    V, ldv = colmajor(out["V"])
    o = _opts(max_sweeps, JSVD_FP64, 0, permute, False)
    field = JSVD_COMPLEX if cplx else JSVD_REAL
    L = _native.lib()
    sz = ctypes.c_size_t(0)
    _native.check(L.jsvd_svd_f32_workspace_size(field, ctypes.byref(o), m, n, ctypes.byref(sz)),
                  "jsvd_svd_f32_workspace_size")
    if work is None:
        work = torch.empty(sz.value, dtype=torch.uint8, device=dev)
    rc = L.jsvd_svd_f32(field, ctypes.byref(o), m, n, Ac.data_ptr(), lda, U.data_ptr(), ldu,
                        out["sigma"].data_ptr(), V.data_ptr(), ldv, work.data_ptr(), work.numel(),
                        out["info"].data_ptr() if out.get("info") is not None else None,
                        _stream_handle(stream))
    _native.check(rc, "jsvd_svd_f32")
    out["U"], out["V"] = U, V
    return out


def ordering(n, stream=None):
    """The device-side parallel pivot ordering as an int32 CUDA tensor
    [n_steps, n_pairs, 2]."""
    torch = _torch()
    nt = n + (n & 1)
    tab = torch.empty((nt - 1, nt // 2, 2), dtype=torch.int32, device="cuda")
    _native.check(_native.lib().jsvd_ordering(int(n), tab.data_ptr(), _stream_handle(stream)),
                  "jsvd_ordering")
    return tab


def probe_fp64_rate(kind, iters, blocks, sink, threads=256, stream=None):
    """Enqueue the FP64-pipe throughput probe (jsvd_probe_fp64_rate): kind 0
    fused multiply-add, 1 IEEE square root, 2 IEEE division; blocks x
    threads x 8 chains x iters operations.  sink: a float64 CUDA tensor of
    at least one element.  The caller times the launch."""
    _native.check(_native.lib().jsvd_probe_fp64_rate(int(kind), int(iters), int(blocks),
                                                     int(threads), sink.data_ptr(),
                                                     _stream_handle(stream)),
                  "jsvd_probe_fp64_rate")


def dgemm(A, B, *, transA=False, alpha=1.0, beta=0.0, C=None, stream=None):
    """C = alpha op(A) B + beta C (jsvd_dgemm) for float64 CUDA tensors, any
    layout (column-major copies are made when needed)."""
    torch = _torch()
    Ac, lda = colmajor(A)
    Bc, ldb = colmajor(B)
    M = A.shape[1] if transA else A.shape[0]
    K = A.shape[0] if transA else A.shape[1]
    N = B.shape[1]
    if B.shape[0] != K:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = colmajor_empty(M, N, torch.float64, A.device)
        beta = 0.0
    Cc, ldc = colmajor(C)
    if Cc.data_ptr() != C.data_ptr():
        raise ValueError("C must be column-major")
    rc = _native.lib().jsvd_dgemm(1 if transA else 0, M, N, K, float(alpha), Ac.data_ptr(), lda,
                                  Bc.data_ptr(), ldb, float(beta), Cc.data_ptr(), ldc,
                                  _stream_handle(stream))
    _native.check(rc, "jsvd_dgemm")
    return C


def zgemm(A, B=None, *, transA=False, herm=False, alpha=1.0, beta=0.0, C=None, stream=None):
    """C = alpha op(A) B + beta C (jsvd_zgemm, the 3M form on split planes)
    for complex128 CUDA tensors; op(A) = A^H when transA.  herm=True gives
    the Hermitian alpha A^H A (B must be None or A, beta 0).  Returns C as a
    complex128 tensor (a new one; C, when given, supplies the beta term)."""
    torch = _torch()
    if herm:
        if B is not None and B is not A:
            raise ValueError("herm=True computes A^H A: B must be None or A")
        if not transA or beta != 0.0:
            raise ValueError("herm=True needs transA=True and beta=0")
        B = A
    M = A.shape[1] if transA else A.shape[0]
    K = A.shape[0] if transA else A.shape[1]
    N = B.shape[1]
    if B.shape[0] != K:
        raise ValueError("inner dimensions differ")
    Ar, lda = colmajor(A.real.contiguous())
    Ai, _ = colmajor(A.imag.contiguous())
    if herm:
        Br, Bi, ldb = Ar, Ai, lda
    else:
        Br, ldb = colmajor(B.real.contiguous())
        Bi, _ = colmajor(B.imag.contiguous())
    Cr = colmajor_empty(M, N, torch.float64, A.device)
    Ci = colmajor_empty(M, N, torch.float64, A.device)
    if C is not None and beta != 0.0:
        Cr.copy_(C.real)
        Ci.copy_(C.imag)
    else:
        beta = 0.0
    rc = _native.lib().jsvd_zgemm(1 if transA else 0, 1 if herm else 0, M, N, K, float(alpha),
                                  Ar.data_ptr(), Ai.data_ptr(), lda, Br.data_ptr(), Bi.data_ptr(),
                                  ldb, float(beta), Cr.data_ptr(), Ci.data_ptr(), max(M, 1),
                                  _stream_handle(stream))
    _native.check(rc, "jsvd_zgemm")
    return torch.complex(Cr, Ci)


# ---------------------------------------------------------------------------
# batched SVD over packed buffers

class BatchedSVD:
    """A prepared jsvd_svd_batched over packed device buffers.

    A is a 1-D CUDA tensor (float64 or complex128) holding the matrices back
    to back, matrix i column-major with lda = m[i] at element offset
    sum_{j<i} m[j] n[j].  Results: U (packed like A), V (matrix i, n[i] x
    n[i], at sum_{j<i} n[j]^2), sigma (sum_{j<i} n[j]), sigma_e, sigma_f,
    info (count * 32 bytes).  The constructor runs jsvd_svd_batched_prepare;
    launch() enqueues the computation (it may be captured in a CUDA graph and
    replayed)."""

    def __init__(self, A, m, n, *, max_sweeps=0, permute=False, compensated=False, want_ef=True):
        import numpy as np
        torch = _torch()
        self.m = np.asarray(m, dtype=np.int64)
        self.n = np.asarray(n, dtype=np.int64)
        self.count = int(self.m.size)
        self.cplx = A.dtype == torch.complex128
        if not self.cplx and A.dtype != torch.float64:
            raise TypeError("A must be float64 or complex128")
        if not A.is_cuda or A.dim() != 1 or not A.is_contiguous():
            raise ValueError("A must be a contiguous 1-D CUDA tensor")
        mn = self.m * self.n
        self.offA = np.concatenate([[0], np.cumsum(mn)[:-1]]) if self.count else np.zeros(0, np.int64)
        self.offV = (np.concatenate([[0], np.cumsum(self.n * self.n)[:-1]]) if self.count
                     else np.zeros(0, np.int64))
        self.offS = np.concatenate([[0], np.cumsum(self.n)[:-1]]) if self.count else np.zeros(0, np.int64)
        if A.numel() < int(mn.sum()):
            raise ValueError("A is smaller than the packed matrices")
        dev = A.device
        self.A = A
        self.U = torch.empty_like(A)
        self.V = torch.empty(int((self.n * self.n).sum()), dtype=A.dtype, device=dev)
        ns = int(self.n.sum())
        self.sigma = torch.empty(ns, dtype=torch.float64, device=dev)
        self.sigma_e = torch.empty(ns, dtype=torch.float64, device=dev) if want_ef else None
        self.sigma_f = torch.empty(ns, dtype=torch.float64, device=dev) if want_ef else None
        self.info = torch.zeros(max(self.count, 1) * _native.INFO_BYTES, dtype=torch.uint8, device=dev)
        self.opts = _opts(max_sweeps, JSVD_FP64, 0, permute, compensated)
        es = 16 if self.cplx else 8
        cnt = self.count
        P = ctypes.c_void_p * max(cnt, 1)
        I64 = ctypes.c_int64 * max(cnt, 1)
        ptrs = lambda base, off, sz: P(*[base + int(o) * sz for o in off])
        self._m = I64(*self.m.tolist())
        self._n = I64(*self.n.tolist())
        self._A = ptrs(A.data_ptr(), self.offA, es)
        self._U = ptrs(self.U.data_ptr(), self.offA, es)
        self._V = ptrs(self.V.data_ptr(), self.offV, es)
        self._s = ptrs(self.sigma.data_ptr(), self.offS, 8)
        self._se = ptrs(self.sigma_e.data_ptr(), self.offS, 8) if want_ef else None
        self._sf = ptrs(self.sigma_f.data_ptr(), self.offS, 8) if want_ef else None
        self._lda = I64(*self.m.tolist())
        self._ldv = I64(*self.n.tolist())
        sz = ctypes.c_size_t(0)
        field = JSVD_COMPLEX if self.cplx else JSVD_REAL
        self.field = field
        L = _native.lib()
        _native.check(L.jsvd_svd_batched_workspace_size(field, ctypes.byref(self.opts), cnt,
                                                        self._m, self._n, ctypes.byref(sz)),
                      "jsvd_svd_batched_workspace_size")
        self.work = torch.empty(max(sz.value, 256), dtype=torch.uint8, device=dev)
        _native.check(L.jsvd_svd_batched_prepare(
            field, ctypes.byref(self.opts), cnt, self._m, self._n, self._A, self._lda, self._U,
            self._lda, self._s, self._se, self._sf, self._V, self._ldv, self.work.data_ptr(),
            self.work.numel(), _stream_handle(None)), "jsvd_svd_batched_prepare")

    warps = None  # warps per block; None: the library's choice for the batch

    def autotune(self, **kw):
        """Time the candidate warps per block on this batch, a couple of
        sweeps each (autotune.tune_batched), and launch with the fastest
        from now on.  Returns the {warps: ms} timings (empty when cached)."""
        from . import autotune
        self.warps, times = autotune.tune_batched(self, **kw)
        return times

    def launch(self, stream=None):
        L = _native.lib()
        if self.warps:
            tune_set(JSVD_TUNE_BATCH_WARPS, self.warps)
        try:
            rc = L.jsvd_svd_batched_launch(self.field, ctypes.byref(self.opts), self.count,
                                           self.work.data_ptr(), self.info.data_ptr(),
                                           _stream_handle(stream))
        finally:
            if self.warps:
                tune_set(JSVD_TUNE_BATCH_WARPS, 0)
        _native.check(rc, "jsvd_svd_batched_launch")
        return self

    def matrix(self, i):
        """(U_i, sigma_i, V_i) views of matrix i's results (column-major)."""
        m, n = int(self.m[i]), int(self.n[i])
        a, v, s = int(self.offA[i]), int(self.offV[i]), int(self.offS[i])
        U = self.U[a:a + m * n].view(n, m).t()
        V = self.V[v:v + n * n].view(n, n).t()
        return U, self.sigma[s:s + n], V


def pack_matrices(mats, device="cuda"):
    """Pack a list of 2-D arrays/tensors (m_i x n_i) column-major into one
    1-D CUDA tensor; returns (A, m, n)."""
    import numpy as np
    torch = _torch()
    ts = [torch.as_tensor(x) for x in mats]
    dtype = torch.complex128 if any(t.is_complex() for t in ts) else torch.float64
    m = np.array([t.shape[0] for t in ts], dtype=np.int64)
    n = np.array([t.shape[1] for t in ts], dtype=np.int64)
    flat = torch.cat([t.to(dtype).t().contiguous().reshape(-1) for t in ts]) if ts else \
        torch.empty(0, dtype=dtype)
    return flat.to(device), m, n


def svd_batched(mats, *, max_sweeps=0, permute=False, compensated=False, stream=None):
    """Batched SVD of a list of matrices (jsvd_svd_batched): returns the
    BatchedSVD after launching it."""
    A, m, n = pack_matrices(mats)
    return BatchedSVD(A, m, n, max_sweeps=max_sweeps, permute=permute,
                      compensated=compensated).launch(stream)


# ---------------------------------------------------------------------------
# differentiated batched SVD

def _packed_cm(t):
    """(count, r, c) tensor -> 1-D float64 CUDA tensor of the column-major
    matrices back to back."""
    return t.transpose(1, 2).contiguous().reshape(-1)


def sign_gauge_batched(U, V, count, m, n, stream=None):
    """In place on packed column-major U (count m n) and V (count n n):
    jsvd_sign_gauge_batched."""
    _native.check(_native.lib().jsvd_sign_gauge_batched(count, m, n, U.data_ptr(), V.data_ptr(),
                                                        _stream_handle(stream)),
                  "jsvd_sign_gauge_batched")


def svd_adjoint_batched(U, s, V, Ubar=None, sbar=None, Vbar=None, stream=None):
    """Abar for count real SVDs (jsvd_svd_adjoint_batched).  U, Ubar:
    (count, m, n); s, sbar: (count, n); V, Vbar: (count, n, n); float64 CUDA
    tensors.  Returns Abar (count, m, n)."""
    torch = _torch()
    count, m, n = U.shape
    Uc, Vc = _packed_cm(U), _packed_cm(V)
    sc = s.contiguous()
    Ubc = _packed_cm(Ubar) if Ubar is not None else None
    Vbc = _packed_cm(Vbar) if Vbar is not None else None
    sbc = sbar.contiguous() if sbar is not None else None
    Ab = torch.empty(count * m * n, dtype=torch.float64, device=U.device)
    p = lambda t: t.data_ptr() if t is not None else None
    rc = _native.lib().jsvd_svd_adjoint_batched(count, m, n, p(Uc), p(sc), p(Vc), p(Ubc), p(sbc),
                                                p(Vbc), Ab.data_ptr(), _stream_handle(stream))
    _native.check(rc, "jsvd_svd_adjoint_batched")
    return Ab.view(count, n, m).transpose(1, 2)


def _diff_svd_class():
    torch = _torch()

    class DifferentiableSVD(torch.autograd.Function):
        """Batched real SVD with a hand-written adjoint: forward is
        jsvd_svd_batched followed by the sign gauge, backward is
        jsvd_svd_adjoint_batched."""

        @staticmethod
        def forward(ctx, A):
            count, m, n = A.shape
            flat = _packed_cm(A.detach().to(torch.float64))
            B = BatchedSVD(flat, [m] * count, [n] * count, want_ef=False).launch()
            sign_gauge_batched(B.U, B.V, count, m, n)
            U = B.U.view(count, n, m).transpose(1, 2)
            S = B.sigma.view(count, n)
            V = B.V.view(count, n, n).transpose(1, 2)
            ctx.save_for_backward(U, S, V)
            ctx.batch = B
            return U, S, V

        @staticmethod
        def backward(ctx, gU, gS, gV):
            U, S, V = ctx.saved_tensors
            return svd_adjoint_batched(U, S, V, gU, gS, gV)

    return DifferentiableSVD


_DIFF = None


def svd_diff(A):
    """(U, S, V) of a (count, m, n) float64 CUDA tensor, differentiable
    through the hand-written adjoint kernel."""
    global _DIFF
    if _DIFF is None:
        _DIFF = _diff_svd_class()
    return _DIFF.apply(A)
