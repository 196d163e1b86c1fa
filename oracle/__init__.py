"""The CPU oracle of the Jacobi SVD hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement of arXiv 2202.08361 in C (jsvd_oracle.c),
loaded through ctypes.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this package; the library under
paper_2202_08361_gb300/ never does.

Functions:
  dsjac2 / zsjac2     batched 2x2 EVD (section 2, Alg. d8jac2 / z8jac2)
  zsjac2_scaled       the scaled eigenvalues lambda' (Eq. e:lamsec)
  pairs               the round-robin parallel ordering (section 4.1 reading)
  vjsvd               one-sided Jacobi SVD after Alg. zvjsvd (section 4.3)
  svd_adjoint         thin real SVD adjoint (Townsend 2016)
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

OK = 0
E_ARG = -1
E_NONFINITE = -2
NOT_CONVERGED = 1

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    if _lib is None:
        # ORC_LIB: a library built by build.build_mutant, for the tests that
        # check that the pins catch a planted mistake (run in a subprocess)
        path = os.environ.get("ORC_LIB") or _build.build()
        L = ctypes.CDLL(path)
        L.orc_dsjac2.argtypes = [ctypes.c_int64, _d, _d, _d, _d, _d, _d, _d, _i32, ctypes.c_int]
        L.orc_dsjac2.restype = None
        L.orc_zsjac2.argtypes = [ctypes.c_int64, _d, _d, _d, _d, _d, _d, _d, _d, _d, _i32,
                                 ctypes.c_int]
        L.orc_zsjac2.restype = None
        L.orc_zsjac2_scaled.argtypes = [ctypes.c_int64, _d, _d, _d, _d, _d, _d]
        L.orc_zsjac2_scaled.restype = None
        _f = ctypes.POINTER(ctypes.c_float)
        L.orc_ssjac2.argtypes = [ctypes.c_int64, _f, _f, _f, _f, _f, _f, _f, _i32]
        L.orc_ssjac2.restype = None
        L.orc_csjac2.argtypes = [ctypes.c_int64, _f, _f, _f, _f, _f, _f, _f, _f, _f, _i32]
        L.orc_csjac2.restype = None
        L.orc_q_zsjac2.argtypes = [ctypes.c_int64, _d, _d, _d, _d, _d, _d, _d, _d, _d]
        L.orc_q_zsjac2.restype = None
        L.orc_q_vjsvd.argtypes = [ctypes.c_int64, ctypes.c_int64, _d, _d, ctypes.c_int64, _d, _d,
                                  _d, _d, _d, _d, ctypes.c_int, _i32]
        L.orc_q_vjsvd.restype = ctypes.c_int
        L.orc_rnF.argtypes = [ctypes.c_int64, _d, _d, _d]
        L.orc_rnF.restype = None
        L.orc_pairs.argtypes = [ctypes.c_int, _i32]
        L.orc_pairs.restype = ctypes.c_int
        L.orc_vjsvd.argtypes = [ctypes.c_int64, ctypes.c_int64, _d, _d, ctypes.c_int64, _d, _d,
                                _d, _d, _d, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int64, ctypes.c_int, _i32, _i64]
        L.orc_vjsvd.restype = ctypes.c_int
        L.orc_dpscl.argtypes = [ctypes.c_int64, _d, _d, _d, _d, ctypes.c_int, ctypes.c_double,
                                ctypes.c_int, ctypes.c_double, ctypes.c_int, _d]
        L.orc_dpscl.restype = ctypes.c_int
        L.orc_svd_adjoint.argtypes = [ctypes.c_int64, ctypes.c_int64, _d, _d, _d, _d, _d, _d, _d]
        L.orc_svd_adjoint.restype = ctypes.c_int
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_vjsvd_batch.argtypes = [ctypes.c_int64, _i64, _i64, _i64, _i64, _i64, _d, _d, _d,
                                      ctypes.c_int, ctypes.c_int, _i32]
        L.orc_vjsvd_batch.restype = ctypes.c_int
        L.orc_svd_adjoint_batch.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _d, _d,
                                            _d, _d, _d, _d, ctypes.c_int]
        L.orc_svd_adjoint_batch.restype = ctypes.c_int
        L.orc_omp_state.argtypes = [_i32]
        L.orc_omp_state.restype = None
        _lib = L
    return _lib


def num_threads():
    """OpenMP threads the oracle's parallel loops use."""
    return int(lib().orc_num_threads())


_BIND = {0: "false", 1: "true", 2: "primary", 3: "close", 4: "spread"}


def omp_state():
    """The OpenMP environment in force for the oracle's loops: dict(threads,
    proc_bind, places, dynamic)."""
    out = np.zeros(4, dtype=np.int32)
    lib().orc_omp_state(out.ctypes.data_as(_i32))
    return {"threads": int(out[0]), "proc_bind": _BIND.get(int(out[1]), str(int(out[1]))),
            "places": int(out[2]), "dynamic": bool(out[3])}


def _dp(a):
    return a.ctypes.data_as(_d) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def ssjac2(a11, a22, a21):
    """Single precision real EVD (binary32 constants of section 2.4):
    (cos phi, sign(a21) tan phi, lambda1, lambda2, zeta_p)."""
    a11, a22, a21 = _f32(a11), _f32(a22), _f32(a21)
    r = a11.size
    out = [np.empty(r, np.float32) for _ in range(4)]
    zp = np.empty(r, np.int32)
    lib().orc_ssjac2(r, _fp(a11), _fp(a22), _fp(a21), *[_fp(o) for o in out],
                     zp.ctypes.data_as(_i32))
    return (*out, zp)


def csjac2(a11, a22, a21r, a21i):
    """Single precision complex EVD: (cos phi, cos(alpha) tan phi,
    sin(alpha) tan phi, lambda1, lambda2, zeta_p)."""
    a11, a22, a21r, a21i = _f32(a11), _f32(a22), _f32(a21r), _f32(a21i)
    r = a11.size
    out = [np.empty(r, np.float32) for _ in range(5)]
    zp = np.empty(r, np.int32)
    lib().orc_csjac2(r, _fp(a11), _fp(a22), _fp(a21r), _fp(a21i), *[_fp(o) for o in out],
                     zp.ctypes.data_as(_i32))
    return (*out, zp)


def dsjac2(a11, a22, a21, nthreads=0):
    """Real symmetric 2x2 EVD of each (a11, a22, a21): returns
    (cos_phi, sign(a21) tan_phi, lambda1, lambda2, zeta_p).  nthreads > 0
    sets the OpenMP threads (else the default)."""
    a11, a22, a21 = _f64(a11), _f64(a22), _f64(a21)
    r = a11.size
    out = [np.empty(r) for _ in range(4)]
    zp = np.empty(r, dtype=np.int32)
    lib().orc_dsjac2(r, _dp(a11), _dp(a22), _dp(a21), *[_dp(o) for o in out],
                     zp.ctypes.data_as(_i32), int(nthreads))
    return (*out, zp)


def zsjac2(a11, a22, a21r, a21i, nthreads=0):
    """Complex Hermitian 2x2 EVD (section 2, Alg. z8jac2): returns (cos_phi,
    cos_alpha tan_phi, sin_alpha tan_phi, lambda1, lambda2, zeta_p)."""
    a11, a22, a21r, a21i = _f64(a11), _f64(a22), _f64(a21r), _f64(a21i)
    r = a11.size
    out = [np.empty(r) for _ in range(5)]
    zp = np.empty(r, dtype=np.int32)
    lib().orc_zsjac2(r, _dp(a11), _dp(a22), _dp(a21r), _dp(a21i), *[_dp(o) for o in out],
                     zp.ctypes.data_as(_i32), int(nthreads))
    return (*out, zp)


def zsjac2_scaled(a11, a22, a21r, a21i):
    """The scaled eigenvalues (lambda1', lambda2') of Eq. e:lamsec."""
    a11, a22, a21r, a21i = _f64(a11), _f64(a22), _f64(a21r), _f64(a21i)
    r = a11.size
    l1, l2 = np.empty(r), np.empty(r)
    lib().orc_zsjac2_scaled(r, _dp(a11), _dp(a22), _dp(a21r), _dp(a21i), _dp(l1), _dp(l2))
    return l1, l2


def pairs(n):
    """The round-robin ordering: int32 array [n_steps, n_pairs, 2] of (p, q)."""
    nt = n + (n & 1)
    K, L = max(nt - 1, 1), max(nt // 2, 1)
    tab = np.zeros((K, L, 2), dtype=np.int32)
    if nt >= 2:
        lib().orc_pairs(n, tab.ctypes.data_as(_i32))
    return tab[: nt - 1] if nt >= 2 else tab[:0]


def vjsvd(A, max_sweeps=100, nthreads=0, permute=False, compensated=False, skr_shift=0,
          max_steps=0):
    """One-sided Jacobi SVD of A (m x n, m >= n; real or complex).  permute
    applies the column swap P of section 2 during the sweeps; compensated
    forms the scaled dot-products by Alg. zdpscl' / ddpscl'; skr_shift > 0
    lowers the per-step rescaling threshold of section 3.2 (Eq. e:skr) by
    2^skr_shift, so that the rescaling branch runs (results unchanged);
    max_steps > 0 stops after that many parallel steps (for timing a bounded
    sample; status then NOT_CONVERGED).

    Returns dict(U, sigma, sigma_e, sigma_f, V, status, sweeps, rotations,
    rescales).  sigma is sorted non-increasingly; A ~= U diag(sigma) V^H.
    """
    A = np.asarray(A)
    m, n = A.shape
    cplx = np.iscomplexobj(A)
    Gr = np.asfortranarray(A.real, dtype=np.float64).copy(order="F")
    Gi = np.asfortranarray(A.imag, dtype=np.float64).copy(order="F") if cplx else None
    Vr = np.zeros((n, n), order="F")
    Vi = np.zeros((n, n), order="F") if cplx else None
    sig, se, sf = np.empty(n), np.empty(n), np.empty(n)
    info = np.zeros(5, dtype=np.int32)
    rot = np.zeros(1, dtype=np.int64)
    rc = lib().orc_vjsvd(m, n, _dp(Gr), _dp(Gi), m, _dp(Vr), _dp(Vi), _dp(sig), _dp(se),
                         _dp(sf), int(max_sweeps), 1 if permute else 0,
                         1 if compensated else 0, int(skr_shift), int(max_steps),
                         int(nthreads),
                         info.ctypes.data_as(_i32),
                         rot.ctypes.data_as(_i64))
    if rc < 0:
        raise ValueError("orc_vjsvd failed with %d" % rc)
    U = Gr + 1j * Gi if cplx else Gr
    V = Vr + 1j * Vi if cplx else Vr
    return dict(U=U, sigma=sig, sigma_e=se, sigma_f=sf,
                V=V, status=int(info[0]), sweeps=int(info[1]), rotations=int(rot[0]),
                rescales=int(info[3]), gs=int(info[4]))


def vjsvd_batch(mats, max_sweeps=100, nthreads=0):
    """Real SVDs of a list of matrices, the OpenMP threads sharing out the
    matrices (each matrix's SVD on one thread).  Returns (sigmas, Us, Vs,
    statuses), lists in the order of mats."""
    m = np.array([a.shape[0] for a in mats], dtype=np.int64)
    n = np.array([a.shape[1] for a in mats], dtype=np.int64)
    offA = np.concatenate([[0], np.cumsum(m * n)[:-1]]).astype(np.int64)
    offV = np.concatenate([[0], np.cumsum(n * n)[:-1]]).astype(np.int64)
    offS = np.concatenate([[0], np.cumsum(n)[:-1]]).astype(np.int64)
    G = np.concatenate([np.asarray(a, dtype=np.float64).ravel(order="F") for a in mats])
    V = np.zeros(int((n * n).sum()))
    sig = np.zeros(int(n.sum()))
    st = np.zeros(len(mats), dtype=np.int32)
    rc = lib().orc_vjsvd_batch(len(mats), m.ctypes.data_as(_i64), n.ctypes.data_as(_i64),
                               offA.ctypes.data_as(_i64), offV.ctypes.data_as(_i64),
                               offS.ctypes.data_as(_i64), _dp(G), _dp(V), _dp(sig),
                               int(max_sweeps), int(nthreads), st.ctypes.data_as(_i32))
    if rc != 0:
        raise ValueError("orc_vjsvd_batch failed with %d" % rc)
    sigmas = [sig[o:o + k] for o, k in zip(offS, n)]
    Us = [G[o:o + a * b].reshape(b, a).T for o, a, b in zip(offA, m, n)]
    Vs = [V[o:o + k * k].reshape(k, k).T for o, k in zip(offV, n)]
    return sigmas, Us, Vs, [int(x) for x in st]


def svd_adjoint_batch(U, s, V, Ubar, sbar, nthreads=0):
    """svd_adjoint for a batch of one shape: U, Ubar [count, m, n], V
    [count, n, n], s, sbar [count, n] (each matrix stored column-major,
    i.e. arrays indexed [i, row, col] are transposed per matrix here).
    Returns Abar [count, m, n]."""
    count, m, n = U.shape
    f = lambda X: np.ascontiguousarray(np.swapaxes(X, 1, 2), dtype=np.float64)  # column-major
    Uc, Vc, Ubc = f(U), f(V), f(Ubar)
    sc, sbc = _f64(s), _f64(sbar)
    Ab = np.zeros((count, n, m))
    rc = lib().orc_svd_adjoint_batch(count, m, n, _dp(Uc), _dp(sc), _dp(Vc), _dp(Ubc), _dp(sbc),
                                     _dp(Ab), int(nthreads))
    if rc != 0:
        raise ValueError("orc_svd_adjoint_batch failed with %d" % rc)
    return np.swapaxes(Ab, 1, 2)


def dpscl(q, p, compensated=False, eq=0, fq=1.0, ep=0, fp=1.0):
    """z = q^* p / (2^(eq + ep) fq fp) by Alg. zdpscl, or Alg. zdpscl' /
    ddpscl' (compensated); q, p real or complex vectors of one length.  The
    default norms make it the dot-product q^* p itself."""
    q = np.asarray(q)
    p = np.asarray(p)
    cplx = np.iscomplexobj(q) or np.iscomplexobj(p)
    qr, pr = _f64(q.real), _f64(p.real)
    qi = _f64(q.imag) if cplx else None
    pi = _f64(p.imag) if cplx else None
    out = np.zeros(2)
    rc = lib().orc_dpscl(len(qr), _dp(qr), _dp(qi), _dp(pr), _dp(pi), int(eq), float(fq), int(ep),
                         float(fp), 1 if compensated else 0, _dp(out))
    if rc != 0:
        raise ValueError("orc_dpscl failed with %d" % rc)
    return complex(out[0], out[1]) if cplx else out[0]


def q_zsjac2(a11, a22, a21r, a21i=None):
    """The binary128 twin of the 2x2 EVD (section 2, binary128 constants):
    (cos phi, Re e^{ia} tan phi, Im e^{ia} tan phi, lambda1, lambda2), each an
    (r, 2) array of (hi, lo) doubles with hi + lo the binary128 value."""
    a11, a22, a21r = _f64(a11), _f64(a22), _f64(a21r)
    a21i = _f64(a21i) if a21i is not None else None
    r = a11.size
    outs = [np.zeros(2 * r) for _ in range(5)]
    lib().orc_q_zsjac2(r, _dp(a11), _dp(a22), _dp(a21r), _dp(a21i), *[_dp(o) for o in outs])
    return tuple(o.reshape(r, 2) for o in outs)


def q_vjsvd(A, max_sweeps=100):
    """The binary128 twin of the one-sided Jacobi SVD (Alg. zvjsvd): dict(
    sigma (n, 2) (hi, lo) pairs, U, V rounded to double, status, sweeps)."""
    A = np.asarray(A)
    m, n = A.shape
    cplx = np.iscomplexobj(A)
    Ar = np.asfortranarray(A.real, dtype=np.float64)
    Ai = np.asfortranarray(A.imag, dtype=np.float64) if cplx else None
    sh, sl = np.zeros(n), np.zeros(n)
    Ur, Vr = np.zeros((m, n), order="F"), np.zeros((n, n), order="F")
    Ui = np.zeros((m, n), order="F") if cplx else None
    Vi = np.zeros((n, n), order="F") if cplx else None
    sw = np.zeros(1, dtype=np.int32)
    rc = lib().orc_q_vjsvd(m, n, _dp(Ar), _dp(Ai), m, _dp(sh), _dp(sl), _dp(Ur), _dp(Ui), _dp(Vr),
                           _dp(Vi), int(max_sweeps), sw.ctypes.data_as(_i32))
    if rc < 0:
        raise ValueError("orc_q_vjsvd failed with %d" % rc)
    U = Ur + 1j * Ui if cplx else Ur
    V = Vr + 1j * Vi if cplx else Vr
    return dict(sigma=np.stack([sh, sl], axis=1), U=U, V=V, status=int(rc), sweeps=int(sw[0]))


def rnF(x):
    """||x||_F as (e, f) = 2^e f by Alg. rnF with one lane: e an integral
    float (-inf for x = 0), f in [1, 2)."""
    x = _f64(x)
    e, f = np.zeros(1), np.zeros(1)
    lib().orc_rnF(x.size, _dp(x), _dp(e), _dp(f))
    return float(e[0]), float(f[0])


def svd_adjoint(U, s, V, Ubar, sbar, Vbar=None):
    """Abar from the thin real SVD adjoint (Townsend 2016)."""
    U = np.asfortranarray(U, dtype=np.float64)
    V = np.asfortranarray(V, dtype=np.float64)
    Ubar = np.asfortranarray(Ubar, dtype=np.float64)
    s = _f64(s)
    sbar = _f64(sbar)
    Vb = np.asfortranarray(Vbar, dtype=np.float64) if Vbar is not None else None
    m, n = U.shape
    Abar = np.zeros((m, n), order="F")
    rc = lib().orc_svd_adjoint(m, n, _dp(U), _dp(s), _dp(V), _dp(Ubar), _dp(sbar), _dp(Vb),
                               _dp(Abar))
    if rc != 0:
        raise ValueError("orc_svd_adjoint failed with %d" % rc)
    return Abar


def sign_gauge(U, V):
    """Flip each (u_j, v_j) so that the largest-magnitude entry of u_j is
    positive (first index on ties).  Real only."""
    U = U.copy()
    V = V.copy()
    idx = np.argmax(np.abs(U), axis=0)
    sg = np.sign(U[idx, np.arange(U.shape[1])])
    sg[sg == 0] = 1.0
    return U * sg, V * sg
