"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method itself: it only draws the
matrices that the library, the tests and the benchmark feed in.  The same
generators serve the CUDA path and the CPU oracle.

Seeds: numpy.random.Generator(PCG64(20220217 + workload_id)), so a workload
is the same on every machine.

Workloads (ids):
  1  real 256 x 128 matrix, i.i.d. N(0, 1)                     (one SVD)
  2  2x2 EVD batches: 2^24 real + 2^24 complex, entries
     sign * (1 + u) * 2^e, u ~ U[0,1), e ~ U{-1074..1023}, 1 % exact zeros
  3  complex 4096 x 2048, A = Q1 diag(s) Q2^H, Haar Q1, Q2, s geometric
     from 1 to 1e-6
  4  10,000 real matrices, n ~ U{16..256}, m ~ U{n..2n}, s geometric with
     condition 1e4, random orthogonal factors
  5  4096 real 64 x 32 matrices, s geometric with condition 1e3,
     w ~ U[0,1)^32, C ~ N(0,1)^(64 x 8) per matrix
"""
import numpy as np

BASE_SEED = 20220217


def rng(workload_id: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + workload_id + 1000 * salt))


# ---------------------------------------------------------------------------
# 2x2 EVD inputs (workload 2)

def wide_range_values(g: np.random.Generator, r: int, zero_frac: float = 0.01) -> np.ndarray:
    """sign * (1 + u) * 2^e with e uniform in [-1074, 1023] (ldexp rounds the
    subnormal ones), sign +-1 equiprobable, each entry exactly 0 w.p. zero_frac."""
    u = g.random(r)
    e = g.integers(-1074, 1024, size=r)
    s = np.where(g.random(r) < 0.5, -1.0, 1.0)
    x = np.ldexp(1.0 + u, e) * s
    x[g.random(r) < zero_frac] = 0.0
    return x


def evd_batch(r: int, complex_: bool, seed_salt: int = 0):
    """SoA streams (a11, a22, a21_re[, a21_im]) of r Hermitian 2x2 matrices."""
    g = rng(2, seed_salt + (1 if complex_ else 0))
    a11 = wide_range_values(g, r)
    a22 = wide_range_values(g, r)
    a21r = wide_range_values(g, r)
    if complex_:
        a21i = wide_range_values(g, r)
        return a11, a22, a21r, a21i
    return a11, a22, a21r


def wide_range_values_f32(g, r, zero_frac=0.01):
    """The binary32 form of wide_range_values: sign * (1 + k 2^-23) * 2^e,
    k ~ U{0..2^23-1}, e ~ U{-149..127} (values below 2^-126 rounded to the
    subnormal grid), each entry exactly 0 with probability zero_frac."""
    k = g.integers(0, 1 << 23, size=r)
    e = g.integers(-149, 128, size=r)
    s = np.where(g.random(r) < 0.5, -1.0, 1.0)
    v = (s * np.ldexp(1.0 + np.ldexp(k.astype(np.float64), -23), e)).astype(np.float32)
    v[g.random(r) < zero_frac] = 0.0
    return v


def evd_batch_f32(r: int, complex_: bool, seed_salt: int = 0):
    """Single precision SoA streams of r Hermitian 2x2 matrices (the binary32
    counterpart of evd_batch)."""
    g = rng(2, 20 + seed_salt + (1 if complex_ else 0))
    cols = [wide_range_values_f32(g, r) for _ in range(4 if complex_ else 3)]
    return tuple(cols)


def evd_prescribed(r: int, complex_: bool, seed_salt: int = 0):
    """Matrices built from prescribed eigenvalues, tan(phi) and cos(alpha)
    as in the paper's EVD test data (Eq. e:2, section 5.1), in FP64 here:
    |lambda_j| <= nu/16 reinterpreted from random bits, tan(phi), cos(alpha)
    uniform in [-1, 1)."""
    g = rng(2, 10 + seed_salt + (1 if complex_ else 0))

    def lam():
        out = np.empty(r)
        filled = 0
        while filled < r:
            bits = g.integers(0, 2**63, size=2 * (r - filled), dtype=np.int64)
            bits ^= g.integers(0, 2, size=bits.size, dtype=np.int64) << 63
            v = bits.view(np.float64)
            v = v[np.isfinite(v) & (np.abs(v) <= np.finfo(np.float64).max / 16)]
            take = min(v.size, r - filled)
            out[filled:filled + take] = v[:take]
            filled += take
        return out

    l1, l2 = lam(), lam()
    t = g.random(r) * 2.0 - 1.0
    c2 = 1.0 / (1.0 + t * t)
    if complex_:
        ca = g.random(r) * 2.0 - 1.0
        sa = np.sqrt(np.maximum(1.0 - ca * ca, 0.0)) * np.where(g.random(r) < 0.5, -1.0, 1.0)
    else:
        ca, sa = np.ones(r), np.zeros(r)
    with np.errstate(over="ignore", invalid="ignore"):
        a11 = c2 * (l1 + l2 * t * t)
        a22 = c2 * (l1 * t * t + l2)
        off = c2 * t * (l1 - l2)
    a21r, a21i = off * ca, off * sa
    ok = np.isfinite(a11) & np.isfinite(a22) & np.isfinite(a21r) & np.isfinite(a21i)
    a11[~ok] = 1.0
    a22[~ok] = 2.0
    a21r[~ok] = 0.5
    a21i[~ok] = 0.0
    if complex_:
        return a11, a22, a21r, a21i
    return a11, a22, a21r


# ---------------------------------------------------------------------------
# SVD inputs

def haar(g: np.random.Generator, m: int, n: int, complex_: bool) -> np.ndarray:
    """m x n matrix with orthonormal columns, Haar-distributed (QR of a
    Gaussian with the R-diagonal phase fix, Mezzadri 2007)."""
    if complex_:
        Z = (g.standard_normal((m, n)) + 1j * g.standard_normal((m, n))) / np.sqrt(2.0)
    else:
        Z = g.standard_normal((m, n))
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R).copy()
    ph = d / np.where(np.abs(d) == 0, 1.0, np.abs(d))
    return Q * ph


def geometric_sigma(n: int, cond: float) -> np.ndarray:
    """sigma_i = cond^{-(i-1)/(n-1)}, i = 1..n (log-equidistributed, as the
    paper's Xi datasets, section 5.1)."""
    if n == 1:
        return np.ones(1)
    return cond ** (-np.arange(n) / (n - 1.0))


def svd_geometric(m: int, n: int, cond: float, complex_: bool, g: np.random.Generator):
    """A = Q1 diag(s) Q2^H, returns (A, s)."""
    s = geometric_sigma(n, cond)
    Q1 = haar(g, m, n, complex_)
    Q2 = haar(g, n, n, complex_)
    A = (Q1 * s) @ Q2.conj().T
    return np.asfortranarray(A), s


def svd_normal(m: int = 256, n: int = 128, seed_salt: int = 0) -> np.ndarray:
    """Workload 1: real m x n, i.i.d. N(0,1), column-major."""
    g = rng(1, seed_salt)
    return np.asfortranarray(g.standard_normal((m, n)))


def svd_complex_geometric(m: int = 4096, n: int = 2048, cond: float = 1e6, seed_salt: int = 0):
    """Workload 3: complex A = Q1 diag(s) Q2^H, s from 1 down to 1/cond."""
    return svd_geometric(m, n, cond, True, rng(3, seed_salt))


def uneven_shapes(count: int = 10000, nmin: int = 16, nmax: int = 256, seed_salt: int = 0):
    """Workload 4 shapes: n ~ U{nmin..nmax}, m ~ U{n..2n}."""
    g = rng(4, seed_salt)
    n = g.integers(nmin, nmax + 1, size=count)
    m = np.array([g.integers(k, 2 * k + 1) for k in n])
    return m.astype(np.int64), n.astype(np.int64)


def uneven_batch(count: int = 10000, nmin: int = 16, nmax: int = 256, cond: float = 1e4,
                 seed_salt: int = 0, indices=None):
    """Workload 4 matrices (list of Fortran-ordered arrays).  `indices`
    selects a subset (each matrix has its own generator, so a subset is
    bit-identical to the same matrices drawn inside the full batch)."""
    m, n = uneven_shapes(count, nmin, nmax, seed_salt)
    idx = range(count) if indices is None else indices
    out = []
    for i in idx:
        g = np.random.Generator(np.random.PCG64([BASE_SEED + 4, seed_salt, int(i)]))
        A, _ = svd_geometric(int(m[i]), int(n[i]), cond, False, g)
        out.append(A)
    return out, m, n


def diff_batch(count: int = 4096, m: int = 64, n: int = 32, cond: float = 1e3, k: int = 8,
               seed_salt: int = 0):
    """Workload 5: (A[count, m, n] column-major per matrix as a C array of
    shape (count, n, m) transposed views, w[count, n], C[count, m, k])."""
    g = rng(5, seed_salt)
    A = np.empty((count, m, n))
    for i in range(count):
        A[i], _ = svd_geometric(m, n, cond, False, g)
    w = g.random((count, n))
    C = g.standard_normal((count, m, k))
    return A, w, C


# ---------------------------------------------------------------------------
# device-side generation of the large batches (workloads 4 and 5)
#
# Drawing 10,000 Haar-factored matrices with numpy takes over a minute, so
# the benchmark draws them on the GPU with torch's seeded CUDA generator:
# for every n, the m x n Gaussians are zero-padded to 2n x n and factored by
# one batched QR (the zero rows stay zero in Q = Z R^-1, so the first m rows
# of Q are the Haar factor of the m x n Gaussian).  The draws are
# reproducible on the same torch build and GPU, not bit-identical to the
# numpy generators above.

def _haar_batch(torch, gen, k, rows, cols, m_rows, device):
    Z = torch.randn((k, rows, cols), generator=gen, dtype=torch.float64, device=device)
    if m_rows is not None:
        r = torch.arange(rows, device=device).view(1, rows, 1)
        Z = Z * (r < m_rows.view(k, 1, 1)).to(Z.dtype)
    Q, R = torch.linalg.qr(Z)
    d = torch.diagonal(R, dim1=-2, dim2=-1)
    sg = torch.where(d < 0, -1.0, 1.0).to(Q.dtype)
    return Q * sg.unsqueeze(1)


def uneven_batch_device(count: int = 10000, nmin: int = 16, nmax: int = 256, cond: float = 1e4,
                        seed_salt: int = 0, device="cuda"):
    """Workload 4 on the device: (A packed column-major 1-D tensor, m, n)."""
    import torch
    m, n = uneven_shapes(count, nmin, nmax, seed_salt)
    off = np.concatenate([[0], np.cumsum(m * n)[:-1]]) if count else np.zeros(0, np.int64)
    A = torch.empty(int((m * n).sum()), dtype=torch.float64, device=device)
    for nv in np.unique(n):
        idx = np.nonzero(n == nv)[0]
        gen = torch.Generator(device=device)
        gen.manual_seed(BASE_SEED + 4 + 7919 * int(nv) + 1000003 * seed_salt)
        k, nv = len(idx), int(nv)
        mt = torch.as_tensor(m[idx], device=device)
        Q1 = _haar_batch(torch, gen, k, 2 * nv, nv, mt, device)
        Q2 = _haar_batch(torch, gen, k, nv, nv, None, device)
        s = torch.as_tensor(geometric_sigma(nv, cond), device=device)
        Ab = (Q1 * s.view(1, 1, nv)) @ Q2.transpose(1, 2)  # (k, 2n, n), zero rows below m
        for t, i in enumerate(idx):
            mi = int(m[i])
            A[int(off[i]):int(off[i]) + mi * nv] = Ab[t, :mi, :].t().reshape(-1)
    return A, m, n


def diff_batch_device(count: int = 4096, m: int = 64, n: int = 32, cond: float = 1e3, k: int = 8,
                      seed_salt: int = 0, device="cuda"):
    """Workload 5 on the device: A (count, m, n) row-major tensor, w (count,
    n), C (count, m, k)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(BASE_SEED + 5 + 1000003 * seed_salt)
    Q1 = _haar_batch(torch, gen, count, m, n, None, device)
    Q2 = _haar_batch(torch, gen, count, n, n, None, device)
    s = torch.as_tensor(geometric_sigma(n, cond), device=device)
    A = (Q1 * s.view(1, 1, n)) @ Q2.transpose(1, 2)
    w = torch.rand((count, n), generator=gen, dtype=torch.float64, device=device)
    C = torch.randn((count, m, k), generator=gen, dtype=torch.float64, device=device)
    return A, w, C


def gram_schmidt_matrix(complex_: bool = False) -> np.ndarray:
    """The 16 x 16 matrix of supplement SM9 (one-based i, j):
    G_ij = 2^(1023 - (j - 1) - |i - j|) for j <= 8 and
    2^(-51 - (j - 1) - |i - j|) for j > 8; the complex variant multiplies
    each entry by a fixed unit phase (seed 9)."""
    n = 16
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    G = np.where(j < 8, np.ldexp(1.0, 1023 - j - abs(i - j)), np.ldexp(1.0, -51 - j - abs(i - j)))
    if complex_:
        G = G * np.exp(1j * np.random.default_rng(9).uniform(0, 2 * np.pi, (n, n)))
    return np.asfortranarray(G)

