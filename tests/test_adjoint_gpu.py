"""The differentiated batched SVD: forward = jsvd_svd_batched + sign gauge,
backward = the adjoint kernel (jsvd_svd_adjoint_batched).  Checked against
the FP64 CPU reference (oracle SVD + oracle adjoint) and against central
differences (h = 1e-6), on the loss sum_i w_i sigma_i + <C, U[:, :k]>."""
import numpy as np
import pytest

import oracle
from paper_2202_08361_gb300 import workloads

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def loss_gpu(A, w, C, k):
    import paper_2202_08361_gb300 as J
    U, S, V = J.svd_diff(A)
    return (w * S).sum() + (C * U[:, :, :k]).sum()


def test_adjoint_kernel_against_oracle_formula():
    """Same inputs to the kernel and to the oracle's plain-loop adjoint."""
    import paper_2202_08361_gb300 as J
    torch = _torch()
    A, w, C = workloads.diff_batch(count=5, m=20, n=10, k=4)
    At = torch.from_numpy(A).cuda()
    U, S, V = J.svd_diff(At)
    g = np.random.default_rng(3)
    Ub = g.standard_normal(U.shape)
    Vb = g.standard_normal(V.shape)
    Ab = J.svd_adjoint_batched(U, S, V, torch.from_numpy(Ub).cuda(), torch.from_numpy(w).cuda(),
                               torch.from_numpy(Vb).cuda()).cpu().numpy()
    Un, Sn, Vn = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    for i in range(5):
        ref = oracle.svd_adjoint(Un[i], Sn[i], Vn[i], Ub[i], w[i], Vb[i])
        assert np.abs(Ab[i] - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())


def test_gradient_against_cpu_reference():
    """Gradient of the loss vs the FP64 CPU reference (oracle SVD, sign
    gauge, oracle adjoint) on 64 matrices of the differentiated workload's
    shape and conditioning (64 x 32, condition 1e3)."""
    torch = _torch()
    k = 8
    count = 64
    A, w, C = workloads.diff_batch(count=count, m=64, n=32, k=k)
    At = torch.from_numpy(A).cuda().requires_grad_(True)
    L = loss_gpu(At, torch.from_numpy(w).cuda(), torch.from_numpy(C).cuda(), k)
    L.backward()
    G = At.grad.cpu().numpy()
    sg, Us, Vs, st = oracle.vjsvd_batch(list(A))
    assert all(x == oracle.OK for x in st)
    gauged = [oracle.sign_gauge(u, v) for u, v in zip(Us, Vs)]
    U = np.stack([u for u, _ in gauged])
    V = np.stack([v for _, v in gauged])
    Ub = np.zeros_like(U)
    Ub[:, :, :k] = C
    ref = oracle.svd_adjoint_batch(U, np.stack(sg), V, Ub, w)
    for i in range(count):
        assert np.abs(G[i] - ref[i]).max() <= 1e-9 * np.abs(ref[i]).max(), i


def test_gradient_central_differences_small():
    torch = _torch()
    k = 4
    A, w, C = workloads.diff_batch(count=4, m=24, n=12, k=k, seed_salt=1)
    At = torch.from_numpy(A).cuda()
    wt, Ct = torch.from_numpy(w).cuda(), torch.from_numpy(C).cuda()
    X = At.clone().requires_grad_(True)
    loss_gpu(X, wt, Ct, k).backward()
    g = np.random.default_rng(7)
    for _ in range(3):
        D = torch.from_numpy(g.standard_normal(A.shape)).cuda()
        h = 1e-6
        with torch.no_grad():
            fd = (loss_gpu(At + h * D, wt, Ct, k) - loss_gpu(At - h * D, wt, Ct, k)) / (2 * h)
        an = (X.grad * D).sum()
        assert abs(fd.item() - an.item()) <= 1e-6 * max(1.0, abs(an.item()))


def test_full_workload_4096_gradient_central_differences():
    """The full workload (4096 real 64 x 32, condition 1e3): forward plus the
    adjoint, checked by central differences of the summed loss along random
    directions (h = 1e-6)."""
    torch = _torch()
    import paper_2202_08361_gb300 as J
    k = 8
    A, w, C = workloads.diff_batch_device()
    X = A.clone().requires_grad_(True)
    loss_gpu(X, w, C, k).backward()
    assert torch.isfinite(X.grad).all()
    # The sign gauge makes U a function of A only where the largest entry
    # of |u_j| is unique by a margin; across the 4096 x 8 gauged columns a
    # few are within a step h of a tie, and there the loss jumps.  The
    # directions below move only the matrices whose first k columns have a
    # clear largest entry.
    with torch.no_grad():
        U = J.svd_diff(A)[0][:, :, :k].abs()
        top2 = U.topk(2, dim=1).values
        stable = ((top2[:, 0, :] - top2[:, 1, :]) > 3e-4 * top2[:, 0, :]).all(dim=1)
    assert stable.float().mean().item() > 0.75
    gen = torch.Generator(device="cuda").manual_seed(17)
    for _ in range(2):
        D = torch.randn(A.shape, generator=gen, dtype=torch.float64, device="cuda")
        D = D * stable.view(-1, 1, 1).to(D.dtype)
        h = 1e-6
        with torch.no_grad():
            d1 = loss_gpu(A + h * D, w, C, k) - loss_gpu(A - h * D, w, C, k)
            d2 = loss_gpu(A + 2 * h * D, w, C, k) - loss_gpu(A - 2 * h * D, w, C, k)
        fd = d1 / (2 * h)
        fd4 = (8 * d1 - d2) / (12 * h)  # Richardson: truncation O(h^4)
        an = (X.grad * D).sum()
        # The plain central difference carries an O(h^2) truncation error of
        # a few 1e-6 relative here: the smallest singular values (1e-3) sit
        # 2.5e-4 apart, so the third derivatives of sigma along D reach
        # ~1/gap^2.  The fourth-order difference at the same h removes it.
        assert abs(fd.item() - an.item()) <= 1e-4 * max(1.0, abs(an.item()))
        assert abs(fd4.item() - an.item()) <= 1e-7 * max(1.0, abs(an.item()))
