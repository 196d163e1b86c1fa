"""The batched uneven SVD (jsvd_svd_batched): every matrix gives the same
bits as jsvd_svd on it alone, whatever the batch, the position in it and
the block shape; parity with the oracle; every matrix of the full 10,000-matrix workload meets the
acceptance bounds, and 50 of them match the oracle; a captured CUDA graph
replays it."""
import numpy as np
import pytest

import oracle
from paper_2202_08361_gb300 import workloads

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


def tol(n):
    return 64 * n * EPS


def _torch():
    import torch
    return torch


def mats_mixed(cplx, seed=0):
    g = np.random.default_rng(seed)
    shapes = [(1, 1), (7, 1), (9, 2), (33, 17), (64, 64), (100, 37), (65, 33), (40, 40), (130, 70)]
    out = []
    for m, n in shapes:
        A, _ = workloads.svd_geometric(m, n, 1e4, cplx, g)
        out.append(A)
    return out


def single(A):
    torch = _torch()
    import paper_2202_08361_gb300 as J
    out = J.svd(torch.from_numpy(np.asfortranarray(A)).cuda())
    torch.cuda.synchronize()
    return out


def same(x, y):
    torch = _torch()
    x, y = x.contiguous(), y.contiguous()
    if x.is_complex():
        x, y = torch.view_as_real(x), torch.view_as_real(y)
    return torch.equal(x.view(torch.int64), y.view(torch.int64))


@pytest.mark.parametrize("cplx", [False, True])
def test_batched_equals_single_bitwise(cplx):
    import paper_2202_08361_gb300 as J
    mats = mats_mixed(cplx, seed=1 + cplx)
    B = J.svd_batched(mats)
    _torch().cuda.synchronize()
    infos = J.decode_info(B.info)
    for i, A in enumerate(mats):
        ref = single(A)
        U, s, V = B.matrix(i)
        assert same(U, ref["U"]) and same(V, ref["V"]) and same(s, ref["sigma"]), i
        assert infos[i] == J.decode_info(ref["info"]), i


@pytest.mark.parametrize("cplx", [False, True])
def test_batched_compensated_equals_single_bitwise(cplx):
    """The compensated option in the batched kernel: the bits of jsvd_svd
    with the same option."""
    import paper_2202_08361_gb300 as J
    torch = _torch()
    mats = mats_mixed(cplx, seed=31 + cplx)
    B = J.svd_batched(mats, compensated=True)
    torch.cuda.synchronize()
    for i, A in enumerate(mats):
        ref = J.svd(torch.from_numpy(np.asfortranarray(A)).cuda(), compensated=True)
        torch.cuda.synchronize()
        U, s, V = B.matrix(i)
        assert same(U, ref["U"]) and same(V, ref["V"]) and same(s, ref["sigma"]), i


@pytest.mark.parametrize("kib", [24, 100, 220])
def test_shared_memory_path_bitwise(kib):
    """Matrices whose G and V fit the shared-memory budget are iterated
    there; the bits do not change, whatever the budget and block shape."""
    import paper_2202_08361_gb300 as J
    torch = _torch()
    mats = mats_mixed(False, seed=5)
    ref = J.svd_batched(mats)
    torch.cuda.synchronize()
    try:
        for w in (2, 8):
            J.tune_set(J.JSVD_TUNE_BATCH_WARPS, w)
            J.tune_set(J.JSVD_TUNE_BATCH_SMEM, kib)
            other = J.svd_batched(mats)
            torch.cuda.synchronize()
            for i in range(len(mats)):
                for a, b in zip(other.matrix(i), ref.matrix(i)):
                    assert same(a, b), (kib, w, i)
        cm = mats_mixed(True, seed=6)
        J.tune_set(J.JSVD_TUNE_BATCH_SMEM, 0)
        cref = J.svd_batched(cm)
        J.tune_set(J.JSVD_TUNE_BATCH_SMEM, kib)
        cother = J.svd_batched(cm)
        torch.cuda.synchronize()
        for i in range(len(cm)):
            for a, b in zip(cother.matrix(i), cref.matrix(i)):
                assert same(a, b), (kib, "complex", i)
    finally:
        J.tune_set(J.JSVD_TUNE_BATCH_WARPS, 0)
        J.tune_set(J.JSVD_TUNE_BATCH_SMEM, 0)


def test_batch_composition_and_block_shape_invariance():
    import paper_2202_08361_gb300 as J
    torch = _torch()
    mats = mats_mixed(False, seed=5)
    ref = J.svd_batched(mats)
    order = list(range(len(mats)))[::-1]
    rev = J.svd_batched([mats[i] for i in order])
    try:
        for w in (1, 4, 16):
            J.tune_set(J.JSVD_TUNE_BATCH_WARPS, w)
            other = J.svd_batched(mats + mats[:3])
            torch.cuda.synchronize()
            for i in range(len(mats)):
                for a, b in zip(other.matrix(i), ref.matrix(i)):
                    assert same(a, b), (w, i)
    finally:
        J.tune_set(J.JSVD_TUNE_BATCH_WARPS, 0)
    for pos, i in enumerate(order):
        for a, b in zip(rev.matrix(pos), ref.matrix(i)):
            assert same(a, b), i


def test_batched_against_oracle():
    import paper_2202_08361_gb300 as J
    mats = mats_mixed(True, seed=9)
    B = J.svd_batched(mats)
    _torch().cuda.synchronize()
    for i, A in enumerate(mats):
        n = A.shape[1]
        U, s, V = (t.cpu().numpy() for t in B.matrix(i))
        o = oracle.vjsvd(A)
        assert np.abs(s - o["sigma"]).max() <= tol(n) * o["sigma"][0]
        res = np.linalg.norm(A - (U * s) @ V.conj().T) / max(np.linalg.norm(A), 1e-300)
        assert res <= tol(n)
        assert np.abs(U.conj().T @ U - np.eye(n)).max() <= tol(n)


def test_batched_edge_cases():
    import paper_2202_08361_gb300 as J
    torch = _torch()
    Z = np.zeros((5, 3))
    N = workloads.svd_normal(6, 3, seed_salt=2)
    N[1, 1] = np.nan
    G = workloads.svd_normal(12, 6, seed_salt=3)
    B = J.svd_batched([Z, N, G], max_sweeps=1)
    torch.cuda.synchronize()
    info = J.decode_info(B.info)
    assert info[0]["status"] == 0 and torch.all(B.matrix(0)[1] == 0)
    assert info[1]["status"] == J.JSVD_E_NONFINITE and torch.all(torch.isnan(B.matrix(1)[1]))
    assert info[2]["status"] == J.JSVD_NOT_CONVERGED and info[2]["sweeps"] == 1
    E = J.svd_batched([])
    assert E.count == 0


def test_full_workload_10000_uneven():
    """The 10,000-matrix uneven workload (n ~ U{16..256}, m ~ U{n..2n},
    condition 1e4): every matrix converges and meets the bounds -- residual,
    both orthogonalities and the prescribed spectrum, checked for all 10,000
    on the GPU (matrices of one n padded to 2n rows with zeros, which change
    none of the measures) -- and 50 of them, among them the smallest and one
    of the largest (n = 256), match the oracle's singular values."""
    import paper_2202_08361_gb300 as J
    torch = _torch()
    A, m, n = workloads.uneven_batch_device()
    B = J.BatchedSVD(A, m, n).launch()
    torch.cuda.synchronize()
    info = J.decode_info(B.info)
    assert all(x["status"] == 0 for x in info)
    worst = {"res": 0.0, "orth": 0.0, "sigma": 0.0}
    for nv in np.unique(n):
        idx = np.nonzero(n == nv)[0]
        nv = int(nv)
        k = len(idx)
        Ap = torch.zeros((k, 2 * nv, nv), dtype=torch.float64, device="cuda")
        Up = torch.zeros_like(Ap)
        Vb = torch.empty((k, nv, nv), dtype=torch.float64, device="cuda")
        Sb = torch.empty((k, nv), dtype=torch.float64, device="cuda")
        for t, i in enumerate(idx):
            mi = int(m[i])
            Ap[t, :mi] = A[int(B.offA[i]):int(B.offA[i]) + mi * nv].view(nv, mi).t()
            U, s, V = B.matrix(int(i))
            Up[t, :mi] = U
            Vb[t] = V
            Sb[t] = s
        I = torch.eye(nv, dtype=torch.float64, device="cuda")
        res = (torch.linalg.norm(Ap - (Up * Sb[:, None, :]) @ Vb.transpose(1, 2), dim=(1, 2))
               / torch.linalg.norm(Ap, dim=(1, 2)))
        ou = (Up.transpose(1, 2) @ Up - I).abs().amax(dim=(1, 2))
        ov = (Vb.transpose(1, 2) @ Vb - I).abs().amax(dim=(1, 2))
        sref = torch.as_tensor(workloads.geometric_sigma(nv, 1e4), device="cuda")
        es = (Sb - sref).abs().amax(dim=1) / sref[0]
        b = tol(nv)
        worst["res"] = max(worst["res"], res.max().item() / b)
        worst["orth"] = max(worst["orth"], max(ou.max().item(), ov.max().item()) / b)
        worst["sigma"] = max(worst["sigma"], es.max().item() / b)
        assert res.max().item() <= b, (nv, res.max().item())
        assert ou.max().item() <= b and ov.max().item() <= b, (nv, ou.max().item(), ov.max().item())
        assert es.max().item() <= b, (nv, es.max().item())
    # the oracle on 50 matrices (the OpenMP threads share them out)
    g = np.random.default_rng(11)
    big = int(np.nonzero(n == n.max())[0][np.argmax(m[n == n.max()])])
    sample = sorted(set(g.choice(len(m), 48, replace=False).tolist()
                        + [int(np.argmin(m * n)), big]))
    assert len(sample) >= 50 and int(n[big]) == 256
    host = [A[int(B.offA[i]):int(B.offA[i]) + int(m[i] * n[i])].view(int(n[i]), int(m[i])).t()
            .cpu().numpy() for i in sample]
    sg, _, _, st = oracle.vjsvd_batch(host)
    assert all(x == oracle.OK for x in st)
    for i, so in zip(sample, sg):
        s = B.matrix(i)[1].cpu().numpy()
        assert np.abs(s - so).max() <= tol(int(n[i])) * so[0], i


@pytest.mark.parametrize("cplx", [False, True])
def test_skipping_unchanged_pairs_bit_identical(cplx):
    """The batched sweeps skip the pairs whose columns have not changed since
    their last meeting (JSVD_TUNE_SVD_SKIP); the results are the bits of the
    run that forms every pair."""
    import paper_2202_08361_gb300 as J
    torch = _torch()
    mats = mats_mixed(cplx, seed=51 + cplx) + workloads.diff_batch(count=6, m=64, n=32, k=8)[0].tolist()
    mats = [np.asarray(a, dtype=np.complex128 if cplx else np.float64) for a in mats]
    outs = []
    try:
        for skip in (0, 1):
            J.tune_set(J.JSVD_TUNE_SVD_SKIP, skip)
            B = J.svd_batched(mats)
            torch.cuda.synchronize()
            outs.append((B.U.clone(), B.V.clone(), B.sigma.clone(), J.decode_info(B.info)))
    finally:
        J.tune_set(J.JSVD_TUNE_SVD_SKIP, 1)
    for a, b in zip(outs[0][:3], outs[1][:3]):
        assert same(a, b)
    assert outs[0][3] == outs[1][3]


def test_cuda_graph_replay():
    import paper_2202_08361_gb300 as J
    torch = _torch()
    mats = mats_mixed(False, seed=21)
    A, m, n = J.pack_matrices(mats)
    B = J.BatchedSVD(A, m, n)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        B.launch(s)  # warm-up outside the capture
    torch.cuda.synchronize()
    ref = [t.clone() for t in (B.U, B.V, B.sigma)]
    B.U.zero_()
    B.sigma.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        B.launch(s)
    graph.replay()
    torch.cuda.synchronize()
    for a, b in zip((B.U, B.V, B.sigma), ref):
        assert same(a, b)


def test_autotune_picks_a_candidate_and_keeps_the_bits(tmp_path, monkeypatch):
    """The autotuner times the candidates on the batch (two sweeps each),
    caches the winner, and the batch launched with it gives the same bits
    as the default."""
    import paper_2202_08361_gb300 as J
    torch = _torch()
    monkeypatch.setenv("JSVD_TUNE_CACHE", str(tmp_path / "tune.json"))
    mats = mats_mixed(False, seed=41) * 3
    A, m, n = J.pack_matrices(mats)
    ref = J.BatchedSVD(A, m, n).launch()
    B = J.BatchedSVD(A, m, n)
    times = B.autotune()
    assert set(times) == {1, 2, 4, 8, 16} and B.warps in times
    assert B.autotune() == {}  # cached
    B.launch()
    torch.cuda.synchronize()
    for a, b in zip((B.U, B.V, B.sigma), (ref.U, ref.V, ref.sigma)):
        assert same(a, b)
