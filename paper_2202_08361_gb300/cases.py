"""Run one named workload once (for profiling and quick checks).

    python -m paper_2202_08361_gb300.cases evd   [--log2 23] [--f32]
    python -m paper_2202_08361_gb300.cases svd   [--m 1024 --n 512 --complex --normal
                                                  --mode fp64|mixed --step 0..5 --reps 1]
    python -m paper_2202_08361_gb300.cases batch [--count 1000] [--shape 64x32]
    python -m paper_2202_08361_gb300.cases diff  [--count 4096]

Each runs the case `--warmup` times and then `--reps` times, synchronising
after each, and prints a short summary line.  Inputs come from the seeded
generators of workloads.py.
"""
import argparse
import os
import sys
import time


def main(argv=None):
    import torch

    import paper_2202_08361_gb300 as J
    from paper_2202_08361_gb300 import workloads

    p = argparse.ArgumentParser()
    p.add_argument("case", choices=["evd", "svd", "batch", "diff"])
    p.add_argument("--log2", type=int, default=23)
    p.add_argument("--f32", action="store_true", help="evd: the binary32 EVD")
    p.add_argument("--m", type=int, default=1024)
    p.add_argument("--n", type=int, default=512)
    p.add_argument("--complex", action="store_true")
    p.add_argument("--normal", action="store_true",
                   help="svd: i.i.d. N(0,1) entries (workload 1) instead of a geometric spectrum")
    p.add_argument("--mode", default="fp64", choices=["fp64", "mixed"])
    p.add_argument("--max-sweeps", type=int, default=0, help="svd: sweep cap (0: the default)")
    p.add_argument("--count", type=int, default=1000)
    p.add_argument("--shape", default=None,
                   help="batch: every matrix m x n (geometric spectrum, condition 1e3) "
                        "instead of the uneven shapes")
    p.add_argument("--warps", type=int, default=0, help="batch: warps per block (0: default)")
    p.add_argument("--smem", type=int, default=-1, help="batch: shared-memory KiB (-1: default)")
    p.add_argument("--step", type=int, default=-1,
                   help="svd: JSVD_TUNE_SVD_STEP form of the sweep steps (-1: the default)")
    p.add_argument("--warmup", type=int, default=1)
    p.add_argument("--reps", type=int, default=1)
    a = p.parse_args(argv)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if a.step >= 0:
        J.tune_set(J.JSVD_TUNE_SVD_STEP, a.step)

    if a.case == "evd":
        r = 1 << a.log2
        gen = workloads.evd_batch_f32 if a.f32 else workloads.evd_batch
        re_ = [torch.from_numpy(x).to(dev) for x in gen(r, False)]
        cx = [torch.from_numpy(x).to(dev) for x in gen(r, True)]
        run = lambda: (J.evd2x2_batched(*re_), J.evd2x2_batched(*cx))
        label = "evd r=2^%d real+complex %s" % (a.log2, "f32" if a.f32 else "f64")
    elif a.case == "svd":
        if a.normal:
            A = workloads.svd_normal(a.m, a.n)
        else:
            A, _ = workloads.svd_geometric(a.m, a.n, 1e6, a.complex, workloads.rng(3, 7))
        At = torch.from_numpy(A).to(dev)
        run = lambda: J.svd(At, mode=a.mode, max_sweeps=a.max_sweeps)
        label = "svd %dx%d %s %s" % (a.m, a.n, "complex" if a.complex else "real", a.mode)
    elif a.case == "batch":
        import numpy as np
        if a.shape:
            # drawn on the host (no device linear algebra, so this also runs
            # under a profiler that hides torch's lazily loaded libraries)
            mm, nn = (int(x) for x in a.shape.split("x"))
            A3 = workloads.diff_batch(count=a.count, m=mm, n=nn)[0]  # (count, m, n) column-major
            A = torch.from_numpy(np.ascontiguousarray(A3.transpose(0, 2, 1))).reshape(-1).to(dev)
            m, n = np.full(a.count, mm), np.full(a.count, nn)
        else:
            A, m, n = workloads.uneven_batch_device(count=a.count, device=dev)
        if a.warps:
            J.tune_set(J.JSVD_TUNE_BATCH_WARPS, a.warps)
        if a.smem >= 0:
            J.tune_set(J.JSVD_TUNE_BATCH_SMEM, a.smem)
        B = J.BatchedSVD(A, m, n)
        run = lambda: B.launch()
        label = "batched %s count=%d" % (a.shape or "uneven", a.count)
    else:
        A, w, C = workloads.diff_batch_device(count=a.count, device=dev)

        def run():
            X = A.clone().requires_grad_(True)
            U, S, V = J.svd_diff(X)
            ((w * S).sum() + (C * U[:, :, :8]).sum()).backward()
        label = "diff count=%d" % a.count
    for _ in range(a.warmup):
        run()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(a.reps):
        run()
    torch.cuda.synchronize(dev)
    print("%s: %.3f ms per run" % (label, 1e3 * (time.perf_counter() - t0) / a.reps))
    return 0


if __name__ == "__main__":
    sys.exit(main())
