#!/usr/bin/env python
"""Benchmark of the Jacobi SVD hot path on GB300; prints ONE JSON line.

Default workload: the batched 2x2 Hermitian EVD (section 2 of the paper),
2^24 real symmetric + 2^24 complex Hermitian FP64 matrices per step in SoA
streams, entries sign*(1+u)*2^e over the whole binary64 range with 1 %
exact zeros.  A step is one pass of both kernels over the resident batch;
metric = 2x2 EVDs per second over the whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank processes its own batch (independent
matrices, no data-path collective: weak scaling); timing is the max over
ranks.  --impl reference times the CPU oracle on the host cores instead.
"""
import os

# The CPU oracle's OpenMP environment, as the paper runs its CPU code
# (threads spread over the cores, one per core, no dynamic adjustment).  Set
# before anything loads an OpenMP runtime: a runtime reads these once, when
# it starts.  The binding in force is read back and reported.
for _k, _v in (("OMP_PROC_BIND", "spread"), ("OMP_PLACES", "cores"), ("OMP_DYNAMIC", "false")):
    os.environ.setdefault(_k, _v)

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import threading  # noqa: E402
import time  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

R_EVD = 1 << 24            # matrices per kernel per step
BYTES_REAL = 60            # 3 x 8 in + 4 x 8 + 4 out
BYTES_CPLX = 76            # 4 x 8 in + 5 x 8 + 4 out
METRIC = "2x2 EVDs/s"
UNIT = "EVD/s"
WORKLOAD = ("batched 2x2 Hermitian EVD, 2^24 real symmetric + 2^24 complex Hermitian FP64 "
            "matrices per step, SoA streams, entries sign*(1+u)*2^e, e~U{-1074..1023}, 1% zeros")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--evd-log2", type=int, default=24,
                   help="log2 of the matrices per kernel per step (24 = the full workload)")
    p.add_argument("--no-svd", action="store_true",
                   help="skip the SVD measurements (C1, C3 plain/mixed, C4, C5)")
    p.add_argument("--c4-loop", type=int, default=120,
                   help="matrices of the 10,000-matrix batch timed through jsvd_svd one by "
                        "one (a random sample scaled by m n^2; 10000 = the whole loop)")
    return p.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def sm_clock_mhz(local_rank):
    """The SM clock nvidia-smi reports now (MHz), or None."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(gpu_index(local_rank)),
                              "--query-gpu=clocks.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=10).stdout
        return float(out.strip().splitlines()[0])
    except Exception:
        return None


def gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


# ---------------------------------------------------------------------------

def kernel_source_sha():
    h = hashlib.sha256()
    for name in ("evd2.cu", "evd2.cuh", "fp64bits.cuh", "fp64soft.cuh"):
        with open(os.path.join(ROOT, "paper_2202_08361_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_pipes(kernel):
    """FP64-pipe, integer-ALU and issue utilisation of the kernel from the
    committed ncu summary, if it was taken on the current kernel source;
    else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "evd2_traffic.json")) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("source_sha") != kernel_source_sha():
        return None
    return rec.get("pipes_active", {}).get(kernel)


def recorded_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "evd2_traffic.json")) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("source_sha") != kernel_source_sha():
        return None
    return rec.get("dram_bytes_per_launch", {}).get(kernel)


def cpu_oracle_evd(r, seed_salt=0):
    """Time the oracle (as it stands) on r real + r complex matrices."""
    import oracle
    from paper_2202_08361_gb300 import workloads
    re_ = workloads.evd_batch(r, False, seed_salt)
    cx = workloads.evd_batch(r, True, seed_salt)
    t0 = time.perf_counter()
    oracle.dsjac2(*re_)
    oracle.zsjac2(*cx)
    dt = time.perf_counter() - t0
    return dt, oracle.num_threads()


def cpu_oracle_svd(A, nthreads=0, max_steps=0):
    """Time the oracle's SVD (as it stands, OpenMP over the pairs of a step)
    on the host matrix A once, all cores (nthreads 0) or nthreads, for at
    most max_steps parallel steps (0: to convergence); (ms, threads, sweeps,
    steps run)."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.vjsvd(A, nthreads=nthreads, max_steps=max_steps)
    dt = time.perf_counter() - t0
    n = A.shape[1]
    nt = n + (n & 1)
    steps = r["sweeps"] * (nt - 1) if max_steps <= 0 else min(max_steps, r["sweeps"] * (nt - 1))
    return 1e3 * dt, (nthreads if nthreads > 0 else oracle.num_threads()), int(r["sweeps"]), steps


def cpu_oracle_evd_threads(r, nthreads, seed_salt=0):
    """cpu_oracle_evd with the oracle's OpenMP loops on nthreads threads."""
    import oracle
    from paper_2202_08361_gb300 import workloads
    re_ = workloads.evd_batch(r, False, seed_salt)
    cx = workloads.evd_batch(r, True, seed_salt)
    t0 = time.perf_counter()
    oracle.dsjac2(*re_, nthreads=nthreads)
    oracle.zsjac2(*cx, nthreads=nthreads)
    return time.perf_counter() - t0, nthreads


def oracle_env():
    """The OpenMP threads and binding in force for the oracle."""
    import oracle
    return oracle.omp_state()



# ---------------------------------------------------------------------------
# the SVD workloads (reported beside the EVD headline)

def _ev(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


# FP64-pipe operations per matrix of the batched EVD in its default division
# placement (evd2.cu: only sqrt(tan2^2 + 1) runs on the FP64 pipe; every
# other division and square root, and all exponent, sign and min/max work,
# run on the integer pipe), counted from evd2.cuh: (adds, multiplies and
# fmas; IEEE square roots).  Real: a11 - a22, fma(tan2, tan2, 1),
# 1 + sqrt(.), fma(tan, tan, 1) for sec^2, two fmas for each lambda'.
# Complex: those 8 plus fma(q, q, 1) and the product by M of Alg. hypot,
# and cos(alpha) tan(phi), sin(alpha) tan(phi).
EVD_FP64_OPS = {"evd2_kernel<real>": (8, 1), "evd2_kernel<complex>": (12, 1)}


def fp64_pipe_rates(torch, J, dev):
    """The FP64 pipe's throughput measured now, on this GPU: fused
    multiply-adds, IEEE square roots and IEEE divisions per second over the
    whole GPU (jsvd_probe_fp64_rate: 8 blocks of 256 threads per SM, 8
    independent chains per thread, best of 3 launches timed with CUDA
    events)."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * 8
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)
    res = {}
    for kind, name, iters in ((0, "fma", 4000), (1, "sqrt", 400), (2, "div", 400)):
        J.probe_fp64_rate(kind, 8, blocks, sink)
        best = None
        for _ in range(3):
            e0, e1 = _ev(torch)
            e0.record(st)
            J.probe_fp64_rate(kind, iters, blocks, sink)
            e1.record(st)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        res[name + "_per_s"] = blocks * 256 * 8 * iters / (best * 1e-3)
    # one warp alone, and one warp on each of an SM's four schedulers (one
    # block of 32 or 128 threads): the time per FP64 instruction of a warp,
    # also in SM clocks at the clock nvidia-smi reports just after
    for warps in (1, 4):
        J.probe_fp64_rate(0, 8, 1, sink, threads=32 * warps)
        e0, e1 = _ev(torch)
        e0.record(st)
        J.probe_fp64_rate(0, 2000, 1, sink, threads=32 * warps)
        e1.record(st)
        torch.cuda.synchronize(dev)
        ns_per_instr = e0.elapsed_time(e1) * 1e6 / (2000 * 8)
        res["warp_fma_issue_ns_%dw" % warps] = ns_per_instr
        clk = sm_clock_mhz(dev.index or 0)
        if clk:
            res["warp_fma_issue_cycles_%dw" % warps] = ns_per_instr * clk * 1e-3
    res["fma_flops"] = 2 * res["fma_per_s"]
    res["sqrt_in_fma"] = res["fma_per_s"] / res["sqrt_per_s"]
    res["div_in_fma"] = res["fma_per_s"] / res["div_per_s"]
    res["method"] = ("jsvd_probe_fp64_rate: %d blocks x 256 threads x 8 independent chains; "
                     "best of 3 CUDA-event-timed launches" % blocks)
    return res


def evd_fp64_roofline(kernel, ms, r, rates):
    """The EVD kernel against the pipe that binds it: FP64-pipe work per
    matrix (counted, the square roots converted to fmas at the measured
    rate ratio) x matrices / kernel time, over the measured fma rate."""
    nf, ns = EVD_FP64_OPS[kernel]
    ops = nf + ns * rates["sqrt_in_fma"]
    achieved = ops * r / (ms * 1e-3)
    return {"bound": "fp64_pipe", "kernel": kernel, "achieved": achieved,
            "peak": rates["fma_per_s"], "unit": "FP64 lane-ops/s (fma equivalents)",
            "frac": achieved / rates["fma_per_s"], "ops_per_matrix": ops,
            "counted": {"add_mul_fma": nf, "ieee_sqrt": ns}, "peak_kind": "measured in this run",
            "avg_launch_ms": ms}


def _svd_lane_ops(m, n, sweeps, rotations, cplx):
    """FP64-pipe lane operations of the sweeps (each add, multiply or fma
    counts one, as the pipe issues them): every visited pair forms its sums
    (3 fma per row real, 8 complex), every rotated pair transforms m + n
    rows (2 fma + 2 mul real; 8 fma + 4 mul complex, Eq. e:transf with the
    complex fma of Eq. e:zfma)."""
    pairs = sweeps * n * (n - 1) // 2
    if cplx:
        return pairs * 8 * m + rotations * 12 * (m + n)
    return pairs * 3 * m + rotations * 4 * (m + n)


def _svd_flops(m, n, sweeps, rotations, cplx):
    """FP64 flops of the sweeps (fma = 2): every visited pair forms its sums
    (3m fma real, 8m complex), every rotated pair transforms m + n rows
    (2 fma + 2 mul real, 8 fma + 4 mul complex)."""
    pairs = sweeps * n * (n - 1) // 2
    if cplx:
        return pairs * 16 * m + rotations * 20 * (m + n)
    return pairs * 6 * m + rotations * 6 * (m + n)


def evd_f32_bench(torch, J, workloads, dev, peaks, reps=50):
    """The single precision EVD on 2^24 real + 2^24 complex binary32
    matrices (jsvd_evd2x2_batched_f32): per-kernel CUDA-event times and the
    HBM fraction (32 / 40 algorithmic bytes per real / complex matrix)."""
    r = 1 << 24
    st = torch.cuda.current_stream(dev)
    res = {}
    for cplx, name, per in ((False, "real", 32), (True, "complex", 40)):
        t = [torch.from_numpy(a).to(dev) for a in workloads.evd_batch_f32(r, cplx)]
        out = J.evd2x2_batched(*t)
        for _ in range(5):
            J.evd2x2_batched(*t, out=out)
        e0, e1 = _ev(torch)
        torch.cuda.synchronize(dev)
        e0.record(st)
        for _ in range(reps):
            J.evd2x2_batched(*t, out=out)
        e1.record(st)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        gbs = per * r / (ms * 1e-3) / 1e9
        res[name] = {"ms": ms, "evd_per_s": r / (ms * 1e-3), "gbs": gbs,
                     "hbm_frac": gbs / peaks["hbm_gbs"], "bytes_per_matrix": per}
        del t, out
    res["workload"] = "2^24 real + 2^24 complex binary32 matrices, entries sign*(1+k 2^-23)*2^e, e~U{-149..127}, 1% zeros"
    return res


def svd_bench(torch, J, workloads, dev, rates, cpu=True, loop_count=120):
    """The SVD workloads beside the EVD headline: per workload the GPU time,
    accuracy, FP64 rate against the measured fma rate, and (cpu) the oracle
    timed on the host cores, all cores and one thread, on the whole workload
    or a stated bounded sample of it."""
    import numpy as np
    out = {}
    DFMA_FLOPS = rates["fma_flops"]
    eps = np.finfo(np.float64).eps
    st = torch.cuda.current_stream(dev)

    def accuracy(A, r):
        n = A.shape[1]
        U, s, V = r["U"], r["sigma"], r["V"]
        I = torch.eye(n, dtype=A.dtype, device=dev)
        res = (torch.linalg.norm(A - (U * s) @ V.conj().T) / torch.linalg.norm(A)).item()
        ou = (U.conj().T @ U - I).abs().max().item()
        ov = (V.conj().T @ V - I).abs().max().item()
        return {"residual": res, "orth_U": ou, "orth_V": ov, "bound_64neps": 64 * n * eps}

    # C1: real 256 x 128, N(0,1)
    A1 = torch.from_numpy(workloads.svd_normal()).to(dev)
    r = J.svd(A1)
    torch.cuda.synchronize(dev)
    reps = 20
    e0, e1 = _ev(torch)
    e0.record(st)
    for _ in range(reps):
        J.svd(A1, out=r)
    e1.record(st)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    info = J.decode_info(r["info"])
    fl = _svd_flops(256, 128, info["sweeps"], info["rotations"], False)
    lo = _svd_lane_ops(256, 128, info["sweeps"], info["rotations"], False)
    c1 = {"ms_per_svd": ms, "sweeps": info["sweeps"], "rotations": info["rotations"],
          "fp64_gflops": fl / ms / 1e6, "fp64_frac": fl / (ms * 1e-3) / DFMA_FLOPS,
          "fp64_pipe_frac": lo / (ms * 1e-3) / rates["fma_per_s"]}
    c1.update(accuracy(A1, r))
    if cpu:
        try:
            co = {"kind": "oracle", "sample": "the same matrix, once, to convergence"}
            for key, thr in (("all_cores", 0), ("one_thread", 1)):
                ms_o, thr_o, sw_o, _ = cpu_oracle_svd(workloads.svd_normal(), nthreads=thr)
                co[key] = {"ms_per_svd": ms_o, "threads": thr_o, "sweeps": sw_o,
                           "gpu_speedup": ms_o / ms}
            c1["cpu_oracle"] = co
        except Exception as exc:  # host-side context only: the GPU figures stand without it
            c1["cpu_oracle"] = {"error": repr(exc)}
    out["C1_real_256x128"] = c1

    # the same matrix in single precision (jsvd_svd_f32)
    A1f = A1.float()
    r = J.svd(A1f)
    torch.cuda.synchronize(dev)
    e0, e1 = _ev(torch)
    e0.record(st)
    for _ in range(reps):
        J.svd(A1f, out=r)
    e1.record(st)
    torch.cuda.synchronize(dev)
    info = J.decode_info(r["info"])
    U, sv, V = r["U"].double(), r["sigma"].double(), r["V"].double()
    I = torch.eye(128, dtype=torch.float64, device=dev)
    A1d = A1f.double()
    out["C1_f32_real_256x128"] = {
        "ms_per_svd": e0.elapsed_time(e1) / reps, "sweeps": info["sweeps"],
        "residual": (torch.linalg.norm(A1d - (U * sv) @ V.T) / torch.linalg.norm(A1d)).item(),
        "orth_U": (U.T @ U - I).abs().max().item(), "orth_V": (V.T @ V - I).abs().max().item(),
        "bound_64neps32": 64 * 128 * 2.0 ** -23}

    # f1: the same 256 x 128 with the compensated dot-products (Alg. ddpscl')
    r = J.svd(A1, compensated=True)
    torch.cuda.synchronize(dev)
    e0, e1 = _ev(torch)
    e0.record(st)
    for _ in range(reps):
        J.svd(A1, out=r, compensated=True)
    e1.record(st)
    torch.cuda.synchronize(dev)
    info = J.decode_info(r["info"])
    f1 = {"ms_per_svd": e0.elapsed_time(e1) / reps, "sweeps": info["sweeps"]}
    f1.update(accuracy(A1, r))
    out["f1_compensated_real_256x128"] = f1

    # f2: wide-exponent column norms (Alg. rnF) of a real 2^21 x 64 matrix
    # (1 GiB, read once): bytes per second against the HBM copy peak
    gen = torch.Generator(device=dev).manual_seed(3)
    Anorm = torch.randn(64, 1 << 21, dtype=torch.float64, device=dev, generator=gen).T
    J.colnorm_ef(Anorm)
    torch.cuda.synchronize(dev)
    e0, e1 = _ev(torch)
    e0.record(st)
    for _ in range(5):
        e_, f_ = J.colnorm_ef(Anorm)
    e1.record(st)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / 5
    nbytes = Anorm.numel() * 8
    ref = torch.linalg.norm(Anorm[:, :4], dim=0)
    got = torch.ldexp(f_[:4], e_[:4].to(torch.int64))
    out["f2_colnorm_ef_real_2p21x64"] = {
        "ms": ms, "gbs": nbytes / (ms * 1e-3) / 1e9,
        "max_rel_diff_vs_torch_norm": ((got - ref).abs() / ref).max().item()}
    del Anorm

    # f4: the 16 x 16 matrix of supplement SM9 (Gram-Schmidt steps, Eq. e:GS)
    G = torch.from_numpy(workloads.gram_schmidt_matrix(False)).to(dev)
    r = J.svd(G)
    torch.cuda.synchronize(dev)
    e0, e1 = _ev(torch)
    e0.record(st)
    for _ in range(reps):
        J.svd(G, out=r)
    e1.record(st)
    torch.cuda.synchronize(dev)
    info = J.decode_info(r["info"])
    out["f4_gram_schmidt_16x16"] = {"ms_per_svd": e0.elapsed_time(e1) / reps,
                                    "sweeps": info["sweeps"], "gs_steps": info["gs_steps"],
                                    "status": info["status"]}

    # C3: complex 4096 x 2048, cond 1e6, plain FP64 and mixed FP32 -> FP64
    A3np, s3 = workloads.svd_complex_geometric()
    A3 = torch.from_numpy(A3np).to(dev)
    from tests.golden import c3_fixture
    fx = c3_fixture.load()
    c3 = {}
    sig = {}
    for mode in ("fp64", "mixed"):
        e0, e1 = _ev(torch)
        torch.cuda.synchronize(dev)
        e0.record(st)
        r = J.svd(A3, mode=mode)
        e1.record(st)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        info = J.decode_info(r["info"])
        d = {"s": ms / 1e3, "sweeps_fp64": info["sweeps"], "sweeps_fp32": info["sweeps_fp32"],
             "rotations": info["rotations"], "status": info["status"]}
        d.update(accuracy(A3, r))
        sig[mode] = r["sigma"].cpu().numpy()
        d["sigma_err_vs_prescribed"] = float(np.abs(sig[mode] - s3).max() / s3[0])
        if fx is not None:
            cols = torch.from_numpy(fx["cols"]).to(dev)
            e = c3_fixture.errors(sig[mode], r["U"][:, cols].cpu().numpy(),
                                  r["V"][:, cols].cpu().numpy(), fx)
            e["input_bit_equal_to_oracle_run"] = c3_fixture.input_matches(A3np, fx)
            e["oracle"] = "tests/golden/c3_oracle_4096x2048.npz (the oracle's FP64 SVD, %d sweeps)" % int(fx["sweeps"])
            d["err_vs_oracle"] = e
        if mode == "fp64":
            fl = _svd_flops(4096, 2048, info["sweeps"], info["rotations"], True)
            lo = _svd_lane_ops(4096, 2048, info["sweeps"], info["rotations"], True)
            d["fp64_tflops"] = fl / (ms * 1e-3) / 1e12
            d["fp64_frac"] = fl / (ms * 1e-3) / DFMA_FLOPS
            d["fp64_pipe_frac"] = lo / (ms * 1e-3) / rates["fma_per_s"]
        c3[mode] = d
        del r
    c3["speedup_mixed_vs_fp64"] = c3["fp64"]["s"] / c3["mixed"]["s"]
    c3["sigma_mixed_vs_fp64_max_rel"] = float(np.abs(sig["mixed"] - sig["fp64"]).max() / s3[0])
    del A3
    if cpu:
        # the oracle's FP64 SVD on the same matrix: a bounded sample (the
        # first parallel steps of the first sweep, where every pair rotates),
        # extrapolated to the oracle's whole run (its sweeps x 2047 steps)
        try:
            full_steps = 2047 * int(fx["sweeps"] if fx is not None else c3["fp64"]["sweeps_fp64"])
            co = {"kind": "oracle", "full_run_steps": full_steps,
                  "sample": "the first K parallel steps of sweep 1 on the same matrix, scaled "
                            "to the full run's steps (later sweeps rotate fewer pairs, so an "
                            "upper estimate)"}
            for key, thr, K in (("all_cores", 0, 512), ("one_thread", 1, 24)):
                ms_o, thr_o, _, steps = cpu_oracle_svd(A3np, nthreads=thr, max_steps=K)
                est = ms_o / steps * full_steps / 1e3
                co[key] = {"threads": thr_o, "steps_timed": steps, "s_timed": ms_o / 1e3,
                           "s_per_step": ms_o / steps / 1e3, "s_full_svd_est": est,
                           "gpu_fp64_speedup_est": est / c3["fp64"]["s"],
                           "gpu_mixed_speedup_est": est / c3["mixed"]["s"]}
            if fx is not None:
                co["measured_full_run_elsewhere"] = {
                    "s": float(fx["seconds"]), "threads": int(fx["threads"]),
                    "where": "the run that wrote the stored oracle result (x86-64 host)"}
            c3["cpu_oracle"] = co
        except Exception as exc:
            c3["cpu_oracle"] = {"error": repr(exc)}
    del A3np
    out["C3_complex_4096x2048"] = c3

    # C4: 10,000 uneven real matrices, one persistent launch vs a per-matrix loop
    A4, m4, n4 = workloads.uneven_batch_device(device=dev)
    B = J.BatchedSVD(A4, m4, n4)
    e0, e1 = _ev(torch)
    torch.cuda.synchronize(dev)
    e0.record(st)
    B.launch()
    e1.record(st)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    infos = J.decode_info(B.info)
    fl = sum(_svd_flops(int(m4[i]), int(n4[i]), infos[i]["sweeps"], infos[i]["rotations"], False)
             for i in range(len(m4)))
    lo4 = sum(_svd_lane_ops(int(m4[i]), int(n4[i]), infos[i]["sweeps"], infos[i]["rotations"],
                            False) for i in range(len(m4)))
    # the per-matrix launch loop: jsvd_svd on each matrix of a random sample,
    # one after another on one stream, scaled to the batch by m n^2
    g = np.random.default_rng(0)
    idx = g.choice(len(m4), loop_count, replace=False) if loop_count < len(m4) else np.arange(len(m4))
    mat = lambda i: A4[int(B.offA[i]):int(B.offA[i] + m4[i] * n4[i])].view(int(n4[i]), int(m4[i])).t()
    J.svd(mat(idx[0]))
    torch.cuda.synchronize(dev)
    e2, e3 = _ev(torch)
    e2.record(st)
    for i in idx:
        J.svd(mat(i))
    e3.record(st)
    torch.cuda.synchronize(dev)
    cost = (m4 * n4 * n4).astype(float)
    loop_meas_s = e2.elapsed_time(e3) / 1e3
    loop_s = loop_meas_s * cost.sum() / cost[idx].sum()
    # the autotuner's choice (each candidate timed on the batch, 2 sweeps)
    import time as _time
    t0 = _time.perf_counter()
    times = B.autotune(use_cache=False)
    tune_s = _time.perf_counter() - t0
    e0, e1 = _ev(torch)
    torch.cuda.synchronize(dev)
    e0.record(st)
    B.launch()
    e1.record(st)
    torch.cuda.synchronize(dev)
    ms_tuned = e0.elapsed_time(e1)
    # the same batch as one captured CUDA graph, replayed (the launch with the
    # tuned warps captured once; each replay redoes the whole batch)
    gs = torch.cuda.Stream(dev)
    gs.wait_stream(st)
    with torch.cuda.stream(gs):
        B.launch(gs)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        B.launch(gs)
    torch.cuda.synchronize(dev)
    reps = 2
    e0, e1 = _ev(torch)
    e0.record(st)
    for _ in range(reps):
        graph.replay()
    e1.record(st)
    torch.cuda.synchronize(dev)
    ms_graph = e0.elapsed_time(e1) / reps
    infos_g = J.decode_info(B.info)
    c4 = {
        "s": ms / 1e3, "matrices_per_s": len(m4) / (ms * 1e-3),
        "autotuned": {"warps": B.warps, "s": ms_tuned / 1e3, "tuning_s": tune_s,
                      "two_sweep_ms": {str(k): v for k, v in times.items()}},
        "graph_replay": {"s": ms_graph / 1e3, "matrices_per_s": len(m4) / (ms_graph * 1e-3),
                         "replays_timed": reps, "warps": B.warps,
                         "converged": int(sum(1 for x in infos_g if x["status"] == 0))},
        "converged": int(sum(1 for x in infos if x["status"] == 0)),
        "sweeps_mean": float(np.mean([x["sweeps"] for x in infos])),
        "fp64_tflops": fl / (ms * 1e-3) / 1e12, "fp64_frac": fl / (ms * 1e-3) / DFMA_FLOPS,
        "fp64_pipe_frac": lo4 / (ms_graph * 1e-3) / rates["fma_per_s"],
        "per_matrix_loop": {"matrices_timed": int(len(idx)), "s_timed": loop_meas_s,
                            "s_full_batch": loop_s,
                            "scaled": bool(len(idx) < len(m4)),
                            "how": "jsvd_svd on each matrix in turn on one stream"
                                   + (", a random sample scaled to the batch by m n^2"
                                      if len(idx) < len(m4) else ", the whole batch")},
        "speedup_graph_vs_loop": loop_s / (ms_graph / 1e3)}
    if cpu:
        # the oracle over matrices of the same random sample, the OpenMP
        # threads sharing out the matrices, scaled to the batch by m n^2
        try:
            import oracle
            co = {"kind": "oracle", "sample": "matrices of the random sample above (all cores: "
                  "all of it, one thread: the first 8), scaled to the batch by m n^2"}
            for key, thr, k in (("all_cores", 0, len(idx)), ("one_thread", 1, 8)):
                sel = idx[:k]
                host = [mat(i).cpu().numpy() for i in sel]
                t0 = _time.perf_counter()
                sg, _, _, stt = oracle.vjsvd_batch(host, nthreads=thr)
                dt = _time.perf_counter() - t0
                est = dt * cost.sum() / cost[sel].sum()
                co[key] = {"threads": thr if thr else oracle.num_threads(),
                           "matrices_timed": int(k), "s_timed": dt, "s_full_batch_est": est,
                           "all_converged": all(x == 0 for x in stt),
                           "gpu_graph_speedup_est": est / (ms_graph / 1e3)}
            c4["cpu_oracle"] = co
        except Exception as exc:
            c4["cpu_oracle"] = {"error": repr(exc)}
    out["C4_uneven_10000"] = c4
    del A4, B, graph

    # C5: differentiated batch, 4096 real 64 x 32, loss sum w sigma + <C, U[:, :8]>
    A5, w5, C5 = workloads.diff_batch_device(device=dev)
    best = None
    for _ in range(3):
        X = A5.clone().requires_grad_(True)
        torch.cuda.synchronize(dev)
        e0, e1 = _ev(torch)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        U, S, V = J.svd_diff(X)
        L = (w5 * S).sum() + (C5 * U[:, :, :8]).sum()
        e2.record(st)
        L.backward()
        e1.record(st)
        torch.cuda.synchronize(dev)
        t = (e0.elapsed_time(e2), e0.elapsed_time(e1))
        best = t if best is None or t[1] < best[1] else best
    c5 = {"forward_ms": best[0], "forward_backward_ms": best[1],
          "matrices_per_s": 4096 / (best[1] * 1e-3)}
    if cpu:
        # the FP64 CPU reference of the same gradient: the oracle's SVD (the
        # threads sharing out the matrices), the sign gauge, the oracle's
        # adjoint; all 4096 matrices on all cores, 256 on one thread
        try:
            import oracle
            G5 = X.grad.cpu().numpy()
            A5h, w5h, C5h = A5.cpu().numpy(), w5.cpu().numpy(), C5.cpu().numpy()
            kk = C5h.shape[2]
            co = {"kind": "oracle", "sample": "all cores: the whole batch; one thread: the "
                  "first 1024 matrices, scaled by 4"}
            for key, thr, k in (("all_cores", 0, A5h.shape[0]), ("one_thread", 1, 1024)):
                t0 = time.perf_counter()
                sg, Us, Vs, stt = oracle.vjsvd_batch(list(A5h[:k]), nthreads=thr)
                g = [oracle.sign_gauge(u, v) for u, v in zip(Us, Vs)]
                U = np.stack([a for a, _ in g])
                V = np.stack([b for _, b in g])
                Ub = np.zeros_like(U)
                Ub[:, :, :kk] = C5h[:k]
                Gref = oracle.svd_adjoint_batch(U, np.stack(sg), V, Ub, w5h[:k], nthreads=thr)
                dt = time.perf_counter() - t0
                co[key] = {"threads": thr if thr else oracle.num_threads(), "matrices_timed": k,
                           "s_timed": dt, "s_full_batch_est": dt * A5h.shape[0] / k,
                           "all_converged": all(x == 0 for x in stt),
                           "gpu_speedup_est": dt * A5h.shape[0] / k / (best[1] * 1e-3)}
                if thr == 0:
                    err = (np.abs(G5[:k] - Gref).max(axis=(1, 2))
                           / np.maximum(np.abs(Gref).max(axis=(1, 2)), 1e-300))
                    c5["grad_err_vs_cpu_reference"] = {
                        "matrices": int(k), "max_rel": float(err.max()),
                        "median_rel": float(np.median(err)),
                        "above_1e-9": int((err > 1e-9).sum()),
                        "measure": "per matrix max|G - G_ref| / max|G_ref|"}
            c5["cpu_oracle"] = co
        except Exception as exc:
            c5["cpu_oracle"] = {"error": repr(exc)}
    out["C5_diff_4096x64x32"] = c5
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    r = 1 << 21  # a bounded sample of the workload per step (1/8 of each batch)
    for _ in range(args.warmup):
        cpu_oracle_evd(r)
    total, cores = 0.0, None
    for _ in range(args.steps):
        dt, cores = cpu_oracle_evd(r)
        total += dt
    value = 2 * r * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_per_step": "2^21 real + 2^21 complex"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "2^21 real + 2^21 complex matrices per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    global R_EVD
    R_EVD = 1 << args.evd_log2
    import numpy as np
    import torch

    import paper_2202_08361_gb300 as J
    from paper_2202_08361_gb300 import dist as D
    from paper_2202_08361_gb300 import workloads

    world, rank, local_rank = D.rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    # inputs resident in HBM before the timed region; each rank its own shard
    host_re = workloads.evd_batch(R_EVD, False, seed_salt=D.evd_seed_salt(rank))
    host_cx = workloads.evd_batch(R_EVD, True, seed_salt=D.evd_seed_salt(rank))
    d_re = [torch.from_numpy(a).to(dev) for a in host_re]
    d_cx = [torch.from_numpy(a).to(dev) for a in host_cx]
    out_re = J.evd2x2_batched(*d_re)
    out_cx = J.evd2x2_batched(*d_cx)
    torch.cuda.synchronize(dev)

    def step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        J.evd2x2_batched(*d_re, out=out_re, stream=stream)
        if evs is not None:
            evs[1].record(stream)
        J.evd2x2_batched(*d_cx, out=out_cx, stream=stream)
        if evs is not None:
            evs[2].record(stream)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)

    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(gpu_index(local_rank))
    clocks.start()
    time.sleep(0.25)
    barrier()
    torch.cuda.synchronize(dev)
    t_start.record(stream)
    for k in range(K):
        step(evs[k])
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    ms_total = t_start.elapsed_time(t_end)
    t_real = sum(e[0].elapsed_time(e[1]) for e in evs) / K
    t_cplx = sum(e[1].elapsed_time(e[2]) for e in evs) / K
    gpu_launches = 2 * K

    value, _, ms_total = D.aggregate_rate(2 * R_EVD * K, ms_total, dist, dev)
    ms_per_step = ms_total / K

    # end to end through the public API a user with host data calls:
    # jsvd_evd2x2_batched_host on pinned host streams, every step.  Pinned
    # streams are mapped, so the kernels read the inputs from and write the
    # outputs to host memory over the host link (the bytes counted below
    # cross it every step); the staged path (copies to a device workspace
    # in pipelined chunks, for unmapped buffers) is timed beside it
    pin = lambda a: torch.from_numpy(a).pin_memory()
    h_re = [pin(a) for a in host_re]
    h_cx = [pin(a) for a in host_cx]
    h_out_re = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in out_re.items()}
    h_out_cx = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in out_cx.items()}
    h2d = sum(t.numel() * t.element_size() for t in h_re + h_cx)
    d2h = sum(t.numel() * t.element_size() for t in list(h_out_re.values()) + list(h_out_cx.values()))
    work_host = torch.empty(J.evd2x2_host_workspace_size(), dtype=torch.uint8, device=dev)

    # the direct path: the real and the complex batch (independent) on two
    # streams, joined back to the timed stream every step (7.6 vs 7.9 ms
    # per step on one stream); the staged path on one stream (two streams
    # sharing the library's pipeline streams measured slower)
    side = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    # each side stream its own workspace (the direct path does not touch it;
    # the staged fallback for unmapped buffers would)
    work_side = [work_host, torch.empty_like(work_host)]

    def e2e_step(staged):
        if staged:
            J.evd2x2_batched_host(*h_re, out=h_out_re, work=work_host, stream=stream)
            J.evd2x2_batched_host(*h_cx, out=h_out_cx, work=work_host, stream=stream)
            return
        fork = torch.cuda.Event()
        fork.record(stream)
        for st, wk, (h, o) in zip(side, work_side, ((h_re, h_out_re), (h_cx, h_out_cx))):
            st.wait_event(fork)
            J.evd2x2_batched_host(*h, out=o, work=wk, stream=st)
            join = torch.cuda.Event()
            join.record(st)
            stream.wait_event(join)

    def e2e_time(staged):
        J.tune_set(J.JSVD_TUNE_EVD_HOST, 1 if staged else 0)
        try:
            for _ in range(2):
                e2e_step(staged)
            torch.cuda.synchronize(dev)
            E = max(args.e2e_steps, 1)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(E):
                e2e_step(staged)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            barrier()
        finally:
            J.tune_set(J.JSVD_TUNE_EVD_HOST, 0)
        return D.aggregate_rate(2 * R_EVD, e0.elapsed_time(e1) / E, dist, dev)

    e2e_value, _, e2e_ms = e2e_time(False)
    e2e_staged_value, _, e2e_staged_ms = e2e_time(True)

    peaks, peak_kind = measured_peaks()
    dom_name, dom_ms, dom_bytes = (("evd2_kernel<complex>", t_cplx, BYTES_CPLX * R_EVD)
                                   if t_cplx >= t_real else
                                   ("evd2_kernel<real>", t_real, BYTES_REAL * R_EVD))
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    traffic = recorded_traffic(dom_name)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": dom_name, "peak_kind": peak_kind,
                "pipes_active": recorded_pipes(dom_name),
                "algorithmic_bytes_per_launch": dom_bytes, "avg_launch_ms": dom_ms}

    # the pipe that binds the EVD: its FP64 work against the FP64 pipe's
    # throughput, measured now on this GPU
    rates = fp64_pipe_rates(torch, J, dev)
    roof_fp64 = {name: evd_fp64_roofline(name, t, R_EVD, rates)
                 for name, t in (("evd2_kernel<real>", t_real), ("evd2_kernel<complex>", t_cplx))}

    svd = None
    if rank == 0 and world == 1 and not args.no_svd:
        svd = svd_bench(torch, J, workloads, dev, rates, cpu=not args.no_cpu_baseline,
                        loop_count=args.c4_loop)
    evd32 = None
    if rank == 0 and world == 1:
        evd32 = evd_f32_bench(torch, J, workloads, dev, peaks)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, cores = cpu_oracle_evd(R_EVD)
        r1 = 1 << 21
        dt1, _ = cpu_oracle_evd_threads(r1, 1)
        cpu = {"value": 2 * R_EVD / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "the full step: 2^24 real + 2^24 complex matrices, once",
               "one_thread": {"value": 2 * r1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": "2^21 real + 2^21 complex matrices, once"},
               "omp": oracle_env()}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "matrices_per_step_per_gpu": 2 * R_EVD,
                           "bytes_per_step_per_gpu": (BYTES_REAL + BYTES_CPLX) * R_EVD,
                           "l2": "inputs larger than L2 (2.28 GB streamed per step), no flush",
                           "parallelism": "independent shards per GPU" if world > 1 else "1 GPU"},
                "roofline": roofline,
                "kernels_ms": {"evd2_kernel<real>": t_real, "evd2_kernel<complex>": t_cplx},
                "hbm_frac_step": (BYTES_REAL + BYTES_CPLX) * R_EVD / (ms_per_step * 1e-3) / 1e9
                / peaks["hbm_gbs"],
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                        "api": "jsvd_evd2x2_batched_host on pinned host streams (the kernel "
                               "reads and writes them in place over the host link), the real "
                               "and complex batches on two streams",
                        "staged": {"value": e2e_staged_value, "ms_per_step": e2e_staged_ms,
                                   "api": "the same call with JSVD_TUNE_EVD_HOST = 1 (copies "
                                          "to a device workspace in pipelined chunks)"}},
                "roofline_fp64_pipe": roof_fp64[dom_name],
                "roofline_fp64_pipe_other": roof_fp64[[k for k in roof_fp64 if k != dom_name][0]],
                "fp64_pipe_rates": rates,
                "cpu_baseline": cpu, "clocks": clk, "gpu_launches": gpu_launches,
                "evd_fp32": evd32, "svd": svd}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
