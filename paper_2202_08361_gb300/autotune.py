"""Launch-shape autotuner for the batched SVD (arithmetic-neutral knobs only:
no choice here changes a result bit).

tune_batched() times the batched kernel with each candidate number of warps
per block on a stratified sample of the batch (every k-th matrix in the
order of cost m n^2, so the sample has the batch's mix of sizes) and
returns the fastest.  Choices are cached in a JSON file (JSVD_TUNE_CACHE,
else ~/.cache/jsvd/tune.json) under the device name, the field, the option
set and a signature of the batch's cost distribution over log2 n.  Without
tuning, the library's own rule (JSVD_TUNE_BATCH_WARPS = 0) applies.
"""
import json
import os

import numpy as np

CANDIDATES = (1, 2, 4, 8, 16)


def signature(m, n, cplx, compensated=False):
    """Field, options, log2 of the count and the share of the sweep cost
    (m n^2) in each octave of n, in 5 % steps."""
    m = np.asarray(m, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    octave = np.clip(np.floor(np.log2(np.maximum(n, 1))).astype(int), 0, 20)
    cost = np.bincount(octave, weights=m * n * n, minlength=21)
    share = np.round(cost / max(cost.sum(), 1.0) * 20).astype(int)
    return "%s|comp%d|lg%d|%s" % ("c" if cplx else "r", int(bool(compensated)),
                                  int(np.log2(max(len(n), 1))), ",".join(map(str, share)))


def cache_path():
    return os.environ.get("JSVD_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "jsvd", "tune.json")


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(table):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home: the choice is still returned


def sample_indices(m, n, size):
    """Every k-th matrix in the order of decreasing m n^2 (at most `size`)."""
    m = np.asarray(m, dtype=np.int64)
    n = np.asarray(n, dtype=np.int64)
    order = np.argsort(-(m * n * n), kind="stable")
    k = max(1, int(np.ceil(len(order) / max(size, 1))))
    return np.sort(order[::k])


def tune_batched(A, m, n, *, compensated=False, candidates=CANDIDATES, sample=1024,
                 use_cache=True, stream=None):
    """The fastest warps per block for the batch (A packed as for
    BatchedSVD).  Returns (warps, {warps: ms on the sample}); the timings
    are empty when the choice came from the cache."""
    import torch

    import paper_2202_08361_gb300 as J
    cplx = A.dtype == torch.complex128
    m = np.asarray(m, dtype=np.int64)
    n = np.asarray(n, dtype=np.int64)
    dev = A.device
    key = "%s|%s" % (torch.cuda.get_device_name(dev), signature(m, n, cplx, compensated))
    table = _load() if use_cache else {}
    if key in table:
        return int(table[key]), {}
    idx = sample_indices(m, n, sample)
    off = np.concatenate([[0], np.cumsum(m * n)[:-1]]) if len(m) else np.zeros(0, np.int64)
    As = torch.cat([A[int(off[i]):int(off[i]) + int(m[i] * n[i])] for i in idx])
    B = J.BatchedSVD(As, m[idx], n[idx], compensated=compensated)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    times = {}
    try:
        for w in candidates:
            J.tune_set(J.JSVD_TUNE_BATCH_WARPS, int(w))
            B.launch(st)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            B.launch(st)
            e1.record(st)
            e1.synchronize()
            times[int(w)] = e0.elapsed_time(e1)
    finally:
        J.tune_set(J.JSVD_TUNE_BATCH_WARPS, 0)
    best = min(times, key=times.get)
    if use_cache:
        table = _load()
        table[key] = best
        _store(table)
    return best, times
