"""Launch-shape autotuner for the batched SVD (arithmetic-neutral knobs only:
no choice here changes a result bit).

tune_batched() times the batched kernel on the whole batch with each
candidate number of warps per block, every run capped at a couple of
sweeps (the persistent kernel's occupancy and load balance are those of the
real run; a subset of the matrices would not fill the GPU the same way),
and returns the fastest.  Choices are cached in a JSON file
(JSVD_TUNE_CACHE, else ~/.cache/jsvd/tune.json) under the device name, the
field, the option set and a signature of the batch's cost distribution over
log2 n.  Without tuning, the library's own rule (JSVD_TUNE_BATCH_WARPS = 0)
applies.
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


def tune_batched(B, *, candidates=CANDIDATES, sweeps=2, use_cache=True, stream=None):
    """The fastest warps per block for the prepared BatchedSVD B.  Returns
    (warps, {warps: ms for `sweeps` sweeps}); the timings are empty when the
    choice came from the cache.  B's outputs are overwritten (a later
    launch recomputes them)."""
    import torch

    import paper_2202_08361_gb300 as J
    from paper_2202_08361_gb300 import _native
    key = "%s|%s" % (torch.cuda.get_device_name(B.A.device),
                     signature(B.m, B.n, B.cplx, bool(B.opts.compensated)))
    table = _load() if use_cache else {}
    if key in table:
        return int(table[key]), {}
    st = stream if stream is not None else torch.cuda.current_stream(B.A.device)
    saved = B.opts.max_sweeps
    times = {}
    try:
        B.opts.max_sweeps = int(sweeps)
        for w in candidates:
            J.tune_set(J.JSVD_TUNE_BATCH_WARPS, int(w))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            rc = _native.lib().jsvd_svd_batched_launch(B.field, J._opts_ref(B.opts), B.count,
                                                       B.work.data_ptr(), B.info.data_ptr(),
                                                       J._stream_handle(st))
            _native.check(rc, "jsvd_svd_batched_launch")
            e1.record(st)
            e1.synchronize()
            times[int(w)] = e0.elapsed_time(e1)
    finally:
        B.opts.max_sweeps = saved
        J.tune_set(J.JSVD_TUNE_BATCH_WARPS, 0)
    best = min(times, key=times.get)
    if use_cache:
        table = _load()
        table[key] = best
        _store(table)
    return best, times
