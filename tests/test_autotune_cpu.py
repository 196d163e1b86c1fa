"""Host logic of the batched-SVD autotuner: the shape signature and the
cache file (no GPU)."""
import json

import numpy as np

from paper_2202_08361_gb300 import autotune, workloads


def test_signature_is_a_cost_histogram():
    m, n = workloads.uneven_shapes(count=2000)
    sig = autotune.signature(m, n, False)
    field, comp, lg, hist = sig.split("|")
    assert (field, comp, lg) == ("r", "comp0", "lg10")
    share = [int(x) for x in hist.split(",")]
    assert sum(share) in (19, 20, 21)          # 5 % steps, rounded
    assert share[7] > share[4]                 # the cost sits in the large n
    assert autotune.signature(m, n, True, True).startswith("c|comp1|")
    # a batch of 64 x 32: all the cost in the octave of 32
    s2 = autotune.signature(np.full(4096, 64), np.full(4096, 32), False)
    assert s2.split("|")[3].split(",")[5] == "20"


def test_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("JSVD_TUNE_CACHE", str(path))
    assert autotune._load() == {}
    autotune._store({"GPU|r|comp0|lg3|x": 4})
    assert json.loads(path.read_text()) == {"GPU|r|comp0|lg3|x": 4}
    assert autotune._load() == {"GPU|r|comp0|lg3|x": 4}
