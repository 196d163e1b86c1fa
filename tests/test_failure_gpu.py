"""Failure detection without a GPU fault: the persistent SVD kernel's grid
barrier is a bounded wait.  Here one block of a cooperative launch never
arrives (a flag that nothing sets), the others give up after a short limit
and report JSVD_E_TIMEOUT through device memory, and the context stays
usable for the next call."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(blocks, absent, rounds, limit_ns):
    import torch
    from paper_2202_08361_gb300 import _native
    st = torch.full((2,), -7, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = _native.lib().jsvd_selftest_barrier(blocks, absent, rounds, limit_ns, st.data_ptr(), None)
    torch.cuda.synchronize()
    return rc, st.cpu().tolist(), time.perf_counter() - t0


def test_wait_runs_out_and_reports_timeout():
    import paper_2202_08361_gb300 as J
    rc, st, dt = _run(8, 3, 5, 200_000_000)  # 0.2 s limit
    assert rc == 0
    assert st[0] == J.JSVD_E_TIMEOUT and st[1] == 0
    assert 0.2 <= dt < 5.0


def test_all_blocks_present_complete():
    import paper_2202_08361_gb300 as J
    rc, st, dt = _run(16, -1, 50, 1_000_000_000)
    assert rc == 0 and st == [J.JSVD_OK, 16 * 50]
    assert dt < 1.0


def test_context_usable_after_timeout():
    import torch
    import paper_2202_08361_gb300 as J
    from paper_2202_08361_gb300 import workloads
    rc, st, _ = _run(4, 0, 1, 100_000_000)
    assert rc == 0 and st[0] == J.JSVD_E_TIMEOUT
    A = workloads.svd_normal(64, 32)
    out = J.svd(torch.from_numpy(A).cuda())
    torch.cuda.synchronize()
    assert J.decode_info(out["info"])["status"] == 0
    s = out["sigma"].cpu().numpy()
    assert np.allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-12)


def test_argument_checks():
    from paper_2202_08361_gb300 import _native
    L = _native.lib()
    assert L.jsvd_selftest_barrier(0, -1, 1, 10**8, None, None) == -1
    assert L.jsvd_selftest_barrier(2, -1, 0, 10**8, None, None) == -3
    assert L.jsvd_selftest_barrier(2, -1, 1, 10, None, None) == -4
    assert L.jsvd_selftest_barrier(2, -1, 1, 10**8, None, None) == -5
