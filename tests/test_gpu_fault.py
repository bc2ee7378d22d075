"""Failure detection without a GPU fault: the tracer's idle wait is bounded.

The host adds phantom unfinished rays (arc_set_fault), so the tracer's count of
live rays never reaches zero and its warps, once out of work, wait for work that
never comes.  With a 0.2 s bound the wait runs out, the kernel sets its timeout
status and returns; the trace reports ARC_E_TIMEOUT, and the same context then
traces normally again."""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_idle_wait_runs_out_and_the_context_recovers():
    import paper_1807_07094_gb300 as P
    w = W.stromgren_32()
    with P.Arc(w.n, w.box_cm, w.params()) as a:
        a.set_fields(w.nH, w.xHI, w.xHeI, w.xHeII, w.T)
        a.add_sources(w.src_pos, w.src_ndot)
        g0, _, b0 = a.trace(1.0)
        g0 = g0.cpu().numpy().copy()
        a.set_fault(live_bias=1, idle_timeout_s=0.2)
        t = time.time()
        with pytest.raises(P.ArcError) as e:
            a.trace(1.0)
        assert e.value.status == P.arc.ARC_E_TIMEOUT
        assert time.time() - t < 30.0
        assert a.stats()["error_word"] & 1            # the kernel's timeout bit
        a.set_fault(0, 10.0)
        g1, _, b1 = a.trace(1.0)
        assert np.array_equal(g1.cpu().numpy(), g0)   # all rays were traced both times
        assert abs(b1[0] - b1[1] - b1[2]) <= 1e-9 * b1[0]
