"""arc_trace_noalloc: the trace entry point that allocates no device memory.

It serves host codes that cannot allocate when they trace: simulation
frameworks that give the whole GPU memory to their own pool allocator at
start-up, where a library's cudaMalloc finds nothing or is not allowed, and
that cannot let a library call cudaFree (which waits for the whole device)
inside their step loop.  Its scratch is a fixed file-scope device array, so it
must give the same rates as arc_trace (the context path, which allocates its
buffers) and must give them again on a second call, since the array keeps the
previous call's contents.  The device's free memory must not change across a
call: the library makes no allocation that torch's allocator would not see.

This file is collected last so that a run stopping at the first failure has
run every other test before it.
"""
import numpy as np
import pytest
import torch

import paper_1807_07094_gb300 as P
from paper_1807_07094_gb300 import arc as A
import workloads as W
from helpers import GAMMA_FLOOR, GAMMA_RTOL, gpu_trace, partly_ionised

pytestmark = pytest.mark.gpu


def _cases():
    w1 = W.stromgren_32()
    w2 = W.cosmic(n=48, nsrc=8, sigma_ln=1.5, seed=4)
    x2 = partly_ionised(w2, seed=8, lo=-4, hi=0)
    return [(w1, (w1.xHI, w1.xHeI, w1.xHeII)), (w2, x2)]


def _close(got, ref):
    for s in range(3):
        r = ref[s]
        if r.max() <= 0:
            assert np.all(got[s] == 0)
            continue
        m = r > GAMMA_FLOOR * r.max()
        assert np.max(np.abs(got[s][m] - r[m]) / r[m]) <= GAMMA_RTOL


@pytest.mark.parametrize("case", [0, 1])
def test_noalloc_matches_context_trace_on_two_calls(case):
    w, xs = _cases()[case]
    ref = gpu_trace(w, *xs)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    fields = [dev(w.nH), dev(xs[0]), dev(xs[1]), dev(xs[2])]
    grid = A.ArcGrid(w.n, w.box_cm)
    params = A.make_params(w.params())
    for call in range(2):
        gamma = torch.full((3, w.n, w.n, w.n), -1.0, dtype=torch.float32, device="cuda")
        heat = torch.full((3, w.n, w.n, w.n), -1.0, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        budget = A.arc_trace_noalloc(grid, params, *fields, w.src_pos, w.src_ndot, gamma, heat,
                                     stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        if call == 1:
            # no cudaMalloc / cudaMallocAsync inside the call: torch's caching
            # allocator cannot see libarc's allocations, the driver's free count
            # can.  (The first call may load the library's device code, and with
            # it the static scratch array, so it is not the one measured.)
            assert torch.cuda.mem_get_info()[0] == free0
        launched, absorbed, escaped, emitted = budget
        assert abs(launched - absorbed - escaped) <= 1e-9 * launched
        assert np.allclose(budget, ref["budget"], rtol=1e-6)
        _close(gamma.cpu().numpy().astype(np.float64), ref["gamma"])
        _close(heat.cpu().numpy().astype(np.float64), ref["heat"])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    w = W.stromgren_32(n=72)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    fields = [dev(w.nH), dev(w.xHI), dev(w.xHeI), dev(w.xHeII)]
    out = torch.zeros((3, 72, 72, 72), dtype=torch.float32, device="cuda")
    with pytest.raises(A.ArcError) as e:
        A.arc_trace_noalloc(A.ArcGrid(72, w.box_cm), A.make_params(w.params()), *fields,
                            w.src_pos, w.src_ndot, out, out.clone())
    assert e.value.status == A.ARC_E_INVALID
    assert "ARC_NOALLOC_MAX_N" in str(e.value)
