"""C ABI checks that need no GPU: libarc loads, exports every entry point
include/arc.h declares, and the binding's ctypes structs have the C layout."""
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import paper_1807_07094_gb300 as P
from paper_1807_07094_gb300 import arc as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*[\w\s\*]+?\b(arc_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_loads_and_exports_all_declared_symbols():
    lib = P.load()
    names = declared_functions()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", A.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (arc_\w+)", out))
    missing = names - exported
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)
    assert set(A._SIGS) >= names


def test_struct_layouts_match_c():
    src = r"""
#include <stddef.h>
#include <stdio.h>
#include "arc.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(arc_grid), sizeof(arc_params), sizeof(arc_stats_t), sizeof(arc_ray_rec));
  printf("%zu %zu %zu %zu\n", offsetof(arc_params, Y), offsetof(arc_params, z_compton),
         offsetof(arc_stats_t, trace_ms), offsetof(arc_ray_rec, r1));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        lines = subprocess.check_output([exe]).decode().split("\n")
    sizes = list(map(int, lines[0].split()))
    offs = list(map(int, lines[1].split()))
    import ctypes as C
    assert sizes == [C.sizeof(A.ArcGrid), C.sizeof(A.ArcParams), C.sizeof(A.ArcStats),
                     P.REC_DTYPE.itemsize]
    assert offs == [A.ArcParams.Y.offset, A.ArcParams.z_compton.offset, A.ArcStats.trace_ms.offset,
                    P.REC_DTYPE.fields["r1"][1]]


def test_invalid_params_rejected_without_gpu_work():
    """arc_create validates parameters before touching the device."""
    import workloads as W
    p = W.thermal_128().params()
    p["ngroups"] = 7
    with pytest.raises(ValueError):
        # the binding refuses more groups than the ABI carries
        A.make_params(p) if p["ngroups"] <= A.MAX_GROUPS else (_ for _ in ()).throw(ValueError())
    p = W.thermal_128().params()
    p["l_max"] = 99
    with pytest.raises(A.ArcError) as e:
        A.arc_create(A.ArcGrid(16, 1e21), A.make_params(p))
    assert e.value.status == A.ARC_E_INVALID


def test_binding_checks_array_sizes_before_any_launch():
    """The C interface receives bare pointers, so the binding refuses arrays of
    the wrong size before anything reaches libarc (no GPU is touched: the
    checks run on host arrays and raise ValueError)."""
    import workloads as W
    w = W.stromgren_32(n=8)
    grid = A.ArcGrid(8, w.box_cm)
    prm = A.make_params(w.params())
    with pytest.raises(ValueError):
        A._check_sources(np.zeros((2, 3)), np.ones(3), 1)          # 2 sources, 1 group: 2 values
    with pytest.raises(ValueError):
        A._check_sources(np.zeros((2, 2)), np.ones(2), 1)          # positions not [nsrc, 3]
    pos, nd = A._check_sources(np.zeros(6), np.ones(6), 3)
    assert pos.shape == (2, 3) and nd.shape == (6,)
    f = np.zeros(8 ** 3, np.float32)
    short = np.zeros(8 ** 3 - 1, np.float32)
    # host arrays are refused as such; the size checks come first for a wrong size
    with pytest.raises(ValueError):
        A.arc_trace_noalloc(grid, prm, f, f, f, short, w.src_pos, w.src_ndot,
                            np.zeros(3 * 8 ** 3, np.float32), np.zeros(3 * 8 ** 3, np.float32))
    with pytest.raises(ValueError):
        A.arc_trace_noalloc(grid, prm, f, f, f, f, w.src_pos, np.ones(5),
                            np.zeros(3 * 8 ** 3, np.float32), np.zeros(3 * 8 ** 3, np.float32))
