"""Thin Python binding of libarc (include/arc.h).

Argument marshalling only: every step of the tracer and the chemistry runs in
the CUDA kernels of libarc.so.  There is no CPU fallback: if the library is
missing or fails to load, every call raises.  PyTorch is used only to hold
device memory and to name the CUDA stream.

Functions keep the C names (arc_create, arc_set_fields, arc_add_sources,
arc_trace, arc_chem_update, arc_step, arc_get_fields, arc_stats, ...).
"""
from __future__ import annotations

import ctypes as C
import json
import os
from typing import Optional

import numpy as np

from . import build as _build

MAX_GROUPS = 4
MAX_LEVEL = 15

ARC_OK, ARC_E_INVALID, ARC_E_OOM, ARC_E_CUDA, ARC_E_TIMEOUT, ARC_E_BUDGET, ARC_E_STATE, \
    ARC_E_OVERFLOW, ARC_E_SUBSTEP = range(9)
STATUS_NAMES = ["ARC_OK", "ARC_E_INVALID", "ARC_E_OOM", "ARC_E_CUDA", "ARC_E_TIMEOUT",
                "ARC_E_BUDGET", "ARC_E_STATE", "ARC_E_OVERFLOW", "ARC_E_SUBSTEP"]
END_SPLIT, END_ESCAPE, END_TERM = 1, 2, 3


class ArcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class ArcGrid(C.Structure):
    _fields_ = [("n", C.c_int), ("box_cm", C.c_double)]


class ArcParams(C.Structure):
    _fields_ = [
        ("ngroups", C.c_int), ("E_group_eV", C.c_double * MAX_GROUPS),
        ("sigma", (C.c_double * MAX_GROUPS) * 3), ("Y", C.c_double), ("phi", C.c_double),
        ("l_base", C.c_int), ("l_max", C.c_int), ("term_frac", C.c_double),
        ("eps_sub", C.c_double), ("x_fp64", C.c_double), ("isothermal", C.c_int),
        ("alpha_B_fixed", C.c_double), ("coll_ion", C.c_int), ("z_compton", C.c_double),
        ("geo_correction", C.c_int), ("thin_approx", C.c_int),
    ]


class ArcStats(C.Structure):
    _fields_ = [
        ("segments", C.c_uint64), ("rays", C.c_uint64), ("splits", C.c_uint64),
        ("terminated", C.c_uint64), ("escaped_rays", C.c_uint64), ("donations", C.c_uint64),
        ("max_level", C.c_uint32), ("error_word", C.c_uint32), ("chem_substeps", C.c_uint64),
        ("chem_fp64_substeps", C.c_uint64), ("chem_capped", C.c_uint64),
        ("trace_ms", C.c_double), ("chem_ms", C.c_double), ("segments_total", C.c_uint64),
        ("traces_total", C.c_uint64), ("surrogate_cells", C.c_uint64), ("fallback_cells", C.c_uint64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


REC_DTYPE = np.dtype([("src", "<u4"), ("level", "u1"), ("end", "u1"), ("pad", "<u2"),
                      ("pix", "<u8"), ("visits", "<u4"), ("r1", "<f4")], align=True)
assert REC_DTYPE.itemsize == 24

_lib = None

# every exported entry point of include/arc.h with its ctypes signature
_SIGS = {
    "arc_create": ([C.POINTER(C.c_void_p), C.POINTER(ArcGrid), C.POINTER(ArcParams), C.c_void_p], C.c_int),
    "arc_set_fields": ([C.c_void_p] + [C.c_void_p] * 5 + [C.c_int], C.c_int),
    "arc_add_sources": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "arc_clear_sources": ([C.c_void_p], C.c_int),
    "arc_trace": ([C.c_void_p, C.c_double, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                   C.POINTER(C.c_double)], C.c_int),
    "arc_chem_update": ([C.c_void_p, C.c_double], C.c_int),
    "arc_step": ([C.c_void_p, C.c_double], C.c_int),
    "arc_get_fields": ([C.c_void_p] + [C.c_void_p] * 4 + [C.c_int], C.c_int),
    "arc_set_records": ([C.c_void_p, C.c_void_p, C.c_int64], C.c_int),
    "arc_get_record_count": ([C.c_void_p, C.POINTER(C.c_int64)], C.c_int),
    "arc_stats": ([C.c_void_p, C.POINTER(ArcStats)], C.c_int),
    "arc_set_tuning": ([C.c_void_p, C.c_int, C.c_int, C.c_int], C.c_int),
    "arc_get_tuning": ([C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "arc_autotune": ([C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_double)], C.c_int),
    "arc_last_error": ([C.c_void_p], C.c_char_p),
    "arc_trace_noalloc": ([C.POINTER(ArcGrid), C.POINTER(ArcParams)] + [C.c_void_p] * 4 +
                          [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.POINTER(C.c_double), C.c_void_p], C.c_int),
    "arc_destroy": ([C.c_void_p], None),
    "arc_set_surrogate": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_double], C.c_int),
    "arc_mlp_trainer_create": ([C.POINTER(C.c_void_p), C.c_int, C.c_void_p], C.c_int),
    "arc_mlp_trainer_set_params": ([C.c_void_p, C.c_void_p], C.c_int),
    "arc_mlp_trainer_get_params": ([C.c_void_p, C.c_void_p], C.c_int),
    "arc_mlp_grad": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_double)], C.c_int),
    "arc_mlp_train_step": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double,
                            C.POINTER(C.c_double)], C.c_int),
    "arc_mlp_trainer_destroy": ([C.c_void_p], None),
    "arc_mlp_eval": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p, C.c_void_p], C.c_int),
    "arc_mlp_features": ([C.c_void_p] * 7 + [C.c_double, C.c_longlong, C.c_void_p, C.c_void_p], C.c_int),
    "arc_rt_timestep": ([C.c_void_p, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "arc_mlp_targets": ([C.c_void_p] * 8 + [C.c_double, C.c_longlong, C.c_void_p], C.c_int),
    "arc_set_emission_mask": ([C.c_void_p, C.c_void_p, C.c_int64], C.c_int),
    "arc_set_thin_radii": ([C.c_void_p, C.c_void_p, C.c_int], C.c_int),
    "arc_get_thin_radii": ([C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_double)], C.c_int),
    "arc_set_fault": ([C.c_void_p, C.c_int64, C.c_double], C.c_int),
}

MLP_NPARAMS = 9412
MLP_NNORM = 36


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libarc.so (building it first if asked).  Raises if it cannot."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise RuntimeError(f"libarc is not built ({path}); run paper_1807_07094_gb300.build")
            _build.build()
        L = C.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(ctx, status):
    if status != ARC_OK:
        msg = load().arc_last_error(ctx).decode() if ctx else "arc_create failed"
        raise ArcError(status, msg)


def make_params(d: dict) -> ArcParams:
    p = ArcParams()
    p.ngroups = int(d["ngroups"])
    for b in range(MAX_GROUPS):
        p.E_group_eV[b] = float(d["E_group_eV"][b]) if b < p.ngroups else 0.0
        for s in range(3):
            p.sigma[s][b] = float(d["sigma"][s][b]) if b < p.ngroups else 0.0
    for k in ("Y", "phi", "term_frac", "eps_sub", "x_fp64", "alpha_B_fixed", "z_compton"):
        setattr(p, k, float(d[k]))
    for k in ("l_base", "l_max", "isothermal", "coll_ion"):
        setattr(p, k, int(d[k]))
    p.geo_correction = int(d.get("geo_corr", 0))
    p.thin_approx = int(d.get("thin_approx", 0))
    return p


def _ptr_and_kind(a):
    """(address, on_device) of a float32 contiguous torch tensor or numpy array."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float32 or not a.is_contiguous():
                raise ValueError("fields must be contiguous float32")
            return a.data_ptr(), 1 if a.is_cuda else 0
    except ImportError:
        pass
    a = np.asarray(a)
    if a.dtype != np.float32 or not a.flags.c_contiguous:
        raise ValueError("fields must be contiguous float32")
    return a.ctypes.data, 0


def current_stream_handle() -> int:
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


class _DevView:
    """__cuda_array_interface__ over a device pointer owned by the context."""

    def __init__(self, ptr: int, shape, typestr="<f4"):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def device_view(ptr: int, shape, dtype="float32"):
    """Zero-copy torch view of a context-owned device buffer."""
    import torch
    ts = {"float32": "<f4"}[dtype]
    return torch.as_tensor(_DevView(ptr, shape, ts), device="cuda")


# ----------------------------------------------------------------- C names
def arc_create(grid: ArcGrid, params: ArcParams, stream: Optional[int] = None) -> int:
    L = load()
    h = C.c_void_p()
    st = L.arc_create(C.byref(h), C.byref(grid), C.byref(params), C.c_void_p(stream or 0))
    _check(None, st)
    return h.value


def arc_destroy(ctx: int) -> None:
    load().arc_destroy(C.c_void_p(ctx))


def arc_set_fields(ctx, nH, xHI, xHeI, xHeII, T) -> None:
    ptrs = [_ptr_and_kind(a) for a in (nH, xHI, xHeI, xHeII, T)]
    kinds = {k for _, k in ptrs}
    if len(kinds) != 1:
        raise ValueError("fields must all be host or all be device arrays")
    _check(ctx, load().arc_set_fields(C.c_void_p(ctx), *[C.c_void_p(p) for p, _ in ptrs], kinds.pop()))


def arc_add_sources(ctx, pos, ndot, ngroups: Optional[int] = None) -> None:
    """pos [nsrc, 3] FP64 grid units, ndot nsrc * ngroups photons/s; give
    ngroups (the context's) to have the size of ndot checked."""
    pos, ndot = _check_sources(pos, ndot, ngroups)
    _check(ctx, load().arc_add_sources(C.c_void_p(ctx), pos.shape[0], pos.ctypes.data, ndot.ctypes.data))


def arc_clear_sources(ctx) -> None:
    _check(ctx, load().arc_clear_sources(C.c_void_p(ctx)))


def arc_trace(ctx, dt: float, budget: bool = True):
    """Returns (gamma_ptr, heat_ptr, budget[4] or None)."""
    g = C.c_void_p()
    h = C.c_void_p()
    b = (C.c_double * 4)() if budget else None
    _check(ctx, load().arc_trace(C.c_void_p(ctx), float(dt), C.byref(g), C.byref(h), b))
    return g.value, h.value, (np.array(list(b)) if budget else None)


def arc_chem_update(ctx, dt: float) -> None:
    _check(ctx, load().arc_chem_update(C.c_void_p(ctx), float(dt)))


def arc_step(ctx, dt: float) -> None:
    _check(ctx, load().arc_step(C.c_void_p(ctx), float(dt)))


def arc_get_fields(ctx, xHI=None, xHeI=None, xHeII=None, T=None) -> None:
    outs = [xHI, xHeI, xHeII, T]
    kinds = set()
    ptrs = []
    for o in outs:
        if o is None:
            ptrs.append(None)
            continue
        p, k = _ptr_and_kind(o)
        kinds.add(k)
        ptrs.append(p)
    if len(kinds) > 1:
        raise ValueError("outputs must all be host or all be device arrays")
    _check(ctx, load().arc_get_fields(C.c_void_p(ctx), *[C.c_void_p(p) if p else None for p in ptrs],
                                      kinds.pop() if kinds else 0))


def arc_set_records(ctx, buf_ptr: int, cap: int) -> None:
    _check(ctx, load().arc_set_records(C.c_void_p(ctx), C.c_void_p(buf_ptr or 0), int(cap)))


def arc_get_record_count(ctx) -> int:
    n = C.c_int64()
    _check(ctx, load().arc_get_record_count(C.c_void_p(ctx), C.byref(n)))
    return int(n.value)


def arc_stats(ctx) -> dict:
    s = ArcStats()
    _check(ctx, load().arc_stats(C.c_void_p(ctx), C.byref(s)))
    return s.as_dict()


def arc_set_tuning(ctx, block_threads=0, blocks_per_sm=0, stack_entries=0) -> None:
    _check(ctx, load().arc_set_tuning(C.c_void_p(ctx), int(block_threads), int(blocks_per_sm),
                                      int(stack_entries)))


NOALLOC_MAX_N = 64
NOALLOC_MAX_SOURCES = 256


def _numel(a) -> int:
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return int(a.numel())
    except ImportError:
        pass
    return int(np.asarray(a).size)


def _check_sources(pos, ndot, ngroups: Optional[int]):
    """pos as [nsrc, 3] FP64 and ndot as nsrc * ngroups FP64 (the C side reads
    exactly that many values and cannot see the arrays' sizes)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    if pos.size % 3 != 0 or (pos.ndim == 2 and pos.shape[1] != 3):
        raise ValueError("source positions must be [nsrc, 3]")
    pos = pos.reshape(-1, 3)
    ndot = np.ascontiguousarray(ndot, dtype=np.float64).reshape(-1)
    if ngroups is not None and ndot.size != pos.shape[0] * int(ngroups):
        raise ValueError(f"ndot must hold nsrc * ngroups = {pos.shape[0]} * {int(ngroups)} values, "
                         f"got {ndot.size}")
    return pos, ndot


def arc_trace_noalloc(grid: ArcGrid, params: ArcParams, nH, xHI, xHeI, xHeII, pos, ndot, gamma, heat,
                      stream: Optional[int] = None):
    """One trace into caller-owned device buffers with no allocation (see
    include/arc.h).  Fields (n^3 each) and outputs (3 n^3 each) are contiguous
    float32 CUDA tensors; returns the budget[4].  Every size is checked here,
    before any launch: the C interface receives bare pointers."""
    n = int(grid.n)
    pos, ndot = _check_sources(pos, ndot, params.ngroups)
    ptrs = []
    for name, a, size in (("nH", nH, n ** 3), ("xHI", xHI, n ** 3), ("xHeI", xHeI, n ** 3),
                          ("xHeII", xHeII, n ** 3), ("gamma", gamma, 3 * n ** 3),
                          ("heat", heat, 3 * n ** 3)):
        p, on_dev = _ptr_and_kind(a)
        if not on_dev:
            raise ValueError("arc_trace_noalloc takes device arrays")
        if _numel(a) != size:
            raise ValueError(f"{name} must hold {size} float32 values for n = {n}, got {_numel(a)}")
        ptrs.append(p)
    b = (C.c_double * 4)()
    st = load().arc_trace_noalloc(C.byref(grid), C.byref(params), *[C.c_void_p(q) for q in ptrs[:4]],
                                  pos.shape[0], pos.ctypes.data, ndot.ctypes.data,
                                  C.c_void_p(ptrs[4]), C.c_void_p(ptrs[5]), b, C.c_void_p(stream or 0))
    if st == ARC_E_INVALID:
        raise ArcError(st, "arc_trace_noalloc refused its arguments (n=%d, %d sources; its fixed "
                       "scratch allows n <= ARC_NOALLOC_MAX_N=%d, sources <= "
                       "ARC_NOALLOC_MAX_SOURCES=%d, l_base <= 2, no thin approximation; positions "
                       "inside the box, finite non-negative luminosities)"
                       % (n, pos.shape[0], NOALLOC_MAX_N, NOALLOC_MAX_SOURCES))
    if st != ARC_OK:
        what = {ARC_E_CUDA: "a CUDA call failed",
                ARC_E_TIMEOUT: "the tracer's bounded wait for work ran out",
                ARC_E_OVERFLOW: "the work queue overflowed",
                ARC_E_BUDGET: "the photon budget did not close to 1e-9"}.get(st, "the trace failed")
        raise ArcError(st, f"arc_trace_noalloc: {what} (n={n}, {pos.shape[0]} sources)")
    return np.array(list(b))


def arc_get_tuning(ctx):
    v = [C.c_int(), C.c_int(), C.c_int()]
    _check(ctx, load().arc_get_tuning(C.c_void_p(ctx), *[C.byref(x) for x in v]))
    return tuple(x.value for x in v)


def arc_autotune(ctx, max_sources: int = 0, reps: int = 1) -> float:
    best = C.c_double()
    _check(ctx, load().arc_autotune(C.c_void_p(ctx), int(max_sources), int(reps), C.byref(best)))
    return best.value


def _f32_host(a, size):
    a = np.ascontiguousarray(a, dtype=np.float32).reshape(-1)
    if a.size != size:
        raise ValueError(f"expected {size} float32 values, got {a.size}")
    return a


def _dev(a):
    p, on_dev = _ptr_and_kind(a)
    if not on_dev:
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return p


def arc_set_surrogate(ctx, params=None, norm=None, tol_x: float = 5e-4, tol_e: float = 1e-2,
                      gate: float = 0.0) -> None:
    if params is None:
        _check(ctx, load().arc_set_surrogate(C.c_void_p(ctx), None, None, 0.0, 0.0, 0.0))
        return
    p = _f32_host(params, MLP_NPARAMS)
    q = _f32_host(norm, MLP_NNORM)
    _check(ctx, load().arc_set_surrogate(C.c_void_p(ctx), p.ctypes.data, q.ctypes.data, float(tol_x), float(tol_e),
                                         float(gate)))


def _mlp_check(st, what):
    if st != ARC_OK:
        raise ArcError(st, what)


class MlpTrainer:
    """GPU trainer of the chemistry surrogate (BF16 tensor-core forward and
    backward passes, FP32 AdamW)."""

    def __init__(self, max_batch: int, stream: Optional[int] = None):
        h = C.c_void_p()
        _mlp_check(load().arc_mlp_trainer_create(C.byref(h), int(max_batch), C.c_void_p(stream or 0)),
                   "arc_mlp_trainer_create")
        self.h = h.value

    def close(self):
        if self.h:
            load().arc_mlp_trainer_destroy(C.c_void_p(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = _f32_host(params, MLP_NPARAMS)
        _mlp_check(load().arc_mlp_trainer_set_params(C.c_void_p(self.h), p.ctypes.data), "set_params")

    def get_params(self) -> np.ndarray:
        p = np.empty(MLP_NPARAMS, np.float32)
        _mlp_check(load().arc_mlp_trainer_get_params(C.c_void_p(self.h), p.ctypes.data), "get_params")
        return p

    def grad(self, X, Y, n: int):
        g = np.empty(MLP_NPARAMS, np.float32)
        loss = C.c_double()
        _mlp_check(load().arc_mlp_grad(C.c_void_p(self.h), C.c_void_p(_dev(X)), C.c_void_p(_dev(Y)), int(n),
                                       g.ctypes.data, C.byref(loss)), "arc_mlp_grad")
        return g, loss.value

    def step(self, X, Y, n: int, lr: float, wd: float = 0.0, want_loss: bool = False):
        loss = C.c_double()
        _mlp_check(load().arc_mlp_train_step(C.c_void_p(self.h), C.c_void_p(_dev(X)), C.c_void_p(_dev(Y)), int(n),
                                             float(lr), float(wd), C.byref(loss) if want_loss else None),
                   "arc_mlp_train_step")
        return loss.value if want_loss else None


def arc_mlp_eval(params, norm, X, Y, stream: Optional[int] = None) -> None:
    p = _f32_host(params, MLP_NPARAMS)
    q = _f32_host(norm, MLP_NNORM)
    n = X.shape[0]
    _mlp_check(load().arc_mlp_eval(p.ctypes.data, q.ctypes.data, C.c_void_p(_dev(X)), n, C.c_void_p(_dev(Y)),
                                   C.c_void_p(stream or 0)), "arc_mlp_eval")


def arc_mlp_features(nH, xHI, xHeI, xHeII, T, gamma, heat, dt: float, X, stream: Optional[int] = None) -> None:
    n = nH.numel()
    _mlp_check(load().arc_mlp_features(*[C.c_void_p(_dev(a)) for a in (nH, xHI, xHeI, xHeII, T, gamma, heat)],
                                       float(dt), n, C.c_void_p(_dev(X)), C.c_void_p(stream or 0)),
               "arc_mlp_features")


def arc_mlp_targets(ctx, nH, x0, T0, gamma, heat, x1, T1, dt: float, Y) -> None:
    """Training targets (corrections to the physics predictor) of n cells;
    runs on the context's stream and synchronises."""
    n = T0.numel()
    _check(ctx, load().arc_mlp_targets(C.c_void_p(ctx), *[C.c_void_p(_dev(a)) for a in (nH, x0, T0, gamma, heat, x1, T1)],
                                       float(dt), n, C.c_void_p(_dev(Y))))


SURROGATE_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "surrogate_cosmic.npz")


def load_surrogate(path: Optional[str] = None):
    """Trained surrogate weights: (params [ARC_MLP_NPARAMS], norm [ARC_MLP_NNORM], meta dict)."""
    d = np.load(path or SURROGATE_FILE)
    params = np.ascontiguousarray(d["params"], np.float32)
    norm = np.ascontiguousarray(d["norm"], np.float32)
    if params.size != MLP_NPARAMS or norm.size != MLP_NNORM:
        raise ValueError("surrogate file does not match the network's shape")
    return params, norm, json.loads(str(d["meta"]))


def arc_last_error(ctx) -> str:
    return load().arc_last_error(C.c_void_p(ctx)).decode()


# ----------------------------------------------------------------- convenience
class Arc:
    """Context owner: ``with Arc(n, box_cm, params_dict) as a: ...``."""

    def __init__(self, n: int, box_cm: float, params: dict, stream: Optional[int] = None):
        self.n = int(n)
        self.ngroups = int(params["ngroups"])
        g = ArcGrid(self.n, float(box_cm))
        self.ctx = arc_create(g, make_params(params), stream)

    def close(self):
        if self.ctx:
            arc_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, nH, xHI, xHeI, xHeII, T):
        for name, a in (("nH", nH), ("xHI", xHI), ("xHeI", xHeI), ("xHeII", xHeII), ("T", T)):
            if _numel(a) != self.n ** 3:
                raise ValueError(f"{name} must hold n^3 = {self.n ** 3} values, got {_numel(a)}")
        arc_set_fields(self.ctx, nH, xHI, xHeI, xHeII, T)

    def add_sources(self, pos, ndot):
        arc_add_sources(self.ctx, pos, ndot, self.ngroups)

    def clear_sources(self):
        arc_clear_sources(self.ctx)

    def trace(self, dt: float = 1.0, budget: bool = True):
        """Returns (gamma, heat) as zero-copy torch views [3,n,n,n] and the budget.

        The rates are written on the context's CUDA stream; with budget=False
        the call does not wait for them, so synchronise that stream (or the
        device) before reading the views from another stream."""
        g, h, b = arc_trace(self.ctx, dt, budget)
        sh = (3, self.n, self.n, self.n)
        return device_view(g, sh), device_view(h, sh), b

    def chem(self, dt: float):
        arc_chem_update(self.ctx, dt)

    def step(self, dt: float):
        arc_step(self.ctx, dt)

    def get_fields(self):
        n3 = (self.n,) * 3
        out = [np.empty(n3, np.float32) for _ in range(4)]
        arc_get_fields(self.ctx, *out)
        return out

    def stats(self) -> dict:
        return arc_stats(self.ctx)

    def set_records(self, buf, cap: int):
        arc_set_records(self.ctx, buf, cap)

    def record_count(self) -> int:
        return arc_get_record_count(self.ctx)

    def set_tuning(self, block_threads=0, blocks_per_sm=0, stack_entries=0):
        arc_set_tuning(self.ctx, block_threads, blocks_per_sm, stack_entries)

    def get_tuning(self):
        return arc_get_tuning(self.ctx)

    def autotune(self, max_sources: int = 0, reps: int = 1) -> float:
        return arc_autotune(self.ctx, max_sources, reps)

    def set_surrogate(self, params=None, norm=None, tol_x: float = 5e-4, tol_e: float = 1e-2, gate: float = 0.0):
        arc_set_surrogate(self.ctx, params, norm, tol_x, tol_e, gate)

    def rt_timestep(self, eps: float = 0.1):
        """(dt_n, dt_I) [s] of Sec. 2.9 from the current state and the last trace."""
        a, b = C.c_double(), C.c_double()
        _check(self.ctx, load().arc_rt_timestep(C.c_void_p(self.ctx), float(eps), C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_emission_mask(self, open_mask=None):
        """Anisotropic escape (Sec. 2.2): open_mask [nsrc, 12*4^l_base] booleans
        in the order sources were added (False blocks that emitted ray); None
        removes the mask."""
        if open_mask is None:
            _check(self.ctx, load().arc_set_emission_mask(C.c_void_p(self.ctx), None, 0))
            return
        m = np.ascontiguousarray(np.asarray(open_mask, dtype=np.uint8).reshape(-1))
        _check(self.ctx, load().arc_set_emission_mask(C.c_void_p(self.ctx), m.ctypes.data, m.size))

    def set_fault(self, live_bias: int = 0, idle_timeout_s: float = 10.0):
        """Failure-detection test aid: phantom unfinished rays and the idle-wait bound."""
        _check(self.ctx, load().arc_set_fault(C.c_void_p(self.ctx), int(live_bias), float(idle_timeout_s)))

    def set_thin_radii(self, radii):
        """Optically thin radius per source [cells] (Sec. 2.6, thin_approx)."""
        r = np.ascontiguousarray(np.asarray(radii, dtype=np.float64).reshape(-1))
        _check(self.ctx, load().arc_set_thin_radii(C.c_void_p(self.ctx), r.ctypes.data, r.size))

    def thin_radii(self, nsrc: int):
        """(radii [nsrc] the last trace measured, photons of its thin fill over dt)."""
        r = np.zeros(nsrc)
        t = C.c_double()
        _check(self.ctx, load().arc_get_thin_radii(C.c_void_p(self.ctx), r.ctypes.data, nsrc, C.byref(t)))
        return r, t.value

    def mlp_targets(self, nH, x0, T0, gamma, heat, x1, T1, dt: float, Y):
        arc_mlp_targets(self.ctx, nH, x0, T0, gamma, heat, x1, T1, dt, Y)
