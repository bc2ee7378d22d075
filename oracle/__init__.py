"""FP64 CPU oracle for the ARC tracer and chemistry (ctypes binding).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the benchmark's ``cpu_baseline`` / reference leg may import this package.  It
shares no code with the CUDA path (``paper_1807_07094_gb300``) and neither
imports the other; both read inputs from ``workloads``.

The arithmetic lives in ``arc_oracle.c`` (plain C, FP64, single thread); this
module only compiles it with gcc, loads it and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "arc_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liborc.so")

MAXG = 4
END_SPLIT, END_ESCAPE, END_TERM, END_BLOCKED = 1, 2, 3, 4


class OrcParams(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("box_cm", C.c_double), ("ngroups", C.c_int),
        ("E_group_eV", C.c_double * MAXG), ("sigma", (C.c_double * MAXG) * 3),
        ("Y", C.c_double), ("phi", C.c_double), ("l_base", C.c_int), ("l_max", C.c_int),
        ("term_frac", C.c_double), ("eps_sub", C.c_double), ("x_fp64", C.c_double),
        ("isothermal", C.c_int), ("alpha_B_fixed", C.c_double), ("coll_ion", C.c_int),
        ("z_compton", C.c_double), ("geo_corr", C.c_int),
    ]


class OrcTraceOpts(C.Structure):
    _fields_ = [("corr_margin", C.c_void_p), ("r_start", C.c_void_p), ("r_thin_out", C.c_void_p),
                ("thin_photons", C.c_void_p), ("open", C.c_void_p)]


REC_DTYPE = np.dtype([("src", "<u4"), ("level", "<i4"), ("pix", "<u8"), ("visits", "<i4"),
                      ("end", "<i4"), ("r0", "<f8"), ("r1", "<f8"), ("geo_margin", "<f8"),
                      ("term_margin", "<f8"), ("exit_margin", "<f8")], align=True)


def build(force: bool = False) -> str:
    """Compile liborc.so with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "arc_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


class use_library:
    """Temporarily route every oracle call to another build of arc_oracle.c
    (used by the mutation tests, which plant a mistake in a copy)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = None
        lib(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def build_variant(src_text: str, out_dir: str) -> str:
    """Compile a modified copy of the oracle source into out_dir."""
    c = os.path.join(out_dir, "arc_oracle.c")
    with open(c, "w") as f:
        f.write(src_text)
    import shutil
    shutil.copy(os.path.join(_HERE, "arc_oracle.h"), out_dir)
    so = os.path.join(out_dir, "liborc_variant.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", so, c, "-lm"])
    return so


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def lib(path: Optional[str] = None):
    global _lib
    if _lib is None:
        if path is None:
            path = build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.orc_pix2vec_nest.argtypes = [C.c_int, C.c_uint64, dp]
        L.orc_vec2pix_nest.argtypes = [C.c_int, dp]
        L.orc_vec2pix_nest.restype = C.c_uint64
        L.orc_r_split.argtypes = [C.POINTER(OrcParams), C.c_int]
        L.orc_r_split.restype = C.c_double
        L.orc_trace.argtypes = [C.POINTER(OrcParams), dp, dp, dp, dp, C.c_int, dp, dp, dp, dp, dp,
                                C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.orc_trace.restype = C.c_int
        L.orc_trace_ex.argtypes = L.orc_trace.argtypes + [C.c_void_p]
        L.orc_trace_ex.restype = C.c_int
        L.orc_trace_opt.argtypes = L.orc_trace.argtypes + [C.POINTER(OrcTraceOpts)]
        L.orc_trace_opt.restype = C.c_int
        L.orc_chem.argtypes = [C.POINTER(OrcParams), C.c_int64, dp, dp, dp, dp, dp, dp, dp,
                               C.c_double, C.POINTER(C.c_int64)]
        L.orc_chem.restype = C.c_int
        L.orc_chem_refined.argtypes = [C.POINTER(OrcParams), C.c_int64, dp, dp, dp, dp, dp, dp, dp,
                                       C.c_double, C.c_int, C.POINTER(C.c_int64)]
        L.orc_chem_refined.restype = C.c_int
        L.orc_rates.argtypes = [C.POINTER(OrcParams), C.c_double, dp]
        L.orc_rt_timestep.argtypes = [C.POINTER(OrcParams), C.c_int64, dp, dp, dp, dp, dp, dp, C.c_double, dp]
        L.orc_rt_timestep.restype = None
        L.orc_cooling.argtypes = [C.POINTER(OrcParams), C.c_double, C.c_double, C.c_double,
                                  C.c_double, C.c_double, C.c_double]
        L.orc_cooling.restype = C.c_double
        L.orc_cooling_terms.argtypes = L.orc_cooling.argtypes + [dp]
        L.orc_cooling_terms.restype = None
        _lib = L
    return _lib


def make_params(d: dict) -> OrcParams:
    p = OrcParams()
    p.n = int(d["n"])
    p.box_cm = float(d["box_cm"])
    p.ngroups = int(d["ngroups"])
    for b in range(MAXG):
        p.E_group_eV[b] = float(d["E_group_eV"][b]) if b < p.ngroups else 0.0
        for s in range(3):
            p.sigma[s][b] = float(d["sigma"][s][b]) if b < p.ngroups else 0.0
    for k in ("Y", "phi", "term_frac", "eps_sub", "x_fp64", "alpha_B_fixed", "z_compton"):
        setattr(p, k, float(d[k]))
    for k in ("l_base", "l_max", "isothermal", "coll_ion"):
        setattr(p, k, int(d[k]))
    p.geo_corr = int(d.get("geo_corr", 0))
    return p


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def pix2vec(level: int, pix: int) -> np.ndarray:
    v = np.zeros(3)
    lib().orc_pix2vec_nest(level, pix, _dptr(v))
    return v


def vec2pix(level: int, v) -> int:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return int(lib().orc_vec2pix_nest(level, _dptr(v)))


def r_split(params: dict, level: int) -> float:
    p = make_params(params)
    return lib().orc_r_split(C.byref(p), level)


def trace(params: dict, nH, xHI, xHeI, xHeII, src_pos, src_ndot, records: bool = False,
          rec_cap: int = 1 << 22, corr_margin: bool = False, r_start=None, open_mask=None):
    """One RT pass.  Returns dict(gamma[3,n,n,n], heat[3,n,n,n], budget[3],
    nseg, nrec, recs (structured array or None), corr_margin, r_thin[nsrc],
    thin_photons).

    r_start: per-source optically thin radius [cells] (Sec. 2.6): the thin
    fill inside it and rays launched at it.  open_mask: [nsrc, 12*4^l_base]
    booleans, False blocks that emitted ray (Sec. 2.2).  r_thin is always the
    next thin radius measured by this pass."""
    p = make_params(params)
    n = p.n
    f = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    nH, xHI, xHeI, xHeII = f(nH), f(xHI), f(xHeI), f(xHeII)
    pos = f(src_pos)
    ndot = f(src_ndot)
    nsrc = pos.size // 3
    gamma = np.zeros(3 * n ** 3)
    heat = np.zeros(3 * n ** 3)
    budget = np.zeros(3)
    nrec = C.c_int64(0)
    nseg = C.c_int64(0)
    recs = np.zeros(rec_cap if records else 0, dtype=REC_DTYPE)
    cm = np.zeros(n ** 3 if corr_margin else 0)
    r_thin = np.zeros(nsrc)
    thin = np.zeros(1)
    o = OrcTraceOpts()
    o.corr_margin = cm.ctypes.data if corr_margin else None
    o.r_thin_out = r_thin.ctypes.data
    o.thin_photons = thin.ctypes.data
    if r_start is not None:
        rs = f(r_start)
        assert rs.size == nsrc
        o.r_start = rs.ctypes.data
    if open_mask is not None:
        om = np.ascontiguousarray(np.asarray(open_mask, dtype=np.uint8).reshape(-1))
        assert om.size == nsrc * 12 * 4 ** p.l_base
        o.open = om.ctypes.data
    rc = lib().orc_trace_opt(C.byref(p), _dptr(nH), _dptr(xHI), _dptr(xHeI), _dptr(xHeII), nsrc,
                             _dptr(pos), _dptr(ndot), _dptr(gamma), _dptr(heat), _dptr(budget),
                             recs.ctypes.data if records else None, rec_cap if records else 0,
                             C.byref(nrec), C.byref(nseg), C.byref(o))
    if rc == -2:
        raise RuntimeError(f"oracle record buffer too small: {nrec.value} > {rec_cap}")
    if rc != 0:
        raise ValueError(f"orc_trace failed ({rc})")
    return dict(gamma=gamma.reshape(3, n, n, n), heat=heat.reshape(3, n, n, n), budget=budget,
                nseg=int(nseg.value), nrec=int(nrec.value),
                recs=recs[: nrec.value] if records else None,
                corr_margin=cm.reshape(n, n, n) if corr_margin else None,
                r_thin=r_thin, thin_photons=float(thin[0]))


def chem(params: dict, nH, xHI, xHeI, xHeII, T, gamma, heat, dt: float, min_sub: int = 0):
    """Chemistry over dt; returns (xHI, xHeI, xHeII, T, nsub, capped) as float64.
    min_sub > 0 also caps every sub-step at dt / min_sub (orc_chem_refined)."""
    p = make_params(params)
    f = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1)).copy()
    nH = f(nH)
    xHI, xHeI, xHeII, T = f(xHI), f(xHeI), f(xHeII), f(T)
    g = f(gamma)
    h = f(heat)
    ncell = nH.size
    assert g.size == 3 * ncell and h.size == 3 * ncell
    nsub = C.c_int64(0)
    if min_sub > 0:
        capped = lib().orc_chem_refined(C.byref(p), ncell, _dptr(nH), _dptr(xHI), _dptr(xHeI), _dptr(xHeII),
                                        _dptr(T), _dptr(g), _dptr(h), float(dt), int(min_sub), C.byref(nsub))
    else:
        capped = lib().orc_chem(C.byref(p), ncell, _dptr(nH), _dptr(xHI), _dptr(xHeI), _dptr(xHeII),
                                _dptr(T), _dptr(g), _dptr(h), float(dt), C.byref(nsub))
    return xHI, xHeI, xHeII, T, int(nsub.value), int(capped)


def rt_timestep(params: dict, nH, xHI, xHeI, xHeII, T, gamma_HI, eps: float):
    """Sec. 2.9: (min dt_n over cells with n_HI sigma d > 0.5, min dt_I) [s]."""
    p = make_params(params)
    f = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    nH, xHI, xHeI, xHeII, T, g = f(nH), f(xHI), f(xHeI), f(xHeII), f(T), f(gamma_HI)
    out = np.zeros(2)
    lib().orc_rt_timestep(C.byref(p), nH.size, _dptr(nH), _dptr(xHI), _dptr(xHeI), _dptr(xHeII), _dptr(T),
                          _dptr(g), float(eps), _dptr(out))
    return float(out[0]), float(out[1])


def rates(params: dict, T: float) -> np.ndarray:
    p = make_params(params)
    out = np.zeros(6)
    lib().orc_rates(C.byref(p), float(T), _dptr(out))
    return out


def cooling(params: dict, T, nH, nHI, nHeI, nHeII, ne) -> float:
    p = make_params(params)
    return float(lib().orc_cooling(C.byref(p), T, nH, nHI, nHeI, nHeII, ne))


COOLING_TERMS = ("ci_HI", "ci_HeI", "ci_HeII", "rec_HII", "rec_HeII", "rec_HeIII", "diel_HeII",
                 "exc_HI", "exc_HeII", "ff", "compton")


def cooling_terms(params: dict, T, nH, nHI, nHeI, nHeII, ne) -> dict:
    """The cooling rate's terms one by one [erg/s/cm^3], named as COOLING_TERMS."""
    p = make_params(params)
    out = np.zeros(len(COOLING_TERMS))
    lib().orc_cooling_terms(C.byref(p), T, nH, nHI, nHeI, nHeII, ne, _dptr(out))
    return dict(zip(COOLING_TERMS, out.tolist()))


def run(params: dict, w, nsteps: int, trace_every: int = 1):
    """Free-running oracle: trace + chemistry per step.  Returns final fields."""
    xHI, xHeI, xHeII, T = (np.asarray(a, np.float64).reshape(-1).copy()
                           for a in (w.xHI, w.xHeI, w.xHeII, w.T))
    hist = []
    for k in range(nsteps):
        tr = trace(params, w.nH, xHI, xHeI, xHeII, w.src_pos, w.src_ndot)
        xHI, xHeI, xHeII, T, nsub, capped = chem(params, w.nH, xHI, xHeI, xHeII, T,
                                                 tr["gamma"], tr["heat"], w.dt_s)
        hist.append(dict(budget=tr["budget"], nseg=tr["nseg"], nsub=nsub))
    n = w.n
    sh = (n, n, n)
    return xHI.reshape(sh), xHeI.reshape(sh), xHeII.reshape(sh), T.reshape(sh), hist
