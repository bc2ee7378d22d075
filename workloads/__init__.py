"""Seeded synthetic inputs for the ARC tracer and chemistry.

This module is shared by the CUDA path's callers (tests, bench) and by the
FP64 oracle's callers.  It holds no arithmetic of the method itself (no ray
tracing, absorption, rate deposition or chemistry): only the workload
recipes -- grids, gas states, source lists -- and the physical input data the
method takes as given, namely the per-group photon-weighted cross sections
and mean energies of a blackbody spectrum (ARC treats each frequency bin as
one frequency carrying a frequency-averaged cross section, Sec. 2.2).

Every generator takes an explicit seed and uses numpy's PCG64.

Workloads (sizes and gas states follow the RT06 tests the paper runs,
Sec. 3, and the 256^3 / 512^3 cosmic-field stand-ins):

* ``stromgren_32``      -- isothermal pure-H Stromgren sphere, 32^3, 1 source.
* ``thermal_128``       -- H+He, 1e5 K blackbody in 3 groups, 128^3, corner source.
* ``cosmic_256``        -- 256^3 lognormal field (sigma_ln 1.5), 1000 sources.
* ``cosmic_512``        -- 512^3 lognormal field (sigma_ln 2.0), 10000 sources.

The cosmic fields stand in for the RT06 Test 4 density grid and halo list,
which are not available: a Gaussian field with P(k) ~ k^-3 is exponentiated
into a lognormal density with the stated mean; sources sit in cells drawn
with probability ~ n_H^2.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

# --- physical constants (CGS) ---------------------------------------------
K_B = 1.380649e-16          # erg/K
EV = 1.602176634e-12        # erg
KPC = 3.0856775814913673e21 # cm
MYR = 3.15576e13            # s (Julian)

# ionisation thresholds [eV] of HI, HeI, HeII (group edges use the same)
E_THRESH = (13.6, 24.6, 54.4)

# Photoionisation cross sections, Osterbrock & Ferland (2006) Table 2.4 fit:
#   sigma(nu) = a_T [beta (nu/nu_T)^-s + (1 - beta) (nu/nu_T)^(-s-1)],  nu >= nu_T
OSTERBROCK_FIT = {
    # species: (E_T [eV], a_T [cm^2], beta, s)
    "HI":   (13.6, 6.30e-18, 1.34, 2.99),
    "HeI":  (24.6, 7.83e-18, 1.66, 2.05),
    "HeII": (54.4, 1.58e-18, 1.34, 2.99),
}
SPECIES = ("HI", "HeI", "HeII")


def cross_section(species: str, e_ev):
    """Photoionisation cross section [cm^2] at photon energy e_ev [eV]."""
    et, a_t, beta, s = OSTERBROCK_FIT[species]
    e = np.asarray(e_ev, dtype=np.float64)
    r = e / et
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        sig = a_t * (beta * r ** (-s) + (1.0 - beta) * r ** (-s - 1.0))
    return np.where(e >= et, sig, 0.0)


def blackbody_groups(t_bb: float = 1.0e5, edges_ev=(13.6, 24.6, 54.4, 544.0),
                     nquad: int = 20000) -> Dict[str, np.ndarray]:
    """Photon-number fractions, mean energies and photon-weighted cross
    sections of a Planck spectrum of temperature ``t_bb`` split into groups.

    Returns dict with ``frac`` [G], ``E`` [G] (eV, energy per photon),
    ``sigma`` [3, G] (cm^2, photon-number weighted, rows HI/HeI/HeII).
    The integrals use composite Simpson quadrature in x = h nu / k T.
    """
    kt_ev = K_B * t_bb / EV
    g = len(edges_ev) - 1
    frac = np.zeros(g)
    emean = np.zeros(g)
    sig = np.zeros((3, g))
    totals = []
    for b in range(g):
        lo, hi = edges_ev[b], edges_ev[b + 1]
        e = np.linspace(lo, hi, nquad + 1)
        e[-1] = hi * (1.0 - 1e-12)          # the group is [lo, hi): the next edge is excluded
        x = e / kt_ev
        nphot = x * x / np.expm1(x)          # photons per unit x (Planck)
        w = np.ones(nquad + 1)
        w[1:-1:2] = 4.0
        w[2:-1:2] = 2.0
        w *= (x[1] - x[0]) / 3.0
        n_b = np.sum(w * nphot)
        totals.append(n_b)
        emean[b] = np.sum(w * nphot * e) / n_b
        for s, sp in enumerate(SPECIES):
            sig[s, b] = np.sum(w * nphot * cross_section(sp, e)) / n_b
    totals = np.array(totals)
    frac = totals / totals.sum()
    return {"frac": frac, "E": emean, "sigma": sig}


@dataclasses.dataclass
class Workload:
    """One synthetic problem: grid, gas, sources, physics switches."""
    name: str
    n: int
    box_cm: float
    Y: float
    ngroups: int
    E_group_eV: np.ndarray          # [G]
    sigma: np.ndarray               # [3, G]
    nH: np.ndarray                  # [n,n,n] float32, C order (i,j,k), k fastest
    xHI: np.ndarray
    xHeI: np.ndarray
    xHeII: np.ndarray
    T: np.ndarray
    src_pos: np.ndarray             # [S,3] float64, grid units (multiples of 2^-12)
    src_ndot: np.ndarray            # [S,G] float64, photons/s per group
    dt_s: float
    nsteps: int
    phi: float = 4.0
    l_base: int = 1
    l_max: int = 14
    term_frac: float = 1e-6
    eps_sub: float = 0.1
    x_fp64: float = 1e-4
    isothermal: int = 0
    alpha_B_fixed: float = 0.0      # > 0: constant case-B recombination coefficient
    coll_ion: int = 1
    z_compton: float = -1.0         # < 0 disables Compton cooling
    seed: int = 0

    def params(self) -> dict:
        """Scalar parameters, in the order both libraries' structs list them."""
        return dict(n=self.n, box_cm=self.box_cm, ngroups=self.ngroups,
                    E_group_eV=list(self.E_group_eV), sigma=[list(r) for r in self.sigma],
                    Y=self.Y, phi=self.phi, l_base=self.l_base, l_max=self.l_max,
                    term_frac=self.term_frac, eps_sub=self.eps_sub, x_fp64=self.x_fp64,
                    isothermal=self.isothermal, alpha_B_fixed=self.alpha_B_fixed,
                    coll_ion=self.coll_ion, z_compton=self.z_compton)

    @property
    def ncell(self) -> int:
        return self.n ** 3

    @property
    def nsrc(self) -> int:
        return int(self.src_pos.shape[0])


def quantise_pos(p):
    """Round positions to multiples of 2^-12 cell so FP32 holds them exactly."""
    return np.round(np.asarray(p, dtype=np.float64) * 4096.0) / 4096.0


def _uniform_gas(n, nH, xHI, xHeI, xHeII, T):
    shape = (n, n, n)
    f = lambda v: np.full(shape, v, dtype=np.float32)
    return f(nH), f(xHI), f(xHeI), f(xHeII), f(T)


def stromgren_32(seed: int = 0, n: int = 32) -> Workload:
    """Isothermal pure-H Stromgren test (RT06 Test 1 scaled to R_s ~ 10 cells)."""
    nH, xHI, xHeI, xHeII, T = _uniform_gas(n, 1e-2, 1.0 - 1e-4, 0.0, 0.0, 1e4)
    sig = np.zeros((3, 1))
    sig[0, 0] = 6.30e-18
    c = n / 2 + 0.5
    return Workload(name=f"stromgren_{n}", n=n, box_cm=2.2 * KPC * n / 32, Y=0.0, ngroups=1,
                    E_group_eV=np.array([13.6]), sigma=sig,
                    nH=nH, xHI=xHI, xHeI=xHeI, xHeII=xHeII, T=T,
                    src_pos=np.array([[c, c, c]]), src_ndot=np.array([[1e48]]),
                    dt_s=1.0 * MYR, nsteps=50, isothermal=1, alpha_B_fixed=2.59e-13,
                    coll_ion=0, z_compton=-1.0, seed=seed)


def thermal_128(seed: int = 0, n: int = 128, box_kpc: float = 6.6) -> Workload:
    """H+He, 1e5 K blackbody in 3 groups, source at the corner cell centre."""
    grp = blackbody_groups(1e5)
    x0 = 1.2e-3
    nH, xHI, xHeI, xHeII, T = _uniform_gas(n, 1e-3, 1.0 - x0, 1.0 - x0, x0, 100.0)
    ndot = 5e48 * grp["frac"]
    return Workload(name=f"thermal_{n}", n=n, box_cm=box_kpc * KPC, Y=0.24, ngroups=3,
                    E_group_eV=grp["E"], sigma=grp["sigma"],
                    nH=nH, xHI=xHI, xHeI=xHeI, xHeII=xHeII, T=T,
                    src_pos=np.array([[0.5, 0.5, 0.5]]), src_ndot=ndot[None, :],
                    dt_s=0.5 * MYR, nsteps=100, z_compton=9.0, seed=seed)


def clump_test3(n: int = 128, box_kpc: float = 6.6, dt_myr: float = 0.05, t_end_myr: float = 15.0) -> Workload:
    """The paper's Test 3 (Sec. 3.4, after RT06): a dense hydrogen clump
    (n = 0.04, 40 K, radius 0.8 kpc, centred at (97, 64, 64) of 128 cells) in
    thin gas (n = 2e-4, 8000 K) of a 6.6 kpc box, lit by one point source of
    3e51 photons/s opposite the clump (1e5 K blackbody in 3 groups).  The
    source sits at the centre of the cell at (0, 64, 64) (0.87-cell shift);
    pure hydrogen, no Compton term; 15 Myr.  At other n the geometry scales."""
    grp = blackbody_groups(1e5)
    s = n / 128.0
    c = np.indices((n, n, n)).transpose(1, 2, 3, 0) + 0.5
    centre = np.array([97.0, 64.0, 64.0]) * s
    R = 0.8 / box_kpc * n
    inside = ((c - centre) ** 2).sum(-1) < R * R
    nH = np.where(inside, 0.04, 2e-4).astype(np.float32)
    T = np.where(inside, 40.0, 8000.0).astype(np.float32)
    x0 = 1.2e-3
    xHI = np.full((n, n, n), 1.0 - x0, np.float32)
    z = np.zeros((n, n, n), np.float32)
    src = np.array([[0.5, 64.5 * s, 64.5 * s]])
    return Workload(name=f"clump_test3_{n}", n=n, box_cm=box_kpc * KPC, Y=0.0, ngroups=3,
                    E_group_eV=grp["E"], sigma=grp["sigma"], nH=nH, xHI=xHI, xHeI=z.copy(), xHeII=z.copy(),
                    T=T, src_pos=src, src_ndot=(3e51 * grp["frac"])[None, :], dt_s=dt_myr * MYR,
                    nsteps=int(round(t_end_myr / dt_myr)), z_compton=-1.0, seed=0)


def gaussian_field_k3(n: int, rng: np.random.Generator) -> np.ndarray:
    """Unit-variance Gaussian random field with P(k) ~ k^-3 (k != 0, |k_i| <= n/2)."""
    w = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(w)
    kx = np.fft.fftfreq(n) * n
    kz = np.fft.rfftfreq(n) * n
    k2 = kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (-0.75)                  # |k|^{-3/2}
    d = np.fft.irfftn(wk * amp, s=(n, n, n), axes=(0, 1, 2))
    d -= d.mean()
    d /= d.std()
    return d


def cosmic_field(n: int, sigma_ln: float, mean_nH: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    d = gaussian_field_k3(n, rng)
    rho = np.exp(sigma_ln * d - 0.5 * sigma_ln ** 2)
    rho *= mean_nH / rho.mean()
    return rho.astype(np.float32)


def place_sources(nH: np.ndarray, nsrc: int, ndot_lo: float, ndot_hi: float,
                  frac: np.ndarray, seed: int, quantise: bool = False):
    """Sources in cells drawn ~ nH^2 (with replacement), jittered by U(-0.4,0.4)
    cells, positions as drawn (FP64; quantise=True rounds them to 2^-12 cell);
    luminosities log-uniform."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    w = nH.astype(np.float64).ravel() ** 2
    w /= w.sum()
    cells = rng.choice(w.size, size=nsrc, replace=True, p=w)
    n = nH.shape[0]
    ijk = np.stack(np.unravel_index(cells, (n, n, n)), axis=1).astype(np.float64)
    pos = ijk + 0.5 + rng.uniform(-0.4, 0.4, size=(nsrc, 3))
    if quantise:
        pos = quantise_pos(pos)
    lum = 10.0 ** rng.uniform(math.log10(ndot_lo), math.log10(ndot_hi), size=nsrc)
    return pos, lum[:, None] * frac[None, :]


def cosmic(n: int = 256, nsrc: int = 1000, sigma_ln: float = 1.5, seed: int = 1807,
           ndot_lo: float = 1e48, ndot_hi: float = 1e51, box_kpc: Optional[float] = None,
           mean_nH: float = 2e-4, quantise: bool = False) -> Workload:
    """Lognormal cosmic-field workload (stand-in for RT06 Test 4)."""
    grp = blackbody_groups(1e5)
    nH = cosmic_field(n, sigma_ln, mean_nH, seed)
    pos, ndot = place_sources(nH, nsrc, ndot_lo, ndot_hi, grp["frac"], seed, quantise)
    if box_kpc is None:
        # 0.5 h^-1 cMpc at z = 9 (h = 0.7) per 256 cells: same cell size at any n
        box_kpc = 500.0 / 0.7 / 10.0 * n / 256
    x0 = 1.2e-3
    shape = (n, n, n)
    return Workload(name=f"cosmic_{n}_{nsrc}", n=n, box_cm=box_kpc * KPC, Y=0.24, ngroups=3,
                    E_group_eV=grp["E"], sigma=grp["sigma"], nH=nH,
                    xHI=np.full(shape, 1 - x0, np.float32), xHeI=np.full(shape, 1 - x0, np.float32),
                    xHeII=np.full(shape, x0, np.float32), T=np.full(shape, 100.0, np.float32),
                    src_pos=pos, src_ndot=ndot, dt_s=0.02 * MYR, nsteps=20,
                    z_compton=9.0, seed=seed)


def cosmic_256(seed: int = 1807, nsrc: int = 1000, n: int = 256) -> Workload:
    return cosmic(n=n, nsrc=nsrc, sigma_ln=1.5, seed=seed)


def cosmic_512(seed: int = 1807, nsrc: int = 10000, n: int = 512) -> Workload:
    w = cosmic(n=n, nsrc=nsrc, sigma_ln=2.0, seed=seed, ndot_lo=1e47, ndot_hi=1e51)
    w.nsteps = 10
    return w


def subset_sources(w: Workload, idx) -> Workload:
    """Same gas, only the sources listed in ``idx``."""
    idx = np.asarray(idx)
    return dataclasses.replace(w, src_pos=w.src_pos[idx], src_ndot=w.src_ndot[idx])


def ionised_bubbles(w: Workload, radius: float, x_in: float = 1e-4, xHeII_in: float = 0.05):
    """The workload's gas with an ionised sphere of ``radius`` cells around
    every source (x_HI = x_HeI = x_in, x_HeII = xHeII_in inside): the state the
    optically thin approximation (Sec. 2.6) is made for.  Returns FP32
    (xHI, xHeI, xHeII)."""
    n = w.n
    if radius >= np.sqrt(3.0) * n:            # every cell is within reach of every source
        inside = np.ones((n, n, n), bool)
    else:
        # distance from each cell centre to its nearest source, slab by slab
        from scipy.spatial import cKDTree
        tree = cKDTree(np.asarray(w.src_pos, np.float64))
        jk = np.indices((n, n)).reshape(2, -1).T + 0.5
        inside = np.zeros((n, n, n), bool)
        for i in range(n):
            pts = np.column_stack([np.full(n * n, i + 0.5), jk])
            d, _ = tree.query(pts, distance_upper_bound=radius)
            inside[i] = (d < radius).reshape(n, n)
    xHI = np.where(inside, x_in, w.xHI).astype(np.float32)
    xHeI = np.where(inside, x_in, w.xHeI).astype(np.float32)
    xHeII = np.where(inside, xHeII_in, w.xHeII).astype(np.float32)
    if w.Y == 0:
        xHeI[:] = 0
        xHeII[:] = 0
    return xHI, xHeI, xHeII


def random_gas(n: int, seed: int, Y: float = 0.24, lo: float = 1e-4, hi: float = 1e-1):
    """Random gas state for chemistry tests: log-uniform nH, random fractions, T."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (n,)
    nH = 10 ** rng.uniform(np.log10(lo), np.log10(hi), shape)
    xHI = 10 ** rng.uniform(-6, 0, shape)
    a = rng.uniform(0, 1, shape)
    b = rng.uniform(0, 1, shape)
    xHeI = np.minimum(a, 1.0)
    xHeII = (1 - xHeI) * b
    T = 10 ** rng.uniform(2, 4.7, shape)
    return [v.astype(np.float32) for v in (nH, xHI, xHeI, xHeII, T)]


def random_rates(n: int, seed: int, gmax: float = 1e-11):
    """Random photoionisation [1/s] and heating [erg/s] rates per species."""
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    g = (10 ** rng.uniform(-6, 0, (3, n)) * gmax)
    g[:, rng.uniform(0, 1, n) < 0.1] = 0.0
    h = g * (10 ** rng.uniform(0, 1.3, (3, n))) * EV
    return g.astype(np.float32), h.astype(np.float32)
