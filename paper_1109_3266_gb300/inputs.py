"""Seeded synthetic inputs for the dose engine: phantoms, materials, spectra,
source geometries and whole problems.

This module only produces input data.  It holds none of the transport method's
arithmetic (no cross sections, no sampling, no tallies) and imports neither the
CUDA library binding nor the CPU oracle; both of those consume what it returns.

Workloads (stand-ins for the paper's water and Zubal phantoms, Sec. 3.1-3.2,
whose measured bowtie map, Boone-Seibert spectrum and phantom data are not
available):
  tiny_water      32^3 x 0.5 cm water, 60 keV, point source 50 cm, 10x10 cm field
  cbct_water      256x256x128 x 0.2 cm water, 120 kVp, 360 projections, SAD 100 cm
  head            256x256x160 x 0.1 cm nested-ellipsoid head, 100 kVp, half fan
  batched         64 requests of mixed water/head phantoms, 64^3..256^3
  served          Poisson stream of head requests
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np


# --------------------------------------------------------------------------
# data records
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Material:
    """Material parameters the closed-form cross sections read.

    z_over_a : electrons per gram divided by Avogadro's number
    a_mol    : molar mass of one formula unit (g/mol)
    z_eff    : effective atomic number
    q0       : form-factor width in 1/Angstrom; 0 selects F^2 = 1 (Thomson)
    density  : nominal density (g/cm^3), used by the phantom generators only
    sq0      : scattering-function width in 1/Angstrom for the Waller-Hartree
               Compton model, S(q)/Z = 1 - exp(-q^2/sq0^2); 0 selects S/Z = 1
    elements : ((Z, atoms per formula unit), ...) for the independent-atom
               Rayleigh form factor (used when the physics asks for it)
    """
    name: str
    z_over_a: float
    a_mol: float
    z_eff: float
    q0: float
    density: float
    sq0: float = 0.55
    elements: tuple = ()


# proposed scattering-function width (the paper's PENELOPE tables are not
# available): S/Z of water's electrons is about 0.4 at sin(theta/2)/lambda = 0.2/A
SQ0 = 0.55


# standard atomic weights (g/mol) of the elements in the materials below
ATOMIC_WEIGHT = {1: 1.008, 6: 12.011, 7: 14.007, 8: 15.999, 11: 22.990, 12: 24.305, 15: 30.974, 16: 32.06,
                 17: 35.45, 18: 39.948, 19: 39.098, 20: 40.078}


def atoms_per_unit(mass_fractions, a_mol):
    """((Z, atoms per formula unit), ...) from mass fractions {Z: w} (normalised
    to 1) for a formula unit of molar mass a_mol."""
    tot = float(sum(mass_fractions.values()))
    return tuple((z, (w / tot) * a_mol / ATOMIC_WEIGHT[z]) for z, w in sorted(mass_fractions.items()))


def _mat(name, z_over_a, z_eff, density, a_mol=None, q0=1.0, sq0=SQ0, mass_fractions=None, elements=None):
    a = a_mol if a_mol is not None else 10.0 / z_over_a
    els = elements if elements is not None else (atoms_per_unit(mass_fractions, a) if mass_fractions else ())
    return Material(name, z_over_a, a, z_eff, q0, density, sq0, els)


# elemental compositions by mass: the ICRU reference tissues and dry air
WATER = _mat("water", 0.5551, 7.42, 1.0, a_mol=18.015, elements=((1, 2.0), (8, 1.0)))
SOFT_TISSUE = _mat("soft_tissue", 0.5494, 7.4, 1.03, mass_fractions={1: 0.101, 6: 0.111, 7: 0.026, 8: 0.762})
BRAIN = _mat("brain", 0.5520, 7.5, 1.04, mass_fractions={1: 0.107, 6: 0.145, 7: 0.022, 8: 0.712, 11: 0.002,
                                                          15: 0.004, 16: 0.002, 17: 0.003, 19: 0.003})
BONE = _mat("bone", 0.5148, 13.8, 1.85, mass_fractions={1: 0.034, 6: 0.155, 7: 0.042, 8: 0.435, 11: 0.001,
                                                        12: 0.002, 15: 0.103, 16: 0.003, 20: 0.225})
AIR = _mat("air", 0.4992, 7.64, 0.0012, mass_fractions={6: 0.000124, 7: 0.755268, 8: 0.231781, 18: 0.012827})


def thomson(m: Material) -> Material:
    """The same material with F^2 = 1 in the Rayleigh angular distribution."""
    return replace(m, q0=0.0)


@dataclass
class Phantom:
    """Voxel grid centred at the origin; arrays have shape (nz, ny, nx) so that
    x runs fastest in memory."""
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    mat: np.ndarray            # uint8
    rho: np.ndarray            # float32, g/cm^3
    materials: List[Material]

    @property
    def nvox(self) -> int:
        return self.nx * self.ny * self.nz


@dataclass
class Source:
    """kind 'static': point source at (0, 0, -sad) aimed along +z.
    kind 'arc': source at sad*(sin b, cos b, 0) aimed at the origin, b on
    [arc0, arc1) at n_proj discrete angles (or uniform if continuous).
    The field [u_lo, u_hi] x [v_lo, v_hi] is given at the centre plane (cm);
    u is lateral, v is along z for 'arc' and along y for 'static'.
    fluence: optional [n_v][n_u] relative beamlet intensities tiling the field
    (Sec. 2.2.4); without it directions are uniform in solid angle."""
    kind: str
    sad: float
    u_lo: float
    u_hi: float
    v_lo: float
    v_hi: float
    n_proj: int = 1
    arc0: float = 0.0
    arc1: float = 2.0 * math.pi
    continuous: bool = False
    fluence: Optional[np.ndarray] = None
    z0: float = 0.0             # 'arc' source height at arc0 and arc1, linear in the angle
    z1: float = 0.0             # (helical trajectory; both 0 for a circle)


@dataclass
class Spectrum:
    """Energy bins [e_lo, e_hi] in keV with relative weights; e_lo == e_hi is a line."""
    e_lo: np.ndarray
    e_hi: np.ndarray
    w: np.ndarray


@dataclass
class Physics:
    e_min: int = 1              # node grid floor = absorption energy (keV)
    e_max: int = 150            # node grid top (keV)
    n_zeta: int = 1024          # surface columns
    majorant_scale: float = 1.0
    mode: str = "full"          # "full" | "max_real" ("primary" is max_real with 1)
    max_real: int = 0
    compton: str = "kn"         # "kn" free-electron Klein-Nishina | "wh" Waller-Hartree (Eq. 2 with S)
    rayleigh: str = "gauss"     # "gauss" F^2 = exp(-q^2/q0^2) | "iaa" independent-atom form factor of the elements


@dataclass
class Problem:
    name: str
    phantom: Phantom
    source: Source
    spectrum: Spectrum
    physics: Physics
    n_hist: int
    n_batches: int
    seed: int
    meta: dict = field(default_factory=dict)


# --------------------------------------------------------------------------
# phantoms
# --------------------------------------------------------------------------
def uniform_box(nx, ny, nz, d, material: Material = WATER, density: Optional[float] = None) -> Phantom:
    rho = np.full((nz, ny, nx), material.density if density is None else density, dtype=np.float32)
    mat = np.zeros((nz, ny, nx), dtype=np.uint8)
    return Phantom(nx, ny, nz, d, d, d, mat, rho, [material])


def slab_phantom(layers, lateral_cm: float = 1000.0, dz: Optional[float] = None) -> Phantom:
    """Slabs stacked along z: layers = [(Material, thickness_cm), ...], one voxel
    per slab when dz is None.  The lateral extent is one wide voxel."""
    mats, rhos, thick = [], [], []
    materials: List[Material] = []
    for m, t in layers:
        if m not in materials:
            materials.append(m)
        n = 1 if dz is None else int(round(t / dz))
        mats += [materials.index(m)] * n
        rhos += [m.density] * n
        thick.append(t)
    if dz is None:
        if len(set(thick)) != 1:
            raise ValueError("one voxel per slab needs equal thicknesses; pass dz")
        dz = thick[0]
    nz = len(mats)
    mat = np.array(mats, dtype=np.uint8).reshape(nz, 1, 1)
    rho = np.array(rhos, dtype=np.float32).reshape(nz, 1, 1)
    return Phantom(1, 1, nz, lateral_cm, lateral_cm, dz, mat, rho, materials)


def head_phantom(nx, ny, nz, d, seed: int, size_ref=(25.6, 25.6, 16.0)) -> Phantom:
    """Nested-ellipsoid head: soft tissue 1.03, a bone shell 0.5 cm under the
    surface of thickness U[0.5, 0.8] cm, brain 1.04, two air sinuses, air
    outside, density x (1 + 0.02 N(0,1)) with N clipped to +-3.  Semi-axes
    (10.0, 12.0, 7.6) cm on a 25.6 x 25.6 x 16 cm box, scaled with the box."""
    rng = np.random.default_rng(seed)
    t_skull = float(rng.uniform(0.5, 0.8))
    sx, sy, sz = nx * d / size_ref[0], ny * d / size_ref[1], nz * d / size_ref[2]
    A, B, C = 10.0 * sx, 12.0 * sy, 7.6 * sz
    x = (np.arange(nx) + 0.5) * d - nx * d / 2.0
    y = (np.arange(ny) + 0.5) * d - ny * d / 2.0
    z = (np.arange(nz) + 0.5) * d - nz * d / 2.0

    def inside(a, b, c, x0=0.0, y0=0.0, z0=0.0):
        # separable quadratic form, broadcast over (z, y, x)
        qx = ((x - x0) / a) ** 2
        qy = ((y - y0) / b) ** 2
        qz = ((z - z0) / c) ** 2
        return (qz[:, None, None] + qy[None, :, None]) + qx[None, None, :] <= 1.0

    scalp = 0.5
    mat = np.zeros((nz, ny, nx), dtype=np.uint8)            # 0 air
    mat[inside(A, B, C)] = 1                                 # soft tissue
    mat[inside(A - scalp, B - scalp, C - scalp)] = 2         # bone shell
    ti = scalp + t_skull
    mat[inside(A - ti, B - ti, C - ti)] = 3                  # brain
    for sgn in (-1.0, 1.0):
        mat[inside(1.5 * sx, 1.0 * sy, 1.0 * sz, sgn * 2.0 * sx, 8.0 * sy, 0.0)] = 0
    materials = [AIR, SOFT_TISSUE, BONE, BRAIN]
    nominal = np.array([m.density for m in materials], dtype=np.float64)
    noise = np.clip(rng.standard_normal((nz, ny, nx)), -3.0, 3.0)
    rho = (nominal[mat] * (1.0 + 0.02 * noise)).astype(np.float32)
    return Phantom(nx, ny, nz, d, d, d, mat, rho, materials)


# --------------------------------------------------------------------------
# spectra
# --------------------------------------------------------------------------
def spectrum_line(e_kev: float) -> Spectrum:
    return Spectrum(np.array([e_kev], float), np.array([e_kev], float), np.array([1.0]))


def spectrum_kramers(kvp: int, mm_al: float, e_min: int = 1) -> Spectrum:
    """Kramers' thick-target law (kvp - E)/E in 1 keV bins [j, j+1), filtered by
    mm_al of aluminium.  The filter uses an input-recipe fit of aluminium's mass
    attenuation, 26300/E^3 + 0.15 cm^2/g (E in keV), density 2.699 g/cm^3; it is
    part of the synthetic spectrum, not of the transport physics."""
    lo = np.arange(e_min, kvp, dtype=float)
    hi = lo + 1.0
    mid = lo + 0.5
    mu_al = 26300.0 / mid ** 3 + 0.15
    w = (kvp - mid) / mid * np.exp(-mu_al * 2.699 * (mm_al / 10.0))
    return Spectrum(lo, hi, w)


# --------------------------------------------------------------------------
# sources
# --------------------------------------------------------------------------
def static_source(sad: float, half_u: float, half_v: float) -> Source:
    return Source("static", sad, -half_u, half_u, -half_v, half_v)


def pencil_source(sad: float = 100.0) -> Source:
    return Source("static", sad, 0.0, 0.0, 0.0, 0.0)


def arc_source(sad, u_lo, u_hi, v_lo, v_hi, n_proj=360, arc0=0.0, arc1=2.0 * math.pi, continuous=False, z0=0.0,
               z1=0.0):
    return Source("arc", sad, u_lo, u_hi, v_lo, v_hi, n_proj, arc0, arc1, continuous, z0=z0, z1=z1)


def helical_source(sad, u_lo, u_hi, v_lo, v_hi, turns, z0, z1, n_proj_per_turn=360, continuous=False):
    """Helical CT: `turns` rotations while the source height goes from z0 to z1."""
    return arc_source(sad, u_lo, u_hi, v_lo, v_hi, int(round(turns * n_proj_per_turn)), 0.0, 2.0 * math.pi * turns,
                      continuous, z0, z1)


def bowtie_fluence(n_u: int = 128, n_v: int = 32, seed: int = 0, t_centre: float = 0.1, t_edge: float = 2.5,
                   mu_al: float = 0.75, noise: float = 0.02) -> np.ndarray:
    """Synthetic air-scan fluence of a full-fan bowtie (stand-in for Fig. 5(a)):
    aluminium thickness growing as the square of the lateral offset, from
    t_centre at the centre to t_edge at the field edge (cm), attenuation
    exp(-mu_al t) with mu_al about aluminium's at 60 keV, times seeded
    multiplicative Gaussian noise of relative size `noise`.  [n_v][n_u], > 0."""
    u = (np.arange(n_u) + 0.5) / n_u * 2.0 - 1.0
    t = t_centre + (t_edge - t_centre) * u * u
    f = np.tile(np.exp(-mu_al * t), (n_v, 1))
    rng = np.random.default_rng(seed)
    f = f * np.clip(1.0 + noise * rng.standard_normal(f.shape), 0.5, 1.5)
    return np.ascontiguousarray(f, dtype=np.float64)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
def tiny_water(n_hist: int = 100_000, n_batches: int = 10, seed: int = 1) -> Problem:
    """32^3 x 0.5 cm water, 60 keV line, point source 50 cm from the centre with a
    10 x 10 cm field at the centre, Thomson Rayleigh, nodes 10-150 keV."""
    ph = uniform_box(32, 32, 32, 0.5, thomson(WATER))
    return Problem("tiny_water", ph, static_source(50.0, 5.0, 5.0), spectrum_line(60.0),
                   Physics(e_min=10, e_max=150), n_hist, n_batches, seed)


def cbct_water(n_hist: int = 1_000_000_000, n_batches: int = 10, seed: int = 2,
               shape=(256, 256, 128), d: float = 0.2, bowtie: bool = False) -> Problem:
    """Water box 256x256x128 x 0.2 cm, 120 kVp Kramers + 2.5 mm Al, full rotation of
    360 projections at SAD 100 cm, 20 x 20 cm field at the centre; with bowtie, the
    field carries a 128 x 32 full-fan bowtie fluence map (Sec. 2.2.4)."""
    nx, ny, nz = shape
    ph = uniform_box(nx, ny, nz, d, WATER)
    src = arc_source(100.0, -10.0, 10.0, -10.0, 10.0, n_proj=360)
    if bowtie:
        src = replace(src, fluence=bowtie_fluence(128, 32, seed=seed))
    return Problem("cbct_water", ph, src, spectrum_kramers(120, 2.5), Physics(e_min=1, e_max=150),
                   n_hist, n_batches, seed)


def head(n_hist: int = 2_000_000_000, n_batches: int = 10, seed: int = 3, phantom_seed: int = 3,
         shape=(256, 256, 160), d: float = 0.1, kvp: int = 100) -> Problem:
    """Nested-ellipsoid head 256x256x160 x 0.1 cm, 100 kVp, half-fan full rotation
    (lateral field -1.0..13.5 cm, axial 16 cm at the centre), SAD 100 cm."""
    nx, ny, nz = shape
    ph = head_phantom(nx, ny, nz, d, phantom_seed)
    src = arc_source(100.0, -1.0, 13.5, -8.0, 8.0, n_proj=360)
    return Problem("head", ph, src, spectrum_kramers(kvp, 2.5), Physics(e_min=1, e_max=150),
                   n_hist, n_batches, seed)


def head_request(phantom: Phantom, seed: int, kvp: int = 100, n_hist: int = 1) -> Problem:
    """A served dose request on a given head phantom: 100 kVp half-fan CBCT,
    transport seed `seed` (the phantom is shared data, the histories are not)."""
    half_z = phantom.nz * phantom.dz / 2.0
    src = arc_source(100.0, -1.0, 13.5, -half_z, half_z, n_proj=360)
    return Problem(f"head_req{seed}", phantom, src, spectrum_kramers(kvp, 2.5), Physics(e_min=1, e_max=150),
                   n_hist, 10, seed)


def batched_requests(n_req: int = 64, seed: int = 4, hist_lo: float = 1e7, hist_hi: float = 1e9,
                     sides=tuple(range(64, 257, 32))) -> List[Problem]:
    """Uneven requests: cube side uniform on {64, 96, ..., 256} voxels of 0.1 cm,
    half water and half head, kVp uniform 80-140 (whole kV), histories
    log-uniform on [hist_lo, hist_hi]; request r uses seed 1000 + r."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_req):
        side = int(rng.choice(sides))
        kvp = int(rng.integers(80, 141))
        nh = int(round(math.exp(rng.uniform(math.log(hist_lo), math.log(hist_hi)))))
        d = 0.1
        if r % 2 == 0:
            ph = uniform_box(side, side, side, d, WATER)
            kind = "water"
        else:
            ph = head_phantom(side, side, side, d, 1000 + r, size_ref=(25.6, 25.6, 25.6))
            kind = "head"
        half = side * d / 2.0
        src = arc_source(100.0, -0.8 * half, 0.8 * half, -0.8 * half, 0.8 * half, n_proj=360)
        out.append(Problem(f"req{r}_{kind}{side}", ph, src, spectrum_kramers(kvp, 2.5),
                           Physics(e_min=1, e_max=150), nh, 10, 1000 + r,
                           meta={"kvp": kvp, "side": side, "kind": kind}))
    return out


def served_arrivals(n_req: int = 200, rate_per_s: float = 4.0, seed: int = 5):
    """Poisson arrival times (s) and per-request seeds 5000 + r."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_req))
    return [(float(t[r]), 5000 + r) for r in range(n_req)]


def scaled(p: Problem, n_hist: Optional[int] = None, n_batches: Optional[int] = None,
           seed: Optional[int] = None, physics: Optional[Physics] = None) -> Problem:
    """The same problem with another history count, batch count, seed or physics."""
    return replace(p, n_hist=p.n_hist if n_hist is None else int(n_hist),
                   n_batches=p.n_batches if n_batches is None else int(n_batches),
                   seed=p.seed if seed is None else int(seed),
                   physics=p.physics if physics is None else physics)
