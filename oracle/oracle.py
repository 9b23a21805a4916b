"""Python face of the CPU oracle (TEST INFRASTRUCTURE).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this module.  It wraps the C oracle (ctd_oracle.c) with ctypes and adds
the batch statistics of Sec. 2.2.1 and the precision measures of Sec. 3.1 in
plain numpy.  It reads problems duck-typed (the attributes of the records in
the package's inputs module) and imports nothing from the product library.
"""
from __future__ import annotations

import ctypes as C
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

from . import build as _build

KEV_TO_J = 1.602176634e-16

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _declare(_lib)
    return _lib


MAX_ELEMENTS = 16


class OrMaterial(C.Structure):
    _fields_ = [("z_over_a", C.c_double), ("a_mol", C.c_double), ("z_eff", C.c_double), ("q0", C.c_double),
                ("sq0", C.c_double), ("n_el", C.c_int), ("el_z", C.c_int * MAX_ELEMENTS),
                ("el_n", C.c_double * MAX_ELEMENTS)]


class OrProblem(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("mat", C.POINTER(C.c_uint8)), ("rho", C.POINTER(C.c_float)),
        ("n_mat", C.c_int), ("mats", C.POINTER(OrMaterial)),
        ("src_kind", C.c_int), ("sad", C.c_double),
        ("u_lo", C.c_double), ("u_hi", C.c_double), ("v_lo", C.c_double), ("v_hi", C.c_double),
        ("n_proj", C.c_int), ("arc0", C.c_double), ("arc1", C.c_double), ("continuous", C.c_int),
        ("z0", C.c_double), ("z1", C.c_double),
        ("fl_nu", C.c_int), ("fl_nv", C.c_int), ("fl_f", C.POINTER(C.c_double)),
        ("nbins", C.c_int), ("e_lo", C.POINTER(C.c_double)), ("e_hi", C.POINTER(C.c_double)),
        ("w", C.POINTER(C.c_double)),
        ("e_min", C.c_int), ("e_max", C.c_int), ("n_zeta", C.c_int), ("majorant_scale", C.c_double),
        ("mode", C.c_int), ("max_real", C.c_int), ("sampling", C.c_int), ("compton", C.c_int),
        ("n_hist", C.c_uint64), ("n_batches", C.c_int), ("seed", C.c_uint64),
    ]


class OrCounts(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("pe", "compton", "rayleigh", "fictitious", "escaped", "missed",
                                          "cutoff", "terminated", "aborted", "steps")] + \
               [(n, C.c_double) for n in ("e_emitted", "e_escaped", "e_deposited")]


COUNT_KEYS = ("pe", "compton", "rayleigh", "fictitious", "escaped", "missed", "cutoff", "terminated",
              "aborted", "steps")


class OrTrack(C.Structure):
    _fields_ = [("end", C.c_int32), ("last_type", C.c_int32), ("steps", C.c_uint32), ("idx", C.c_uint32),
                ("e_end", C.c_double), ("margin", C.c_double), ("margin_loc", C.c_double),
                ("margin_kind", C.c_int32), ("pad", C.c_int32)]


# numpy view of or_track records
TRACK_DTYPE = np.dtype([("end", np.int32), ("last_type", np.int32), ("steps", np.uint32), ("idx", np.uint32),
                        ("e_end", np.float64), ("margin", np.float64), ("margin_loc", np.float64),
                        ("margin_kind", np.int32), ("pad", np.int32)])
END_NAMES = ("pe", "cutoff", "escaped", "missed", "terminated", "aborted")
MARGIN_NAMES = ("none", "accept", "entry", "escape", "boundary", "type", "cutoff")


def _declare(L):
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
    L.or_uniform.restype = C.c_double
    L.or_uniform.argtypes = [C.c_uint32]
    for n in ("or_mu_pe", "or_mu_compton", "or_mu_rayleigh", "or_mu_compton_wh"):
        getattr(L, n).restype = C.c_double
        getattr(L, n).argtypes = [C.POINTER(OrMaterial), C.c_double]
    L.or_sigma_kn.restype = C.c_double
    L.or_sigma_kn.argtypes = [C.c_double]
    L.or_sigma_wh.restype = C.c_double
    L.or_sigma_wh.argtypes = [C.c_double, C.c_double]
    L.or_build_wh_surface.argtypes = [C.c_double, C.c_int, C.c_int, C.c_int, dp]
    L.or_allocate.argtypes = [C.c_uint64, C.c_int, dp, C.POINTER(C.c_uint64)]
    L.or_log_f32.restype = C.c_float
    L.or_log_f32.argtypes = [C.c_float]
    L.or_eval_log_f32.argtypes = [C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_size_t]
    L.or_eval_sincos_f32.argtypes = [C.POINTER(C.c_float)] * 3 + [C.c_size_t]
    L.or_eval_uniform_f32.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_float), C.c_size_t]
    for n in ("or_setup_create_f64", "or_setup_create_f32"):
        getattr(L, n).restype = P
        getattr(L, n).argtypes = [C.POINTER(OrProblem)]
    L.or_setup_destroy.argtypes = [P]
    for n in ("or_transport_f64", "or_transport_f32"):
        getattr(L, n).argtypes = [P, C.c_uint64, C.c_uint64, dp, C.POINTER(OrCounts)]
    for n in ("or_track_f64", "or_track_f32"):
        getattr(L, n).argtypes = [P, C.c_uint64, C.c_uint64, C.c_void_p]
    L.or_setup_sizes.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.or_setup_tables.argtypes = [P, dp, dp]
    L.or_setup_surfaces.argtypes = [P, dp, dp]
    L.or_build_kn_surface.argtypes = [C.c_int, C.c_int, C.c_int, dp]
    L.or_build_rayleigh_surface.argtypes = [C.c_double, C.c_int, C.c_int, C.c_int, dp]
    L.or_build_rayleigh_iaa_surface.argtypes = [C.POINTER(OrMaterial), C.c_int, C.c_int, C.c_int, dp]
    L.or_ff_atom2.restype = C.c_double
    L.or_ff_atom2.argtypes = [C.c_int, C.c_double]
    for n in ("or_ff_mol2", "or_sigma_rayleigh_iaa", "or_mu_rayleigh_iaa"):
        getattr(L, n).restype = C.c_double
        getattr(L, n).argtypes = [C.POINTER(OrMaterial), C.c_double]
    L.or_sample_mu_f64.argtypes = [P, C.c_int, C.c_int, C.c_double, C.c_int, C.c_uint64, C.c_uint64, dp]
    L.or_sample_mu_f32.argtypes = [P, C.c_int, C.c_int, C.c_double, C.c_uint64, C.c_uint64, dp]
    L.or_alias_build.argtypes = [C.c_int, dp, C.POINTER(C.c_uint32), C.POINTER(C.c_int32)]
    L.or_alias_counts.argtypes = [C.c_int, C.POINTER(C.c_uint32), C.POINTER(C.c_int32), C.c_uint64, C.c_uint64,
                                  C.POINTER(C.c_uint64)]
    L.or_mh_counts.argtypes = [C.c_int, dp, C.c_int, C.c_uint64, C.c_uint64, C.POINTER(C.c_uint64)]
    L.or_mh_chains.argtypes = [C.c_int, dp, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64, C.POINTER(C.c_uint64)]
    L.or_rotate_f64.argtypes = [dp, C.c_double, C.c_double]
    L.or_rotate_f32.argtypes = [C.POINTER(C.c_float), C.c_float, C.c_float]


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


# --------------------------------------------------------------------------
# small wrappers used by the pins
# --------------------------------------------------------------------------
def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return list(o)


def uniform(x: int) -> float:
    return lib().or_uniform(x)


def material_struct(m, iaa=False) -> OrMaterial:
    """The C record of a material; iaa=True carries its elements (independent-atom
    Rayleigh form factor)."""
    s = OrMaterial(m.z_over_a, m.a_mol, m.z_eff, m.q0, m.sq0)
    if iaa:
        if not 0 < len(m.elements) <= MAX_ELEMENTS:
            raise ValueError(f"material {m.name}: 1..{MAX_ELEMENTS} elements needed for the IAA form factor")
        s.n_el = len(m.elements)
        for i, (z, n) in enumerate(m.elements):
            s.el_z[i] = int(z)
            s.el_n[i] = float(n)
    return s


def mu_pe(m, e):
    return lib().or_mu_pe(C.byref(material_struct(m)), e)


def mu_compton(m, e):
    return lib().or_mu_compton(C.byref(material_struct(m)), e)


def mu_rayleigh(m, e):
    return lib().or_mu_rayleigh(C.byref(material_struct(m)), e)


def sigma_kn(e):
    return lib().or_sigma_kn(e)


def sigma_wh(e, sq0):
    """Waller-Hartree total per electron (cm^2), Simpson over mu."""
    return lib().or_sigma_wh(e, sq0)


def mu_compton_wh(m, e):
    return lib().or_mu_compton_wh(C.byref(material_struct(m)), e)


def ff_atom2(z, x2):
    """Squared form factor of element z at x^2 = (sin(theta/2)/lambda)^2, 1/Angstrom^2."""
    return lib().or_ff_atom2(int(z), float(x2))


def ff_mol2(m, x2):
    """Independent-atom molecular F^2 of material m at x^2."""
    return lib().or_ff_mol2(C.byref(material_struct(m, iaa=True)), float(x2))


def sigma_rayleigh_iaa(m, e):
    """Rayleigh total per formula unit (cm^2) with the IAA form factor, Simpson over mu."""
    return lib().or_sigma_rayleigh_iaa(C.byref(material_struct(m, iaa=True)), e)


def mu_rayleigh_iaa(m, e):
    return lib().or_mu_rayleigh_iaa(C.byref(material_struct(m, iaa=True)), e)


def rayleigh_iaa_surface(m, e_min, n_e, n_zeta):
    out = np.empty((n_e, n_zeta), dtype=np.float64)
    lib().or_build_rayleigh_iaa_surface(C.byref(material_struct(m, iaa=True)), e_min, n_e, n_zeta,
                                        _ptr(out, C.c_double))
    return out


def allocate(n: int, w) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros(len(w), dtype=np.uint64)
    rc = lib().or_allocate(n, len(w), _ptr(w, C.c_double), _ptr(out, C.c_uint64))
    if rc != 0:
        raise ValueError("allocation failed")
    return out


def log_f32(u):
    u = np.ascontiguousarray(u, dtype=np.float32)
    out = np.empty_like(u)
    lib().or_eval_log_f32(_ptr(u, C.c_float), _ptr(out, C.c_float), u.size)
    return out


def uniform_f32(x):
    """The uniform mapping of 32-bit words, as binary32."""
    x = np.ascontiguousarray(x, dtype=np.uint32)
    out = np.empty(x.size, dtype=np.float32)
    lib().or_eval_uniform_f32(_ptr(x, C.c_uint32), _ptr(out, C.c_float), x.size)
    return out


def sincos_turns_f32(t):
    t = np.ascontiguousarray(t, dtype=np.float32)
    c = np.empty_like(t)
    s = np.empty_like(t)
    lib().or_eval_sincos_f32(_ptr(t, C.c_float), _ptr(c, C.c_float), _ptr(s, C.c_float), t.size)
    return c, s


def rotate(u, mu, t_phi, precision=64):
    if precision == 64:
        a = np.array(u, dtype=np.float64)
        lib().or_rotate_f64(_ptr(a, C.c_double), mu, t_phi)
    else:
        a = np.array(u, dtype=np.float32)
        lib().or_rotate_f32(_ptr(a, C.c_float), np.float32(mu), np.float32(t_phi))
    return a


def alias_table(f):
    """Walker/Vose alias table of intensities f: (thresholds uint32, aliases int32)."""
    f = np.ascontiguousarray(f, dtype=np.float64).ravel()
    thr = np.empty(f.size, dtype=np.uint32)
    al = np.empty(f.size, dtype=np.int32)
    if lib().or_alias_build(f.size, _ptr(f, C.c_double), _ptr(thr, C.c_uint32), _ptr(al, C.c_int32)) != 0:
        raise ValueError("unusable intensities")
    return thr, al


def alias_counts(thr, al, n, seed):
    out = np.zeros(thr.size, dtype=np.uint64)
    lib().or_alias_counts(thr.size, _ptr(np.ascontiguousarray(thr), C.c_uint32),
                          _ptr(np.ascontiguousarray(al), C.c_int32), n, seed, _ptr(out, C.c_uint64))
    return out


def mh_counts(f, n, seed, i0=0):
    """Beamlet counts of the paper's Metropolis-Hastings chain (Algorithm A1)."""
    f = np.ascontiguousarray(f, dtype=np.float64).ravel()
    out = np.zeros(f.size, dtype=np.uint64)
    lib().or_mh_counts(f.size, _ptr(f, C.c_double), i0, n, seed, _ptr(out, C.c_uint64))
    return out


def mh_chains(f, n, seed, chains, i0=0):
    """Beamlet counts of Algorithm A1 run as `chains` chains (one per GPU thread)."""
    f = np.ascontiguousarray(f, dtype=np.float64).ravel()
    out = np.zeros(f.size, dtype=np.uint64)
    lib().or_mh_chains(f.size, _ptr(f, C.c_double), i0, n, seed, chains, _ptr(out, C.c_uint64))
    return out


def kn_surface(e_min, n_e, n_zeta):
    out = np.empty((n_e, n_zeta), dtype=np.float64)
    lib().or_build_kn_surface(e_min, n_e, n_zeta, _ptr(out, C.c_double))
    return out


def rayleigh_surface(q0, e_min, n_e, n_zeta):
    out = np.empty((n_e, n_zeta), dtype=np.float64)
    lib().or_build_rayleigh_surface(q0, e_min, n_e, n_zeta, _ptr(out, C.c_double))
    return out


def wh_surface(sq0, e_min, n_e, n_zeta):
    out = np.empty((n_e, n_zeta), dtype=np.float64)
    lib().or_build_wh_surface(sq0, e_min, n_e, n_zeta, _ptr(out, C.c_double))
    return out


# --------------------------------------------------------------------------
# problem set-up and transport
# --------------------------------------------------------------------------
_MODES = {"full": 0, "max_real": 1}
_COMPTON = {"kn": 0, "wh": 1}


class Setup:
    """Tables, majorant, surfaces and batch layout of one problem, in one precision."""

    def __init__(self, problem, precision: int = 64, sampling: str = "surface"):
        if precision not in (32, 64):
            raise ValueError("precision is 32 or 64")
        ph, src, sp, phy = problem.phantom, problem.source, problem.spectrum, problem.physics
        self.problem = problem
        self.precision = precision
        self._mat = np.ascontiguousarray(ph.mat, dtype=np.uint8).ravel()
        self._rho = np.ascontiguousarray(ph.rho, dtype=np.float32).ravel()
        iaa = getattr(phy, 'rayleigh', 'gauss') == 'iaa'
        self._mats = (OrMaterial * len(ph.materials))(*[material_struct(m, iaa) for m in ph.materials])
        self._elo = np.ascontiguousarray(sp.e_lo, dtype=np.float64)
        self._ehi = np.ascontiguousarray(sp.e_hi, dtype=np.float64)
        self._w = np.ascontiguousarray(sp.w, dtype=np.float64)
        mode = _MODES[phy.mode]
        p = OrProblem()
        p.nx, p.ny, p.nz = ph.nx, ph.ny, ph.nz
        p.dx, p.dy, p.dz = ph.dx, ph.dy, ph.dz
        p.mat, p.rho = _ptr(self._mat, C.c_uint8), _ptr(self._rho, C.c_float)
        p.n_mat, p.mats = len(ph.materials), self._mats
        p.src_kind = 0 if src.kind == "static" else 1
        p.sad = src.sad
        p.u_lo, p.u_hi, p.v_lo, p.v_hi = src.u_lo, src.u_hi, src.v_lo, src.v_hi
        p.n_proj, p.arc0, p.arc1, p.continuous = src.n_proj, src.arc0, src.arc1, int(src.continuous)
        p.z0, p.z1 = getattr(src, "z0", 0.0), getattr(src, "z1", 0.0)
        fl = getattr(src, "fluence", None)
        if fl is not None:
            self._fl = np.ascontiguousarray(fl, dtype=np.float64)
            p.fl_nv, p.fl_nu = self._fl.shape
            p.fl_f = _ptr(self._fl, C.c_double)
        p.nbins = len(self._w)
        p.e_lo, p.e_hi, p.w = _ptr(self._elo, C.c_double), _ptr(self._ehi, C.c_double), _ptr(self._w, C.c_double)
        p.e_min, p.e_max, p.n_zeta = phy.e_min, phy.e_max, phy.n_zeta
        p.majorant_scale, p.mode, p.max_real = phy.majorant_scale, mode, phy.max_real
        p.sampling = 0 if sampling == "surface" else 1
        self.compton = getattr(phy, "compton", "kn")
        p.compton = _COMPTON[self.compton]
        p.n_hist, p.n_batches, p.seed = problem.n_hist, problem.n_batches, problem.seed
        self._p = p
        fn = lib().or_setup_create_f64 if precision == 64 else lib().or_setup_create_f32
        self.handle = fn(C.byref(p))
        if not self.handle:
            raise ValueError("oracle set-up rejected the problem")
        ne, nz, nm = C.c_int(), C.c_int(), C.c_int()
        lib().or_setup_sizes(self.handle, C.byref(ne), C.byref(nz), C.byref(nm))
        self.n_e, self.n_zeta, self.n_mat = ne.value, nz.value, nm.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.or_setup_destroy(h)
            self.handle = None

    def tables(self):
        cum = np.empty((self.n_mat, self.n_e, 3), dtype=np.float64)
        mm = np.empty(self.n_e, dtype=np.float64)
        lib().or_setup_tables(self.handle, _ptr(cum, C.c_double), _ptr(mm, C.c_double))
        return cum, mm

    def surfaces(self):
        """C surfaces ([n_e][n_zeta], or [n_mat][n_e][n_zeta] for Waller-Hartree) and R surfaces."""
        shape = (self.n_mat, self.n_e, self.n_zeta) if self.compton == "wh" else (self.n_e, self.n_zeta)
        cs = np.empty(shape, dtype=np.float64)
        rs = np.empty((self.n_mat, self.n_e, self.n_zeta), dtype=np.float64)
        lib().or_setup_surfaces(self.handle, _ptr(cs, C.c_double), _ptr(rs, C.c_double))
        return cs, rs

    def sample_mu(self, kind: str, material: int, e_kev: float, n: int, seed: int, exact: bool = False):
        out = np.empty(n, dtype=np.float64)
        k = 0 if kind == "compton" else 1
        if self.precision == 64:
            rc = lib().or_sample_mu_f64(self.handle, k, material, e_kev, int(exact), seed, n, _ptr(out, C.c_double))
        else:
            if exact:
                raise ValueError("exact samplers run in binary64 only")
            rc = lib().or_sample_mu_f32(self.handle, k, material, e_kev, seed, n, _ptr(out, C.c_double))
        if rc != 0:
            raise ValueError("sampler rejected its arguments")
        return out

    def transport(self, h0: int, h1: int, threads: int = 1):
        """Energy deposited per voxel (keV) and counts for histories [h0, h1)."""
        nvox = self._rho.size
        fn = lib().or_transport_f64 if self.precision == 64 else lib().or_transport_f32
        threads = max(1, min(int(threads), max(1, (h1 - h0) // 64)))
        edges = np.linspace(h0, h1, threads + 1).astype(np.int64)
        parts = [(int(edges[i]), int(edges[i + 1])) for i in range(threads)]
        bufs = [np.zeros(nvox, dtype=np.float64) for _ in parts]
        cnts = [OrCounts() for _ in parts]

        def work(i):
            a, b = parts[i]
            rc = fn(self.handle, a, b, _ptr(bufs[i], C.c_double), C.byref(cnts[i]))
            if rc != 0:
                raise ValueError("oracle transport rejected its arguments")

        if threads == 1:
            work(0)
        else:
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(work, range(threads)))
        edep = bufs[0]
        for b in bufs[1:]:
            edep += b
        counts = {k: sum(getattr(c, k) for c in cnts) for k in COUNT_KEYS}
        for k in ("e_emitted", "e_escaped", "e_deposited"):
            counts[k] = float(sum(getattr(c, k) for c in cnts))
        return edep, counts


    def track(self, h0: int, h1: int, threads: int = 1) -> np.ndarray:
        """Per-history records of histories [h0, h1) (TRACK_DTYPE): how each ended,
        its steps, the voxel and type of its last real interaction, the energy of
        the event that ended it and, in binary64, its decision margins."""
        assert TRACK_DTYPE.itemsize == C.sizeof(OrTrack)
        out = np.zeros(h1 - h0, dtype=TRACK_DTYPE)
        fn = lib().or_track_f64 if self.precision == 64 else lib().or_track_f32
        threads = max(1, min(int(threads), max(1, (h1 - h0) // 64)))
        edges = np.linspace(h0, h1, threads + 1).astype(np.int64)

        def work(i):
            a, b = int(edges[i]), int(edges[i + 1])
            if a < b and fn(self.handle, a, b, out[a - h0:].ctypes.data) != 0:
                raise ValueError("oracle transport rejected its arguments")

        if threads == 1:
            work(0)
        else:
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(work, range(threads)))
        return out

    def transport_ranges(self, ranges, threads: int = 1):
        """Transport a list of history ranges [(h0, h1), ...] on `threads` threads,
        each thread with one deposit buffer for all its ranges; returns the summed
        deposits and counts."""
        nvox = self._rho.size
        fn = lib().or_transport_f64 if self.precision == 64 else lib().or_transport_f32
        threads = max(1, min(int(threads), len(ranges)))
        bufs = [np.zeros(nvox, dtype=np.float64) for _ in range(threads)]
        cnts = [OrCounts() for _ in range(threads)]

        def work(i):
            for a, b in ranges[i::threads]:
                if fn(self.handle, a, b, _ptr(bufs[i], C.c_double), C.byref(cnts[i])) != 0:
                    raise ValueError("oracle transport rejected its arguments")

        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(work, range(threads)))
        edep = bufs[0]
        for b in bufs[1:]:
            edep += b
        counts = {k: sum(getattr(c, k) for c in cnts) for k in COUNT_KEYS}
        for k in ("e_emitted", "e_escaped", "e_deposited"):
            counts[k] = float(sum(getattr(c, k) for c in cnts))
        return edep, counts


# --------------------------------------------------------------------------
# batch statistics (Sec. 2.2.1) and precision measures (Sec. 3.1)
# --------------------------------------------------------------------------
def batch_sizes(n_hist: int, n_batches: int):
    lo, rem = divmod(n_hist, n_batches)
    return [lo + 1 if b < rem else lo for b in range(n_batches)]


def voxel_mass_kg(phantom) -> np.ndarray:
    v = phantom.dx * phantom.dy * phantom.dz
    return np.asarray(phantom.rho, dtype=np.float64).ravel() * v / 1000.0


def dose_per_history(edep_kev, mass_kg, n):
    """Gy per source history from keV deposited by n histories; 0 where the mass is 0."""
    out = np.zeros_like(edep_kev)
    ok = mass_kg > 0
    out[ok] = edep_kev[ok] * KEV_TO_J / (mass_kg[ok] * n)
    return out


def batch_statistics(d_batches: np.ndarray):
    """Mean over batches and the standard error of that mean (Sec. 2.2.1):
    D = mean_b d_b, s^2 = sum_b (d_b - D)^2 / (N_b (N_b - 1))."""
    nb = d_batches.shape[0]
    D = d_batches.mean(axis=0)
    s2 = ((d_batches - D) ** 2).sum(axis=0) / (nb * (nb - 1))
    return D, np.sqrt(s2)


def avg_rsd(D, s, rho, frac: float = 0.1, rho_min: float = 0.1):
    """Mean of s/D over voxels with D > frac * D_max and density >= rho_min,
    with D_max taken over the same density mask."""
    rho = np.asarray(rho, dtype=np.float64).ravel()
    dense = rho >= rho_min
    if not dense.any():
        return float("nan")
    dmax = D[dense].max()
    if not dmax > 0:
        return float("nan")
    m = dense & (D > frac * dmax)
    return float(np.mean(s[m] / D[m]))


def paper_sigma_bar(D, s, rho, rho_min: float = 0.1):
    """The paper's measure (Sec. 3.1): s/D_max averaged where D > 0.2 D_max."""
    rho = np.asarray(rho, dtype=np.float64).ravel()
    dense = rho >= rho_min
    dmax = D[dense].max()
    m = dense & (D > 0.2 * dmax)
    return float(np.mean(s[m] / dmax))


@dataclass
class Result:
    dose: np.ndarray          # Gy per history, mean over batches
    std: np.ndarray           # standard error of the mean
    counts: dict
    edep: np.ndarray          # keV summed over all batches
    d_batches: np.ndarray     # per-batch dose per history


def run(problem, precision: int = 64, sampling: str = "surface", threads: int = None,
        setup: Setup = None) -> Result:
    """The whole method on the CPU: N_b batches, statistics after all batches."""
    if threads is None:
        threads = os.cpu_count() or 1
    s = setup if setup is not None else Setup(problem, precision, sampling)
    mass = voxel_mass_kg(problem.phantom)
    sizes = batch_sizes(problem.n_hist, problem.n_batches)
    d_b = np.zeros((problem.n_batches, mass.size), dtype=np.float64)
    edep_total = np.zeros(mass.size, dtype=np.float64)
    counts = None
    h = 0
    for b, n in enumerate(sizes):
        edep, c = s.transport(h, h + n, threads)
        h += n
        d_b[b] = dose_per_history(edep, mass, n)
        edep_total += edep
        counts = c if counts is None else {k: counts[k] + c[k] for k in counts}
    D, sd = batch_statistics(d_b)
    return Result(D, sd, counts, edep_total, d_b)


def efficiency(sigma_bar: float, t_seconds: float) -> float:
    """Simulation efficiency of Sec. 3.1: eps = 1 / (sigma_bar^2 T)."""
    return 1.0 / (sigma_bar * sigma_bar * t_seconds)
