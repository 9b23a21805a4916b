"""Python binding of the dose engine's C ABI (include/ctd.h).

Argument marshalling only: every step of the transport runs in the CUDA
library libctd.so, built in-tree by paper_1109_3266_gb300.build.  The
functions keep the C names.  If the library is missing, loading raises;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libctd.so")

CTD_OK = 0
STATUS = {0: "CTD_OK", 1: "CTD_EINVAL", 2: "CTD_ENOMEM", 3: "CTD_ECUDA", 4: "CTD_EBUSY", 5: "CTD_ETIMEOUT",
          6: "CTD_ECANCELLED", 7: "CTD_ENOTFOUND"}
CTD_SRC_STATIC, CTD_SRC_ARC = 0, 1
CTD_MODE_FULL, CTD_MODE_MAX_REAL = 0, 1


class CtdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class ctd_options(C.Structure):
    _fields_ = [("device", C.c_int), ("stream", C.c_void_p), ("blocks_per_sm", C.c_int),
                ("threads_per_block", C.c_int), ("chunk", C.c_int), ("flight_cap", C.c_int),
                ("multi_blocks_per_sm", C.c_int), ("serve_max_active", C.c_int),
                ("serve_round_histories", C.c_double), ("serve_reserve_bytes", C.c_double),
                ("shared_launch", C.c_int), ("l2_persist", C.c_int), ("plain_overlap", C.c_int),
                ("batch_lanes", C.c_int)]


class ctd_material(C.Structure):
    _fields_ = [("z_over_a", C.c_double), ("a_mol", C.c_double), ("z_eff", C.c_double), ("q0", C.c_double),
                ("sq0", C.c_double)]


class ctd_source(C.Structure):
    _fields_ = [("kind", C.c_int), ("sad_cm", C.c_double), ("u_lo_cm", C.c_double), ("u_hi_cm", C.c_double),
                ("v_lo_cm", C.c_double), ("v_hi_cm", C.c_double), ("n_proj", C.c_int), ("arc0_rad", C.c_double),
                ("arc1_rad", C.c_double), ("continuous", C.c_int), ("z0_cm", C.c_double), ("z1_cm", C.c_double)]


class ctd_physics(C.Structure):
    _fields_ = [("e_min_kev", C.c_int), ("e_max_kev", C.c_int), ("n_zeta", C.c_int), ("majorant_scale", C.c_double),
                ("mode", C.c_int), ("max_real", C.c_int), ("compton_model", C.c_int)]


class ctd_run_stats(C.Structure):
    _fields_ = [("histories", C.c_uint64), ("n_batches", C.c_int)] + \
               [(n, C.c_uint64) for n in ("pe", "compton", "rayleigh", "fictitious", "escaped", "missed", "cutoff",
                                          "terminated", "aborted", "steps")] + \
               [(n, C.c_double) for n in ("e_emitted_kev", "e_escaped_kev", "e_deposited_kev", "avg_rsd",
                                          "paper_sigma_bar", "d_max", "t_total_s", "t_transport_s")] + \
               [("transport_launches", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ctd_request(C.Structure):
    _fields_ = [("batch_histories", C.c_uint64), ("n_histories_max", C.c_uint64), ("rsd_target", C.c_double),
                ("min_batches", C.c_int), ("seed", C.c_uint64)]


class ctd_req_status(C.Structure):
    _fields_ = [("state", C.c_int), ("batches", C.c_int), ("histories", C.c_uint64), ("avg_rsd", C.c_double),
                ("paper_sigma_bar", C.c_double), ("t_queued_s", C.c_double), ("t_latency_s", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_CANCELLED, REQ_FAILED = range(5)


class ctd_tune_result(C.Structure):
    _fields_ = [("blocks_per_sm", C.c_int), ("chunk", C.c_int), ("flight_cap", C.c_int), ("n_tried", C.c_int),
                ("histories_per_s", C.c_double), ("baseline_per_s", C.c_double), ("threads_per_block", C.c_int),
                ("shared_launch", C.c_int), ("multi_blocks_per_sm", C.c_int), ("batch_lanes", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

_lib = None


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise CtdError(3, f"CUDA library not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P, dp, fp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_float)
        L.ctd_last_error.restype = C.c_char_p
        L.ctd_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(ctd_options)]
        L.ctd_destroy.argtypes = [P]
        L.ctd_create_phantom.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                         C.POINTER(C.c_uint8), fp, C.c_int, C.POINTER(ctd_material),
                                         C.POINTER(C.c_int32)]
        L.ctd_destroy_phantom.argtypes = [P, C.c_int32]
        L.ctd_set_physics.argtypes = [P, C.c_int32, C.POINTER(ctd_physics)]
        L.ctd_set_material_elements.argtypes = [P, C.c_int32, C.c_int, C.c_int, C.POINTER(C.c_int), dp]
        L.ctd_set_source.argtypes = [P, C.c_int32, C.POINTER(ctd_source)]
        L.ctd_set_spectrum.argtypes = [P, C.c_int32, dp, dp, dp, C.c_int]
        L.ctd_run.argtypes = [P, C.c_int32, C.c_uint64, C.c_uint64, C.c_int]
        L.ctd_run_range.argtypes = [P, C.c_int32, C.c_uint64, C.c_uint64, C.c_int, C.c_uint64, C.c_uint64, C.c_int]
        L.ctd_trace_range.argtypes = [P, C.c_int32, C.c_uint64, C.c_uint64, C.c_int, C.c_uint64, C.c_uint64, P]
        L.ctd_mh_beamlets.argtypes = [P, C.c_int, dp, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64,
                                      C.POINTER(C.c_uint64)]
        L.ctd_shard_begin.argtypes = [P, C.c_int32, C.c_uint64, C.c_uint64, C.c_int]
        L.ctd_shard_batch.argtypes = [P, C.c_int32, C.c_int, C.c_uint64, C.c_uint64, P]
        L.ctd_shard_fold.argtypes = [P, C.c_int32, C.c_int, P]
        L.ctd_shard_counts.argtypes = [P, C.c_int32, C.POINTER(C.c_uint64), dp]
        L.ctd_shard_finish.argtypes = [P, C.c_int32, C.POINTER(C.c_uint64), dp]
        L.ctd_get_dose_and_stddev.argtypes = [P, C.c_int32, dp, dp, C.c_size_t, C.POINTER(ctd_run_stats)]
        L.ctd_get_edep.argtypes = [P, C.c_int32, dp, C.c_size_t]
        L.ctd_get_tables.argtypes = [P, C.c_int32, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     dp, dp, dp, dp]
        L.ctd_sample_mu.argtypes = [P, C.c_int32, C.c_int, C.c_int, C.c_double, C.c_uint64, C.c_uint64, dp]
        L.ctd_eval_math.argtypes = [P, C.c_int, fp, fp, C.c_size_t]
        L.ctd_avg_rsd_noalloc.argtypes = [P, P, P, C.c_size_t, P, P]
        L.ctd_run_batch.argtypes = [P, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                    C.c_int]
        L.ctd_submit.argtypes = [P, C.c_int32, C.POINTER(ctd_request), C.POINTER(C.c_int64)]
        L.ctd_serve_step.argtypes = [P, C.POINTER(C.c_int)]
        L.ctd_serve_wait.argtypes = [P, C.c_double, C.POINTER(C.c_int)]
        L.ctd_poll.argtypes = [P, C.c_int64, C.POINTER(ctd_req_status)]
        L.ctd_wait.argtypes = [P, C.c_int64, C.c_double, C.POINTER(ctd_req_status)]
        L.ctd_cancel.argtypes = [P, C.c_int64]
        L.ctd_autotune.argtypes = [P, C.c_int32, C.c_uint64, C.c_uint64, C.POINTER(ctd_tune_result)]
        L.ctd_autotune_batch.argtypes = [P, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_uint64),
                                         C.POINTER(C.c_uint64), C.c_int, C.c_double, C.POINTER(ctd_tune_result)]
        L.ctd_probe_memory.argtypes = [P, C.c_int, C.c_uint64, C.c_uint64, dp]
        L.ctd_set_fluence.argtypes = [P, C.c_int32, C.c_int, C.c_int, dp]
        L.ctd_spectrum_kramers.argtypes = [C.c_int, C.c_double, C.c_int, dp, dp, dp, C.POINTER(C.c_int)]
        L.ctd_material_columns.argtypes = [C.POINTER(ctd_material), C.c_int, C.POINTER(C.c_int), dp, C.c_int,
                                           C.c_int, C.c_int, dp]
        L.ctd_allocate_histories.argtypes = [C.c_uint64, C.c_int, dp, C.POINTER(C.c_uint64)]
        L.ctd_alias_table.argtypes = [C.c_int, dp, C.POINTER(C.c_uint32), C.POINTER(C.c_int32)]
        L.ctd_angular_surface.argtypes = [C.c_int, C.POINTER(ctd_material), C.c_int, C.POINTER(C.c_int), dp,
                                          C.c_int, C.c_int, C.c_int, dp]
        L.ctd_get_fluence_table.argtypes = [P, C.c_int32, C.POINTER(C.c_int), C.POINTER(C.c_uint32),
                                            C.POINTER(C.c_int32)]
        _lib = L
    return _lib


def _check(rc):
    if rc != CTD_OK:
        raise CtdError(rc, lib().ctd_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# --------------------------------------------------------------------------- C names
def ctd_create(device=0, stream=None, blocks_per_sm=0, threads_per_block=0, chunk=0, flight_cap=0,
               multi_blocks_per_sm=0, serve_max_active=0, serve_round_histories=0.0, shared_launch=0,
               serve_reserve_bytes=0.0, l2_persist=0, plain_overlap=0, batch_lanes=0):
    """Context handle.  stream: a CUDA stream handle (int), e.g. torch's current stream.
    shared_launch: batched and served forms share one multi-request launch per
    batch (1) instead of one chain of single-request launches per request (0).
    l2_persist: plain-form launches keep the tally (1) or the voxel words (2) persisting
    in L2 (-1 or 0: neither).  plain_overlap: ctd_run alternates its batches between
    two streams with a tally each (1; 0 or -1: one stream)."""
    opt = ctd_options(device, stream or None, blocks_per_sm, threads_per_block, chunk, flight_cap, multi_blocks_per_sm,
                      serve_max_active, float(serve_round_histories), float(serve_reserve_bytes), int(shared_launch),
                      int(l2_persist), int(plain_overlap), int(batch_lanes))
    h = C.c_void_p()
    _check(lib().ctd_create(C.byref(h), C.byref(opt)))
    return h


def ctd_destroy(ctx):
    _check(lib().ctd_destroy(ctx))


def ctd_create_phantom(ctx, nx, ny, nz, dx, dy, dz, mat, density, materials):
    """materials: records with z_over_a, a_mol, z_eff, q0."""
    mat = np.ascontiguousarray(mat, dtype=np.uint8).ravel()
    density = np.ascontiguousarray(density, dtype=np.float32).ravel()
    n = nx * ny * nz
    if mat.size != n or density.size != n:
        raise CtdError(1, "voxel arrays must hold nx*ny*nz values")
    ms = (ctd_material * len(materials))(*[ctd_material(m.z_over_a, m.a_mol, m.z_eff, m.q0, m.sq0)
                                            for m in materials])
    out = C.c_int32()
    _check(lib().ctd_create_phantom(ctx, nx, ny, nz, dx, dy, dz, mat.ctypes.data_as(C.POINTER(C.c_uint8)),
                                    density.ctypes.data_as(C.POINTER(C.c_float)), len(materials), ms, C.byref(out)))
    return out.value


def ctd_destroy_phantom(ctx, ph):
    _check(lib().ctd_destroy_phantom(ctx, ph))


CTD_COMPTON_KN, CTD_COMPTON_WH = 0, 1


def ctd_set_physics(ctx, ph, e_min_kev=1, e_max_kev=150, n_zeta=1024, majorant_scale=1.0, mode="full", max_real=0,
                    compton="kn"):
    """compton: "kn" (free-electron Klein-Nishina) or "wh" (Waller-Hartree)."""
    m = {"full": CTD_MODE_FULL, "max_real": CTD_MODE_MAX_REAL}[mode] if isinstance(mode, str) else int(mode)
    c = {"kn": CTD_COMPTON_KN, "wh": CTD_COMPTON_WH}[compton] if isinstance(compton, str) else int(compton)
    p = ctd_physics(e_min_kev, e_max_kev, n_zeta, majorant_scale, m, max_real, c)
    _check(lib().ctd_set_physics(ctx, ph, C.byref(p)))


def ctd_set_material_elements(ctx, ph, material, elements):
    """Independent-atom Rayleigh form factor for one material: elements is
    ((Z, atoms per formula unit), ...); empty restores the analytic form factor."""
    n, z, cnt = _element_arrays(elements)
    _check(lib().ctd_set_material_elements(ctx, ph, int(material), n, z, _dp(cnt)))


def ctd_set_source(ctx, ph, kind, sad_cm, u_lo_cm, u_hi_cm, v_lo_cm, v_hi_cm, n_proj=1, arc0_rad=0.0,
                   arc1_rad=2 * np.pi, continuous=False, z0_cm=0.0, z1_cm=0.0):
    """z0_cm, z1_cm: arc source height at arc0 and arc1 (helical trajectory)."""
    k = {"static": CTD_SRC_STATIC, "arc": CTD_SRC_ARC}[kind] if isinstance(kind, str) else int(kind)
    s = ctd_source(k, sad_cm, u_lo_cm, u_hi_cm, v_lo_cm, v_hi_cm, n_proj, arc0_rad, arc1_rad, int(continuous),
                   float(z0_cm), float(z1_cm))
    _check(lib().ctd_set_source(ctx, ph, C.byref(s)))


def ctd_set_spectrum(ctx, ph, e_lo, e_hi, w):
    e_lo = np.ascontiguousarray(e_lo, dtype=np.float64)
    e_hi = np.ascontiguousarray(e_hi, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    _check(lib().ctd_set_spectrum(ctx, ph, _dp(e_lo), _dp(e_hi), _dp(w), len(w)))


def ctd_run(ctx, ph, n_histories, seed, n_batches):
    _check(lib().ctd_run(ctx, ph, int(n_histories), int(seed), int(n_batches)))


def ctd_run_batch(ctx, phantoms, n_histories, seeds, n_batches):
    """Batched form: every request's batch b in one shared launch."""
    n = len(phantoms)
    ph = (C.c_int32 * n)(*phantoms)
    nh = (C.c_uint64 * n)(*[int(x) for x in n_histories])
    sd = (C.c_uint64 * n)(*[int(x) for x in seeds])
    _check(lib().ctd_run_batch(ctx, n, ph, nh, sd, int(n_batches)))


def ctd_submit(ctx, ph, batch_histories, rsd_target, seed, n_histories_max=0, min_batches=0):
    """Queue a served request; returns its id."""
    r = ctd_request(int(batch_histories), int(n_histories_max), float(rsd_target), int(min_batches), int(seed))
    out = C.c_int64()
    _check(lib().ctd_submit(ctx, ph, C.byref(r), C.byref(out)))
    return out.value


def ctd_serve_wait(ctx, timeout_s):
    """Step the served form until something changed or timeout_s passed; returns the
    number of requests still queued or running."""
    n = C.c_int()
    _check(lib().ctd_serve_wait(ctx, float(timeout_s), C.byref(n)))
    return n.value


def ctd_serve_step(ctx):
    """One round of the served form; returns the number of requests still queued or running."""
    n = C.c_int()
    _check(lib().ctd_serve_step(ctx, C.byref(n)))
    return n.value


def ctd_poll(ctx, req_id):
    st = ctd_req_status()
    _check(lib().ctd_poll(ctx, int(req_id), C.byref(st)))
    return st.as_dict()


def ctd_wait(ctx, req_id, timeout_s):
    st = ctd_req_status()
    _check(lib().ctd_wait(ctx, int(req_id), float(timeout_s), C.byref(st)))
    return st.as_dict()


def ctd_cancel(ctx, req_id):
    _check(lib().ctd_cancel(ctx, int(req_id)))


def ctd_autotune(ctx, ph, n_probe, seed=1):
    """Pick the fastest launch shape for this phantom's problem; returns the choice."""
    r = ctd_tune_result()
    _check(lib().ctd_autotune(ctx, ph, int(n_probe), int(seed), C.byref(r)))
    return r.as_dict()


def ctd_autotune_batch(ctx, phantoms, n_histories, seeds, n_batches, probe_fraction=0.05):
    """Pick the batched form's launch design and shape for these requests (kept in the
    context); returns the choice."""
    n = len(phantoms)
    ph = (C.c_int32 * n)(*phantoms)
    nh = (C.c_uint64 * n)(*[int(x) for x in n_histories])
    sd = (C.c_uint64 * n)(*[int(x) for x in seeds])
    r = ctd_tune_result()
    _check(lib().ctd_autotune_batch(ctx, n, ph, nh, sd, int(n_batches), float(probe_fraction), C.byref(r)))
    return r.as_dict()


def ctd_run_range(ctx, ph, n_histories, seed, n_batches, h_begin, h_end, clear=True):
    _check(lib().ctd_run_range(ctx, ph, int(n_histories), int(seed), int(n_batches), int(h_begin), int(h_end),
                               int(bool(clear))))


def ctd_shard_begin(ctx, ph, n_histories, seed, n_batches):
    _check(lib().ctd_shard_begin(ctx, ph, int(n_histories), int(seed), int(n_batches)))


def ctd_shard_batch(ctx, ph, batch, local_begin, local_end, tally_dev):
    """Add local histories [local_begin, local_end) of `batch` to the device buffer at
    address tally_dev (nvox doubles, e.g. a torch tensor's data_ptr())."""
    _check(lib().ctd_shard_batch(ctx, ph, int(batch), int(local_begin), int(local_end), int(tally_dev)))


def ctd_shard_fold(ctx, ph, batch, tally_dev):
    """Fold the summed batch tally at device address tally_dev; leaves it zeroed."""
    _check(lib().ctd_shard_fold(ctx, ph, int(batch), int(tally_dev)))


def ctd_shard_counts(ctx, ph):
    """This rank's counts (10 uint64) and emitted/escaped energies (2 doubles)."""
    c = np.zeros(10, dtype=np.uint64)
    e = np.zeros(2, dtype=np.float64)
    _check(lib().ctd_shard_counts(ctx, ph, c.ctypes.data_as(C.POINTER(C.c_uint64)), _dp(e)))
    return c, e


def ctd_shard_finish(ctx, ph, counts, energies):
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    e = np.ascontiguousarray(energies, dtype=np.float64)
    _check(lib().ctd_shard_finish(ctx, ph, c.ctypes.data_as(C.POINTER(C.c_uint64)), _dp(e)))


# ctd_track records as numpy sees them
TRACK_DTYPE = np.dtype([("code", np.uint32), ("steps", np.uint32), ("idx", np.uint32), ("e_end_kev", np.float32)])
END_NAMES = ("pe", "cutoff", "escaped", "missed", "terminated", "aborted")


def ctd_trace_range(ctx, ph, n_histories, seed, n_batches, h_begin, h_end):
    """Per-history records of histories [h_begin, h_end): a structured array with
    end (0 photoelectric, 1 cutoff, 2 escaped, 3 missed, 4 terminated, 5 aborted,
    -1 never ended), last_type (0 PE, 1 Compton, 2 Rayleigh, -1 none), steps, idx
    and e_end (keV)."""
    raw = np.zeros(int(h_end) - int(h_begin), dtype=TRACK_DTYPE)
    _check(lib().ctd_trace_range(ctx, ph, int(n_histories), int(seed), int(n_batches), int(h_begin), int(h_end),
                                 raw.ctypes.data if raw.size else None))
    out = np.zeros(raw.size, dtype=[("end", np.int32), ("last_type", np.int32), ("steps", np.uint32),
                                    ("idx", np.uint32), ("e_end", np.float64)])
    out["end"] = (raw["code"] & 0xff).astype(np.int32) - 1
    out["last_type"] = ((raw["code"] >> 8) & 0xff).astype(np.int32) - 1
    out["steps"] = raw["steps"]
    out["idx"] = raw["idx"]
    out["e_end"] = raw["e_end_kev"]
    return out


def ctd_get_dose_and_stddev(ctx, ph, nvox, want_arrays=True):
    """(dose, stddev, stats) -- Gy per history, standard error, stats dict."""
    st = ctd_run_stats()
    if want_arrays:
        dose = np.empty(nvox, dtype=np.float64)
        sd = np.empty(nvox, dtype=np.float64)
        _check(lib().ctd_get_dose_and_stddev(ctx, ph, _dp(dose), _dp(sd), nvox, C.byref(st)))
        return dose, sd, st.as_dict()
    _check(lib().ctd_get_dose_and_stddev(ctx, ph, None, None, 0, C.byref(st)))
    return None, None, st.as_dict()


def ctd_get_edep(ctx, ph, nvox):
    out = np.empty(nvox, dtype=np.float64)
    _check(lib().ctd_get_edep(ctx, ph, _dp(out), nvox))
    return out


def ctd_get_tables(ctx, ph, compton="kn"):
    """Tables as the device holds them; C surfaces [n_e][n_zeta], or
    [n_mat][n_e][n_zeta] for a phantom set to the Waller-Hartree model."""
    ne, nz, nm = C.c_int(), C.c_int(), C.c_int()
    _check(lib().ctd_get_tables(ctx, ph, C.byref(ne), C.byref(nz), C.byref(nm), None, None, None, None))
    ne, nz, nm = ne.value, nz.value, nm.value
    cum = np.empty((nm, ne, 3))
    mm = np.empty(ne)
    cs = np.empty((nm, ne, nz) if compton == "wh" else (ne, nz))
    rs = np.empty((nm, ne, nz))
    _check(lib().ctd_get_tables(ctx, ph, None, None, None, _dp(cum), _dp(mm), _dp(cs), _dp(rs)))
    return cum, mm, cs, rs


def ctd_sample_mu(ctx, ph, kind, material, e_kev, seed, n):
    out = np.empty(n, dtype=np.float64)
    k = {"compton": 0, "rayleigh": 1}[kind] if isinstance(kind, str) else int(kind)
    _check(lib().ctd_sample_mu(ctx, ph, k, material, e_kev, seed, n, _dp(out)))
    return out


def ctd_eval_math(ctx, fn, x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.size * (2 if fn == 1 else 1), dtype=np.float32)
    _check(lib().ctd_eval_math(ctx, fn, x.ctypes.data_as(C.POINTER(C.c_float)),
                               out.ctypes.data_as(C.POINTER(C.c_float)), x.size))
    return out


def ctd_avg_rsd_noalloc(dose_dev, stddev_dev, density_dev, nvox, result_dev, stream=None):
    """Allocation-free avg RSD of device arrays (integer device addresses, e.g.
    torch's data_ptr()); writes avg RSD, sigma_bar and D_max to 3 device doubles
    at result_dev, asynchronously on stream.  For callers that cannot allocate
    device memory at that point (inside stream capture, or under a host-owned
    memory pool); it uses a fixed scratch array inside the library instead."""
    _check(lib().ctd_avg_rsd_noalloc(dose_dev, stddev_dev, density_dev, int(nvox), result_dev, stream or None))


# --------------------------------------------------------------------------- problem helpers
def load_problem(ctx, problem, physics=True):
    """Create the phantom of an inputs.Problem and set its source, spectrum and physics."""
    ph_ = problem.phantom
    h = ctd_create_phantom(ctx, ph_.nx, ph_.ny, ph_.nz, ph_.dx, ph_.dy, ph_.dz, ph_.mat, ph_.rho, ph_.materials)
    s = problem.source
    ctd_set_source(ctx, h, s.kind, s.sad, s.u_lo, s.u_hi, s.v_lo, s.v_hi, s.n_proj, s.arc0, s.arc1, s.continuous,
                   getattr(s, "z0", 0.0), getattr(s, "z1", 0.0))
    sp = problem.spectrum
    ctd_set_spectrum(ctx, h, sp.e_lo, sp.e_hi, sp.w)
    if getattr(s, "fluence", None) is not None:
        ctd_set_fluence(ctx, h, s.fluence)
    if physics:
        p = problem.physics
        ctd_set_physics(ctx, h, p.e_min, p.e_max, p.n_zeta, p.majorant_scale, p.mode, p.max_real,
                        getattr(p, "compton", "kn"))
        if getattr(p, "rayleigh", "gauss") == "iaa":
            for m, mat in enumerate(ph_.materials):
                ctd_set_material_elements(ctx, h, m, mat.elements)
    return h


def ctd_spectrum_kramers(kvp, mm_al, e_min=1):
    """Kramers' spectrum with aluminium filtration on 1 keV bins: (e_lo, e_hi, w)."""
    n = C.c_int()
    _check(lib().ctd_spectrum_kramers(int(kvp), float(mm_al), int(e_min), None, None, None, C.byref(n)))
    lo, hi, w = (np.empty(n.value) for _ in range(3))
    _check(lib().ctd_spectrum_kramers(int(kvp), float(mm_al), int(e_min), _dp(lo), _dp(hi), _dp(w), C.byref(n)))
    return lo, hi, w


def _element_arrays(elements):
    n = len(elements)
    z = (C.c_int * max(n, 1))(*[int(e[0]) for e in elements])
    cnt = np.ascontiguousarray([float(e[1]) for e in elements] or [0.0], dtype=np.float64)
    return n, z, cnt


def ctd_material_columns(material, e_min_kev=1, e_max_kev=150, compton="kn", elements=()):
    """Host physics: the binary64 node-table columns [n_e][3] of one material
    (photoelectric, + Compton, + Rayleigh); elements select the independent-atom
    Rayleigh form factor."""
    m = ctd_material(material.z_over_a, material.a_mol, material.z_eff, material.q0, material.sq0)
    c = {"kn": CTD_COMPTON_KN, "wh": CTD_COMPTON_WH}[compton] if isinstance(compton, str) else int(compton)
    n, z, cnt = _element_arrays(elements)
    out = np.empty((e_max_kev - e_min_kev + 1, 3), dtype=np.float64)
    _check(lib().ctd_material_columns(C.byref(m), n, z, _dp(cnt), int(e_min_kev), int(e_max_kev), c, _dp(out)))
    return out


def ctd_angular_surface(kind, material, e_min_kev=1, e_max_kev=150, n_zeta=1024, elements=()):
    """Host physics: the binary64 surface rows [n_e][n_zeta]; kind "kn" (C surface),
    "rayleigh" (R surface; elements select the independent-atom form factor) or
    "wh" (Waller-Hartree C surface)."""
    k = {"kn": 0, "rayleigh": 1, "wh": 2}[kind] if isinstance(kind, str) else int(kind)
    m = ctd_material(material.z_over_a, material.a_mol, material.z_eff, material.q0, material.sq0)
    n, z, cnt = _element_arrays(elements)
    out = np.empty((e_max_kev - e_min_kev + 1, n_zeta), dtype=np.float64)
    _check(lib().ctd_angular_surface(k, C.byref(m), n, z, _dp(cnt), int(e_min_kev), int(e_max_kev), int(n_zeta),
                                     _dp(out)))
    return out


def ctd_allocate_histories(n, w):
    """Host logic: n histories over spectrum bins of weights w by largest remainder."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.empty(w.size, dtype=np.uint64)
    _check(lib().ctd_allocate_histories(int(n), w.size, _dp(w), out.ctypes.data_as(C.POINTER(C.c_uint64))))
    return out


def ctd_alias_table(f):
    """Host logic: the Walker alias table (thresholds uint32, aliases int32) of intensities f."""
    f = np.ascontiguousarray(f, dtype=np.float64).ravel()
    thr = np.empty(f.size, dtype=np.uint32)
    al = np.empty(f.size, dtype=np.int32)
    _check(lib().ctd_alias_table(f.size, _dp(f), thr.ctypes.data_as(C.POINTER(C.c_uint32)),
                                 al.ctypes.data_as(C.POINTER(C.c_int32))))
    return thr, al


def ctd_set_fluence(ctx, ph, f):
    """Fluence map f[n_v][n_u] over the source's field (None removes it)."""
    if f is None:
        _check(lib().ctd_set_fluence(ctx, ph, 0, 0, None))
        return
    f = np.ascontiguousarray(f, dtype=np.float64)
    if f.ndim != 2:
        raise CtdError(1, "fluence map must be [n_v][n_u]")
    _check(lib().ctd_set_fluence(ctx, ph, f.shape[1], f.shape[0], _dp(f)))


def ctd_mh_beamlets(ctx, f, n, seed, chains, i0=0):
    """Beamlet visit counts of the paper's Metropolis-Hastings sampler (Algorithm A1) run on
    the device as `chains` chains, one per thread."""
    f = np.ascontiguousarray(f, dtype=np.float64).ravel()
    out = np.zeros(f.size, dtype=np.uint64)
    _check(lib().ctd_mh_beamlets(ctx, f.size, _dp(f), int(i0), int(n), int(seed), int(chains),
                                 out.ctypes.data_as(C.POINTER(C.c_uint64))))
    return out


def ctd_get_fluence_table(ctx, ph):
    """The fluence map's alias table: (thresholds uint32, aliases int32)."""
    n = C.c_int()
    _check(lib().ctd_get_fluence_table(ctx, ph, C.byref(n), None, None))
    thr = np.empty(n.value, dtype=np.uint32)
    al = np.empty(n.value, dtype=np.int32)
    _check(lib().ctd_get_fluence_table(ctx, ph, None, thr.ctypes.data_as(C.POINTER(C.c_uint32)),
                                       al.ctypes.data_as(C.POINTER(C.c_int32))))
    return thr, al


def run_problem(ctx, problem, handle=None):
    """Run a problem end to end: (dose, stddev, stats, handle)."""
    h = handle if handle is not None else load_problem(ctx, problem)
    ctd_run(ctx, h, problem.n_hist, problem.seed, problem.n_batches)
    dose, sd, st = ctd_get_dose_and_stddev(ctx, h, problem.phantom.nvox)
    return dose, sd, st, h


PROBE_L2_RED, PROBE_GATHER4, PROBE_VOXEL = 0, 1, 2


def ctd_probe_memory(ctx, kind, n_slots, n_ops):
    """Rate (operations/s) of random binary64 L2 reductions (kind 0), 4-byte
    gathers (1) or voxel gathers (2) over n_slots slots."""
    r = C.c_double()
    _check(lib().ctd_probe_memory(ctx, int(kind), C.c_uint64(n_slots), C.c_uint64(n_ops), C.byref(r)))
    return r.value
