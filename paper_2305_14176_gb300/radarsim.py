"""Thin ctypes binding of libradarsim.so (C ABI in include/radarsim.h).

Argument marshalling only: every step of the simulation runs in the library's
CUDA kernels.  Functions carry the C names.  Pointers may be host numpy arrays
or device tensors (anything with ``data_ptr()`` or ``ctypes.data``).
There is no fallback: if the library is missing, importing raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Dict, Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libradarsim.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "radarsim.h")

SIM_OK = 0
SIM_E_INVALID = -1
SIM_E_NOMEM = -2
SIM_E_BUSY = -3
SIM_E_TIMEOUT = -4
SIM_E_NOT_READY = -5
SIM_E_UNKNOWN_TICKET = -6
SIM_E_CUDA = -7
SIM_E_DEVICE = -8

SIM_WIN_NONE, SIM_WIN_HANN_PERIODIC, SIM_WIN_HANN_SYMMETRIC, SIM_WIN_HANN_NOZERO = 0, 1, 2, 3
SIM_PREC_FP32_DIRECT, SIM_PREC_BF16, SIM_PREC_BF16_SPLIT, SIM_PREC_FP16, SIM_PREC_FP16_SPLIT = 0, 1, 2, 3, 4
SIM_OUT_SIGNAL, SIM_OUT_SPECTRUM, SIM_OUT_LABELS = 1, 2, 4
SIM_MODEL_SEPARABLE, SIM_MODEL_EXACT = 0, 1
PRECISION_NAMES = {"fp32": SIM_PREC_FP32_DIRECT, "bf16": SIM_PREC_BF16, "bf16_split": SIM_PREC_BF16_SPLIT,
                   "fp16": SIM_PREC_FP16, "fp16_split": SIM_PREC_FP16_SPLIT}


class sim_radar_params(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32),
                ("carrier_hz", ctypes.c_double), ("bandwidth_hz", ctypes.c_double),
                ("sweep_time_s", ctypes.c_double), ("chirp_period_s", ctypes.c_double),
                ("n_samples", ctypes.c_int32), ("n_chirps", ctypes.c_int32),
                ("n_tx", ctypes.c_int32), ("n_rx", ctypes.c_int32),
                ("element_spacing_m", ctypes.c_double), ("n_angle", ctypes.c_int32),
                ("window", ctypes.c_int32 * 3), ("precision", ctypes.c_int32),
                ("outputs", ctypes.c_int32), ("max_rays", ctypes.c_int64),
                ("model", ctypes.c_int32), ("pattern_exp", ctypes.c_int32),
                ("tdm_slot_s", ctypes.c_double)]


class sim_rays(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("range_rt_m", ctypes.c_void_p), ("amplitude", ctypes.c_void_p),
                ("radial_velocity_mps", ctypes.c_void_p), ("azimuth_rad", ctypes.c_void_p),
                ("elevation_rad", ctypes.c_void_p), ("phase0_rad", ctypes.c_void_p)]


class sim_meta(ctypes.Structure):
    _fields_ = [("object_id", ctypes.c_void_p), ("material_id", ctypes.c_void_p), ("n_hits", ctypes.c_void_p)]


class sim_span_rule(ctypes.Structure):
    _fields_ = [("object_id", ctypes.c_int32), ("material_id", ctypes.c_int32), ("min_hits", ctypes.c_int32),
                ("max_hits", ctypes.c_int32), ("exclude", ctypes.c_int32)]


class sim_geometry(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_triangles", ctypes.c_int64),
                ("vertices", ctypes.c_void_p), ("triangles", ctypes.c_void_p),
                ("tx_pos", ctypes.c_void_p), ("rx_pos", ctypes.c_void_p),
                ("ref_tx", ctypes.c_double * 3), ("ref_rx", ctypes.c_double * 3)]


class sim_hits(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_void_p), ("triangle", ctypes.c_void_p), ("u", ctypes.c_void_p),
                ("v", ctypes.c_void_p)]


class sim_tuning(ctypes.Structure):
    _fields_ = [("splits", ctypes.c_int32), ("fft_range_points", ctypes.c_int32),
                ("fft_doppler_strip", ctypes.c_int32), ("fft_angle_strip", ctypes.c_int32),
                ("ray_sum_ms", ctypes.c_float), ("fft_ms", ctypes.c_float)]


class SimError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {sim_status_string(code)} ({code})" if what else sim_status_string(code))


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libradarsim.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, U64P = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)
    lib.sim_create.argtypes = [ctypes.POINTER(sim_radar_params), ctypes.POINTER(ctypes.c_void_p)]
    lib.sim_submit.argtypes = [P, ctypes.POINTER(sim_rays), ctypes.POINTER(sim_meta), U64P]
    lib.sim_fetch.argtypes = [P, ctypes.c_uint64, P, P, P, I32]
    lib.sim_destroy.argtypes = [P]
    lib.sim_scene_bytes.argtypes = [P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    lib.sim_status_string.argtypes = [ctypes.c_int]
    lib.sim_status_string.restype = ctypes.c_char_p
    lib.sim_engine_configure.argtypes = [I64, I32, I32]
    lib.sim_last_stage_ms.argtypes = [P, ctypes.POINTER(ctypes.c_float), I32]
    lib.sim_last_kernel_count.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
    lib.sim_last_expansion_terms.argtypes = [P, ctypes.POINTER(ctypes.c_uint32)]
    lib.sim_selftest_umma.argtypes = [I32, I32, I32, I64, P, P, P, P]
    lib.sim_selftest_umma_pair.argtypes = [I32, I32, I64, P, P, P, P]
    lib.sim_selftest_wait.argtypes = [I32, ctypes.POINTER(ctypes.c_int32), P]
    lib.sim_raysum_noalloc.argtypes = [ctypes.POINTER(sim_radar_params), ctypes.POINTER(sim_rays), P, P]
    lib.sim_run_batch.argtypes = [I32, P, ctypes.POINTER(sim_rays), ctypes.POINTER(sim_meta), P, P, P,
                                  ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)]
    lib.sim_run_batch.restype = ctypes.c_int
    lib.sim_autotune.argtypes = [P, I64, ctypes.POINTER(sim_tuning)]
    lib.sim_decompose.argtypes = [P, ctypes.POINTER(sim_rays), ctypes.POINTER(sim_meta), I32,
                                  ctypes.POINTER(sim_span_rule), P, P, ctypes.c_float]
    lib.sim_decompose.restype = ctypes.c_int
    lib.sim_snapshot_paths.argtypes = [P, ctypes.POINTER(sim_rays), ctypes.POINTER(sim_hits),
                                       ctypes.POINTER(sim_geometry), P]
    lib.sim_snapshot_run.argtypes = [P, ctypes.POINTER(sim_rays), ctypes.POINTER(sim_meta),
                                     ctypes.POINTER(sim_hits), ctypes.POINTER(sim_geometry), P, P, P]
    lib.sim_tuning_save.argtypes = [ctypes.c_char_p]
    lib.sim_tuning_load.argtypes = [ctypes.c_char_p]
    for f in ("sim_autotune", "sim_tuning_save", "sim_tuning_load", "sim_tuning_clear", "sim_tuning_count"):
        getattr(lib, f).restype = ctypes.c_int
    for f in ("sim_create", "sim_submit", "sim_fetch", "sim_destroy", "sim_engine_configure",
              "sim_last_stage_ms", "sim_last_kernel_count", "sim_last_expansion_terms", "sim_selftest_umma",
              "sim_raysum_noalloc"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


lib = _load()


def header_functions(path: str = HEADER) -> Sequence[str]:
    """Names of the functions include/radarsim.h declares."""
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sim_[a-z_0-9]+)\s*\(", src)))


def _addr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


# ------------------------------------------------------------------ the C entry points

def sim_status_string(code: int) -> str:
    return lib.sim_status_string(int(code)).decode()


def sim_engine_configure(memory_budget_bytes: int = 0, slots: int = 2, max_queue: int = 64) -> int:
    return lib.sim_engine_configure(int(memory_budget_bytes), int(slots), int(max_queue))


def sim_scene_bytes(ctx, n_rays: int) -> int:
    """Device bytes one admitted scene of n_rays rays holds on this context."""
    b = ctypes.c_int64(0)
    rc = lib.sim_scene_bytes(ctx, int(n_rays), ctypes.byref(b))
    if rc != SIM_OK:
        raise SimError(rc, "sim_scene_bytes")
    return int(b.value)


def sim_create(params: sim_radar_params) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    rc = lib.sim_create(ctypes.byref(params), ctypes.byref(ctx))
    if rc != SIM_OK:
        raise SimError(rc, "sim_create")
    return ctx


def sim_submit(ctx, rays: sim_rays, meta: Optional[sim_meta] = None) -> int:
    t = ctypes.c_uint64()
    rc = lib.sim_submit(ctx, ctypes.byref(rays), ctypes.byref(meta) if meta is not None else None,
                        ctypes.byref(t))
    if rc != SIM_OK:
        raise SimError(rc, "sim_submit")
    return int(t.value)


def sim_fetch(ctx, ticket: int, spectrum=None, signal=None, labels=None, timeout_ms: int = -1) -> int:
    """Returns the status code (SIM_OK, SIM_E_TIMEOUT, ...) without raising."""
    return lib.sim_fetch(ctx, ctypes.c_uint64(ticket), _addr(spectrum), _addr(signal), _addr(labels),
                         int(timeout_ms))


def sim_selftest_umma(f16: int, m: int, n: int, k: int, a, b, d, stream=None) -> int:
    """D = A B^T through the tensor-core tile path (see include/radarsim.h)."""
    return lib.sim_selftest_umma(int(f16), int(m), int(n), int(k), _addr(a), _addr(b), _addr(d),
                                 _addr(stream) if stream is not None else None)


def sim_selftest_umma_pair(f16: int, n: int, k: int, a, b, d, stream=None) -> int:
    """D[256][N] = A B^T through the two-SM tensor-core tile (see include/radarsim.h)."""
    return lib.sim_selftest_umma_pair(int(f16), int(n), int(k), _addr(a), _addr(b), _addr(d),
                                      _addr(stream) if stream is not None else None)


def sim_selftest_wait(limit_ms: int, stream=None):
    """(status, waited_ms) of a bounded wait that nothing ends (see include/radarsim.h)."""
    w = ctypes.c_int32(0)
    rc = lib.sim_selftest_wait(int(limit_ms), ctypes.byref(w), _addr(stream) if stream is not None else None)
    return int(rc), int(w.value)


def sim_raysum_noalloc(params: sim_radar_params, rays: sim_rays, signal, stream=None) -> int:
    """Beat-signal cube into a device buffer with no device allocation (see the header)."""
    return lib.sim_raysum_noalloc(ctypes.byref(params), ctypes.byref(rays), _addr(signal),
                                  _addr(stream) if stream is not None else None)


def sim_run_batch(ctxs, rays, metas, spectra=None, signals=None, labels=None):
    """One batched device pipeline over several scenes (see include/radarsim.h).
    ctxs: list of sim_ctx handles; rays / metas: lists of sim_rays / sim_meta; spectra,
    signals, labels: lists of output buffers (or None).  Returns (status, device_ms, kernels)."""
    n = len(ctxs)
    carr = (ctypes.c_void_p * n)(*[c.value if hasattr(c, "value") else c for c in ctxs])
    rarr = (sim_rays * n)(*rays)
    marr = (sim_meta * n)(*metas)

    def ptrs(bufs):
        if bufs is None:
            return None
        return (ctypes.c_void_p * n)(*[_addr(b) for b in bufs])

    ms = ctypes.c_float()
    kc = ctypes.c_int32()
    rc = lib.sim_run_batch(n, carr, rarr, marr, ptrs(spectra), ptrs(signals), ptrs(labels), ctypes.byref(ms),
                           ctypes.byref(kc))
    return int(rc), float(ms.value), int(kc.value)


def span_rule(object_id=-1, material_id=-1, min_hits=0, max_hits=-1, exclude=False) -> sim_span_rule:
    return sim_span_rule(int(object_id), int(material_id), int(min_hits), int(max_hits), int(bool(exclude)))


def sim_decompose(ctx, rays: sim_rays, meta: sim_meta, rules, span_spectra=None, span_labels=None,
                  threshold: float = 0.0) -> int:
    """Per-span spectra and span labels (see include/radarsim.h); returns the status."""
    n = len(rules)
    rarr = (sim_span_rule * n)(*rules)
    sp = None if span_spectra is None else (ctypes.c_void_p * n)(*[_addr(x) for x in span_spectra])
    return lib.sim_decompose(ctx, ctypes.byref(rays), ctypes.byref(meta) if meta is not None else None, n, rarr,
                             sp, _addr(span_labels), float(threshold))


def make_geometry(arrays: Dict[str, object], ref_tx, ref_rx):
    """(sim_geometry, sim_hits) over arrays keyed vertices [N_c][V][3] f64, triangles [T][3] i32,
    tx_pos [n_tx][3] f64, rx_pos [n_rx][3] f64, hit_offset [n+1] i64, hit_triangle i32, hit_u,
    hit_v f32 (numpy or torch; the caller keeps them alive)."""
    vert, tri = arrays["vertices"], arrays["triangles"]
    g = sim_geometry(int(vert.shape[1]), int(tri.shape[0]), _addr(vert), _addr(tri), _addr(arrays["tx_pos"]),
                     _addr(arrays["rx_pos"]))
    for c in range(3):
        g.ref_tx[c] = float(ref_tx[c])
        g.ref_rx[c] = float(ref_rx[c])
    h = sim_hits(_addr(arrays["hit_offset"]), _addr(arrays["hit_triangle"]), _addr(arrays["hit_u"]),
                 _addr(arrays["hit_v"]))
    return g, h


def sim_snapshot_paths(ctx, rays: sim_rays, hits: sim_hits, geom: sim_geometry, paths) -> int:
    return lib.sim_snapshot_paths(ctx, ctypes.byref(rays), ctypes.byref(hits), ctypes.byref(geom), _addr(paths))


def sim_snapshot_run(ctx, rays: sim_rays, meta: sim_meta, hits: sim_hits, geom: sim_geometry, spectrum=None,
                     signal=None, labels=None) -> int:
    return lib.sim_snapshot_run(ctx, ctypes.byref(rays), ctypes.byref(meta) if meta is not None else None,
                                ctypes.byref(hits), ctypes.byref(geom), _addr(spectrum), _addr(signal),
                                _addr(labels))


def sim_autotune(ctx, n_rays: int) -> sim_tuning:
    t = sim_tuning()
    rc = lib.sim_autotune(ctx, int(n_rays), ctypes.byref(t))
    if rc != SIM_OK:
        raise SimError(rc, "sim_autotune")
    return t


def sim_tuning_save(path: str) -> int:
    return lib.sim_tuning_save(path.encode())


def sim_tuning_load(path: str) -> int:
    return lib.sim_tuning_load(path.encode())


def sim_tuning_clear() -> int:
    return lib.sim_tuning_clear()


def sim_tuning_count() -> int:
    return lib.sim_tuning_count()


def sim_destroy(ctx) -> int:
    return lib.sim_destroy(ctx)


def sim_last_stage_ms(ctx):
    buf = (ctypes.c_float * 7)()
    rc = lib.sim_last_stage_ms(ctx, buf, 7)
    if rc != SIM_OK:
        raise SimError(rc, "sim_last_stage_ms")
    names = ("ingest", "prep", "ray_sum", "ray_sum_reduce", "fft", "labels", "total")
    return dict(zip(names, list(buf)))


def sim_last_kernel_count(ctx) -> int:
    c = ctypes.c_int32()
    rc = lib.sim_last_kernel_count(ctx, ctypes.byref(c))
    if rc != SIM_OK:
        raise SimError(rc, "sim_last_kernel_count")
    return int(c.value)


def sim_last_expansion_terms(ctx) -> set:
    """The route mask of sim_last_expansion_terms as a set of its bits: P for a chunk expanded
    with P Taylor terms, 16 + P with P Chebyshev terms (P = 4, 6, 8), 0 for a chunk that took
    the per-chirp or pair-sum form; empty when no ray sum chose an expansion."""
    m = ctypes.c_uint32()
    rc = lib.sim_last_expansion_terms(ctx, ctypes.byref(m))
    if rc != SIM_OK:
        raise SimError(rc, "sim_last_expansion_terms")
    return {b for b in range(32) if (m.value >> b) & 1}


# ------------------------------------------------------------------ marshalling helpers

def make_params(radar, precision: int = SIM_PREC_FP32_DIRECT,
                outputs: int = SIM_OUT_SIGNAL | SIM_OUT_SPECTRUM | SIM_OUT_LABELS,
                max_rays: int = 1 << 21, model: int = SIM_MODEL_SEPARABLE) -> sim_radar_params:
    """sim_radar_params from any object with the radar attribute names of the ABI."""
    p = sim_radar_params()
    p.struct_size = ctypes.sizeof(sim_radar_params)
    p.carrier_hz = radar.carrier_hz
    p.bandwidth_hz = radar.bandwidth_hz
    p.sweep_time_s = radar.sweep_time_s
    p.chirp_period_s = radar.chirp_period_s
    p.n_samples = radar.n_samples
    p.n_chirps = radar.n_chirps
    p.n_tx = radar.n_tx
    p.n_rx = radar.n_rx
    p.element_spacing_m = radar.element_spacing_m
    p.n_angle = radar.n_angle
    for i in range(3):
        p.window[i] = int(radar.window[i])
    p.precision = int(precision)
    p.outputs = int(outputs)
    p.max_rays = int(max_rays)
    p.model = int(model)
    p.pattern_exp = int(getattr(radar, "pattern_exp", 0))
    p.tdm_slot_s = float(getattr(radar, "tdm_slot_s", 0.0))
    return p


def make_rays(arrays: Dict[str, object], n: int):
    """(sim_rays, sim_meta) over arrays keyed by the ABI field names."""
    r = sim_rays(int(n), _addr(arrays["range_rt_m"]), _addr(arrays["amplitude"]),
                 _addr(arrays["radial_velocity_mps"]), _addr(arrays["azimuth_rad"]),
                 _addr(arrays["elevation_rad"]), _addr(arrays["phase0_rad"]))
    m = sim_meta(_addr(arrays.get("object_id")), _addr(arrays.get("material_id")), _addr(arrays.get("n_hits")))
    return r, m


class Context:
    """Owns one sim_ctx; submit/fetch with numpy (host) or torch (device) arrays."""

    def __init__(self, radar, precision=SIM_PREC_FP32_DIRECT,
                 outputs=SIM_OUT_SIGNAL | SIM_OUT_SPECTRUM | SIM_OUT_LABELS, max_rays=1 << 21,
                 model=SIM_MODEL_SEPARABLE):
        if isinstance(precision, str):
            precision = PRECISION_NAMES[precision]
        self.radar = radar
        self.outputs = outputs
        self.ctx = sim_create(make_params(radar, precision, outputs, max_rays, model))
        self.nv = radar.n_tx * radar.n_rx
        na = radar.n_angle or max(16, 1 << (self.nv - 1).bit_length())
        self.signal_shape = (self.nv, radar.n_chirps, radar.n_samples)
        self.cube_shape = (na, radar.n_chirps, radar.n_samples)

    def submit(self, arrays: Dict[str, object], n: Optional[int] = None) -> int:
        if n is None:
            n = len(arrays["range_rt_m"])
        r, m = make_rays(arrays, n)
        return sim_submit(self.ctx, r, m)

    def fetch(self, ticket, spectrum=None, signal=None, labels=None, timeout_ms=-1) -> int:
        return sim_fetch(self.ctx, ticket, spectrum, signal, labels, timeout_ms)

    def close(self):
        if self.ctx is not None:
            sim_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
