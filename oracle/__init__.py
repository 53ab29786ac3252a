"""FP64 CPU oracle (ctypes binding over ``oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product library
never does.  It is a plain, slow restatement of the paper's signal model
(arXiv 2305.14176, Sec. II-A Eqs. 1-4, Sec. II-C Eq. 5, Sec. II-E Eq. 7) in
FP64, independent of the CUDA path: no shared code, headers, tables or
constants.

Functions and the passage each follows:
  signal        Eq. 2 with Eq. 1 and Eq. 3, separable reading (beat cube s[k,m,n])
  signal_at     the same sum at chosen (k, m, n)
  spectrum      Eq. 4, naive windowed DFT along range, Doppler, then angle (zero padded)
  cell_dtft     Eq. 4 applied ray by ray (linearity, Eq. 5): windowed DTFT per cell
  bins, labels  Sec. II-C (decomposition by object id) and its automatic annotation
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# RADAR_ORACLE_LIB points at another build of oracle.c (the pin-sensitivity test's mutants)
_LIB_PATH = os.environ.get("RADAR_ORACLE_LIB", os.path.join(_HERE, "liboracle.so"))
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (FP64, no contraction, no fast-math)."""
    if "RADAR_ORACLE_LIB" in os.environ:
        return _LIB_PATH
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src),
                                                   os.path.getmtime(os.path.join(_HERE, "oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-std=c11", "-D_GNU_SOURCE", "-Wall", "-o", tmp, src, "-lm", "-lpthread"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Radar(ctypes.Structure):
    _fields_ = [("carrier_hz", ctypes.c_double), ("bandwidth_hz", ctypes.c_double),
                ("sweep_time_s", ctypes.c_double), ("chirp_period_s", ctypes.c_double),
                ("n_samples", ctypes.c_int32), ("n_chirps", ctypes.c_int32),
                ("n_tx", ctypes.c_int32), ("n_rx", ctypes.c_int32),
                ("element_spacing_m", ctypes.c_double), ("n_angle", ctypes.c_int32),
                ("window", ctypes.c_int32 * 3), ("model", ctypes.c_int32), ("pattern_exp", ctypes.c_int32),
                ("tdm_slot_s", ctypes.c_double)]


class _Rays(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("range_rt_m", ctypes.c_void_p),
                ("amplitude", ctypes.c_void_p), ("radial_velocity_mps", ctypes.c_void_p),
                ("azimuth_rad", ctypes.c_void_p), ("elevation_rad", ctypes.c_void_p),
                ("phase0_rad", ctypes.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_signal.argtypes = [P, P, P, ctypes.c_int]
            lib.orc_signal_at.argtypes = [P, P, ctypes.c_int64, P, P, ctypes.c_int]
            lib.orc_spectrum.argtypes = [P, P, P, ctypes.c_int]
            lib.orc_cell_dtft.argtypes = [P, P, ctypes.c_int64, P, P, ctypes.c_int]
            lib.orc_window.argtypes = [P, ctypes.c_int, P]
            lib.orc_bins.argtypes = [P, P, P, P, P, P, P]
            lib.orc_labels.argtypes = [P, P, P, P]
            lib.orc_cell_object_energy.argtypes = [P, P, P, P, P, P]
            lib.orc_cell_object_energy.restype = ctypes.c_int64
            lib.orc_sin_rep.argtypes = [ctypes.c_double]
            lib.orc_sin_rep.restype = ctypes.c_double
            lib.orc_cos_rep.argtypes = [ctypes.c_double]
            lib.orc_cos_rep.restype = ctypes.c_double
            lib.orc_default_threads.restype = ctypes.c_int
            lib.orc_paths.argtypes = [P, P, P, P, ctypes.c_int]
            lib.orc_signal_geom.argtypes = [P, P, P, P, ctypes.c_int]
            lib.orc_signal_geom_at.argtypes = [P, P, P, ctypes.c_int64, P, P, ctypes.c_int]
            _lib = lib
    return _lib


def _radar(radar) -> _Radar:
    r = _Radar()
    r.carrier_hz = radar.carrier_hz
    r.bandwidth_hz = radar.bandwidth_hz
    r.sweep_time_s = radar.sweep_time_s
    r.chirp_period_s = radar.chirp_period_s
    r.n_samples = radar.n_samples
    r.n_chirps = radar.n_chirps
    r.n_tx = radar.n_tx
    r.n_rx = radar.n_rx
    r.element_spacing_m = radar.element_spacing_m
    r.n_angle = radar.n_angle
    for i in range(3):
        r.window[i] = int(radar.window[i])
    r.model = int(getattr(radar, "model", 0))
    r.pattern_exp = int(getattr(radar, "pattern_exp", 0))
    r.tdm_slot_s = float(getattr(radar, "tdm_slot_s", 0.0))
    return r


class _RayRef:
    """Keeps contiguous typed copies alive while the C call runs."""

    def __init__(self, rays):
        self.d = np.ascontiguousarray(rays.range_rt_m, np.float64)
        self.a = np.ascontiguousarray(rays.amplitude, np.float32)
        self.v = np.ascontiguousarray(rays.radial_velocity_mps, np.float32)
        self.az = np.ascontiguousarray(rays.azimuth_rad, np.float32)
        self.el = np.ascontiguousarray(rays.elevation_rad, np.float32)
        self.p0 = np.ascontiguousarray(rays.phase0_rad, np.float32)
        self.obj = np.ascontiguousarray(rays.object_id, np.int32)
        self.s = _Rays(self.d.shape[0], self.d.ctypes.data, self.a.ctypes.data, self.v.ctypes.data,
                       self.az.ctypes.data, self.el.ctypes.data, self.p0.ctypes.data)


class _Geometry(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_triangles", ctypes.c_int64),
                ("vertices", ctypes.c_void_p), ("triangles", ctypes.c_void_p),
                ("tx_pos", ctypes.c_void_p), ("rx_pos", ctypes.c_void_p),
                ("ref_tx", ctypes.c_double * 3), ("ref_rx", ctypes.c_double * 3),
                ("hit_offset", ctypes.c_void_p), ("hit_triangle", ctypes.c_void_p),
                ("hit_u", ctypes.c_void_p), ("hit_v", ctypes.c_void_p)]


class _GeomRef:
    """Contiguous typed copies of a scene's mesh, antennas and hit lists for one C call."""

    def __init__(self, radar, rays, hits, geom):
        self.vert = np.ascontiguousarray(geom.vertices, np.float64)
        self.tri = np.ascontiguousarray(geom.triangles, np.int32)
        self.tx = np.ascontiguousarray(geom.tx_pos, np.float64)
        self.rx = np.ascontiguousarray(geom.rx_pos, np.float64)
        self.off = np.ascontiguousarray(hits.offset, np.int64)
        self.ht = np.ascontiguousarray(hits.triangle, np.int32)
        self.hu = np.ascontiguousarray(hits.u, np.float32)
        self.hv = np.ascontiguousarray(hits.v, np.float32)
        assert self.vert.shape[0] == radar.n_chirps and self.vert.shape[2] == 3
        assert self.tx.shape == (radar.n_tx, 3) and self.rx.shape == (radar.n_rx, 3)
        assert self.off.shape[0] == rays.n + 1 and np.all(np.diff(self.off) >= 1)
        assert np.all((self.tri >= 0) & (self.tri < self.vert.shape[1]))
        assert np.all((self.ht >= 0) & (self.ht < self.tri.shape[0]))
        g = _Geometry()
        g.n_vertices = self.vert.shape[1]
        g.n_triangles = self.tri.shape[0]
        g.vertices, g.triangles = self.vert.ctypes.data, self.tri.ctypes.data
        g.tx_pos, g.rx_pos = self.tx.ctypes.data, self.rx.ctypes.data
        for c in range(3):
            g.ref_tx[c] = float(geom.ref_tx[c])
            g.ref_rx[c] = float(geom.ref_rx[c])
        g.hit_offset, g.hit_triangle = self.off.ctypes.data, self.ht.ctypes.data
        g.hit_u, g.hit_v = self.hu.ctypes.data, self.hv.ctypes.data
        self.s = g


def _ptr(a: np.ndarray):
    return a.ctypes.data


def threads() -> int:
    return int(_load().orc_default_threads())


def signal(radar, rays, nthreads: int = 0) -> np.ndarray:
    """complex128[N_v, N_c, N_s]: Eq. 2 summed over all rays."""
    lib = _load()
    rp, rr = _radar(radar), _RayRef(rays)
    out = np.zeros((radar.n_virtual, radar.n_chirps, radar.n_samples, 2), np.float64)
    lib.orc_signal(ctypes.byref(rp), ctypes.byref(rr.s), _ptr(out), nthreads)
    return out[..., 0] + 1j * out[..., 1]


def signal_at(radar, rays, flat_idx, nthreads: int = 0) -> np.ndarray:
    """complex128[len(flat_idx)]: the Eq. 2 sum at flat indices (k*N_c + m)*N_s + n."""
    lib = _load()
    rp, rr = _radar(radar), _RayRef(rays)
    idx = np.ascontiguousarray(flat_idx, np.int64)
    out = np.zeros((idx.shape[0], 2), np.float64)
    lib.orc_signal_at(ctypes.byref(rp), ctypes.byref(rr.s), idx.shape[0], _ptr(idx), _ptr(out), nthreads)
    return out[:, 0] + 1j * out[:, 1]


def spectrum(radar, sig: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """complex128[N_a, N_c, N_s]: Eq. 4 with windows and angle zero padding, naive DFTs."""
    lib = _load()
    rp = _radar(radar)
    s = np.ascontiguousarray(np.stack([sig.real, sig.imag], axis=-1), np.float64)
    out = np.zeros((radar.n_angle, radar.n_chirps, radar.n_samples, 2), np.float64)
    lib.orc_spectrum(ctypes.byref(rp), _ptr(s), _ptr(out), nthreads)
    return out[..., 0] + 1j * out[..., 1]


def cell_dtft(radar, rays, flat_cells, nthreads: int = 0) -> np.ndarray:
    """complex128[len(flat_cells)]: spectrum cells from the rays directly (windowed DTFT).
    The separable model only: the exact model's n m term does not factor over the axes."""
    if int(getattr(radar, "model", 0)) != 0:
        raise ValueError("cell_dtft needs the separable signal model")
    lib = _load()
    rp, rr = _radar(radar), _RayRef(rays)
    cells = np.ascontiguousarray(flat_cells, np.int64)
    out = np.zeros((cells.shape[0], 2), np.float64)
    lib.orc_cell_dtft(ctypes.byref(rp), ctypes.byref(rr.s), cells.shape[0], _ptr(cells), _ptr(out), nthreads)
    return out[:, 0] + 1j * out[:, 1]


def window(radar, axis: int) -> np.ndarray:
    lib = _load()
    rp = _radar(radar)
    n = (radar.n_samples, radar.n_chirps, radar.n_virtual)[axis]
    out = np.zeros(n, np.float64)
    lib.orc_window(ctypes.byref(rp), axis, _ptr(out))
    return out


def bins(radar, rays):
    """dict of per-ray x_r, x_d, x_a (FP64), flat cell index and fixed-point energy."""
    lib = _load()
    rp, rr = _radar(radar), _RayRef(rays)
    n = rr.d.shape[0]
    out = {k: np.zeros(n, np.float64) for k in ("x_r", "x_d", "x_a")}
    out["cell"] = np.zeros(n, np.int64)
    out["energy"] = np.zeros(n, np.int64)
    lib.orc_bins(ctypes.byref(rp), ctypes.byref(rr.s), _ptr(out["x_r"]), _ptr(out["x_d"]),
                 _ptr(out["x_a"]), _ptr(out["cell"]), _ptr(out["energy"]))
    return out


def labels(radar, rays) -> np.ndarray:
    """int32[N_a, N_c, N_s]: per cell the object id with the most ray energy (ties to the
    smallest id), -1 where no ray falls."""
    lib = _load()
    rp, rr = _radar(radar), _RayRef(rays)
    out = np.zeros((radar.n_angle, radar.n_chirps, radar.n_samples), np.int32)
    lib.orc_labels(ctypes.byref(rp), ctypes.byref(rr.s), _ptr(rr.obj), _ptr(out))
    return out


def cell_object_energy(radar, rays):
    """(cell int64[m], obj int32[m], energy int64[m]) sorted by (cell, obj)."""
    lib = _load()
    rp, rr = _radar(radar), _RayRef(rays)
    n = rr.d.shape[0]
    cell = np.zeros(max(n, 1), np.int64)
    obj = np.zeros(max(n, 1), np.int32)
    e = np.zeros(max(n, 1), np.int64)
    m = lib.orc_cell_object_energy(ctypes.byref(rp), ctypes.byref(rr.s), _ptr(rr.obj), _ptr(cell),
                                   _ptr(obj), _ptr(e))
    return cell[:m], obj[:m], e[:m]


def sin_rep(x: float) -> float:
    return float(_load().orc_sin_rep(float(x)))


def cos_rep(x: float) -> float:
    return float(_load().orc_cos_rep(float(x)))


def span_mask(rule, object_id=None, material_id=None, n_hits=None) -> np.ndarray:
    """Rays of a span (Sec. II-C filter rules): every set field of the rule must match."""
    n = len(object_id) if object_id is not None else len(n_hits)
    m = np.ones(n, bool)
    if rule["object_id"] >= 0:
        m &= np.asarray(object_id) == rule["object_id"]
    if rule["material_id"] >= 0:
        m &= np.asarray(material_id) == rule["material_id"]
    if rule["min_hits"] > 0 or rule["max_hits"] >= 0:
        h = np.asarray(n_hits)
        m &= h >= rule["min_hits"]
        if rule["max_hits"] >= 0:
            m &= h <= rule["max_hits"]
    if rule.get("exclude", 0):
        m = ~m
    return m


def span_labels(spectra, threshold: float) -> np.ndarray:
    """Per cell the span with the largest |X_h|^2 among spans whose |X_h|^2 is at least
    threshold^2 times the largest |X|^2 of all spans and cells (ties to the lower span),
    -1 where none passes.  `spectra` is [H, ...]; powers are (x*x) + (y*y) in the spectra's
    own real dtype, each operation rounded separately, so complex64 spectra give FP32
    decisions."""
    x, y = np.ascontiguousarray(spectra.real), np.ascontiguousarray(spectra.imag)
    ft = x.dtype.type
    p = (x * x) + (y * y)
    floor = (ft(threshold) * ft(threshold)) * p.max()
    ok = (p >= floor) & (p > 0)
    masked = np.where(ok, p, -1.0)
    lab = np.argmax(masked, axis=0).astype(np.int32)
    lab[~ok.any(axis=0)] = -1
    return lab


def paths(radar, rays, hits, geom, nthreads: int = 0) -> np.ndarray:
    """float64[n][N_c][N_v]: path length of each ray at each chirp snapshot and virtual
    channel (Eq. 6 hit positions, Eq. 7 antenna displacement)."""
    lib = _load()
    rp, rr, gr = _radar(radar), _RayRef(rays), _GeomRef(radar, rays, hits, geom)
    out = np.zeros((rays.n, radar.n_chirps, radar.n_virtual), np.float64)
    lib.orc_paths(ctypes.byref(rp), ctypes.byref(rr.s), ctypes.byref(gr.s), _ptr(out), nthreads)
    return out


def signal_geom(radar, rays, hits, geom, nthreads: int = 0) -> np.ndarray:
    """complex128[N_v][N_c][N_s]: Eq. 2 over the per-(ray, chirp, channel) path lengths."""
    lib = _load()
    rp, rr, gr = _radar(radar), _RayRef(rays), _GeomRef(radar, rays, hits, geom)
    out = np.zeros((radar.n_virtual, radar.n_chirps, radar.n_samples, 2), np.float64)
    lib.orc_signal_geom(ctypes.byref(rp), ctypes.byref(rr.s), ctypes.byref(gr.s), _ptr(out), nthreads)
    return out[..., 0] + 1j * out[..., 1]


def signal_geom_at(radar, rays, hits, geom, flat_idx, nthreads: int = 0) -> np.ndarray:
    lib = _load()
    rp, rr, gr = _radar(radar), _RayRef(rays), _GeomRef(radar, rays, hits, geom)
    idx = np.ascontiguousarray(flat_idx, np.int64)
    out = np.zeros((idx.shape[0], 2), np.float64)
    lib.orc_signal_geom_at(ctypes.byref(rp), ctypes.byref(rr.s), ctypes.byref(gr.s), idx.shape[0], _ptr(idx),
                           _ptr(out), nthreads)
    return out[:, 0] + 1j * out[:, 1]
