"""Seeded synthetic radar scenes: the inputs shared by the oracle tests and the GPU path.

This module holds no arithmetic of the simulation method itself.  It only
draws rays (round-trip path length, amplitude, radial velocity, azimuth,
elevation, start phase, object id) from the workload recipes and returns the
raw radar parameters of each workload.  The paper's own scenes (a pedestrian
mesh, a measured corridor) are not available; these seeded scenes stand in for
them with the shapes, sizes and value distributions stated below.

Random numbers come from a counter-based generator: SplitMix64's output
function (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to ``seed_key + (i + 1) * golden_gamma`` for
element ``i`` of a named stream, so every value depends only on
(seed, stream, index) and any prefix or sub-range can be regenerated.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)

# window codes (same numbering as the C ABI's sim_window enum)
WIN_NONE = 0
WIN_HANN_PERIODIC = 1
WIN_HANN_SYMMETRIC = 2
WIN_HANN_NOZERO = 3


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def u64(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """``n`` 64-bit counter-based draws of (seed, stream), elements start..start+n-1."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([(seed & 0xFFFFFFFFFFFFFFFF)], dtype=np.uint64)
                   ^ (np.uint64(stream & 0xFFFFFFFF) * _STREAM_MUL))[0]
        idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        return _mix(key + idx * _GOLDEN)


def uniform(seed: int, stream: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Uniform doubles in [lo, hi): the top 53 bits of each draw."""
    x = (u64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * x


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """Standard normals by the Box-Muller transform over two uniform streams."""
    u1 = ((u64(seed, stream, n) >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u2 = (u64(seed, stream + 0x10000, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def randint(seed: int, stream: int, n: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform on [lo, hi] (inclusive), by multiply-shift of the top 32 bits."""
    span = np.uint64(hi - lo + 1)
    top = u64(seed, stream, n) >> np.uint64(32)
    with np.errstate(over="ignore"):
        return (lo + ((top * span) >> np.uint64(32)).astype(np.int64)).astype(np.int32)


@dataclasses.dataclass
class Radar:
    """Raw FMCW radar parameters (SI units).  Nothing here is derived."""
    carrier_hz: float
    bandwidth_hz: float
    sweep_time_s: float
    chirp_period_s: float
    n_samples: int
    n_chirps: int
    n_tx: int
    n_rx: int
    element_spacing_m: float = 0.0        # 0 means half a carrier wavelength
    n_angle: int = 16
    window: tuple = (WIN_HANN_PERIODIC, WIN_HANN_PERIODIC, WIN_HANN_NOZERO)
    model: int = 0                        # 0 separable signal model, 1 exact (range migration)
    pattern_exp: int = 0                  # antenna pattern (cos az cos el)^q; 0 isotropic
    tdm_slot_s: float = 0.0               # TDM-MIMO: transmitter t's chirp j starts at j T_d + t slot

    @property
    def n_virtual(self) -> int:
        return self.n_tx * self.n_rx

    def replace(self, **kw) -> "Radar":
        return dataclasses.replace(self, **kw)


@dataclasses.dataclass
class Rays:
    """Structure-of-arrays ray list, in the dtypes of the C ABI."""
    range_rt_m: np.ndarray          # f64, round-trip path length d_i
    amplitude: np.ndarray           # f32
    radial_velocity_mps: np.ndarray  # f32, > 0 receding
    azimuth_rad: np.ndarray         # f32
    elevation_rad: np.ndarray       # f32
    phase0_rad: np.ndarray          # f32
    object_id: np.ndarray           # i32
    material_id: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return int(self.range_rt_m.shape[0])

    def take(self, idx) -> "Rays":
        mat = None if self.material_id is None else self.material_id[idx]
        return Rays(self.range_rt_m[idx], self.amplitude[idx], self.radial_velocity_mps[idx],
                    self.azimuth_rad[idx], self.elevation_rad[idx], self.phase0_rad[idx],
                    self.object_id[idx], mat)

    @staticmethod
    def concat(parts: List["Rays"]) -> "Rays":
        f = lambda name: np.concatenate([getattr(p, name) for p in parts])
        return Rays(f("range_rt_m"), f("amplitude"), f("radial_velocity_mps"), f("azimuth_rad"),
                    f("elevation_rad"), f("phase0_rad"), f("object_id"))

    def arrays(self) -> Dict[str, np.ndarray]:
        return {k: getattr(self, k) for k in ("range_rt_m", "amplitude", "radial_velocity_mps",
                                              "azimuth_rad", "elevation_rad", "phase0_rad",
                                              "object_id")}


# ---------------------------------------------------------------- radar configurations

def radar_tiny() -> Radar:
    """77 GHz, 512 MHz over 25.6 us, chirp period 40 us, 1x4 ULA at lambda/2, 64 x 128."""
    return Radar(77e9, 512e6, 25.6e-6, 40e-6, n_samples=128, n_chirps=64, n_tx=1, n_rx=4,
                 n_angle=16)


def radar_automotive(n_chirps: int = 256, n_samples: int = 512, n_tx: int = 3, n_rx: int = 4) -> Radar:
    """77 GHz, 1 GHz over 51.2 us, chirp period 60 us, 3x4 TDM-MIMO (12 virtual), 256 x 512."""
    nv = n_tx * n_rx
    na = max(16, 1 << (nv - 1).bit_length())
    return Radar(77e9, 1e9, 51.2e-6, 60e-6, n_samples=n_samples, n_chirps=n_chirps,
                 n_tx=n_tx, n_rx=n_rx, n_angle=na)


def radar_imaging() -> Radar:
    """Imaging radar: 12x16 = 192 virtual channels, 512 chirps x 1024 samples,
    1 GHz over 102.4 us, chirp period 120 us, angle FFT of 256."""
    return Radar(77e9, 1e9, 102.4e-6, 120e-6, n_samples=1024, n_chirps=512, n_tx=12, n_rx=16,
                 n_angle=256)


# ---------------------------------------------------------------- scene recipes

_DEG = math.pi / 180.0


def _amplitude(seed: int, stream: int, rng_m: np.ndarray) -> np.ndarray:
    """a = sqrt(RCS)/R^2 with RCS log-normal (mu 0, sigma 1 in ln m^2)."""
    rcs = np.exp(normal(seed, stream, rng_m.shape[0]))
    return np.sqrt(rcs) / (rng_m * rng_m)


def _finish(seed: int, stream: int, rng_m, vel, az, obj) -> Rays:
    n = rng_m.shape[0]
    return Rays(
        range_rt_m=(2.0 * rng_m).astype(np.float64),
        amplitude=_amplitude(seed, stream, rng_m).astype(np.float32),
        radial_velocity_mps=vel.astype(np.float32),
        azimuth_rad=az.astype(np.float32),
        elevation_rad=np.zeros(n, np.float32),
        phase0_rad=uniform(seed, stream + 1, n, 0.0, 2.0 * math.pi).astype(np.float32),
        object_id=obj.astype(np.int32),
    )


def uniform_rays(seed: int, n: int, n_objects: int = 3, r_lo: float = 1.0, r_hi: float = 30.0,
                 v_max: float = 15.0, az_max_deg: float = 60.0, stream0: int = 0) -> Rays:
    """Rays uniform over range [r_lo, r_hi] m, velocity +-v_max, azimuth +-az_max_deg,
    object id uniform on 0..n_objects-1 (the tiny-scene recipe)."""
    rng_m = uniform(seed, stream0 + 1, n, r_lo, r_hi)
    vel = uniform(seed, stream0 + 2, n, -v_max, v_max)
    az = uniform(seed, stream0 + 3, n, -az_max_deg * _DEG, az_max_deg * _DEG)
    obj = randint(seed, stream0 + 4, n, 0, n_objects - 1)
    return _finish(seed, stream0 + 10, rng_m, vel, az, obj)


def cluster_rays(seed: int, n_rays: int, n_objects: int = 20, clutter_frac: float = 0.1,
                 range_centre=(3.0, 30.0), min_per_obj: int = 2000, max_per_obj: int = 20000) -> Rays:
    """Object clusters plus clutter (the automotive recipe).

    ``n_objects`` weights are drawn U[min_per_obj, max_per_obj] and scaled by the
    largest-remainder method so the object rays total (1 - clutter_frac) * n_rays;
    the rest are clutter rays labelled id 0 and drawn as in :func:`uniform_rays`.
    Each object j (id j+1) has a centre with range U(range_centre), velocity
    U(-15, 15) m/s and azimuth U(-60, 60) deg; its rays are Gaussian about the
    centre with sigma 0.5 m, 0.2 m/s and 1 deg, ranges clamped to >= 0.5 m.
    """
    n_clutter = int(round(clutter_frac * n_rays))
    n_obj_rays = n_rays - n_clutter
    w = uniform(seed, 100, n_objects, min_per_obj, max_per_obj)
    quota = w / w.sum() * n_obj_rays
    counts = np.floor(quota).astype(np.int64)
    rem = n_obj_rays - int(counts.sum())
    order = np.argsort(-(quota - counts), kind="stable")
    counts[order[:rem]] += 1
    rc = uniform(seed, 101, n_objects, range_centre[0], range_centre[1])
    vc = uniform(seed, 102, n_objects, -15.0, 15.0)
    ac = uniform(seed, 103, n_objects, -60 * _DEG, 60 * _DEG)
    obj = np.repeat(np.arange(1, n_objects + 1, dtype=np.int64), counts)
    centre = obj - 1
    rng_m = np.maximum(rc[centre] + 0.5 * normal(seed, 110, n_obj_rays), 0.5)
    vel = vc[centre] + 0.2 * normal(seed, 111, n_obj_rays)
    az = ac[centre] + 1.0 * _DEG * normal(seed, 112, n_obj_rays)
    objects = _finish(seed, 120, rng_m, vel, az, obj)
    if n_clutter == 0:
        return objects
    clutter = uniform_rays(seed, n_clutter, n_objects=1, stream0=200)
    clutter.object_id[:] = 0
    return Rays.concat([objects, clutter])


# ---------------------------------------------------------------- moving triangle scenes

@dataclasses.dataclass
class Geometry:
    """Animated triangle mesh and antenna positions (x forward, y left, z up; metres)."""
    vertices: np.ndarray   # f64 [N_c][V][3]: vertex positions at t = j T_d
    triangles: np.ndarray  # i32 [T][3] vertex indices
    tx_pos: np.ndarray     # f64 [n_tx][3]
    rx_pos: np.ndarray     # f64 [n_rx][3]
    ref_tx: np.ndarray     # f64 [3]: antennas the rays were traced between
    ref_rx: np.ndarray     # f64 [3]


@dataclasses.dataclass
class Hits:
    """Per-ray hit lists in CSR form, first hit first."""
    offset: np.ndarray     # i64 [n + 1]
    triangle: np.ndarray   # i32 [H]
    u: np.ndarray          # f32 [H] barycentric coordinates
    v: np.ndarray          # f32 [H]

    @property
    def n_hits(self) -> np.ndarray:
        return np.diff(self.offset).astype(np.int32)


_BOX_TRIS = np.array([[0, 1, 2], [0, 2, 3], [4, 6, 5], [4, 7, 6], [0, 4, 5], [0, 5, 1],
                      [1, 5, 6], [1, 6, 2], [2, 6, 7], [2, 7, 3], [3, 7, 4], [3, 4, 0]], np.int32)


def _rot_z(angle: np.ndarray, xyz: np.ndarray) -> np.ndarray:
    c, s = np.cos(angle), np.sin(angle)
    return np.stack([c * xyz[..., 0] - s * xyz[..., 1], s * xyz[..., 0] + c * xyz[..., 1], xyz[..., 2]], -1)


def moving_scene(seed: int, radar: Radar, n_rays: int, n_objects: int = 8, bounce_frac: float = 0.2,
                 r_range=(3.0, 30.0), v_max: float = 15.0, yaw_max: float = 1.0):
    """A scene of boxes moving and turning in front of the radar, standing in for the ray
    tracer's output: rays with their traced path length, hit lists on the boxes (a fraction
    first bouncing off a static ground plane), and the mesh animated over the N_c chirps.

    The virtual array lies along -y: transmitter t at y = -t N_rx s, receiver r at y = -r s,
    s the element spacing (lambda / 2 by default); rays were traced between transmitter 0
    and receiver 0 at the origin.  Box j (id j + 1): size U(0.5, 4.5) x U(0.5, 2) x
    U(0.5, 1.8) m, centre at range U(r_range), azimuth U(+-60 deg), height U(-0.5, 0.5) m,
    radial velocity U(+-v_max), tangential U(+-2) m/s, yaw rate U(+-yaw_max) rad/s.  Rays
    pick a box uniformly, a triangle uniformly and a uniform point on it; with probability
    bounce_frac the ray first hits the ground (z = -1.5 m) half way to that point.
    Amplitude sqrt(RCS) / R^2 with R = d / 2, start phase U[0, 2 pi).  The label inputs
    (v, az, el) are the traced ray's: half the path-length rate between the first two
    snapshots, and the direction of its first hit at snapshot 0."""
    lam = 299792458.0 / radar.carrier_hz
    sp = radar.element_spacing_m or lam / 2
    tx = np.zeros((radar.n_tx, 3))
    tx[:, 1] = -np.arange(radar.n_tx) * radar.n_rx * sp
    rx = np.zeros((radar.n_rx, 3))
    rx[:, 1] = -np.arange(radar.n_rx) * sp
    size = np.stack([uniform(seed, 300, n_objects, 0.5, 4.5), uniform(seed, 301, n_objects, 0.5, 2.0),
                     uniform(seed, 302, n_objects, 0.5, 1.8)], -1)
    rng = uniform(seed, 303, n_objects, *r_range)
    azc = uniform(seed, 304, n_objects, -60 * _DEG, 60 * _DEG)
    zc = uniform(seed, 305, n_objects, -0.5, 0.5)
    centre = np.stack([rng * np.cos(azc), rng * np.sin(azc), zc], -1)
    los = centre / np.linalg.norm(centre, axis=1, keepdims=True)
    side = np.stack([-np.sin(azc), np.cos(azc), np.zeros(n_objects)], -1)
    vel = los * uniform(seed, 306, n_objects, -v_max, v_max)[:, None] + side * uniform(seed, 307, n_objects, -2, 2)[:, None]
    yaw0 = uniform(seed, 308, n_objects, -math.pi, math.pi)
    yaw_rate = uniform(seed, 309, n_objects, -yaw_max, yaw_max)
    corners = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                        [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], np.float64) * 0.5
    offs = corners[None] * size[:, None, :]                                  # [obj][8][3]
    t = np.arange(radar.n_chirps) * radar.chirp_period_s
    ang = yaw0[None, :, None] + yaw_rate[None, :, None] * t[:, None, None]   # [j][obj][1]
    boxes = (centre[None, :, None, :] + vel[None, :, None, :] * t[:, None, None, None]
             + _rot_z(np.broadcast_to(ang, (radar.n_chirps, n_objects, 8)), np.broadcast_to(offs, (radar.n_chirps, n_objects, 8, 3))))
    ground = np.array([[0.0, -100.0, -1.5], [150.0, -100.0, -1.5], [150.0, 100.0, -1.5], [0.0, 100.0, -1.5]])
    verts = np.concatenate([boxes.reshape(radar.n_chirps, -1, 3),
                            np.broadcast_to(ground, (radar.n_chirps, 4, 3))], 1).astype(np.float64)
    g0 = 8 * n_objects
    tris = np.concatenate([(_BOX_TRIS[None] + 8 * np.arange(n_objects)[:, None, None]).reshape(-1, 3),
                           np.array([[g0, g0 + 1, g0 + 2], [g0, g0 + 2, g0 + 3]])]).astype(np.int32)
    # object hits
    obj = randint(seed, 310, n_rays, 0, n_objects - 1)
    tri = (12 * obj + randint(seed, 311, n_rays, 0, 11)).astype(np.int32)
    u = uniform(seed, 312, n_rays)
    v = uniform(seed, 313, n_rays)
    fold = u + v > 1.0
    u, v = np.where(fold, 1.0 - u, u), np.where(fold, 1.0 - v, v)
    u, v = u.astype(np.float32), v.astype(np.float32)

    def on_tri(j, tr, uu, vv):
        V = verts[j]
        a, b, c = V[tris[tr, 0]], V[tris[tr, 1]], V[tris[tr, 2]]
        uu = uu.astype(np.float64)[:, None]
        vv = vv.astype(np.float64)[:, None]
        return (1.0 - uu - vv) * a + uu * b + vv * c

    p_obj0 = on_tri(0, tri, u, v)
    bounce = uniform(seed, 314, n_rays) < bounce_frac
    # ground point half way (static plane): barycentric coordinates on one of its two triangles
    gx, gy = 0.5 * p_obj0[:, 0], 0.5 * p_obj0[:, 1]
    s_, t_ = gx / 150.0, (gy + 100.0) / 200.0                                 # unit-square coordinates
    lower = s_ >= t_                                                         # triangle (g0, g0+1, g0+2)
    gtri = np.where(lower, len(tris) - 2, len(tris) - 1).astype(np.int32)
    gu = np.where(lower, s_ - t_, s_).astype(np.float32)
    gv = np.where(lower, t_, t_ - s_).astype(np.float32)
    nh = np.where(bounce, 2, 1)
    offset = np.concatenate([[0], np.cumsum(nh)]).astype(np.int64)
    H = int(offset[-1])
    htri = np.empty(H, np.int32)
    hu = np.empty(H, np.float32)
    hv = np.empty(H, np.float32)
    first = offset[:-1]
    htri[first] = np.where(bounce, gtri, tri)
    hu[first] = np.where(bounce, gu, u)
    hv[first] = np.where(bounce, gv, v)
    second = first[bounce] + 1
    htri[second] = tri[bounce]
    hu[second] = u[bounce]
    hv[second] = v[bounce]
    hits = Hits(offset, htri, hu, hv)

    def polyline(j):
        pts_first = on_tri(j, htri[first], hu[first], hv[first])
        pts_last = on_tri(j, htri[offset[1:] - 1], hu[offset[1:] - 1], hv[offset[1:] - 1])
        inner = np.where(bounce, np.linalg.norm(pts_last - pts_first, axis=1), 0.0)
        return (np.linalg.norm(pts_first - tx[0], axis=1) + inner + np.linalg.norm(pts_last - rx[0], axis=1),
                pts_first)

    d0, pf = polyline(0)
    d1, _ = polyline(1) if radar.n_chirps > 1 else (d0, None)
    az = np.arctan2(pf[:, 1], pf[:, 0])
    el = np.arctan2(pf[:, 2], np.hypot(pf[:, 0], pf[:, 1]))
    rays = Rays(range_rt_m=d0.astype(np.float64),
                amplitude=_amplitude(seed, 315, 0.5 * d0).astype(np.float32),
                radial_velocity_mps=((d1 - d0) / (2.0 * radar.chirp_period_s)).astype(np.float32),
                azimuth_rad=az.astype(np.float32), elevation_rad=el.astype(np.float32),
                phase0_rad=uniform(seed, 317, n_rays, 0.0, 2.0 * math.pi).astype(np.float32),
                object_id=(obj + 1).astype(np.int32), material_id=nh.astype(np.int32))
    geom = Geometry(verts, tris, tx, rx, tx[0].copy(), rx[0].copy())
    return rays, hits, geom


# ---------------------------------------------------------------- named workloads

def tiny_scene(seed: int = 0, n_rays: int = 2000):
    """Tiny scene: 1x4 ULA, 64 chirps x 128 samples, 2,000 uniform rays, ids 0..2."""
    return radar_tiny(), uniform_rays(seed, n_rays, n_objects=3)


def automotive_scene(seed: int = 1000, n_rays: int = 200_000, radar: Optional[Radar] = None):
    """Automotive frame: 3x4 TDM-MIMO, 256 chirps x 512 samples, 200k rays in
    20 Gaussian object clusters plus 10 % clutter (id 0)."""
    return (radar or radar_automotive()), cluster_rays(seed, n_rays)


def imaging_scene(seed: int, n_rays: int):
    """Imaging frame: 192 virtual channels, 512 x 1024, object centres 3..120 m."""
    return radar_imaging(), cluster_rays(seed, n_rays, range_centre=(3.0, 120.0))


def batch_scenes(seed: int = 3000, n_scenes: int = 64, r_lo: int = 10_000, r_hi: int = 500_000,
                 ray_scale: float = 1.0):
    """Uneven batch: ray counts log-uniform [r_lo, r_hi], chirps in {128,256,512},
    samples in {256,512}, virtual channels in {4,12}; automotive ray law."""
    lr = uniform(seed, 1, n_scenes, math.log(r_lo), math.log(r_hi))
    nc = randint(seed, 2, n_scenes, 0, 2)
    ns = randint(seed, 3, n_scenes, 0, 1)
    nv = randint(seed, 4, n_scenes, 0, 1)
    out = []
    for s in range(n_scenes):
        r = max(1, int(round(math.exp(lr[s]) * ray_scale)))
        radar = radar_automotive(n_chirps=(128, 256, 512)[nc[s]], n_samples=(256, 512)[ns[s]],
                                 n_tx=(1, 3)[nv[s]], n_rx=4)
        out.append((radar, cluster_rays(seed * 1000 + s, r, min_per_obj=max(1, r // 100),
                                        max_per_obj=max(2, r // 10))))
    return out
