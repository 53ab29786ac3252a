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
