"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test checks the oracle against something it does not compute the same
way: the signal model of Eq. 2 written in physical time, textbook FMCW
resolutions, the library FFT, closed-form window transforms (Harris 1978),
Parseval's theorem, linearity (Eq. 5), and hand-built label cases.
"""
import json
import math
import os

import mpmath
import numpy as np
import pytest

import oracle
import scenegen
from scenegen import Radar, Rays, WIN_NONE, WIN_HANN_PERIODIC, WIN_HANN_SYMMETRIC, WIN_HANN_NOZERO

C = 299792458.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def one_ray(d, a=1.0, v=0.0, az=0.0, el=0.0, phi0=0.0, obj=0):
    f32 = lambda x: np.array([x], np.float32)
    return Rays(np.array([d], np.float64), f32(a), f32(v), f32(az), f32(el), f32(phi0),
                np.array([obj], np.int32))


def rect(radar):
    return radar.replace(window=(WIN_NONE, WIN_NONE, WIN_NONE))


def small_radar(**kw):
    base = dict(carrier_hz=77e9, bandwidth_hz=512e6, sweep_time_s=25.6e-6, chirp_period_s=40e-6,
                n_samples=32, n_chirps=16, n_tx=1, n_rx=4, n_angle=4)
    base.update(kw)
    return Radar(**base)


# ------------------------------------------------------------------ Eq. 2 in physical time

def brute_signal(radar, rays):
    """Eq. 2 written out with t_n = n T_c / N_s, tau_i(j) = (d + 2 v j T_d)/c, mu = B/T_c,
    dropping only the range-migration product mu * t * (tau_i(j) - tau_i(0)); the channel
    term is the far-field path difference k s sin(az) cos(el) of Eq. 7, lambda = c / f_c."""
    lam = C / radar.carrier_hz
    s_m = radar.element_spacing_m or lam / 2
    mu = radar.bandwidth_hz / radar.sweep_time_s
    out = np.zeros((radar.n_virtual, radar.n_chirps, radar.n_samples), np.complex128)
    t = np.arange(radar.n_samples) * radar.sweep_time_s / radar.n_samples
    for i in range(rays.n):
        d = float(rays.range_rt_m[i])
        v = float(rays.radial_velocity_mps[i])
        az, el = float(rays.azimuth_rad[i]), float(rays.elevation_rad[i])
        for k in range(radar.n_virtual):
            for j in range(radar.n_chirps):
                tau0 = d / C
                tauj = (d + 2.0 * v * j * radar.chirp_period_s) / C
                ph = (2 * math.pi * (mu * t * tau0 + radar.carrier_hz * tauj)
                      + float(rays.phase0_rad[i])
                      + 2 * math.pi * k * s_m * math.sin(az) * math.cos(el) / lam)
                out[k, j] += float(rays.amplitude[i]) * np.exp(1j * ph)
    return out


def brute_signal_exact(radar, rays):
    """Eq. 2 written out in physical time with nothing dropped: mu t_n tau_i(j) + f_c tau_i(j),
    tau_i(j) = (d + 2 v j T_d) / c, plus the far-field channel term and phi0."""
    lam = C / radar.carrier_hz
    s_m = radar.element_spacing_m or lam / 2
    mu = radar.bandwidth_hz / radar.sweep_time_s
    out = np.zeros((radar.n_virtual, radar.n_chirps, radar.n_samples), np.complex128)
    t = np.arange(radar.n_samples) * radar.sweep_time_s / radar.n_samples
    for i in range(rays.n):
        d = float(rays.range_rt_m[i])
        v = float(rays.radial_velocity_mps[i])
        az, el = float(rays.azimuth_rad[i]), float(rays.elevation_rad[i])
        for k in range(radar.n_virtual):
            for j in range(radar.n_chirps):
                tauj = (d + 2.0 * v * j * radar.chirp_period_s) / C
                ph = (2 * math.pi * (mu * t * tauj + radar.carrier_hz * tauj) + float(rays.phase0_rad[i])
                      + 2 * math.pi * k * s_m * math.sin(az) * math.cos(el) / lam)
                out[k, j] += float(rays.amplitude[i]) * np.exp(1j * ph)
    return out


def test_exact_model_matches_eq2_brute_force():
    """The exact signal model keeps the range-migration product of Eq. 2."""
    radar = small_radar(n_samples=16, n_chirps=8, n_tx=2, n_rx=2, model=1)
    rays = scenegen.uniform_rays(seed=13, n=5, v_max=40.0)
    ref = brute_signal_exact(radar, rays)
    got = oracle.signal(radar, rays)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
    # it differs from the separable model exactly when rays move
    sep = oracle.signal(radar.replace(model=0), rays)
    assert np.abs(got - sep).max() > 1e-3 * np.abs(ref).max()
    still = rays.take(slice(None))
    still.radial_velocity_mps = np.zeros_like(rays.radial_velocity_mps)
    assert np.array_equal(oracle.signal(radar, still), oracle.signal(radar.replace(model=0), still))
    idx = np.arange(0, ref.size, 7)
    assert np.array_equal(oracle.signal_at(radar, rays, idx), got.reshape(-1)[idx])


def test_antenna_pattern_matches_eq2_brute_force():
    """The antenna gain A(az, el) of Eq. 2, modelled as (cos az cos el)^q, scales each
    ray's amplitude; the brute force applies it with the library cosine."""
    for q in (1, 4, 16):
        radar = small_radar(n_samples=16, n_chirps=8, n_tx=2, n_rx=2, pattern_exp=q)
        rays = scenegen.uniform_rays(seed=17 + q, n=6)
        rays.elevation_rad[:] = scenegen.uniform(5, q, 6, -0.4, 0.4).astype(np.float32)
        gain = (np.cos(rays.azimuth_rad.astype(np.float64)) * np.cos(rays.elevation_rad.astype(np.float64))) ** q
        # brute_signal reads float32 amplitudes: scale its per-ray terms in FP64
        ref = sum(gain[i] * brute_signal(radar, rays.take(slice(i, i + 1))) for i in range(rays.n))
        got = oracle.signal(radar, rays)
        assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max(), q
        assert np.array_equal(oracle.signal(radar.replace(pattern_exp=0), rays),
                              oracle.signal(small_radar(n_samples=16, n_chirps=8, n_tx=2, n_rx=2), rays))


def test_antenna_pattern_weights_the_labels():
    """Two rays in one cell (az = 0, so elevation leaves the angle bin alone): the stronger
    raw ray at a steep elevation wins without the pattern and loses with it."""
    radar = small_radar(n_samples=32, n_chirps=16, n_angle=4)
    d = 5 * C / radar.bandwidth_hz
    rays = Rays.concat([one_ray(d, a=0.5, el=0.0, obj=1), one_ray(d, a=1.0, el=1.2, obj=2)])
    assert oracle.labels(radar, rays)[0, 0, 5] == 2
    q = 4
    pr = radar.replace(pattern_exp=q)
    L = oracle.labels(pr, rays)
    assert L[0, 0, 5] == 1 and np.sum(L >= 0) == 1
    cell, obj, e = oracle.cell_object_energy(pr, rays)
    got = {int(o): int(x) for o, x in zip(obj, e)}
    assert got[1] == 2 ** 30                      # boresight: gain exactly 1
    mpmath.mp.prec = 100
    g = mpmath.cos(mpmath.mpf(float(np.float32(1.2)))) ** q
    assert abs(got[2] - g * g * 2 ** 32) <= 1.0


def test_signal_matches_eq2_brute_force():
    radar = small_radar(n_samples=16, n_chirps=8, n_tx=2, n_rx=2)
    rays = scenegen.uniform_rays(seed=11, n=6)
    rays.elevation_rad[:] = np.float32(0.2)
    ref = brute_signal(radar, rays)
    got = oracle.signal(radar, rays)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()


def test_signal_explicit_spacing_matches_brute_force():
    radar = small_radar(n_samples=8, n_chirps=4, element_spacing_m=0.0031)
    rays = scenegen.uniform_rays(seed=12, n=4)
    ref = brute_signal(radar, rays)
    got = oracle.signal(radar, rays)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()


# ------------------------------------------------------------------ textbook resolutions

@pytest.mark.parametrize("qr,qd,qa", [(5, 3, 1), (0, 0, 0), (17, -2, -1), (31, 7, 2)])
def test_single_ray_on_grid_is_one_cell(qr, qd, qa):
    """Rectangular windows, N_a = N_v: a ray at range q_r c/(2B), velocity
    q_d lambda/(2 N_c T_d) and sin(az) = q_a lambda/(N_a s) is a single DFT cell of value
    a e^{i(2 pi f_c d/c + phi0)} N_v N_c N_s (FMCW range and velocity resolution)."""
    radar = rect(small_radar())
    lam = C / radar.carrier_hz
    d = 2.0 * qr * C / (2.0 * radar.bandwidth_hz)
    v = qd * lam / (2.0 * radar.n_chirps * radar.chirp_period_s)
    az = math.asin(qa * lam / (radar.n_angle * lam / 2.0))
    a, phi0 = 0.75, 1.1
    rays = one_ray(d, a=a, v=v, az=az, phi0=phi0)
    X = oracle.spectrum(radar, oracle.signal(radar, rays))
    cell = (qa % radar.n_angle, qd % radar.n_chirps, qr % radar.n_samples)
    n_total = radar.n_virtual * radar.n_chirps * radar.n_samples
    phase = 2 * math.pi * radar.carrier_hz * d / C + float(np.float32(phi0))
    expect = float(np.float32(a)) * n_total * np.exp(1j * phase)
    assert abs(X[cell] - expect) <= 1e-5 * abs(expect)
    rest = X.copy()
    rest[cell] = 0
    assert np.abs(rest).max() <= 1e-5 * abs(expect)


def test_analytic_bins_hit_their_cell():
    radar = scenegen.radar_automotive()
    lam = C / radar.carrier_hz
    q = np.array([0, 1, 100, 511, 512 + 3, 7])
    qd = np.array([0, -1, 17, 127, -128, 300])
    qa = np.array([0, 1, -3, 7, -8, 5])
    d = 2.0 * q * C / (2.0 * radar.bandwidth_hz)
    v = qd * lam / (2.0 * radar.n_chirps * radar.chirp_period_s)
    az = np.arcsin(qa * 2.0 / radar.n_angle)
    n = len(q)
    rays = Rays(d, np.ones(n, np.float32), v.astype(np.float32), az.astype(np.float32),
                np.zeros(n, np.float32), np.zeros(n, np.float32), np.zeros(n, np.int32))
    b = oracle.bins(radar, rays)
    exp_cell = ((qa % 16) * radar.n_chirps + (qd % radar.n_chirps)) * radar.n_samples + (q % radar.n_samples)
    assert np.array_equal(b["cell"], exp_cell)
    assert np.allclose(b["x_r"], q, atol=1e-9)
    assert np.allclose(b["x_d"], qd, atol=1e-4)
    assert np.allclose(b["x_a"], qa, atol=1e-5)


# ------------------------------------------------------------------ DFT and windows

def textbook_window(kind, n):
    if kind == WIN_NONE:
        return np.ones(n)
    if kind == WIN_HANN_PERIODIC:
        return np.hanning(n + 1)[:-1]
    if kind == WIN_HANN_SYMMETRIC:
        return np.hanning(n)
    return np.hanning(n + 2)[1:-1]


@pytest.mark.parametrize("wins", [(WIN_HANN_PERIODIC, WIN_HANN_PERIODIC, WIN_HANN_NOZERO),
                                  (WIN_NONE, WIN_HANN_SYMMETRIC, WIN_HANN_PERIODIC)])
def test_spectrum_matches_numpy_fft(wins):
    radar = small_radar(n_tx=3, n_rx=2, n_angle=16, window=wins)
    rays = scenegen.uniform_rays(seed=5, n=40)
    s = oracle.signal(radar, rays)
    w = [textbook_window(wins[0], radar.n_samples), textbook_window(wins[1], radar.n_chirps),
         textbook_window(wins[2], radar.n_virtual)]
    for ax in range(3):
        assert np.allclose(oracle.window(radar, ax), w[ax], rtol=0, atol=1e-15)
    sw = s * w[2][:, None, None] * w[1][None, :, None] * w[0][None, None, :]
    ref = np.fft.fft(np.fft.fft(np.fft.fft(sw, axis=2), axis=1), n=radar.n_angle, axis=0)
    got = oracle.spectrum(radar, s)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_two_oracle_paths_agree():
    radar, rays = scenegen.tiny_scene(seed=3, n_rays=300)
    X = oracle.spectrum(radar, oracle.signal(radar, rays))
    cells = scenegen.randint(3, 77, 600, 0, X.size - 1).astype(np.int64)
    Y = oracle.cell_dtft(radar, rays, cells)
    ref = X.reshape(-1)[cells]
    assert np.linalg.norm(Y - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.abs(Y - ref).max() <= 1e-12 * np.abs(X).max()


def test_signal_at_matches_full_cube():
    radar, rays = scenegen.tiny_scene(seed=4, n_rays=100)
    s = oracle.signal(radar, rays)
    idx = scenegen.randint(4, 9, 50, 0, s.size - 1).astype(np.int64)
    assert np.array_equal(oracle.signal_at(radar, rays, idx), s.reshape(-1)[idx])


def test_hann_on_grid_peak_and_neighbours():
    """Periodic Hann on range and Doppler, on-grid ray: the peak is a N/2 per axis and
    each neighbour -a N/4 per axis; every other cell is zero."""
    radar = small_radar(n_angle=4, window=(WIN_HANN_PERIODIC, WIN_HANN_PERIODIC, WIN_NONE))
    lam = C / radar.carrier_hz
    qr, qd = 9, 5
    d = qr * C / radar.bandwidth_hz
    v = qd * lam / (2.0 * radar.n_chirps * radar.chirp_period_s)
    X = oracle.spectrum(radar, oracle.signal(radar, one_ray(d, a=1.0, v=v)))
    A = X[0] * np.exp(-1j * np.angle(X[0, qd, qr]))  # remove the carrier phase
    nv, nc, ns = radar.n_virtual, radar.n_chirps, radar.n_samples
    tol = 1e-5 * nv * nc * ns
    expect = np.zeros((nc, ns))
    for dd, wd in ((-1, -0.25), (0, 0.5), (1, -0.25)):
        for dr, wr in ((-1, -0.25), (0, 0.5), (1, -0.25)):
            expect[(qd + dd) % nc, (qr + dr) % ns] = nv * nc * ns * wd * wr
    assert np.abs(A - expect).max() <= tol


def dirichlet(delta, L):
    delta = np.asarray(delta, np.float64)
    num = np.sin(np.pi * L * delta)
    den = np.sin(np.pi * delta)
    with np.errstate(invalid="ignore", divide="ignore"):
        g = np.where(np.abs(den) < 1e-15, L * np.cos(np.pi * (L - 1) * delta) ** 0, num / den)
    return np.exp(1j * np.pi * delta * (L - 1)) * g


def test_zero_padded_angle_no_zero_hann_closed_form():
    """N_v = 12 channels zero padded to 16 with the Hann window on L + 2 points without
    its zero end points: X[q] = W(nu - q/N_a) with
    W(d) = G(d)/2 - e^{2 pi i/(L+1)} G(d + 1/(L+1))/4 - e^{-2 pi i/(L+1)} G(d - 1/(L+1))/4,
    G the L-point Dirichlet kernel."""
    radar = small_radar(n_samples=8, n_chirps=4, n_tx=3, n_rx=4, n_angle=16,
                        window=(WIN_NONE, WIN_NONE, WIN_HANN_NOZERO))
    L = 12
    az = 0.3
    rays = one_ray(2.0, a=1.0, az=az)
    nu = 0.5 * math.sin(float(np.float32(az)))
    X = oracle.spectrum(radar, oracle.signal(radar, rays))
    x_r = radar.bandwidth_hz * 2.0 / C  # range cycles; take the cell nearest it
    qr = int(round(x_r)) % radar.n_samples
    carrier = np.exp(2j * np.pi * (radar.carrier_hz * 2.0 / C))
    rr = sum(np.exp(2j * np.pi * n * (x_r - qr) / radar.n_samples) for n in range(radar.n_samples))
    dd = radar.n_chirps  # v = 0: Doppler DFT is N_c at bin 0
    q = np.arange(16)
    delta = nu - q / 16.0
    b = 1.0 / (L + 1)
    W = 0.5 * dirichlet(delta, L) - 0.25 * np.exp(2j * np.pi * b) * dirichlet(delta + b, L) \
        - 0.25 * np.exp(-2j * np.pi * b) * dirichlet(delta - b, L)
    expect = carrier * rr * dd * W
    got = X[:, 0, qr]
    assert np.abs(got - expect).max() <= 1e-9 * np.abs(expect).max()


def test_hann_sidelobe_and_scalloping_match_harris():
    """Sweeping a ray across one range bin in 1/32 steps samples the periodic-Hann
    response: its highest sidelobe and its scalloping loss are Harris's tabulated values."""
    g = json.load(open(os.path.join(GOLDEN, "hann_window_harris1978.json")))
    radar = Radar(77e9, 512e6, 25.6e-6, 40e-6, n_samples=128, n_chirps=1, n_tx=1, n_rx=1,
                  n_angle=1, window=(WIN_HANN_PERIODIC, WIN_NONE, WIN_NONE))
    q0 = 40
    offs = np.arange(32) / 32.0
    d = (q0 + offs) * C / radar.bandwidth_hz
    peak_on = None
    worst_side = -1e9
    peaks = []
    for i, dd in enumerate(d):
        X = np.abs(oracle.spectrum(radar, oracle.signal(radar, one_ray(float(dd)))))[0, 0]
        if i == 0:
            peak_on = X[q0]
        peaks.append(max(X[q0], X[q0 + 1]))
        side = np.concatenate([X[:q0 - 1], X[q0 + 3:]])  # outside the main lobe (+-2 bins)
        worst_side = max(worst_side, 20 * np.log10(side.max() / peak_on))
    scallop = 20 * np.log10(peak_on / min(peaks))
    assert abs(worst_side - g["highest_sidelobe_db"]) < 0.1
    assert abs(scallop - g["scalloping_loss_db"]) < 0.01
    assert abs(peak_on / radar.n_samples - g["coherent_gain"]) < 1e-12


# ------------------------------------------------------------------ linearity and invariants

def test_linearity_and_phase_flip():
    """Eq. 5: the cube of a union of ray sets is the sum of their cubes; scaling the
    amplitudes scales it; adding pi to every start phase negates it."""
    radar = small_radar(n_samples=16, n_chirps=8)
    A = scenegen.uniform_rays(seed=21, n=30)
    B = scenegen.uniform_rays(seed=22, n=17)
    sA, sB = oracle.signal(radar, A), oracle.signal(radar, B)
    sAB = oracle.signal(radar, Rays.concat([A, B]))
    assert np.abs(sAB - (sA + sB)).max() <= 1e-12 * np.abs(sAB).max()
    A2 = A.take(slice(None))
    A2.amplitude = (A.amplitude * np.float32(2.0)).astype(np.float32)
    assert np.abs(oracle.signal(radar, A2) - 2 * sA).max() <= 1e-12 * np.abs(sA).max()
    A3 = A.take(slice(None))
    A3.phase0_rad = (A.phase0_rad.astype(np.float64) + math.pi).astype(np.float32)
    # phase0 is f32, so pi is added to within half an f32 ulp: a relative error of ~1e-6
    assert np.abs(oracle.signal(radar, A3) + sA).max() <= 2e-6 * np.abs(sA).max()
    XA = oracle.spectrum(radar, sA)
    XB = oracle.spectrum(radar, sB)
    XAB = oracle.spectrum(radar, sAB)
    assert np.abs(XAB - XA - XB).max() <= 1e-12 * np.abs(XAB).max()


def test_parseval_rect_window_with_zero_padding():
    radar = rect(small_radar(n_tx=3, n_rx=2, n_angle=8))
    rays = scenegen.uniform_rays(seed=8, n=25)
    s = oracle.signal(radar, rays)
    X = oracle.spectrum(radar, s)
    lhs = np.sum(np.abs(X) ** 2)
    rhs = radar.n_angle * radar.n_chirps * radar.n_samples * np.sum(np.abs(s) ** 2)
    assert abs(lhs - rhs) <= 1e-12 * rhs


def test_permutation_invariance():
    radar, rays = scenegen.tiny_scene(seed=9, n_rays=500)
    perm = np.argsort(scenegen.uniform(9, 55, rays.n))
    rp = rays.take(perm)
    assert np.array_equal(oracle.labels(radar, rays), oracle.labels(radar, rp))
    idx = np.arange(0, 4 * 64 * 128, 97)
    a, b = oracle.signal_at(radar, rays, idx), oracle.signal_at(radar, rp, idx)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_empty_scene():
    radar = scenegen.radar_tiny()
    empty = scenegen.uniform_rays(seed=0, n=0)
    assert np.all(oracle.signal(radar, empty) == 0)
    assert np.all(oracle.labels(radar, empty) == -1)


# ------------------------------------------------------------------ labels

def test_labels_hand_built_cells():
    """Cells with known energies: sums per object, ties to the smallest id, zero-energy
    rays still label their cell, empty cells are -1."""
    radar = small_radar(n_samples=32, n_chirps=16, n_angle=4)
    lam = C / radar.carrier_hz

    def ray_at(qr, qd, a, obj):
        d = qr * C / radar.bandwidth_hz
        v = qd * lam / (2.0 * radar.n_chirps * radar.chirp_period_s)
        return one_ray(d, a=a, v=v, obj=obj)

    u = 1.0 / 65536.0  # a = k u gives energy rint(a^2 2^32) = k^2 exactly
    rays = Rays.concat([
        ray_at(3, 2, 3 * u, 1), ray_at(3, 2, 3 * u, 1), ray_at(3, 2, 4 * u, 2),   # 18 vs 16 -> 1
        ray_at(7, 1, 5 * u, 4), ray_at(7, 1, 4 * u, 2), ray_at(7, 1, 3 * u, 2),   # 25 vs 25 -> 2
        ray_at(9, 9, 0.0, 7), ray_at(9, 9, 0.0, 5),                               # 0 vs 0 -> 5
        ray_at(1, 0, 2 * u, 0), ray_at(1, 0, 1 * u, 3),                           # clutter id 0 wins
    ])
    L = oracle.labels(radar, rays)
    assert L[0, 2, 3] == 1 and L[0, 1, 7] == 2 and L[0, 9, 9] == 5 and L[0, 0, 1] == 0
    mask = np.ones_like(L, bool)
    for c in [(0, 2, 3), (0, 1, 7), (0, 9, 9), (0, 0, 1)]:
        mask[c] = False
    assert np.all(L[mask] == -1)
    cell, obj, e = oracle.cell_object_energy(radar, rays)
    got = {(int(c), int(o)): int(x) for c, o, x in zip(cell, obj, e)}
    flat = lambda qd, qr: qd * radar.n_samples + qr
    assert got[(flat(2, 3), 1)] == 18 and got[(flat(2, 3), 2)] == 16
    assert got[(flat(1, 7), 4)] == 25 and got[(flat(1, 7), 2)] == 25
    assert got[(flat(9, 9), 7)] == 0 and got[(flat(0, 1), 0)] == 4


def test_energy_quantisation_and_cap():
    radar = small_radar()
    amps = np.array([0.0, 1.0, 2.0 ** -16, 0.3, 12.0, 40.0, 1e-6], np.float32)
    n = len(amps)
    rays = Rays(np.full(n, 3.0), amps, np.zeros(n, np.float32), np.zeros(n, np.float32),
                np.zeros(n, np.float32), np.zeros(n, np.float32), np.zeros(n, np.int32))
    e = oracle.bins(radar, rays)["energy"]
    for a, got in zip(amps, e):
        x = mpmath.mpf(float(a)) ** 2 * 2 ** 32
        ref = min(int(mpmath.nint(x)), 2 ** 41)
        assert got == ref


def test_bins_aliasing_wraps_like_the_dft():
    """A ray beyond the unambiguous range lands where its DFT peak does."""
    radar = rect(small_radar())
    d = (radar.n_samples + 5) * C / radar.bandwidth_hz
    rays = one_ray(d)
    X = np.abs(oracle.spectrum(radar, oracle.signal(radar, rays)))
    peak = np.unravel_index(np.argmax(X), X.shape)
    cell = int(oracle.bins(radar, rays)["cell"][0])
    assert np.ravel_multi_index(peak, X.shape) == cell


# ------------------------------------------------------------------ polynomial sine / cosine

def test_sin_cos_rep_within_two_ulp_of_exact():
    mpmath.mp.prec = 200
    xs = np.concatenate([np.linspace(-math.pi, math.pi, 4001),
                         scenegen.uniform(1, 2, 2000, -math.pi, math.pi),
                         [0.0, -0.0, math.pi / 2, -math.pi / 2, math.pi / 4, 1e-300, 3 * math.pi / 4]])
    for x in xs:
        x = float(x)
        for f, g in ((oracle.sin_rep, mpmath.sin), (oracle.cos_rep, mpmath.cos)):
            ref = g(mpmath.mpf(x))
            got = f(x)
            ulp = math.ulp(float(ref)) if float(ref) != 0 else 5e-324
            assert abs(mpmath.mpf(got) - ref) <= 2.0 * ulp + 1e-300, (x, got)
    assert oracle.sin_rep(0.0) == 0.0 and oracle.cos_rep(0.0) == 1.0


def test_span_selection_and_segmentation_rules():
    """Sec. II-C filter rules select exactly the rays they name; the segmentation labels the
    strongest span above the threshold and nothing below it."""
    obj = np.array([1, 1, 2, 3, 2, 0], np.int32)
    mat = np.array([0, 1, 0, 1, 2, 0], np.int32)
    hits = np.array([1, 2, 1, 3, 2, 1], np.int32)
    rule = lambda **kw: dict(dict(object_id=-1, material_id=-1, min_hits=0, max_hits=-1, exclude=0), **kw)
    assert oracle.span_mask(rule(object_id=1), obj, mat, hits).tolist() == [1, 1, 0, 0, 0, 0]
    assert oracle.span_mask(rule(min_hits=2), obj, mat, hits).tolist() == [0, 1, 0, 1, 1, 0]
    assert oracle.span_mask(rule(object_id=2, min_hits=1, max_hits=1), obj, mat, hits).tolist() == [0, 0, 1, 0, 0, 0]
    assert oracle.span_mask(rule(material_id=0, exclude=1), obj, mat, hits).tolist() == [0, 1, 0, 1, 1, 0]
    spectra = np.array([[3.0, 0.1, 0.0, 2.0], [1.0, 0.2, 0.0, 2.0]], np.complex128)
    assert oracle.span_labels(spectra, 0.2).tolist() == [0, -1, -1, 0]  # 0.2 floor: 0.36 of power 9
    assert oracle.span_labels(spectra, 0.0).tolist() == [0, 1, -1, 0]


# ------------------------------------------------------------------ TDM-MIMO slot offsets

def brute_signal_tdm(radar, rays, exact):
    """Eq. 2 in physical time for a TDM-MIMO frame: transmitter t sends chirp j at
    j T_d + t T_slot, so tau_i(j, t) = (d + 2 v (j T_d + t T_slot)) / c.  The separable model
    keeps mu t_n tau_i(0) in the beat term, the exact one mu t_n tau_i(j, t)."""
    lam = C / radar.carrier_hz
    s_m = radar.element_spacing_m or lam / 2
    mu = radar.bandwidth_hz / radar.sweep_time_s
    out = np.zeros((radar.n_virtual, radar.n_chirps, radar.n_samples), np.complex128)
    t = np.arange(radar.n_samples) * radar.sweep_time_s / radar.n_samples
    for i in range(rays.n):
        d = float(rays.range_rt_m[i])
        v = float(rays.radial_velocity_mps[i])
        az, el = float(rays.azimuth_rad[i]), float(rays.elevation_rad[i])
        for k in range(radar.n_virtual):
            tx = k // radar.n_rx
            for j in range(radar.n_chirps):
                tau = (d + 2.0 * v * (j * radar.chirp_period_s + tx * radar.tdm_slot_s)) / C
                beat = tau if exact else d / C
                ph = (2 * math.pi * (mu * t * beat + radar.carrier_hz * tau) + float(rays.phase0_rad[i])
                      + 2 * math.pi * k * s_m * math.sin(az) * math.cos(el) / lam)
                out[k, j] += float(rays.amplitude[i]) * np.exp(1j * ph)
    return out


@pytest.mark.parametrize("model", [0, 1])
def test_tdm_slot_offsets_match_eq2_brute_force(model):
    radar = small_radar(n_samples=16, n_chirps=8, n_tx=3, n_rx=2, n_angle=8, tdm_slot_s=13.3e-6, model=model)
    rays = scenegen.uniform_rays(seed=23 + model, n=5, v_max=40.0)
    ref = brute_signal_tdm(radar, rays, exact=bool(model))
    got = oracle.signal(radar, rays)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
    idx = np.arange(0, ref.size, 5)
    assert np.array_equal(oracle.signal_at(radar, rays, idx), got.reshape(-1)[idx])
    # the offsets only act on moving rays, and only on transmitters t > 0
    off = oracle.signal(radar.replace(tdm_slot_s=0.0), rays)
    assert np.array_equal(got[: radar.n_rx], off[: radar.n_rx])
    assert np.abs(got - off).max() > 1e-2 * np.abs(ref).max()


def test_tdm_two_oracle_paths_agree():
    """The per-cell DTFT path with its own angle sum equals DFT(signal) under TDM offsets."""
    radar = small_radar(n_samples=16, n_chirps=8, n_tx=3, n_rx=2, n_angle=8, tdm_slot_s=20e-6,
                        window=(WIN_HANN_PERIODIC, WIN_HANN_PERIODIC, WIN_HANN_NOZERO))
    rays = scenegen.uniform_rays(seed=29, n=7, v_max=30.0)
    X = oracle.spectrum(radar, oracle.signal(radar, rays))
    cells = np.arange(0, X.size, 3)
    got = oracle.cell_dtft(radar, rays, cells)
    assert np.abs(got - X.reshape(-1)[cells]).max() <= 1e-12 * np.abs(X).max()


# ------------------------------------------------------------------ virtual snapshots (Eq. 6, Eq. 7)

def polyline_paths(radar, hits, geom):
    """Path of every ray at every snapshot j and channel (t, r), measured directly: transmitter t
    to the hits at snapshot j (each the barycentric point of its triangle's vertices then) and
    on to receiver r."""
    V, T = geom.vertices, geom.triangles
    n = hits.offset.shape[0] - 1
    out = np.zeros((n, radar.n_chirps, radar.n_virtual))
    for i in range(n):
        hs = range(int(hits.offset[i]), int(hits.offset[i + 1]))
        for j in range(radar.n_chirps):
            pts = []
            for h in hs:
                a, b, c = (V[j, T[hits.triangle[h], q]] for q in range(3))
                u, v = float(hits.u[h]), float(hits.v[h])
                pts.append(np.einsum("q,qc->c", [1.0 - u - v, u, v], np.stack([a, b, c])))
            inner = sum(np.linalg.norm(pts[q + 1] - pts[q]) for q in range(len(pts) - 1))
            for k in range(radar.n_virtual):
                t, r = divmod(k, radar.n_rx)
                out[i, j, k] = (np.linalg.norm(pts[0] - geom.tx_pos[t]) + inner
                                + np.linalg.norm(pts[-1] - geom.rx_pos[r]))
    return out


def test_snapshot_paths_match_polylines():
    """Eq. 6 moves each hit with its triangle and Eq. 7 swaps the antenna legs: with the traced
    length equal to the snapshot-0 polyline, every path is the polyline at snapshot j between
    transmitter t and receiver r.  A traced length carrying an extra delta shifts every path
    by exactly that delta (Eq. 7 only replaces the two antenna legs)."""
    radar = scenegen.radar_automotive(n_chirps=8, n_samples=16)
    rays, hits, geom = scenegen.moving_scene(3, radar, 40, bounce_frac=0.4)
    assert np.any(hits.n_hits == 2) and np.any(hits.n_hits == 1)
    ref = polyline_paths(radar, hits, geom)
    got = oracle.paths(radar, rays, hits, geom)
    assert np.abs(got - ref).max() <= 1e-10
    assert np.ptp(got[:, :, 0], axis=1).max() > 0.01      # the boxes move over the frame
    shifted = rays.take(slice(None))
    shifted.range_rt_m = rays.range_rt_m + 0.37
    assert np.abs(oracle.paths(radar, shifted, hits, geom) - got - 0.37).max() <= 1e-12


def _one_triangle_scene(radar, verts0, vel, hit_uv, d_offset=0.0):
    tri = np.array([[0, 1, 2]], np.int32)
    t = np.arange(radar.n_chirps) * radar.chirp_period_s
    verts = verts0[None] + vel[None, None, :] * t[:, None, None]
    z = np.zeros(3)
    geom = scenegen.Geometry(verts, tri, np.zeros((radar.n_tx, 3)), np.zeros((radar.n_rx, 3)), z, z)
    n = len(hit_uv)
    hits = scenegen.Hits(np.arange(n + 1, dtype=np.int64), np.zeros(n, np.int32),
                         np.array([u for u, _ in hit_uv], np.float32), np.array([v for _, v in hit_uv], np.float32))
    return geom, hits


def test_barycentric_corners_are_the_vertices():
    radar = small_radar(n_samples=16, n_chirps=4, n_tx=1, n_rx=1, n_angle=1)
    verts0 = np.array([[10.0, 1.0, 0.5], [12.0, -2.0, 0.0], [9.0, 0.0, 3.0]])
    vel = np.array([3.0, -1.0, 0.5])
    geom, hits = _one_triangle_scene(radar, verts0, vel, [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0)])
    rays = Rays(2 * np.linalg.norm(verts0, axis=1), np.ones(3, np.float32), np.zeros(3, np.float32),
                np.zeros(3, np.float32), np.zeros(3, np.float32), np.zeros(3, np.float32), np.zeros(3, np.int32))
    P = oracle.paths(radar, rays, hits, geom)[:, :, 0]
    for q in range(3):
        for j in range(radar.n_chirps):
            ref = 2 * np.linalg.norm(verts0[q] + vel * j * radar.chirp_period_s)
            assert abs(P[q, j] - ref) <= 1e-12 * ref


def test_radial_motion_reduces_to_the_exact_model():
    """A triangle moving along the line of sight of its hit point at speed v, antennas at the
    origin: the path is d + 2 v j T_d and the signal equals Eq. 2 with tau_i(j) in both terms."""
    radar = small_radar(n_samples=32, n_chirps=16, n_tx=1, n_rx=1, n_angle=1)
    verts0 = np.array([[20.0, 3.0, 1.0], [21.0, 2.0, 0.0], [20.5, 4.0, -1.0]])
    uv = (0.25, 0.35)
    p0 = (1 - uv[0] - uv[1]) * verts0[0] + uv[0] * verts0[1] + uv[1] * verts0[2]
    v = 7.5
    geom, hits = _one_triangle_scene(radar, verts0, v * p0 / np.linalg.norm(p0), [uv])
    d = 2 * np.linalg.norm(p0)
    rays = one_ray(d, a=0.7, v=v, phi0=1.1)
    got = oracle.signal_geom(radar, rays, hits, geom)
    ref = oracle.signal(radar.replace(model=1), rays)
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()
    ref_bf = brute_signal_exact(radar, rays)
    assert np.abs(got - ref_bf).max() <= 1e-8 * np.abs(ref).max()


def test_far_field_limit_of_eq7():
    """A static scatterer 2 km away: the channel-to-channel path step of the array along -y is
    s sin(az) cos(el) to within aperture^2 / R."""
    radar = scenegen.radar_automotive(n_chirps=2, n_samples=16)
    lam = C / radar.carrier_hz
    s = lam / 2
    az, el = 0.4, -0.1
    dirv = np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    p0 = 2000.0 * dirv
    verts0 = p0[None] + np.array([[0.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    geom, hits = _one_triangle_scene(radar, verts0, np.zeros(3), [(0.0, 0.0)])
    geom.tx_pos[:, 1] = -np.arange(radar.n_tx) * radar.n_rx * s
    geom.rx_pos[:, 1] = -np.arange(radar.n_rx) * s
    rays = one_ray(2 * 2000.0)
    P = oracle.paths(radar, rays, hits, geom)[0, 0]
    k = np.arange(radar.n_virtual)
    aperture = radar.n_virtual * s
    assert np.abs((P - P[0]) - k * s * math.sin(az) * math.cos(el)).max() <= aperture ** 2 / 2000.0
    assert np.abs((P - P[0]) - k * s * math.sin(az) * math.cos(el)).max() > 0.0
