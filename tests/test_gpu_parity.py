"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Signal and spectrum: max |error| / max |oracle| and RMS error within the bound
of the ray-sum arithmetic (`gpu_helpers.TOL`): the 1e-5 target for FP32 and
split precision, a rounding bound below the 2e-3 target for single-pass FP16.
Single-pass BF16 misses its 2e-3 target on large frames; its cases assert its
rounding bound only and say so in their ids.  Labels and bins: bit exact.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import scenegen
from scenegen import Radar, Rays
from paper_2305_14176_gb300 import radarsim as rs
from gpu_helpers import TOL, TOL_RMS, prec_params, rel_max, rel_rms, run

pytestmark = pytest.mark.gpu

C = 299792458.0
PRECISIONS = prec_params(rs.SIM_PREC_FP32_DIRECT, rs.SIM_PREC_BF16_SPLIT, rs.SIM_PREC_FP16_SPLIT, rs.SIM_PREC_BF16,
                         rs.SIM_PREC_FP16)


@pytest.fixture(scope="module")
def tiny():
    radar, rays = scenegen.tiny_scene(seed=0)
    sig = oracle.signal(radar, rays)
    return radar, rays, sig, oracle.spectrum(radar, sig), oracle.labels(radar, rays)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("device_inputs", [True, False])
def test_tiny_scene_full_cube(tiny, precision, device_inputs):
    radar, rays, ref_sig, ref_spec, ref_lab = tiny
    rc, sig, spec, lab = run(radar, rays, precision, device_inputs)
    assert rc == rs.SIM_OK, rs.sim_status_string(rc)
    tol, trms = TOL[precision], TOL_RMS[precision]
    assert rel_max(sig, ref_sig) <= tol and rel_rms(sig, ref_sig) <= trms
    assert rel_max(spec, ref_spec) <= tol and rel_rms(spec, ref_spec) <= trms
    assert np.array_equal(lab, ref_lab)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("shape,n", [((16, 2, 1, 3, 4), 1), ((32, 4, 1, 3, 4), 255),
                                     ((64, 8, 2, 3, 8), 257), ((128, 128, 3, 4, 16), 700),
                                     ((256, 32, 1, 1, 1), 33), ((2048, 2, 1, 1, 1), 301),
                                     ((4096, 4, 1, 2, 2), 97),
                                     # three 128-row tiles in one channel each: the second
                                     # two-SM tile's odd CTA lies wholly past the last row
                                     ((64, 128, 1, 3, 4), 400),
                                     # wider arrays: 16, 24 and 64 virtual channels, angle FFTs
                                     # of 32 and 64 (zero padding 24 -> 32)
                                     ((64, 16, 4, 4, 32), 211), ((32, 8, 3, 8, 32), 150),
                                     ((16, 4, 8, 8, 64), 99), ((128, 32, 2, 8, 64), 173)])
def test_ragged_shapes(precision, shape, n):
    ns, nc, ntx, nrx, na = shape
    radar = Radar(77e9, 512e6, 25.6e-6, 40e-6, n_samples=ns, n_chirps=nc, n_tx=ntx, n_rx=nrx, n_angle=na)
    rays = scenegen.uniform_rays(seed=ns + n, n=n, n_objects=5)
    ref = oracle.signal(radar, rays)
    rc, sig, spec, lab = run(radar, rays, precision)
    assert rc == rs.SIM_OK
    tol = TOL[precision]
    assert rel_max(sig, ref) <= tol
    assert rel_max(spec, oracle.spectrum(radar, ref)) <= tol
    assert np.array_equal(lab, oracle.labels(radar, rays))


@pytest.mark.parametrize("precision", PRECISIONS)
def test_empty_scene(precision):
    radar = scenegen.radar_tiny()
    rays = scenegen.uniform_rays(seed=0, n=0)
    rc, sig, spec, lab = run(radar, rays, precision)
    assert rc == rs.SIM_OK
    assert np.all(sig == 0) and np.all(spec == 0) and np.all(lab == -1)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_automotive_radar_subsampled(precision):
    """The automotive frame's radar (12 x 256 x 512, N_a 16) with 3,000 of its rays:
    signal at 4,096 sampled points, spectrum at sampled and peak cells, labels whole."""
    radar, rays = scenegen.automotive_scene(seed=1000, n_rays=3000)
    rc, sig, spec, lab = run(radar, rays, precision)
    assert rc == rs.SIM_OK
    idx = scenegen.randint(7, 1, 4096, 0, sig.size - 1).astype(np.int64)
    ref = oracle.signal_at(radar, rays, idx)
    tol, trms = TOL[precision], TOL_RMS[precision]
    assert rel_max(sig.reshape(-1)[idx], ref) <= tol and rel_rms(sig.reshape(-1)[idx], ref) <= trms
    flat = np.abs(spec.reshape(-1))
    cells = np.unique(np.concatenate([np.argsort(-flat)[:16],
                                      scenegen.randint(7, 2, 240, 0, flat.size - 1)])).astype(np.int64)
    refc = oracle.cell_dtft(radar, rays, cells)
    assert rel_max(spec.reshape(-1)[cells], refc) <= tol
    assert np.array_equal(lab, oracle.labels(radar, rays))


@pytest.fixture(scope="module")
def imaging():
    """The imaging radar (12 x 16 = 192 virtual channels, angle FFT of 256, 512 chirps x 1024
    samples) with 2,000 of its rays, and the oracle's values at sampled outputs: 4,096 signal
    points and 256 spectrum cells (the analytic cells of the 32 strongest rays among them), and
    the labels whole."""
    radar, rays = scenegen.imaging_scene(seed=4100, n_rays=2000)
    n_sig = radar.n_virtual * radar.n_chirps * radar.n_samples
    n_cell = radar.n_angle * radar.n_chirps * radar.n_samples
    idx = scenegen.randint(41, 1, 4096, 0, n_sig - 1).astype(np.int64)
    strong = np.argsort(-rays.amplitude)[:32]
    cells = np.unique(np.concatenate([oracle.bins(radar, rays)["cell"][strong],
                                      scenegen.randint(41, 2, 224, 0, n_cell - 1)])).astype(np.int64)
    return (radar, rays, idx, oracle.signal_at(radar, rays, idx), cells, oracle.cell_dtft(radar, rays, cells),
            oracle.labels(radar, rays))


@pytest.mark.parametrize("precision", PRECISIONS)
def test_imaging_radar_shape(imaging, precision):
    """Every precision at the imaging radar's shape: the angle FFT over 192 channels zero padded
    to 256, a 1024-sample range FFT beside a 512-chirp Doppler FFT; sampled outputs against the
    oracle (the 1.1 GB spectrum stays on the device, only the sampled cells come back)."""
    radar, rays, idx, ref_sig, cells, ref_cells, ref_lab = imaging
    ctx = rs.Context(radar, precision=precision)
    try:
        arr = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.arrays().items()}
        sig = torch.full(ctx.signal_shape + (2,), float("nan"), dtype=torch.float32, device="cuda")
        spec = torch.full(ctx.cube_shape + (2,), float("nan"), dtype=torch.float32, device="cuda")
        lab = torch.full(ctx.cube_shape, -7, dtype=torch.int32, device="cuda")
        rc = ctx.fetch(ctx.submit(arr, rays.n), spec, sig, lab)
        assert rc == rs.SIM_OK, rs.sim_status_string(rc)
        torch.cuda.synchronize()
        s = sig.reshape(-1, 2)[torch.from_numpy(idx).cuda()].double().cpu().numpy()
        x = spec.reshape(-1, 2)[torch.from_numpy(cells).cuda()].double().cpu().numpy()
        peak = int(torch.argmax(spec.reshape(-1, 2).square().sum(1)).item())
        xp = spec.reshape(-1, 2)[peak].double().cpu().numpy()
        labels = lab.cpu().numpy()
    finally:
        ctx.close()
    tol, trms = TOL[precision], TOL_RMS[precision]
    got_s = s[:, 0] + 1j * s[:, 1]
    assert rel_max(got_s, ref_sig) <= tol and rel_rms(got_s, ref_sig) <= trms
    got_x = x[:, 0] + 1j * x[:, 1]
    assert rel_max(got_x, ref_cells) <= tol and rel_rms(got_x, ref_cells) <= trms
    # the strongest cell of the whole spectrum, against the oracle's closed form there
    ref_peak = oracle.cell_dtft(radar, rays, np.array([peak], np.int64))
    assert rel_max(np.array([xp[0] + 1j * xp[1]]), ref_peak) <= tol
    assert np.array_equal(labels, ref_lab)
    assert (labels >= 0).any()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_automotive_frame_full_size(precision):
    """The full automotive frame (200,000 rays) in the launch configuration the benchmark
    times: signal at sampled points, four spectrum cells (the peak among them), labels whole."""
    radar, rays = scenegen.automotive_scene(seed=1000)
    rc, sig, spec, lab = run(radar, rays, precision)
    assert rc == rs.SIM_OK
    idx = scenegen.randint(8, 1, 256, 0, sig.size - 1).astype(np.int64)
    ref = oracle.signal_at(radar, rays, idx)
    tol, trms = TOL[precision], TOL_RMS[precision]
    assert rel_rms(sig.reshape(-1)[idx], ref) <= trms
    assert rel_max(sig.reshape(-1)[idx], ref) <= tol
    flat = np.abs(spec.reshape(-1))
    cells = np.array([int(np.argmax(flat)), 12345, 777777, int(flat.size - 1)], np.int64)
    refc = oracle.cell_dtft(radar, rays, cells)
    assert rel_max(spec.reshape(-1)[cells], refc, norm=np.abs(refc).max()) <= tol
    assert np.array_equal(lab, oracle.labels(radar, rays))


def _boundary_rays(radar, seed):
    """Rays whose range, Doppler or angle coordinate sits within a few ulp of a bin edge."""
    lam = C / radar.carrier_hz
    out = []
    oid = 0
    rng = np.random.default_rng(seed)
    for q in (0, 3, 17, radar.n_samples - 1, radar.n_samples + 2):
        d0 = (q + 0.5) * C / radar.bandwidth_hz
        for k in range(-3, 4):
            d = d0
            for _ in range(abs(k)):
                d = np.nextafter(d, np.inf if k > 0 else -np.inf)
            out.append((d, 0.0, 0.0, oid)); oid += 1
    for q in (-3, 0, 5, radar.n_chirps // 2 - 1):
        v0 = np.float32((q + 0.5) * lam / (2 * radar.n_chirps * radar.chirp_period_s))
        for k in range(-3, 4):
            v = v0
            for _ in range(abs(k)):
                v = np.nextafter(v, np.float32(np.inf if k > 0 else -np.inf))
            out.append((40 * C / radar.bandwidth_hz, float(v), 0.0, oid)); oid += 1
    for q in (-2, 0, 1, 3):
        a0 = np.float32(math.asin((q + 0.5) / (radar.n_angle * 0.5)))
        for k in range(-3, 4):
            a = a0
            for _ in range(abs(k)):
                a = np.nextafter(a, np.float32(np.inf if k > 0 else -np.inf))
            out.append((80 * C / radar.bandwidth_hz, 0.0, float(a), oid)); oid += 1
    n = len(out)
    return Rays(np.array([o[0] for o in out]), rng.uniform(0.1, 1.0, n).astype(np.float32),
                np.array([o[1] for o in out], np.float32), np.array([o[2] for o in out], np.float32),
                np.zeros(n, np.float32), np.zeros(n, np.float32), np.array([o[3] for o in out], np.int32))


def test_bin_edges_are_bit_exact():
    radar = scenegen.radar_automotive(n_chirps=64, n_samples=128)
    rays = _boundary_rays(radar, 3)
    ref = oracle.labels(radar, rays)
    rc, _, _, lab = run(radar, rays, rs.SIM_PREC_FP32_DIRECT,
                        outputs=rs.SIM_OUT_SPECTRUM | rs.SIM_OUT_LABELS)
    assert rc == rs.SIM_OK
    assert np.array_equal(lab, ref)
    # the cells really do straddle edges: both sides occur among the nudged rays
    b = oracle.bins(radar, rays)
    assert np.any(np.abs(b["x_r"] - np.round(b["x_r"] - 0.5) - 0.5) < 1e-12)


def test_invalid_rays_rejected():
    radar, rays = scenegen.tiny_scene(seed=1, n_rays=50)
    bad = rays.take(slice(None))
    bad.range_rt_m = bad.range_rt_m.copy()
    bad.range_rt_m[7] = np.nan
    ctx = rs.Context(radar)
    try:
        with pytest.raises(rs.SimError) as e:  # host arrays: rejected at submit
            ctx.submit(bad.arrays(), bad.n)
        assert e.value.code == rs.SIM_E_INVALID
        arr = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in bad.arrays().items()}
        t = ctx.submit(arr, bad.n)  # device arrays: the prep kernel flags them
        assert ctx.fetch(t) == rs.SIM_E_INVALID
        with pytest.raises(rs.SimError):
            ctx.submit(rays.arrays(), (1 << 21) + 1)
        neg = rays.take(slice(None))
        neg.object_id = neg.object_id.copy()
        neg.object_id[0] = -4
        with pytest.raises(rs.SimError):
            ctx.submit(neg.arrays(), neg.n)
    finally:
        ctx.close()


def test_unknown_ticket_and_poll():
    radar, rays = scenegen.automotive_scene(seed=5, n_rays=20000)
    ctx = rs.Context(radar)
    try:
        assert ctx.fetch(123456789) == rs.SIM_E_UNKNOWN_TICKET
        t = ctx.submit(rays.arrays(), rays.n)
        rc = ctx.fetch(t, timeout_ms=0)
        assert rc in (rs.SIM_E_NOT_READY, rs.SIM_OK)
        if rc != rs.SIM_OK:
            assert ctx.fetch(t, timeout_ms=-1) == rs.SIM_OK
        assert ctx.fetch(t) == rs.SIM_E_UNKNOWN_TICKET
    finally:
        ctx.close()


def test_linearity_on_gpu():
    """Eq. 5: the cube of A and B together equals the sum of their cubes."""
    radar = scenegen.radar_tiny()
    A = scenegen.uniform_rays(seed=31, n=600)
    B = scenegen.uniform_rays(seed=32, n=400)
    _, sA, _, _ = run(radar, A)
    _, sB, _, _ = run(radar, B)
    _, sAB, _, _ = run(radar, Rays.concat([A, B]))
    assert rel_max(sAB, sA + sB) <= 1e-5


def test_exact_model_direct_sum():
    """Eq. 2 with the range-migration product, on the direct-sum path."""
    radar, rays = scenegen.tiny_scene(seed=6, n_rays=800)
    radar = radar.replace(model=1)
    ref = oracle.signal(radar, rays)
    ctx = rs.Context(radar, precision=rs.SIM_PREC_FP32_DIRECT, model=rs.SIM_MODEL_EXACT)
    try:
        rc, sig, spec, lab = run(radar, rays, rs.SIM_PREC_FP32_DIRECT, ctx=ctx)
    finally:
        ctx.close()
    assert rc == rs.SIM_OK
    assert rel_max(sig, ref) <= 1e-5 and rel_rms(sig, ref) <= 1e-5
    assert rel_max(spec, oracle.spectrum(radar, ref)) <= 1e-5
    assert np.array_equal(lab, oracle.labels(radar, rays))
    # a moving automotive scene at full radar size, sampled
    radar2, rays2 = scenegen.automotive_scene(seed=44, n_rays=5000)
    radar2 = radar2.replace(model=1)
    ctx = rs.Context(radar2, precision=rs.SIM_PREC_FP32_DIRECT, model=rs.SIM_MODEL_EXACT)
    try:
        rc, sig2, _, _ = run(radar2, rays2, rs.SIM_PREC_FP32_DIRECT, ctx=ctx)
    finally:
        ctx.close()
    idx = scenegen.randint(44, 3, 2048, 0, sig2.size - 1).astype(np.int64)
    ref2 = oracle.signal_at(radar2, rays2, idx)
    assert rel_max(sig2.reshape(-1)[idx], ref2) <= 1e-5


@pytest.mark.parametrize("precision", PRECISIONS)
def test_antenna_pattern(precision):
    """Eq. 2's antenna gain (cos az cos el)^q scales every ray on every path; the labels,
    decided on the weighted energies, stay bit exact."""
    radar, rays = scenegen.tiny_scene(seed=9, n_rays=900)
    radar = radar.replace(pattern_exp=6)
    ref = oracle.signal(radar, rays)
    rc, sig, spec, lab = run(radar, rays, precision)
    assert rc == rs.SIM_OK
    tol, trms = TOL[precision], TOL_RMS[precision]
    assert rel_max(sig, ref) <= tol and rel_rms(sig, ref) <= trms
    assert rel_max(spec, oracle.spectrum(radar, ref)) <= tol
    assert np.array_equal(lab, oracle.labels(radar, rays))
    # a crowded cube where the gain moves 27 of 323 labels
    crowded = Radar(77e9, 512e6, 25.6e-6, 40e-6, n_samples=32, n_chirps=4, n_tx=1, n_rx=3, n_angle=4,
                    pattern_exp=6)
    rays = scenegen.uniform_rays(seed=77, n=700, n_objects=5)
    rc, _, _, lab = run(crowded, rays, precision)
    assert rc == rs.SIM_OK
    ref_lab = oracle.labels(crowded, rays)
    assert np.array_equal(lab, ref_lab)
    assert np.sum(ref_lab != oracle.labels(crowded.replace(pattern_exp=0), rays)) == 27


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("shape", [(64, 32, 3, 4, 16), (32, 128, 3, 2, 8)])
def test_tdm_slot_offsets(precision, shape):
    """TDM-MIMO slot offsets: transmitter t's chirps start t T_slot later, on every path
    (the second shape fills whole 128-chirp tiles, the tensor core's single-channel tiles)."""
    ns, nc, ntx, nrx, na = shape
    radar = Radar(77e9, 512e6, 25.6e-6, 40e-6, n_samples=ns, n_chirps=nc, n_tx=ntx, n_rx=nrx, n_angle=na,
                  tdm_slot_s=13.3e-6)
    rays = scenegen.uniform_rays(seed=ns + nc, n=700, n_objects=4, v_max=30.0)
    ref = oracle.signal(radar, rays)
    rc, sig, spec, lab = run(radar, rays, precision)
    assert rc == rs.SIM_OK
    tol, trms = TOL[precision], TOL_RMS[precision]
    assert rel_max(sig, ref) <= tol and rel_rms(sig, ref) <= trms
    assert rel_max(spec, oracle.spectrum(radar, ref)) <= tol
    assert np.array_equal(lab, oracle.labels(radar, rays))
    # the offsets change the cube well beyond the tolerance
    assert rel_max(oracle.signal(radar.replace(tdm_slot_s=0.0), rays), ref) > 100 * tol


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("shape", [(64, 32, 3, 4, 16, 30.0), (128, 64, 4, 2, 8, 30.0), (64, 32, 3, 4, 16, 5.0)])
def test_tdm_exact_model(precision, shape):
    """Exact Eq. 2 with TDM slot offsets on every path: on tensor cores the slot term n t eps_t
    joins the per-tile expansion (transmitters about their centre); at 30 m/s six Chebyshev terms
    (four single pass on the narrower case), at 5 m/s four Taylor terms."""
    ns, nc, ntx, nrx, na, v_max = shape
    radar = Radar(77e9, 512e6, 25.6e-6, 40e-6, n_samples=ns, n_chirps=nc, n_tx=ntx, n_rx=nrx, n_angle=na,
                  tdm_slot_s=9.1e-6, model=1)
    rays = scenegen.uniform_rays(seed=71 + ns, n=600, n_objects=4, v_max=v_max)
    ref = oracle.signal(radar, rays)
    ctx = rs.Context(radar, precision=precision, model=rs.SIM_MODEL_EXACT)
    try:
        rc, sig, spec, lab = run(radar, rays, precision, ctx=ctx)
        route = rs.sim_last_expansion_terms(ctx.ctx)
    finally:
        ctx.close()
    assert rc == rs.SIM_OK, rs.sim_status_string(rc)
    # the FP32 direct sum chooses no term count; route bits: P Taylor, 16 + P Chebyshev terms
    split = precision in (rs.SIM_PREC_BF16_SPLIT, rs.SIM_PREC_FP16_SPLIT)
    expect = {(64, 30.0): {22} if split else {20}, (128, 30.0): {22}, (64, 5.0): {4}}[(ns, v_max)]
    assert route == (set() if precision == rs.SIM_PREC_FP32_DIRECT else expect)
    tol, trms = TOL[precision], TOL_RMS[precision]
    assert rel_max(sig, ref) <= tol and rel_rms(sig, ref) <= trms
    assert rel_max(spec, oracle.spectrum(radar, ref)) <= tol
    assert np.array_equal(lab, oracle.labels(radar, rays))
    # both couplings matter: without the slot term, or without the migration, the cube is off
    assert rel_max(oracle.signal(radar.replace(tdm_slot_s=0.0), rays), ref) > 1e-4
    assert rel_max(oracle.signal(radar.replace(model=0), rays), ref) > 1e-4


@pytest.mark.filterwarnings("ignore:invalid value encountered in cast")  # a failed fetch's outputs are undefined
@pytest.mark.parametrize("precision", [rs.SIM_PREC_BF16_SPLIT, rs.SIM_PREC_FP16])
def test_tdm_exact_model_beyond_the_expansion_is_reported(precision):
    """With TDM slots the exact model has no per-chirp tensor form, so a migration beyond the
    eight-term bound is an error (invalid rays) rather than a silent approximation; the same
    context then computes an ordinary scene."""
    radar = Radar(77e9, 512e6, 25.6e-6, 40e-6, n_samples=64, n_chirps=32, n_tx=3, n_rx=4, n_angle=16,
                  tdm_slot_s=9.1e-6, model=1)
    fast = scenegen.uniform_rays(seed=72, n=300, n_objects=4, v_max=2000.0)
    slow = scenegen.uniform_rays(seed=73, n=300, n_objects=4, v_max=15.0)
    ctx = rs.Context(radar, precision=precision, model=rs.SIM_MODEL_EXACT)
    try:
        rc, _, _, _ = run(radar, fast, precision, ctx=ctx)
        assert rc == rs.SIM_E_INVALID
        rc, sig, _, _ = run(radar, slow, precision, ctx=ctx)
        assert rc == rs.SIM_OK
        ref = oracle.signal(radar, slow)
        assert rel_max(sig, ref) <= TOL[precision]
    finally:
        ctx.close()


@pytest.mark.parametrize("precision", prec_params(rs.SIM_PREC_BF16_SPLIT, rs.SIM_PREC_FP16_SPLIT, rs.SIM_PREC_BF16,
                                                   rs.SIM_PREC_FP16))
def test_exact_model_tensor_core(precision):
    """The exact model on tensor cores: per chirp, samples x channels tiles."""
    radar, rays = scenegen.tiny_scene(seed=16, n_rays=900)
    radar = radar.replace(model=1)
    ref = oracle.signal(radar, rays)
    ctx = rs.Context(radar, precision=precision, model=rs.SIM_MODEL_EXACT)
    try:
        rc, sig, spec, lab = run(radar, rays, precision, ctx=ctx)
    finally:
        ctx.close()
    assert rc == rs.SIM_OK, rs.sim_status_string(rc)
    tol, trms = TOL[precision], TOL_RMS[precision]
    assert rel_max(sig, ref) <= tol and rel_rms(sig, ref) <= trms
    assert rel_max(spec, oracle.spectrum(radar, ref)) <= tol
    assert np.array_equal(lab, oracle.labels(radar, rays))
    # channels past a 16-column tile, samples below one 128-sample tile, and a ragged ray count
    small = Radar(77e9, 512e6, 25.6e-6, 40e-6, n_samples=64, n_chirps=8, n_tx=3, n_rx=7, n_angle=32, model=1)
    rays2 = scenegen.uniform_rays(seed=61, n=333, v_max=30.0)
    ref2 = oracle.signal(small, rays2)
    ctx = rs.Context(small, precision=precision, model=rs.SIM_MODEL_EXACT)
    try:
        rc, sig2, _, _ = run(small, rays2, precision, ctx=ctx)
    finally:
        ctx.close()
    assert rc == rs.SIM_OK
    assert rel_max(sig2, ref2) <= tol and rel_rms(sig2, ref2) <= trms


@pytest.mark.parametrize("precision", prec_params(rs.SIM_PREC_BF16_SPLIT, rs.SIM_PREC_FP16_SPLIT, rs.SIM_PREC_BF16,
                                                   rs.SIM_PREC_FP16))
@pytest.mark.parametrize("case", ["narrow_tile", "beyond_expansion", "short_chirp"])
def test_exact_model_tensor_core_regimes(precision, case):
    """The exact model's per-tile expansion of the range-migration phase in its edge regimes:
    the narrowest two-SM tile (32 samples, 16 columns of B per CTA, 43 chirps per tile: six
    Chebyshev terms); a velocity whose migration phase no eight-term expansion bounds (the device hands
    the scene to the per-chirp kernel); and 16 samples (per-chirp kernel chosen on the host,
    no term choice)."""
    ns, nc, ntx, nrx, na, v_max = {"narrow_tile": (32, 16, 1, 3, 4, 15.0),
                                   "beyond_expansion": (64, 32, 1, 4, 16, 2000.0),
                                   "short_chirp": (16, 32, 2, 2, 4, 15.0)}[case]
    radar = Radar(77e9, 512e6, 25.6e-6, 40e-6, n_samples=ns, n_chirps=nc, n_tx=ntx, n_rx=nrx, n_angle=na, model=1)
    rays = scenegen.uniform_rays(seed=ns * nc + ntx, n=517, n_objects=4, v_max=v_max)
    ref = oracle.signal(radar, rays)
    ctx = rs.Context(radar, precision=precision, model=rs.SIM_MODEL_EXACT)
    try:
        rc, sig, spec, lab = run(radar, rays, precision, ctx=ctx)
        route = rs.sim_last_expansion_terms(ctx.ctx)
    finally:
        ctx.close()
    assert rc == rs.SIM_OK, rs.sim_status_string(rc)
    assert route == {"narrow_tile": {22}, "beyond_expansion": {0}, "short_chirp": set()}[case]
    tol, trms = TOL[precision], TOL_RMS[precision]
    assert rel_max(sig, ref) <= tol and rel_rms(sig, ref) <= trms
    assert rel_max(spec, oracle.spectrum(radar, ref)) <= tol
    assert np.array_equal(lab, oracle.labels(radar, rays))
    # the migration term matters here: the separable model misses the cube by far more
    assert rel_max(oracle.signal(radar.replace(model=0), rays), ref) > 10 * tol


@pytest.mark.parametrize("precision", prec_params(rs.SIM_PREC_FP16_SPLIT, rs.SIM_PREC_BF16))
@pytest.mark.parametrize("shape", [(4096, 4, 1, 2, 2), (64, 2, 1, 1, 1), (256, 512, 2, 2, 4)])
def test_exact_model_tensor_core_size_extremes(precision, shape):
    """The expansion at the edges of the radar sizes: 4096 samples (16 column tiles of 256),
    two chirps with one channel (the tile's rows are mostly past M), and 512 chirps of four
    channels (64 chirps per 256-row tile, six terms)."""
    ns, nc, ntx, nrx, na = shape
    radar = Radar(77e9, 512e6, 25.6e-6, 40e-6, n_samples=ns, n_chirps=nc, n_tx=ntx, n_rx=nrx, n_angle=na, model=1)
    rays = scenegen.uniform_rays(seed=ns + nc, n=150, n_objects=3, v_max=15.0)
    ref = oracle.signal(radar, rays)
    ctx = rs.Context(radar, precision=precision, model=rs.SIM_MODEL_EXACT)
    try:
        rc, sig, _, lab = run(radar, rays, precision, ctx=ctx)
    finally:
        ctx.close()
    assert rc == rs.SIM_OK, rs.sim_status_string(rc)
    assert rel_max(sig, ref) <= TOL[precision] and rel_rms(sig, ref) <= TOL_RMS[precision]
    assert np.array_equal(lab, oracle.labels(radar, rays))


@pytest.mark.parametrize("precision", prec_params(rs.SIM_PREC_BF16_SPLIT, rs.SIM_PREC_FP16_SPLIT, rs.SIM_PREC_BF16,
                                                   rs.SIM_PREC_FP16))
@pytest.mark.parametrize("v_max,split_route,single_route", [(3.0, 4, 4), (7.0, 20, 4), (25.0, 22, 22), (70.0, 24, 24),
                                                          (2000.0, 0, 0)])
def test_exact_model_each_term_count(precision, v_max, split_route, single_route):
    """Every route of the exact model's expansion (Sec. II-A, Eq. 2): the velocity sets the
    expansion variable theta = 2 pi n_h max|eps| m_h (0.042, 0.099, 0.35, 0.99, 28 on this
    radar of 64 samples and 4 channels).  The device takes four Taylor terms where they meet
    the tolerance (route bit 4), else the fewest Chebyshev (Jacobi-Anger) terms that do: four,
    six (five rays and two zero K slots per stage) or eight (bits 20, 22, 24), else the
    per-chirp kernel (bit 0).  The single-pass tolerance is ten times looser, so 7 m/s still
    takes Taylor terms there."""
    radar = Radar(77e9, 512e6, 25.6e-6, 40e-6, n_samples=64, n_chirps=32, n_tx=1, n_rx=4, n_angle=16, model=1)
    rays = scenegen.uniform_rays(seed=90 + int(v_max) % 97, n=517, n_objects=4, v_max=v_max)
    ref = oracle.signal(radar, rays)
    ctx = rs.Context(radar, precision=precision, model=rs.SIM_MODEL_EXACT)
    try:
        rc, sig, spec, lab = run(radar, rays, precision, ctx=ctx)
        route = rs.sim_last_expansion_terms(ctx.ctx)
    finally:
        ctx.close()
    assert rc == rs.SIM_OK, rs.sim_status_string(rc)
    split = precision in (rs.SIM_PREC_BF16_SPLIT, rs.SIM_PREC_FP16_SPLIT)
    assert route == {split_route if split else single_route}
    tol, trms = TOL[precision], TOL_RMS[precision]
    assert rel_max(sig, ref) <= tol and rel_rms(sig, ref) <= trms
    assert rel_max(spec, oracle.spectrum(radar, ref)) <= tol
    assert np.array_equal(lab, oracle.labels(radar, rays))


@pytest.mark.parametrize("precision", [rs.SIM_PREC_FP16_SPLIT, rs.SIM_PREC_BF16_SPLIT])
def test_exact_model_tensor_core_automotive_sampled(precision):
    """Full automotive radar size (four expansion terms): at FP16 hi + lo the third and fourth
    terms go single pass (their bound times the FP16 rounding is below 2e-6), at BF16 hi + lo
    they keep their lo operands."""
    radar, rays = scenegen.automotive_scene(seed=45, n_rays=50_000)
    radar = radar.replace(model=1)
    ctx = rs.Context(radar, precision=precision, model=rs.SIM_MODEL_EXACT)
    try:
        rc, sig, _, lab = run(radar, rays, precision, ctx=ctx)
    finally:
        ctx.close()
    assert rc == rs.SIM_OK
    idx = scenegen.randint(45, 3, 1024, 0, sig.size - 1).astype(np.int64)
    ref = oracle.signal_at(radar, rays, idx)
    assert rel_max(sig.reshape(-1)[idx], ref) <= 1e-5 and rel_rms(sig.reshape(-1)[idx], ref) <= 1e-5
    assert np.array_equal(lab, oracle.labels(radar, rays))
