"""GPU parity of virtual snapshots (Sec. II-D, Eq. 6) and antenna displacement (Sec. II-E,
Eq. 7): per-(ray, chirp, channel) path lengths and the signal, spectrum and labels built on
them, through the C ABI, against the FP64 oracle on seeded moving-box scenes."""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from paper_2305_14176_gb300 import radarsim as rs
from gpu_helpers import TOL, TOL_RMS, prec_params, rel_max, rel_rms, to_c

pytestmark = pytest.mark.gpu


def _arrays(rays, hits, geom, device):
    a = dict(rays.arrays())
    a["material_id"] = rays.material_id
    a.update(vertices=geom.vertices, triangles=geom.triangles, tx_pos=geom.tx_pos, rx_pos=geom.rx_pos,
             hit_offset=hits.offset, hit_triangle=hits.triangle, hit_u=hits.u, hit_v=hits.v)
    a = {k: np.ascontiguousarray(v) for k, v in a.items()}
    if device:
        a = {k: torch.from_numpy(v).cuda() for k, v in a.items()}
    return a


def snapshot(radar, rays, hits, geom, device=True, paths=False, outputs=None, precision=rs.SIM_PREC_FP32_DIRECT,
             routes=None):
    """routes (a list, optional) receives the call's expansion route (sim_last_expansion_terms)."""
    outputs = outputs or (rs.SIM_OUT_SIGNAL | rs.SIM_OUT_SPECTRUM | rs.SIM_OUT_LABELS)
    ctx = rs.Context(radar, precision=precision, outputs=outputs)
    try:
        a = _arrays(rays, hits, geom, device)
        r, m = rs.make_rays(a, rays.n)
        g, h = rs.make_geometry(a, geom.ref_tx, geom.ref_rx)
        if paths:
            out = torch.zeros((rays.n, radar.n_chirps, radar.n_virtual), dtype=torch.float64,
                              device="cuda" if device else "cpu")
            rc = rs.sim_snapshot_paths(ctx.ctx, r, h, g, out)
            torch.cuda.synchronize()
            return rc, out.cpu().numpy()
        sig = torch.zeros(ctx.signal_shape + (2,), dtype=torch.float32, device="cuda")
        spec = torch.zeros(ctx.cube_shape + (2,), dtype=torch.float32, device="cuda")
        lab = torch.zeros(ctx.cube_shape, dtype=torch.int32, device="cuda")
        rc = rs.sim_snapshot_run(ctx.ctx, r, m, h, g, spec, sig, lab)
        torch.cuda.synchronize()
        if routes is not None:
            routes.append(rs.sim_last_expansion_terms(ctx.ctx))
        return rc, to_c(sig), to_c(spec), lab.cpu().numpy()
    finally:
        ctx.close()


@pytest.mark.parametrize("device", [True, False])
def test_paths_match_oracle(device):
    radar = scenegen.radar_automotive(n_chirps=16, n_samples=32)
    rays, hits, geom = scenegen.moving_scene(21, radar, 300, bounce_frac=0.3)
    rc, got = snapshot(radar, rays, hits, geom, device=device, paths=True)
    assert rc == rs.SIM_OK, rs.sim_status_string(rc)
    ref = oracle.paths(radar, rays, hits, geom)
    # reference legs in float-float (~48 bits), antenna offsets (<= 1.6 cm here) from them in
    # FP32: ~3e-7 of the offset, 5 nm
    assert np.abs(got - ref).max() <= 2e-8
    assert np.abs(got[:, :, 0] - ref[:, :, 0]).max() <= 1e-9   # the reference pair itself: no FP32 offset


def test_paths_far_and_translated():
    """Far targets (100-250 m) in a scene moved 2.9 km from the origin: the per-chirp legs are
    float-float relative to the reference transmitter, so neither the range nor the absolute
    position costs accuracy."""
    radar = scenegen.radar_automotive(n_chirps=16, n_samples=32)
    rays, hits, g0 = scenegen.moving_scene(22, radar, 300, bounce_frac=0.3, r_range=(100.0, 250.0))
    shift = np.array([1500.0, -2500.0, 30.0])
    geom = scenegen.Geometry(g0.vertices + shift, g0.triangles, g0.tx_pos + shift, g0.rx_pos + shift,
                             g0.ref_tx + shift, g0.ref_rx + shift)
    rc, got = snapshot(radar, rays, hits, geom, paths=True)
    assert rc == rs.SIM_OK, rs.sim_status_string(rc)
    ref = oracle.paths(radar, rays, hits, geom)
    assert ref.min() > 150.0                                    # round trips of 100 m and more
    assert np.abs(got - ref).max() <= 2e-8
    assert np.abs(got[:, :, 0] - ref[:, :, 0]).max() <= 1e-9
    # the translation changes the oracle's FP64 rounding only
    assert np.abs(ref - oracle.paths(radar, rays, hits, g0)).max() <= 1e-9


PRECISIONS = prec_params(rs.SIM_PREC_FP32_DIRECT, rs.SIM_PREC_FP16_SPLIT, rs.SIM_PREC_BF16_SPLIT, rs.SIM_PREC_FP16,
                         rs.SIM_PREC_BF16)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("shape", [(32, 16, 3, 4, 16), (64, 8, 1, 4, 16), (16, 4, 2, 3, 8), (128, 64, 2, 2, 4)])
def test_signal_spectrum_labels_match_oracle(shape, precision):
    """Every precision: FP32 sums directly; the tensor-core precisions expand each tile about
    its centre with each row's own phase words (N_s = 16 is summed directly at any precision).
    The scenes' largest 2 pi n_h |S - S_ref| (0.25, 0.14, -, 0.54) take six, six, no and eight
    Chebyshev terms at hi + lo (route bits 22, 22, -, 24), and six, four, no and six single
    pass."""
    ns, nc, ntx, nrx, na = shape
    radar = scenegen.Radar(77e9, 1e9, 51.2e-6, 60e-6, n_samples=ns, n_chirps=nc, n_tx=ntx, n_rx=nrx, n_angle=na)
    rays, hits, geom = scenegen.moving_scene(ns + nc, radar, 333, n_objects=5, bounce_frac=0.3)
    routes = []
    rc, sig, spec, lab = snapshot(radar, rays, hits, geom, precision=precision, routes=routes)
    assert rc == rs.SIM_OK, rs.sim_status_string(rc)
    split = precision in (rs.SIM_PREC_BF16_SPLIT, rs.SIM_PREC_FP16_SPLIT)
    terms = ({32: {22}, 64: {22}, 16: set(), 128: {24}} if split else {32: {22}, 64: {20}, 16: set(), 128: {22}})[ns]
    assert routes == [set() if precision == rs.SIM_PREC_FP32_DIRECT else terms]
    ref = oracle.signal_geom(radar, rays, hits, geom)
    tol, trms = TOL[precision], TOL_RMS[precision]
    assert rel_max(sig, ref) <= tol and rel_rms(sig, ref) <= trms
    assert rel_max(spec, oracle.spectrum(radar, ref)) <= tol
    assert np.array_equal(lab, oracle.labels(radar, rays))
    # host inputs give the same bits
    rc, sig_h, _, _ = snapshot(radar, rays, hits, geom, device=False, precision=precision)
    assert rc == rs.SIM_OK and np.array_equal(sig_h, sig)


@pytest.mark.parametrize("precision", [rs.SIM_PREC_FP16_SPLIT, rs.SIM_PREC_FP16])
def test_fast_boxes_take_the_pair_sum(precision):
    """Boxes at up to 3 km/s move a path by ~4 m across a 256-row tile's eleven chirps: the
    steps' spread 2 pi n_h |S - S_ref| is ~40 rad, far beyond eight Chebyshev terms, so the
    chunk's bound sends it to the FP32 pair sum (route bit 0) and the result is the FP32
    path's."""
    radar = scenegen.radar_automotive(n_chirps=16, n_samples=64)
    rays, hits, geom = scenegen.moving_scene(27, radar, 300, n_objects=4, bounce_frac=0.3, v_max=3000.0)
    routes = []
    rc, sig, spec, lab = snapshot(radar, rays, hits, geom, precision=precision, routes=routes)
    assert rc == rs.SIM_OK, rs.sim_status_string(rc)
    assert routes == [{0}]
    ref = oracle.signal_geom(radar, rays, hits, geom)
    assert rel_max(sig, ref) <= TOL[rs.SIM_PREC_FP32_DIRECT] and rel_rms(sig, ref) <= TOL_RMS[rs.SIM_PREC_FP32_DIRECT]
    assert rel_max(spec, oracle.spectrum(radar, ref)) <= TOL[rs.SIM_PREC_FP32_DIRECT]
    assert np.array_equal(lab, oracle.labels(radar, rays))


@pytest.mark.parametrize("precision", [rs.SIM_PREC_FP32_DIRECT, rs.SIM_PREC_FP16_SPLIT])
def test_automotive_size_in_two_chunks_sampled(precision):
    """256 chirps x 512 samples x 12 channels; 240,000 rays need two chunks of phase words
    (224,512 rays fill the 3 GiB of a chunk; the second chunk adds to the first, on tensor cores
    too)."""
    radar = scenegen.radar_automotive()
    rays, hits, geom = scenegen.moving_scene(1234, radar, 240_000, n_objects=20)
    routes = []
    rc, sig, spec, lab = snapshot(radar, rays, hits, geom, precision=precision, routes=routes)
    assert rc == rs.SIM_OK, rs.sim_status_string(rc)
    if precision == rs.SIM_PREC_FP32_DIRECT:
        assert routes == [set()]
    else:  # each chunk picks its own expansion; these road-speed boxes need four terms
        assert routes[0] and routes[0] <= {4, 20}
    idx = scenegen.randint(1234, 9, 384, 0, sig.size - 1).astype(np.int64)
    ref = oracle.signal_geom_at(radar, rays, hits, geom, idx)
    assert rel_max(sig.reshape(-1)[idx], ref) <= 1e-5
    assert rel_rms(sig.reshape(-1)[idx], ref) <= 1e-5
    assert np.array_equal(lab, oracle.labels(radar, rays))


def test_invalid_geometry_is_an_error():
    radar = scenegen.radar_automotive(n_chirps=4, n_samples=16)
    rays, hits, geom = scenegen.moving_scene(5, radar, 50)
    bad = scenegen.Hits(hits.offset, hits.triangle.copy(), hits.u, hits.v)
    bad.triangle[7] = geom.triangles.shape[0]          # one past the last triangle
    assert snapshot(radar, rays, bad, geom)[0] == rs.SIM_E_INVALID
    tris = geom.triangles.copy()
    tris[0, 1] = geom.vertices.shape[1] + 5            # a vertex index past the mesh
    g2 = scenegen.Geometry(geom.vertices, tris, geom.tx_pos, geom.rx_pos, geom.ref_tx, geom.ref_rx)
    hits0 = scenegen.Hits(hits.offset, np.zeros_like(hits.triangle), hits.u, hits.v)
    assert snapshot(radar, rays, hits0, g2)[0] == rs.SIM_E_INVALID
    off = hits.offset.copy()
    off[10] = off[11]                                  # ray 10 left without hits
    assert snapshot(radar, rays, scenegen.Hits(off, hits.triangle, hits.u, hits.v), geom)[0] == rs.SIM_E_INVALID
    # the tensor-core precisions run snapshots too
    assert snapshot(radar, rays, hits, geom, precision=rs.SIM_PREC_BF16_SPLIT)[0] == rs.SIM_OK
    # and a good call still works afterwards
    assert snapshot(radar, rays, hits, geom)[0] == rs.SIM_OK
