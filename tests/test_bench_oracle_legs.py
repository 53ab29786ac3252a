"""The oracle legs of bench.py on tiny scenes (host only): each leg's sampled values are the
full oracle's at the same indices, and the error the bench line reports is zero on the
oracle's own output and sees a planted change."""
import numpy as np

import bench
import oracle
import scenegen


def _complex_as_f32_pairs(x: np.ndarray) -> np.ndarray:
    return np.stack([x.real, x.imag], -1).astype(np.float32)


def test_signal_leg_samples_the_full_oracle_and_error_is_exact_on_it():
    radar = scenegen.radar_automotive(n_chirps=16, n_samples=32)
    _, rays = scenegen.automotive_scene(seed=41, n_rays=300, radar=radar)
    rate, n_pts, dt, cores, idx, ref = bench.cpu_oracle_rate(radar, rays, seconds=0.05, seed=5)
    full = oracle.signal(radar, rays)
    assert rate > 0 and cores >= 1 and n_pts == idx.shape[0] == ref.shape[0]
    assert np.allclose(ref, full.reshape(-1)[idx], rtol=0, atol=1e-12 * np.abs(full).max())
    lab = oracle.labels(radar, rays)
    err = bench.result_error(radar, rays, _complex_as_f32_pairs(full), lab, idx, ref)
    assert err["labels_exact"] and err["max_rel"] < 1e-6 and err["rms_rel"] < 1e-6
    bad = _complex_as_f32_pairs(full)
    bad.reshape(-1, 2)[idx[0], 0] += np.float32(1e-3 * np.abs(full).max())
    lab2 = lab.copy()
    lab2.reshape(-1)[0] = 12345
    err2 = bench.result_error(radar, rays, bad, lab2, idx, ref)
    assert err2["max_rel"] > 5e-4 and not err2["labels_exact"]


def test_snapshot_leg_samples_the_full_snapshot_oracle():
    radar = scenegen.radar_automotive(n_chirps=8, n_samples=32)
    rays, hits, geom = scenegen.moving_scene(42, radar, 120, bounce_frac=0.3)
    rate, n_pts, dt, cores, idx, ref = bench.cpu_snapshot_rate(radar, rays, hits, geom, seconds=0.05, seed=6)
    full = oracle.signal_geom(radar, rays, hits, geom)
    assert rate > 0 and n_pts == idx.shape[0]
    assert np.allclose(ref, full.reshape(-1)[idx], rtol=0, atol=1e-12 * np.abs(full).max())


def test_decompose_leg_samples_each_span_at_its_rays_bins():
    radar = scenegen.radar_automotive(n_chirps=16, n_samples=32)
    _, rays = scenegen.automotive_scene(seed=43, n_rays=400, radar=radar)
    ids = np.unique(rays.object_id)
    rate, per, dt, cores, cells, refs = bench.cpu_decompose_rate(radar, rays, ids, seconds=0.05, seed=7)
    assert rate > 0 and len(cells) == len(refs) == len(ids)
    for o, c, ref in zip(ids, cells, refs):
        sub = rays.take(np.nonzero(rays.object_id == o)[0])
        assert set(c.tolist()) <= set(oracle.bins(radar, sub)["cell"].tolist())
        spec = oracle.spectrum(radar, oracle.signal(radar, sub))
        assert np.allclose(ref, spec.reshape(-1)[c], rtol=0, atol=1e-9 * np.abs(spec).max())


def test_traffic_comes_only_from_a_capture_of_the_current_sources(tmp_path, monkeypatch):
    """roofline.traffic is read from the capture table row whose source hash matches the
    kernel's current sources; a row captured from other sources gives no figure."""
    import bench
    cur = bench.kernel_source_hash("umma_sum_kernel")
    table = tmp_path / "traffic.md"
    table.write_text("| kernel | precision | rays | bytes | sources | note |\n|---|---|---|---|---|---|\n"
                     f"| umma_sum_kernel | fp16_split | 200000 | 12345 | {cur} | current |\n"
                     "| umma_sum_kernel | bf16 | 200000 | 999 | 0000000000000000 | stale |\n")
    monkeypatch.setattr(bench, "TRAFFIC_TABLE", str(table))
    assert bench.captured_traffic("umma_sum_kernel", "fp16_split", 200000)[0] == 12345
    assert bench.captured_traffic("umma_sum_kernel", "fp16_split", 100000)[0] is None
    nbytes, note = bench.captured_traffic("umma_sum_kernel", "bf16", 200000)
    assert nbytes is None and "changed" in note
