"""The autotuner's table: JSON save / load round trip and validation, without a GPU."""
import json

from paper_2305_14176_gb300 import radarsim as rs


def test_tuning_table_round_trip(tmp_path):
    rs.sim_tuning_clear()
    src = tmp_path / "in.json"
    rows = [dict(n_virtual=12, n_chirps=256, n_samples=512, n_angle=16, precision=4, ray_bucket=18, splits=19,
                 fft_range_points=2048, fft_doppler_strip=16, fft_angle_strip=32),
            dict(n_virtual=4, n_chirps=64, n_samples=128, n_angle=16, precision=2, ray_bucket=11, splits=7,
                 fft_range_points=0, fft_doppler_strip=8, fft_angle_strip=0),
            dict(n_virtual=4, n_chirps=64, n_samples=128, n_angle=16, precision=2, ray_bucket=12, splits=-3,
                 fft_range_points=0, fft_doppler_strip=8, fft_angle_strip=0),   # invalid: skipped
            dict(n_virtual=4, n_chirps=64, n_samples=128, n_angle=16, precision=2, ray_bucket=13, splits=3,
                 fft_range_points=0, fft_doppler_strip=3, fft_angle_strip=0),   # odd strip: skipped
            dict(n_virtual=4, n_chirps=64, n_samples=128, n_angle=16, precision=2, ray_bucket=14, splits=3,
                 fft_range_points=1000, fft_doppler_strip=8, fft_angle_strip=0)]  # not a power of two: skipped
    with open(src, "w") as f:
        f.write("[\n" + ",\n".join("  " + json.dumps(r) for r in rows) + "\n]\n")
    assert rs.sim_tuning_load(str(src)) == rs.SIM_OK
    assert rs.sim_tuning_count() == 2
    out = tmp_path / "out.json"
    assert rs.sim_tuning_save(str(out)) == rs.SIM_OK
    back = json.load(open(out))
    assert sorted(map(lambda d: tuple(sorted(d.items())), back)) == \
        sorted(map(lambda d: tuple(sorted(d.items())), rows[:2]))
    assert rs.sim_tuning_load(str(tmp_path / "missing.json")) == rs.SIM_E_INVALID
    rs.sim_tuning_clear()
    assert rs.sim_tuning_count() == 0
