"""The C ABI library without a GPU: it loads, exports every declared entry point,
and its host-side parameter checks reject bad input before touching CUDA."""
import ctypes
import subprocess

import pytest

import scenegen
from paper_2305_14176_gb300 import radarsim as rs


def test_library_exports_every_declared_function():
    declared = rs.header_functions()
    assert {"sim_create", "sim_submit", "sim_fetch", "sim_destroy", "sim_status_string"} <= set(declared)
    for name in declared:
        assert hasattr(rs.lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", rs.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(declared) <= exported
    # nothing but the C ABI leaks out
    assert all(s.startswith("sim_") for s in exported), sorted(s for s in exported if not s.startswith("sim_"))


def test_status_strings():
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert rs.sim_status_string(code) not in ("", "unknown status")
    assert rs.sim_status_string(42) == "unknown status"


def _params(**kw):
    p = rs.make_params(scenegen.radar_tiny(), max_rays=1000)
    for k, v in kw.items():
        if k == "window":
            for i in range(3):
                p.window[i] = v[i]
        else:
            setattr(p, k, v)
    return p


@pytest.mark.parametrize("bad", [
    dict(struct_size=8), dict(carrier_hz=0.0), dict(bandwidth_hz=float("nan")), dict(sweep_time_s=-1.0),
    dict(n_samples=100), dict(n_samples=8), dict(n_chirps=3), dict(n_chirps=8192), dict(n_tx=0),
    dict(n_tx=64, n_rx=32), dict(n_angle=2), dict(n_angle=24), dict(window=(0, 9, 0)),
    dict(precision=7), dict(outputs=0), dict(outputs=8), dict(max_rays=0), dict(max_rays=(1 << 21) + 1),
    dict(element_spacing_m=-0.001), dict(n_samples=4096, n_chirps=4096, n_angle=1024),
    dict(model=2), dict(model=1, precision=2, tdm_slot_s=1e-5, n_samples=16), dict(pattern_exp=17),
    dict(pattern_exp=-1),
    dict(tdm_slot_s=-1e-6), dict(tdm_slot_s=float("nan")), dict(tdm_slot_s=2.0),
])
def test_create_rejects_bad_params_without_a_gpu(bad):
    ctx = ctypes.c_void_p()
    rc = rs.lib.sim_create(ctypes.byref(_params(**bad)), ctypes.byref(ctx))
    assert rc == rs.SIM_E_INVALID
    assert ctx.value is None


def test_null_arguments():
    assert rs.lib.sim_create(None, None) == rs.SIM_E_INVALID
    assert rs.lib.sim_submit(None, None, None, None) == rs.SIM_E_INVALID
    assert rs.lib.sim_fetch(None, ctypes.c_uint64(1), None, None, None, 0) == rs.SIM_E_INVALID
    assert rs.lib.sim_destroy(None) == rs.SIM_E_INVALID
    assert rs.sim_engine_configure(-5, 4, 8) == rs.SIM_E_INVALID
    assert rs.sim_engine_configure(0, 0, 8) == rs.SIM_E_INVALID
    assert rs.lib.sim_selftest_wait(0, None, None) == rs.SIM_E_INVALID
    assert rs.lib.sim_selftest_wait(2000, None, None) == rs.SIM_E_INVALID
    mask = ctypes.c_uint32(7)
    assert rs.lib.sim_last_expansion_terms(None, ctypes.byref(mask)) == rs.SIM_E_INVALID
    assert mask.value == 7  # untouched
    count = ctypes.c_int32(-1)
    assert rs.lib.sim_last_kernel_count(None, ctypes.byref(count)) == rs.SIM_E_INVALID
    assert rs.lib.sim_scene_bytes(None, 10, None) == rs.SIM_E_INVALID


def test_expansion_route_names():
    """The bench's names for the route bits of sim_last_expansion_terms: P for Taylor terms,
    16 + P for Chebyshev terms, 0 for the per-chirp (or pair-sum) route."""
    import bench
    assert bench.expansion_names({4}) == ["taylor4"]
    assert bench.expansion_names({20, 22, 24}) == ["chebyshev4", "chebyshev6", "chebyshev8"]
    assert bench.expansion_names({0, 4}) == ["per-chirp", "taylor4"]
    assert bench.expansion_names(set()) == []
