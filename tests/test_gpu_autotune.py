"""Autotuner on the device: it picks a valid launch shape (the built-in plan or a forced
split count), later runs use it, and the results still match the oracle and repeat bit for
bit."""
import numpy as np
import pytest

import oracle
import scenegen
from paper_2305_14176_gb300 import radarsim as rs
from gpu_helpers import TOL, rel_max, run

pytestmark = pytest.mark.gpu


def test_autotune_then_run():
    rs.sim_tuning_clear()
    radar, rays = scenegen.automotive_scene(seed=21, n_rays=20_000)
    ctx = rs.Context(radar, precision=rs.SIM_PREC_FP16_SPLIT)
    try:
        t = rs.sim_autotune(ctx.ctx, rays.n)
        # 0 keeps the built-in plan (stream-K at hi + lo), timed first; a forced split count
        # is stored only when it beat that plan
        assert t.splits >= 0 and t.ray_sum_ms > 0 and t.fft_ms > 0
        assert rs.sim_tuning_count() == 1
        rc1, s1, x1, l1 = run(radar, rays, rs.SIM_PREC_FP16_SPLIT, ctx=ctx)
        rc2, s2, x2, l2 = run(radar, rays, rs.SIM_PREC_FP16_SPLIT, ctx=ctx)
        assert rc1 == rc2 == rs.SIM_OK
        assert np.array_equal(s1, s2) and np.array_equal(x1, x2) and np.array_equal(l1, l2)
        idx = scenegen.randint(3, 1, 1024, 0, s1.size - 1).astype(np.int64)
        ref = oracle.signal_at(radar, rays, idx)
        assert rel_max(s1.reshape(-1)[idx], ref) <= TOL[rs.SIM_PREC_FP16_SPLIT]
        assert np.array_equal(l1, oracle.labels(radar, rays))
    finally:
        ctx.close()
        rs.sim_tuning_clear()
