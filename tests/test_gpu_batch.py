"""Batched pipeline: uneven scenes in one persistent tensor-core launch, graph-captured.
Each scene must give exactly the bits it gives alone through sim_submit/sim_fetch, on
the eager first run and on graph replays, and match the oracle within tolerance."""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from paper_2305_14176_gb300 import radarsim as rs
from gpu_helpers import TOL, prec_params, rel_max, run, to_c

pytestmark = pytest.mark.gpu


def _outputs(ctx):
    sig = torch.full(ctx.signal_shape + (2,), float("nan"), dtype=torch.float32, device="cuda")
    spec = torch.full(ctx.cube_shape + (2,), float("nan"), dtype=torch.float32, device="cuda")
    lab = torch.full(ctx.cube_shape, -7, dtype=torch.int32, device="cuda")
    return spec, sig, lab


@pytest.mark.parametrize("precision", prec_params(rs.SIM_PREC_FP16_SPLIT, rs.SIM_PREC_BF16_SPLIT, rs.SIM_PREC_BF16))
def test_batch_equals_alone_bitwise_and_replays(precision):
    scenes = scenegen.batch_scenes(seed=3000, n_scenes=10, ray_scale=0.05)
    scenes.append(scenegen.tiny_scene(seed=3))
    ctxs = [rs.Context(radar, precision=precision) for radar, _ in scenes]
    try:
        alone = [run(radar, rays, precision) for radar, rays in scenes]
        rays_s, metas, outs, keep = [], [], [], []
        for (radar, rays), ctx in zip(scenes, ctxs):
            arr = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.arrays().items()}
            r, m = rs.make_rays(arr, rays.n)
            rays_s.append(r)
            metas.append(m)
            keep.append(arr)
        for rep in range(3):  # eager + capture, then two graph replays
            outs = [_outputs(c) for c in ctxs]
            rc, ms, kernels = rs.sim_run_batch([c.ctx for c in ctxs], rays_s, metas,
                                               [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])
            assert rc == rs.SIM_OK, rs.sim_status_string(rc)
            assert ms > 0 and kernels > len(scenes)
            torch.cuda.synchronize()
            for i, (spec, sig, lab) in enumerate(outs):
                rc0, s0, x0, l0 = alone[i]
                assert rc0 == rs.SIM_OK
                assert np.array_equal(to_c(sig), s0), (rep, i)
                assert np.array_equal(to_c(spec), x0), (rep, i)
                assert np.array_equal(lab.cpu().numpy(), l0), (rep, i)
        # and the small scene against the oracle
        radar, rays = scenes[-1]
        ref = oracle.signal(radar, rays)
        assert rel_max(to_c(outs[-1][1]), ref) <= TOL[precision]
    finally:
        for c in ctxs:
            c.close()


def test_batch_rejects_mixed_precision_and_direct():
    radar, rays = scenegen.tiny_scene(seed=1, n_rays=100)
    a = rs.Context(radar, precision=rs.SIM_PREC_FP16_SPLIT)
    b = rs.Context(radar, precision=rs.SIM_PREC_BF16_SPLIT)
    d = rs.Context(radar, precision=rs.SIM_PREC_FP32_DIRECT)
    try:
        r, m = rs.make_rays(rays.arrays(), rays.n)
        assert rs.sim_run_batch([a.ctx, b.ctx], [r, r], [m, m])[0] == rs.SIM_E_INVALID
        assert rs.sim_run_batch([d.ctx], [r], [m])[0] == rs.SIM_E_INVALID
    finally:
        for c in (a, b, d):
            c.close()
