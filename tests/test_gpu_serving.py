"""Serving: scenes in flight together give the results they give alone; admission by
memory budget queues, admits as memory frees, and refuses what cannot fit."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

import scenegen
from paper_2305_14176_gb300 import radarsim as rs
from gpu_helpers import run, to_c

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _mixed_scenes():
    out = []
    for i, (nc, ns, ntx) in enumerate([(256, 512, 3), (128, 256, 1), (64, 128, 1), (512, 256, 3),
                                       (256, 256, 3), (128, 512, 1)]):
        radar = scenegen.radar_automotive(n_chirps=nc, n_samples=ns, n_tx=ntx)
        rays = scenegen.cluster_rays(500 + i, [40_000, 3_000, 500, 25_000, 9_000, 17_000][i],
                                     min_per_obj=100, max_per_obj=2000)
        out.append((radar, rays))
    out.append(scenegen.tiny_scene(seed=77))
    return out


@pytest.mark.parametrize("precision", [rs.SIM_PREC_FP16_SPLIT, rs.SIM_PREC_FP32_DIRECT])
def test_mix_equals_alone_bitwise(precision):
    scenes = _mixed_scenes()
    alone = [run(radar, rays, precision) for radar, rays in scenes]
    ctxs = [rs.Context(radar, precision=precision) for radar, _ in scenes]
    try:
        tickets = []
        for (radar, rays), ctx in zip(scenes, ctxs):
            arr = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.arrays().items()}
            tickets.append(ctx.submit(arr, rays.n))  # all in flight before any fetch
        order = np.argsort(scenegen.uniform(5, 1, len(scenes)))  # fetch in a shuffled order
        for i in order:
            ctx = ctxs[i]
            sig = torch.zeros(ctx.signal_shape + (2,), dtype=torch.float32, device="cuda")
            spec = torch.zeros(ctx.cube_shape + (2,), dtype=torch.float32, device="cuda")
            lab = torch.zeros(ctx.cube_shape, dtype=torch.int32, device="cuda")
            assert ctx.fetch(tickets[i], spec, sig, lab) == rs.SIM_OK
            rc, s0, x0, l0 = alone[i]
            assert rc == rs.SIM_OK
            assert np.array_equal(to_c(sig), s0), i
            assert np.array_equal(to_c(spec), x0), i
            assert np.array_equal(lab.cpu().numpy(), l0), i
    finally:
        for c in ctxs:
            c.close()


_ADMISSION = textwrap.dedent("""
    import sys, numpy as np, torch
    sys.path.insert(0, {root!r})
    import scenegen
    from paper_2305_14176_gb300 import radarsim as rs
    torch.cuda.init()
    # budget for one and a half automotive scenes of 20k rays (their size from the engine's own
    # plan, measured in another process), at most 3 queued
    one = {one}
    assert rs.sim_engine_configure(int(1.5 * one), 4, 3) == rs.SIM_OK
    radar, rays = scenegen.automotive_scene(seed=9, n_rays=20_000)
    ctx = rs.Context(radar, precision=rs.SIM_PREC_FP16_SPLIT)
    assert rs.sim_engine_configure(0, 4, 3) == rs.SIM_E_INVALID  # too late: engine running
    tickets = [ctx.submit(rays.arrays(), rays.n) for _ in range(4)]   # 1 admitted, 3 queued
    try:
        ctx.submit(rays.arrays(), rays.n)
        raise SystemExit("queue overflow not refused")
    except rs.SimError as e:
        assert e.code == rs.SIM_E_BUSY, e.code
    big = scenegen.radar_imaging()
    bctx = rs.Context(big, precision=rs.SIM_PREC_FP16_SPLIT)
    try:
        bctx.submit(rays.arrays(), rays.n)   # 2.7 GB of cube alone exceeds the budget
        raise SystemExit("oversize scene not refused")
    except rs.SimError as e:
        assert e.code == rs.SIM_E_BUSY, e.code
    # the last ticket cannot be admitted before the earlier results are fetched: no wait
    assert ctx.fetch(tickets[-1], None, None, None, -1) == rs.SIM_E_BUSY
    first = None
    for t in tickets:                    # in order: each fetch admits the next queued scene
        sig = torch.zeros(ctx.signal_shape + (2,), dtype=torch.float32, device="cuda")
        assert ctx.fetch(t, None, sig, None) == rs.SIM_OK
        if first is None:
            first = sig.clone()
        else:
            assert torch.equal(first, sig)
    print("admission ok")
""")


_SCENE_BYTES = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import scenegen
    from paper_2305_14176_gb300 import radarsim as rs
    radar, rays = scenegen.automotive_scene(seed=9, n_rays=20_000)
    ctx = rs.Context(radar, precision=rs.SIM_PREC_FP16_SPLIT)
    print(rs.sim_scene_bytes(ctx.ctx, rays.n))
""")


def test_admission_by_memory_budget():
    r = subprocess.run([sys.executable, "-c", _SCENE_BYTES.format(root=ROOT)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    one = int(r.stdout.strip().splitlines()[-1])
    assert 50e6 < one < 400e6, one
    src = _ADMISSION.format(root=ROOT, one=one)
    r = subprocess.run([sys.executable, "-c", src], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "admission ok" in r.stdout, r.stdout + r.stderr


def test_fetch_timeout_keeps_ticket():
    radar, rays = scenegen.automotive_scene(seed=12, n_rays=200_000)
    ctx = rs.Context(radar, precision=rs.SIM_PREC_FP32_DIRECT)  # ~0.1 s on the device
    try:
        t = ctx.submit(rays.arrays(), rays.n)
        rc = ctx.fetch(t, timeout_ms=1)
        assert rc in (rs.SIM_E_TIMEOUT, rs.SIM_OK)
        if rc == rs.SIM_E_TIMEOUT:
            assert ctx.fetch(t, timeout_ms=-1) == rs.SIM_OK
    finally:
        ctx.close()
