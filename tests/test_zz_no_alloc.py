"""sim_raysum_noalloc: the ray sum for callers that cannot allocate device memory.

It must give the signal that sim_submit/sim_fetch give for the same scene, within
the tolerance of the precision, on two calls in a row (the static scratch array
keeps the first call's contents when the second starts), and the FP64 oracle's
signal within the same tolerance.  The exact model (Eq. 2 with range migration)
takes another route here on the tensor-core precisions (the per-chirp product),
so it is checked the same way.  This file is collected last so that a run
stopping at the first failure has run everything else first.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from paper_2305_14176_gb300 import radarsim as rs
from gpu_helpers import TOL, TOL_RMS, rel_max, rel_rms, run, to_c

pytestmark = pytest.mark.gpu


def _noalloc_signal(radar, rays, precision, stream, model=rs.SIM_MODEL_SEPARABLE):
    params = rs.make_params(radar, precision=precision, outputs=rs.SIM_OUT_SIGNAL, model=model)
    arr = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.arrays().items()}
    r, _ = rs.make_rays(arr, rays.n)
    nv = radar.n_tx * radar.n_rx
    sig = torch.full((nv, radar.n_chirps, radar.n_samples, 2), float("nan"), dtype=torch.float32, device="cuda")
    rc = rs.sim_raysum_noalloc(params, r, sig, stream)
    torch.cuda.synchronize()
    return rc, to_c(sig)


def _submit_fetch_signal(radar, rays, precision, model):
    ctx = rs.Context(radar, precision=precision, outputs=rs.SIM_OUT_SIGNAL, model=model)
    try:
        rc, ref, _, _ = run(radar, rays, precision, outputs=rs.SIM_OUT_SIGNAL, ctx=ctx)
    finally:
        ctx.close()
    return rc, ref


def _check_twice(radar, rays, precision, model=rs.SIM_MODEL_SEPARABLE, n_oracle=512, seed=0):
    stream = torch.cuda.current_stream().cuda_stream
    rc, ref = _submit_fetch_signal(radar, rays, precision, model)
    assert rc == rs.SIM_OK
    # an oracle check on sampled outputs: the comparison with sim_submit/sim_fetch alone would
    # only carry correctness over from the other path
    idx = scenegen.randint(seed, 9, n_oracle, 0, ref.size - 1).astype(np.int64)
    orc = oracle.signal_at(radar, rays, idx)
    for _ in range(2):
        rc, got = _noalloc_signal(radar, rays, precision, stream, model)
        assert rc == rs.SIM_OK, rs.sim_status_string(rc)
        assert rel_max(got, ref) <= TOL[precision]
        assert rel_rms(got, ref) <= TOL_RMS[precision]
        g = got.reshape(-1)[idx]
        assert rel_max(g, orc) <= TOL[precision] and rel_rms(g, orc) <= TOL_RMS[precision]


@pytest.mark.parametrize("precision", [rs.SIM_PREC_BF16_SPLIT, rs.SIM_PREC_FP16_SPLIT, rs.SIM_PREC_FP32_DIRECT])
def test_noalloc_matches_submit_fetch_twice(precision):
    scenes = [scenegen.automotive_scene(seed=1000, n_rays=200_000), scenegen.tiny_scene(seed=4)]
    if precision == rs.SIM_PREC_FP32_DIRECT:
        scenes = [scenegen.automotive_scene(seed=1000, n_rays=20_000), scenegen.tiny_scene(seed=4)]
    for k, (radar, rays) in enumerate(scenes):
        _check_twice(radar, rays, precision, seed=k)


@pytest.mark.parametrize("precision", [rs.SIM_PREC_BF16_SPLIT, rs.SIM_PREC_FP16_SPLIT])
def test_noalloc_exact_model_matches_submit_fetch_twice(precision):
    """The exact model without TDM slots on the tensor-core precisions: the no-alloc call runs
    the per-chirp product, sim_submit the per-tile expansion; both must agree with each other
    and with the oracle's exact Eq. 2."""
    for k, (radar, rays) in enumerate([scenegen.tiny_scene(seed=5, n_rays=1500),
                                       scenegen.automotive_scene(seed=1001, n_rays=20_000)]):
        radar = radar.replace(model=1)
        _check_twice(radar, rays, precision, model=rs.SIM_MODEL_EXACT, seed=10 + k)


def test_noalloc_rejects_oversize_and_host_pointers():
    stream = torch.cuda.current_stream().cuda_stream
    radar, rays = scenegen.tiny_scene(seed=1, n_rays=100)
    params = rs.make_params(radar, precision=rs.SIM_PREC_BF16_SPLIT, outputs=rs.SIM_OUT_SIGNAL)
    host = rays.arrays()
    r, _ = rs.make_rays(host, rays.n)
    sig = torch.empty((4, 64, 128, 2), dtype=torch.float32, device="cuda")
    assert rs.sim_raysum_noalloc(params, r, sig, stream) == rs.SIM_E_INVALID  # host rays
    arr = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in host.items()}
    r, _ = rs.make_rays(arr, (1 << 18) + 1)
    assert rs.sim_raysum_noalloc(params, r, sig, stream) == rs.SIM_E_INVALID  # too many rays
    img = scenegen.radar_imaging()
    r, _ = rs.make_rays(arr, rays.n)
    big = torch.empty(16, dtype=torch.float32, device="cuda")  # never written: rejected first
    assert rs.sim_raysum_noalloc(rs.make_params(img, precision=rs.SIM_PREC_BF16_SPLIT,
                                                outputs=rs.SIM_OUT_SIGNAL), r, big, stream) == rs.SIM_E_INVALID
    # the exact model with TDM slots has no allocation-free tensor-core form
    tdm = rs.make_params(radar.replace(tdm_slot_s=9.1e-6), precision=rs.SIM_PREC_BF16_SPLIT,
                         outputs=rs.SIM_OUT_SIGNAL, model=rs.SIM_MODEL_EXACT)
    assert rs.sim_raysum_noalloc(tdm, r, big, stream) == rs.SIM_E_INVALID
    # a host output buffer is refused too
    host_sig = np.zeros((4, 64, 128, 2), np.float32)
    assert rs.sim_raysum_noalloc(params, r, host_sig, stream) == rs.SIM_E_INVALID
