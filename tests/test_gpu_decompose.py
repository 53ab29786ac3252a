"""Decomposition by ray meta data (Sec. II-C, Eq. 5): per-span spectra against the oracle on
the span's rays, parts of a partition adding up to the whole scene, and span labels against the
labels of the oracle's own span spectra, exact on every cell whose decision is not within the
spectra's stated error of the threshold or of a tie."""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from paper_2305_14176_gb300 import radarsim as rs
from gpu_helpers import TOL, prec_params, rel_max, to_c
from span_bands import decisive_cells

pytestmark = pytest.mark.gpu


def _scene(seed, n, automotive=False):
    if automotive:
        radar, rays = scenegen.automotive_scene(seed=seed, n_rays=n)
    else:
        radar, rays = scenegen.tiny_scene(seed=seed, n_rays=n)
        rays.object_id = scenegen.randint(seed, 50, n, 0, 3)
    mat = scenegen.randint(seed, 51, n, 0, 2)
    hits = scenegen.randint(seed, 52, n, 1, 3)
    return radar, rays, mat, hits


RULES = [dict(object_id=1, material_id=-1, min_hits=0, max_hits=-1, exclude=0),      # "the pedestrian"
         dict(object_id=-1, material_id=-1, min_hits=2, max_hits=-1, exclude=0),     # multi-path ghosts
         dict(object_id=2, material_id=-1, min_hits=1, max_hits=1, exclude=0),       # line of sight of 2
         dict(object_id=-1, material_id=0, min_hits=0, max_hits=-1, exclude=1)]      # not material 0

# the automotive frame: spans of a few of its 20 objects and of its multi-path rays
RULES_AUTO = [dict(object_id=3, material_id=-1, min_hits=0, max_hits=-1, exclude=0),
              dict(object_id=7, material_id=-1, min_hits=0, max_hits=-1, exclude=0),
              dict(object_id=-1, material_id=-1, min_hits=3, max_hits=-1, exclude=0),
              dict(object_id=11, material_id=-1, min_hits=1, max_hits=1, exclude=0),
              dict(object_id=0, material_id=1, min_hits=0, max_hits=-1, exclude=0)]


def _decompose(radar, rays, mat, hits, rules, precision, threshold):
    ctx = rs.Context(radar, precision=precision)
    try:
        arr = dict(rays.arrays(), material_id=mat, n_hits=hits)
        arr = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in arr.items()}
        r, m = rs.make_rays(arr, rays.n)
        spans = [torch.full(ctx.cube_shape + (2,), float("nan"), dtype=torch.float32, device="cuda")
                 for _ in rules]
        labels = torch.full(ctx.cube_shape, -7, dtype=torch.int32, device="cuda")
        rc = rs.sim_decompose(ctx.ctx, r, m, [rs.span_rule(**q) for q in rules], spans, labels, threshold)
        assert rc == rs.SIM_OK, rs.sim_status_string(rc)
        torch.cuda.synchronize()
        return spans, labels.cpu().numpy()
    finally:
        ctx.close()


def _check_spans_and_labels(radar, rays, mat, hits, rules, precision, threshold, max_band_frac):
    spans, lab = _decompose(radar, rays, mat, hits, rules, precision, threshold)
    got = np.stack([to_c(x) for x in spans])
    refs = []
    for q, x in zip(rules, got):
        mask = oracle.span_mask(q, rays.object_id, mat, hits)
        assert mask.any()
        ref = oracle.spectrum(radar, oracle.signal(radar, rays.take(mask)))
        refs.append(ref)
        assert rel_max(x, ref, norm=max(np.abs(ref).max(), 1e-30)) <= TOL[precision]
    refs = np.stack(refs)
    # the labels of the oracle's own spectra (FP64 powers), compared exactly on every cell
    # whose decision the stated error of the spectra (TOL of each span's peak) cannot move
    want = oracle.span_labels(refs, threshold)
    err = TOL[precision] * np.abs(refs).reshape(len(rules), -1).max(axis=1)
    safe = decisive_cells(refs, threshold, err)
    assert 1.0 - safe.mean() <= max_band_frac, 1.0 - safe.mean()
    assert np.array_equal(lab[safe], want[safe])
    # and the cells left out still carry a valid decision: -1 or a span at or near the top
    assert np.isin(lab[~safe], np.arange(-1, len(rules))).all()
    assert (want >= 0).any() and (want < 0).any()
    # the segmentation kernel itself: the rule applied in FP32 to this call's own spectra gives
    # its labels bit for bit (same precision, same operations)
    spans32 = np.stack([x.cpu().numpy()[..., 0] + 1j * x.cpu().numpy()[..., 1] for x in spans]).astype(np.complex64)
    assert np.array_equal(lab, oracle.span_labels(spans32, threshold))


@pytest.mark.parametrize("precision", [rs.SIM_PREC_FP32_DIRECT, rs.SIM_PREC_FP16_SPLIT])
def test_span_spectra_and_labels(precision):
    radar, rays, mat, hits = _scene(21, 1500)
    _check_spans_and_labels(radar, rays, mat, hits, RULES, precision, 0.05, max_band_frac=0.01)


@pytest.mark.parametrize("precision", [rs.SIM_PREC_FP32_DIRECT, rs.SIM_PREC_FP16_SPLIT])
def test_span_labels_automotive_frame(precision):
    """An automotive frame of 20,000 rays (12 channels x 256 chirps x 512 samples): five spans
    (three objects, a line-of-sight rule, a material rule on the clutter) and the multi-path
    rays; labels against the oracle's spectra of each span."""
    radar, rays, mat, hits = _scene(1500, 20_000, automotive=True)
    _check_spans_and_labels(radar, rays, mat, hits, RULES_AUTO, precision, 0.05, max_band_frac=0.01)


def test_partition_parts_add_up_to_the_scene():
    """Eq. 5: spans that partition the rays (object 1 and its complement) sum to the full spectrum."""
    radar, rays, mat, hits = _scene(22, 1200)
    ctx = rs.Context(radar, precision=rs.SIM_PREC_FP32_DIRECT)
    try:
        arr = {k: np.ascontiguousarray(v) for k, v in dict(rays.arrays(), material_id=mat, n_hits=hits).items()}
        r, m = rs.make_rays(arr, rays.n)
        rules = [rs.span_rule(object_id=1), rs.span_rule(object_id=1, exclude=True)]
        spans = [np.zeros(ctx.cube_shape + (2,), np.float32) for _ in rules]
        assert rs.sim_decompose(ctx.ctx, r, m, rules, spans, None, 0.0) == rs.SIM_OK
        whole = np.zeros(ctx.cube_shape + (2,), np.float32)
        t = ctx.submit(arr, rays.n)
        assert ctx.fetch(t, whole) == rs.SIM_OK
        parts = sum(x[..., 0].astype(np.float64) + 1j * x[..., 1] for x in spans)
        full = whole[..., 0].astype(np.float64) + 1j * whole[..., 1]
        assert rel_max(parts, full) <= 1e-5
    finally:
        ctx.close()


@pytest.mark.parametrize("precision", prec_params(rs.SIM_PREC_FP32_DIRECT, rs.SIM_PREC_FP16_SPLIT, rs.SIM_PREC_BF16))
@pytest.mark.parametrize("model", [rs.SIM_MODEL_SEPARABLE, rs.SIM_MODEL_EXACT])
@pytest.mark.parametrize("n_rays", [1400, 40_000])
def test_span_part_is_the_scene_of_its_rays(precision, model, n_rays):
    """A span's rays are packed in ray order and summed alone, so its spectrum is the spectrum
    of a scene holding only those rays; an empty span gives zeros.  The FP32 direct sum and the
    exact model plan a span as they plan a scene, so there it is bit for bit; the separable
    tensor-core sum plans a span for a share of the GPU (fewer split-K parts), so it differs
    from the scene alone by the rounding of that grouping of FP32 sums only.  Either way two calls give
    the same bits.  The exact model's packed spans carry the range-migration words too."""
    radar, rays, mat, hits = _scene(24, n_rays)
    radar = radar.replace(model=model)
    ctx = rs.Context(radar, precision=precision, model=model)
    same_plan = precision == rs.SIM_PREC_FP32_DIRECT or model == rs.SIM_MODEL_EXACT
    try:
        arr = {k: np.ascontiguousarray(v) for k, v in dict(rays.arrays(), material_id=mat, n_hits=hits).items()}
        r, m = rs.make_rays(arr, rays.n)
        rules = [dict(object_id=2, material_id=-1, min_hits=0, max_hits=-1, exclude=0),
                 dict(object_id=-1, material_id=1, min_hits=2, max_hits=-1, exclude=0),
                 dict(object_id=9, material_id=-1, min_hits=0, max_hits=-1, exclude=0)]   # no such object
        spans = [np.full(ctx.cube_shape + (2,), np.nan, np.float32) for _ in rules]
        assert rs.sim_decompose(ctx.ctx, r, m, [rs.span_rule(**q) for q in rules], spans, None, 0.0) == rs.SIM_OK
        again = [np.full(ctx.cube_shape + (2,), np.nan, np.float32) for _ in rules]
        assert rs.sim_decompose(ctx.ctx, r, m, [rs.span_rule(**q) for q in rules], again, None, 0.0) == rs.SIM_OK
        for x, y in zip(spans, again):
            assert np.array_equal(x, y)
        for q, x in zip(rules[:2], spans[:2]):
            mask = oracle.span_mask(q, rays.object_id, mat, hits)
            sub = {k: np.ascontiguousarray(v[mask]) for k, v in arr.items()}
            alone = np.zeros(ctx.cube_shape + (2,), np.float32)
            t = ctx.submit(sub, int(mask.sum()))
            assert ctx.fetch(t, alone) == rs.SIM_OK
            if same_plan:
                assert np.array_equal(x, alone)
            else:
                # the tensor core's FP32 accumulation (not round-to-nearest) regrouped: a few 1e-6
                # at split precision, whose chains end every 16 stages in an FP32 running sum; a
                # single-pass chain holds all of a split's rays, so fewer splits there move the
                # result by a few 1e-5 (its operands alone err by ~3e-4 and ~2.5e-3)
                split = precision in (rs.SIM_PREC_FP16_SPLIT, rs.SIM_PREC_BF16_SPLIT)
                assert rel_max(to_c(torch.from_numpy(x)), to_c(torch.from_numpy(alone))) <= (1e-5 if split else 1e-4)
        assert not spans[2].any()
    finally:
        ctx.close()


@pytest.mark.parametrize("precision", [rs.SIM_PREC_FP32_DIRECT, rs.SIM_PREC_FP16_SPLIT])
def test_host_and_device_spectra_give_the_same_bits(precision):
    """Spectra copied to host memory and to device memory, empty spans included, carry the same
    bits, and so do the labels."""
    radar, rays, mat, hits = _scene(26, 6000)
    ctx = rs.Context(radar, precision=precision)
    try:
        arr = {k: np.ascontiguousarray(v) for k, v in dict(rays.arrays(), material_id=mat, n_hits=hits).items()}
        r, m = rs.make_rays(arr, rays.n)
        rules = [rs.span_rule(**q) for q in RULES] + [rs.span_rule(object_id=9)]  # the last one is empty
        host = [np.full(ctx.cube_shape + (2,), np.nan, np.float32) for _ in rules]
        lab_h = np.full(ctx.cube_shape, -7, np.int32)
        assert rs.sim_decompose(ctx.ctx, r, m, rules, host, lab_h, 0.1) == rs.SIM_OK
        dev = [torch.full(ctx.cube_shape + (2,), float("nan"), dtype=torch.float32, device="cuda") for _ in rules]
        lab_d = torch.full(ctx.cube_shape, -7, dtype=torch.int32, device="cuda")
        assert rs.sim_decompose(ctx.ctx, r, m, rules, dev, lab_d, 0.1) == rs.SIM_OK
        torch.cuda.synchronize()
        for x, y in zip(host, dev):
            assert np.array_equal(x, y.cpu().numpy())
        assert not host[-1].any()
        assert np.array_equal(lab_h, lab_d.cpu().numpy())
    finally:
        ctx.close()


def test_rules_needing_missing_meta_are_rejected():
    radar, rays, mat, hits = _scene(23, 100)
    ctx = rs.Context(radar, precision=rs.SIM_PREC_FP32_DIRECT)
    try:
        r, m = rs.make_rays(rays.arrays(), rays.n)  # no material or hit arrays
        assert rs.sim_decompose(ctx.ctx, r, m, [rs.span_rule(min_hits=2)]) == rs.SIM_E_INVALID
        assert rs.sim_decompose(ctx.ctx, r, m, [rs.span_rule(material_id=1)]) == rs.SIM_E_INVALID
        assert rs.sim_decompose(ctx.ctx, r, m, [rs.span_rule(min_hits=3, max_hits=2)]) == rs.SIM_E_INVALID
        assert rs.sim_decompose(ctx.ctx, r, m, [rs.span_rule(object_id=1)], threshold=2.0) == rs.SIM_E_INVALID
    finally:
        ctx.close()


def test_concurrent_calls_on_one_context():
    """Four threads decompose on one context at once: one call holds the context's scratch,
    the others allocate their own for their duration; every call gives the bits of a call made
    alone, and a later call reuses the scratch."""
    import threading
    radar, rays, mat, hits = _scene(25, 3000)
    ctx = rs.Context(radar, precision=rs.SIM_PREC_FP16_SPLIT)
    try:
        arr = {k: np.ascontiguousarray(v) for k, v in dict(rays.arrays(), material_id=mat, n_hits=hits).items()}
        r, m = rs.make_rays(arr, rays.n)
        rules = [rs.span_rule(**q) for q in RULES]

        def call():
            out = [np.zeros(ctx.cube_shape + (2,), np.float32) for _ in rules]
            lab = np.zeros(ctx.cube_shape, np.int32)
            return rs.sim_decompose(ctx.ctx, r, m, rules, out, lab, 0.1), out, lab

        rc0, ref, lab0 = call()
        assert rc0 == rs.SIM_OK
        results = [None] * 4

        def worker(k):
            results[k] = call()

        threads = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for rc, out, lab in results + [call()]:
            assert rc == rs.SIM_OK
            assert all(np.array_equal(a, b) for a, b in zip(out, ref))
            assert np.array_equal(lab, lab0)
    finally:
        ctx.close()
