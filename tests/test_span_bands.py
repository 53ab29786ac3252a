"""CPU check of the decision band the span-label tests use: perturbing the oracle's span spectra
by any error within the band's bound leaves the segmentation (Sec. II-C) of every decisive cell
unchanged, and the band is a small fraction of the cells."""
import numpy as np

import oracle
import scenegen
from span_bands import decisive_cells

RULES = [dict(object_id=1, material_id=-1, min_hits=0, max_hits=-1, exclude=0),
         dict(object_id=-1, material_id=-1, min_hits=2, max_hits=-1, exclude=0),
         dict(object_id=2, material_id=-1, min_hits=1, max_hits=1, exclude=0)]


def test_perturbation_within_bound_keeps_decisive_labels():
    radar, rays = scenegen.tiny_scene(seed=21, n_rays=1200)
    rays.object_id = scenegen.randint(21, 50, rays.n, 0, 3)
    mat = scenegen.randint(21, 51, rays.n, 0, 2)
    hits = scenegen.randint(21, 52, rays.n, 1, 3)
    refs = np.stack([oracle.spectrum(radar, oracle.signal(radar, rays.take(oracle.span_mask(q, rays.object_id,
                                                                                             mat, hits))))
                     for q in RULES])
    thr = 0.05
    want = oracle.span_labels(refs, thr)
    for tol in (1e-5, 1e-3):
        err = tol * np.abs(refs).reshape(len(RULES), -1).max(axis=1)
        safe = decisive_cells(refs, thr, err)
        assert safe.mean() >= 0.99 if tol == 1e-5 else safe.mean() < 1.0
        rng = np.random.default_rng(7)
        for _ in range(3):
            mag = rng.uniform(0.0, 1.0, refs.shape) * err[:, None, None, None]
            ph = rng.uniform(0.0, 2 * np.pi, refs.shape)
            got = oracle.span_labels(refs + mag * np.exp(1j * ph), thr)
            assert np.array_equal(got[safe], want[safe])
        # errors past the bound do move some of the undecided cells
        if tol == 1e-3:
            mag = 30.0 * err[:, None, None, None]
            got = oracle.span_labels(refs + mag * np.exp(1j * rng.uniform(0.0, 2 * np.pi, refs.shape)), thr)
            assert not np.array_equal(got, want)
