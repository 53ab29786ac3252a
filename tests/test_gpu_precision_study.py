"""Precision study: the automotive frame scaled to 1,000,000 rays, every ray-sum variant
against the FP64 oracle at 512 sampled signal points (all rays each) and labels whole.
The table is also written to $RADARSIM_ARTIFACT_DIR/precision_study.json when that variable
names a folder."""
import json
import os

import numpy as np
import pytest

import oracle
import scenegen
from paper_2305_14176_gb300 import radarsim as rs
from gpu_helpers import TOL, TOL_RMS, rel_max, rel_rms, run

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_precision_study_one_million_rays():
    radar, rays = scenegen.automotive_scene(seed=2000, n_rays=1_000_000)
    idx = scenegen.randint(2000, 7, 512, 0, radar.n_virtual * radar.n_chirps * radar.n_samples - 1)
    idx = idx.astype(np.int64)
    ref = oracle.signal_at(radar, rays, idx)
    ref_lab = oracle.labels(radar, rays)
    table = {}
    for name, prec in rs.PRECISION_NAMES.items():
        rc, sig, _, lab = run(radar, rays, prec, outputs=rs.SIM_OUT_SIGNAL | rs.SIM_OUT_LABELS)
        assert rc == rs.SIM_OK
        got = sig.reshape(-1)[idx]
        table[name] = {"max_rel": rel_max(got, ref), "rms_rel": rel_rms(got, ref),
                       "labels_exact": bool(np.array_equal(lab, ref_lab))}
    out = os.environ.get("RADARSIM_ARTIFACT_DIR", "")
    if out and os.path.isdir(out):
        with open(os.path.join(out, "precision_study.json"), "w") as f:
            json.dump({"rays": rays.n, "points": int(idx.size), "variants": table}, f, indent=1)
    for name, prec in rs.PRECISION_NAMES.items():
        r = table[name]
        assert r["labels_exact"], name
        assert r["max_rel"] <= TOL[prec] and r["rms_rel"] <= TOL_RMS[prec], (name, r)
