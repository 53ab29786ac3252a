"""Precision study: the automotive frame scaled to 1,000,000 rays, every ray-sum variant
against the FP64 oracle at 512 sampled signal points (all rays each) and labels whole.
The table is also written to $RADARSIM_ARTIFACT_DIR/precision_study.json when that variable
names a folder, with each variant's stated target and whether it meets it.

Every variant but single-pass BF16 must meet its stated target (1e-5 for FP32 and split
precision, 2e-3 for single-pass FP16).  Single-pass BF16 misses its 2e-3 target at this size;
a test of its own, named for that, checks that it stays within its rounding bound."""
import json
import os

import numpy as np
import pytest

import oracle
import scenegen
from paper_2305_14176_gb300 import radarsim as rs
from gpu_helpers import MEETS_TARGET, TARGET, TOL, TOL_RMS, rel_max, rel_rms, run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def study():
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
        mx, rms = rel_max(got, ref), rel_rms(got, ref)
        table[name] = {"max_rel": mx, "rms_rel": rms, "labels_exact": bool(np.array_equal(lab, ref_lab)),
                       "target": TARGET[prec], "meets_target": bool(mx <= TARGET[prec] and rms <= TARGET[prec])}
    out = os.environ.get("RADARSIM_ARTIFACT_DIR", "")
    if out and os.path.isdir(out):
        with open(os.path.join(out, "precision_study.json"), "w") as f:
            json.dump({"rays": rays.n, "points": int(idx.size), "variants": table}, f, indent=1)
    return table


@pytest.mark.parametrize("name", [n for n, p in rs.PRECISION_NAMES.items() if MEETS_TARGET[p]])
def test_variant_meets_its_target_at_one_million_rays(study, name):
    prec = rs.PRECISION_NAMES[name]
    r = study[name]
    assert r["labels_exact"], name
    assert r["max_rel"] <= TOL[prec] <= TARGET[prec] and r["rms_rel"] <= TOL_RMS[prec] <= TARGET[prec], (name, r)
    assert r["meets_target"]


def test_bf16_single_pass_misses_2e3_target_within_its_rounding_bound(study):
    """BF16 single pass is not counted as meeting its 2e-3 target: it measures about 2.5e-3
    max and 2.3e-3 RMS here.  What is asserted is its rounding bound (3 x 2^-9 max,
    1.5 x 2^-9 RMS) and exact labels."""
    r = study["bf16"]
    assert r["labels_exact"]
    assert r["max_rel"] <= TOL[rs.SIM_PREC_BF16] and r["rms_rel"] <= TOL_RMS[rs.SIM_PREC_BF16], r
    assert not MEETS_TARGET[rs.SIM_PREC_BF16]
