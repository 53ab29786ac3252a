"""Shared helpers of the GPU tests: run a scene through the C ABI and compare."""
import numpy as np
import torch

from paper_2305_14176_gb300 import radarsim as rs

# Each ray-sum arithmetic's stated target, normwise (max |err| / max |ref|, and RMS): 1e-5 for
# the FP32 direct sum and for split precision (hi + lo operands), 2e-3 for single-pass BF16/FP16.
TARGET = {rs.SIM_PREC_FP32_DIRECT: 1e-5, rs.SIM_PREC_BF16_SPLIT: 1e-5, rs.SIM_PREC_FP16_SPLIT: 1e-5,
          rs.SIM_PREC_BF16: 2e-3, rs.SIM_PREC_FP16: 2e-3}

# The bounds the tests assert.  FP32 and split precision assert their target.  Single-pass FP16
# asserts a bound tighter than its target, from its rounding: each real operand component keeps
# 11 significand bits, a relative error of at most 2^-12; two operands per term and errors adding
# in quadrature over incoherent rays give an RMS near 2^-12 and a maximum of about twice that,
# so 3 x 2^-12 (max) and 1.5 x 2^-12 (RMS), both below 2e-3.
# Single-pass BF16 MISSES its 2e-3 target on frames of many rays: with 8 significand bits per
# component the same argument gives ~2^-9 = 1.95e-3 per term, and the automotive frame measures
# 2.5e-3 max and 2.3e-3 RMS.  Its tests assert only that rounding bound (3 x 2^-9 max,
# 1.5 x 2^-9 RMS) and carry "misses-2e-3-target" in their names (see `prec_params`).
TOL = {rs.SIM_PREC_FP32_DIRECT: 1e-5, rs.SIM_PREC_BF16_SPLIT: 1e-5, rs.SIM_PREC_FP16_SPLIT: 1e-5,
       rs.SIM_PREC_BF16: 3 * 2.0 ** -9, rs.SIM_PREC_FP16: 3 * 2.0 ** -12}
TOL_RMS = {rs.SIM_PREC_FP32_DIRECT: 1e-5, rs.SIM_PREC_BF16_SPLIT: 1e-5, rs.SIM_PREC_FP16_SPLIT: 1e-5,
           rs.SIM_PREC_BF16: 1.5 * 2.0 ** -9, rs.SIM_PREC_FP16: 1.5 * 2.0 ** -12}
MEETS_TARGET = {p: TOL[p] <= TARGET[p] and TOL_RMS[p] <= TARGET[p] for p in TARGET}

PREC_ID = {rs.SIM_PREC_FP32_DIRECT: "fp32", rs.SIM_PREC_BF16_SPLIT: "bf16_split",
           rs.SIM_PREC_FP16_SPLIT: "fp16_split", rs.SIM_PREC_FP16: "fp16",
           rs.SIM_PREC_BF16: "bf16-single-pass-misses-2e-3-target"}


def prec_params(*precisions):
    """pytest parameters for precisions, named so that a variant that misses its stated target
    says so in every test id it appears in."""
    import pytest
    return [pytest.param(p, id=PREC_ID[p]) for p in precisions]


def to_c(x: torch.Tensor) -> np.ndarray:
    a = x.cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


def run(radar, rays, precision=rs.SIM_PREC_FP32_DIRECT, device_inputs=True,
        outputs=rs.SIM_OUT_SIGNAL | rs.SIM_OUT_SPECTRUM | rs.SIM_OUT_LABELS, ctx=None):
    """Returns (status, signal complex128, spectrum complex128, labels int32) via the C ABI."""
    own = ctx is None
    if own:
        ctx = rs.Context(radar, precision=precision, outputs=outputs)
    try:
        arr = rays.arrays()
        if device_inputs:
            arr = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in arr.items()}
        else:
            arr = {k: np.ascontiguousarray(v) for k, v in arr.items()}
        sig = torch.zeros(ctx.signal_shape + (2,), dtype=torch.float32, device="cuda") \
            if outputs & rs.SIM_OUT_SIGNAL else None
        spec = torch.zeros(ctx.cube_shape + (2,), dtype=torch.float32, device="cuda") \
            if outputs & rs.SIM_OUT_SPECTRUM else None
        lab = torch.zeros(ctx.cube_shape, dtype=torch.int32, device="cuda") \
            if outputs & rs.SIM_OUT_LABELS else None
        t = ctx.submit(arr, rays.n)
        rc = ctx.fetch(t, spec, sig, lab)
        torch.cuda.synchronize()
        return (rc, None if sig is None else to_c(sig), None if spec is None else to_c(spec),
                None if lab is None else lab.cpu().numpy())
    finally:
        if own:
            ctx.close()


def rel_max(got, ref, norm=None):
    norm = np.abs(ref).max() if norm is None else norm
    return float(np.abs(got - ref).max() / norm) if norm > 0 else float(np.abs(got - ref).max())


def rel_rms(got, ref):
    n = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / n) if n > 0 else float(np.linalg.norm(got - ref))
