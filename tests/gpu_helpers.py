"""Shared helpers of the GPU tests: run a scene through the C ABI and compare."""
import numpy as np
import torch

from paper_2305_14176_gb300 import radarsim as rs

# Normwise tolerances (max |err| / max |ref|, and RMS) per ray-sum arithmetic.
# FP32 and split precision: 1e-5.  Single-pass operands carry their format's rounding:
# each real operand component is rounded to 8 (BF16) or 11 (FP16) significand bits,
# a relative error of at most 2^-9 (2^-12); two operands per term and errors adding in
# quadrature over incoherent rays give an RMS near 2^-9 (2^-12) and a maximum of about
# twice that, so the bounds below are 1.5x (RMS) and 3x (max) the unit roundoff.
TOL = {rs.SIM_PREC_FP32_DIRECT: 1e-5, rs.SIM_PREC_BF16_SPLIT: 1e-5, rs.SIM_PREC_FP16_SPLIT: 1e-5,
       rs.SIM_PREC_BF16: 3 * 2.0 ** -9, rs.SIM_PREC_FP16: 3 * 2.0 ** -12}
TOL_RMS = {rs.SIM_PREC_FP32_DIRECT: 1e-5, rs.SIM_PREC_BF16_SPLIT: 1e-5, rs.SIM_PREC_FP16_SPLIT: 1e-5,
           rs.SIM_PREC_BF16: 1.5 * 2.0 ** -9, rs.SIM_PREC_FP16: 1.5 * 2.0 ** -12}


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
