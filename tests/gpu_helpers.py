"""Shared helpers of the GPU tests: run a scene through the C ABI and compare."""
import numpy as np
import torch

from paper_2305_14176_gb300 import radarsim as rs

# normwise tolerance on signal and spectrum per ray-sum arithmetic
TOL = {rs.SIM_PREC_FP32_DIRECT: 1e-5, rs.SIM_PREC_BF16_SPLIT: 1e-5, rs.SIM_PREC_FP16_SPLIT: 1e-5,
       rs.SIM_PREC_BF16: 2e-3, rs.SIM_PREC_FP16: 2e-3}


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
