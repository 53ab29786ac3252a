"""The tensor-core tile path (shared-memory operand layout, descriptors, tcgen05
pipeline, tensor-memory drain) on plain matrices, against an FP64 matmul of the
same 16-bit operands."""
import pytest
import torch

from paper_2305_14176_gb300 import radarsim as rs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("f16,m,n,k", [
    (0, 128, 256, 64),     # one pipeline stage, one tile
    (0, 128, 32, 64),      # narrowest tile
    (1, 128, 256, 64),     # FP16 operands
    (0, 300, 64, 2048),    # ragged rows, many stages
    (0, 256, 512, 4096),   # two column tiles
    (1, 130, 512, 1002),   # ragged K tail
    (2, 128, 256, 64),     # BF16 with the descriptor's negate-B bit: D = -A B^T
    (3, 200, 64, 512),     # FP16, negate-B
])
def test_tile_matches_fp64_matmul(f16, m, n, k):
    g = torch.Generator().manual_seed(m * 7 + n * 3 + k)
    dt = torch.float16 if f16 & 1 else torch.bfloat16
    A = torch.randn(m, k, generator=g).to(dt)
    B = torch.randn(n, k, generator=g).to(dt)
    ref = A.double() @ B.double().T
    if f16 & 2:
        ref = -ref
    D = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
    Ad, Bd = A.cuda(), B.cuda()
    rc = rs.sim_selftest_umma(f16, m, n, k, Ad, Bd, D, torch.cuda.current_stream().cuda_stream)
    assert rc == rs.SIM_OK, rs.sim_status_string(rc)
    err = (D.cpu().double() - ref).abs().max().item() / ref.abs().max().item()
    # FP32 accumulation in tensor memory rounds each K=16 step; observed ~1e-6 per 1e3 K
    assert err < 1e-5, err
