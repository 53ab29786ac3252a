"""The two-SM tensor-core tile (tcgen05.mma.cta_group::2 across a CTA pair, operands split
over both CTAs' shared memory, barriers across the pair) on plain matrices, against an FP64
matmul of the same 16-bit operands."""
import pytest
import torch

from paper_2305_14176_gb300 import radarsim as rs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("f16,n,k", [(0, 256, 64), (0, 32, 64), (1, 128, 64), (0, 256, 4096), (1, 64, 1002)])
def test_pair_tile_matches_fp64_matmul(f16, n, k):
    g = torch.Generator().manual_seed(n * 3 + k)
    dt = torch.float16 if f16 else torch.bfloat16
    A = torch.randn(256, k, generator=g).to(dt)
    B = torch.randn(n, k, generator=g).to(dt)
    ref = A.double() @ B.double().T
    D = torch.full((256, n), float("nan"), dtype=torch.float32, device="cuda")
    rc = rs.sim_selftest_umma_pair(f16, n, k, A.cuda(), B.cuda(), D, torch.cuda.current_stream().cuda_stream)
    assert rc == rs.SIM_OK, rs.sim_status_string(rc)
    err = (D.cpu().double() - ref).abs().max().item() / ref.abs().max().item()
    assert err < 1e-5, err


def test_bounded_wait_runs_out_and_reports():
    """A pipeline wait that nothing ends expires after its limit, the kernel reports it in its
    status word (SIM_E_DEVICE) and the context stays usable."""
    rc, waited = rs.sim_selftest_wait(50)
    assert rc == rs.SIM_E_DEVICE
    assert 45 <= waited <= 1000
    # the next call on the same context works
    A = torch.randn(256, 64).to(torch.bfloat16)
    B = torch.randn(32, 64).to(torch.bfloat16)
    D = torch.zeros((256, 32), dtype=torch.float32, device="cuda")
    assert rs.sim_selftest_umma_pair(0, 32, 64, A.cuda(), B.cuda(), D) == rs.SIM_OK
    ref = A.double() @ B.double().T
    assert (D.cpu().double() - ref).abs().max().item() <= 1e-5 * ref.abs().max().item()
