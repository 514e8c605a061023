"""lcf_gram_noalloc: the windowed Gram for callers that cannot allocate.

Some callers of this library cannot call cudaMalloc (a real-time thread that
must not wait on the allocator, a host framework that owns all device
memory).  lcf_gram_noalloc gives them the Gram stage with its scratch in a
static per-device array.  This test calls it through the C ABI twice in a row
on the same packet and checks both results against the Gram the regular
plan computes (lcf_debug_gram), within the Gram tolerance the parity tests
use.  It runs alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

GRAM_TOL = 1e-6


def rel_fro(a, b):
    return max(float(np.linalg.norm(a[k] - b[k]) / np.linalg.norm(b[k])) for k in range(b.shape[0]))


@pytest.mark.parametrize("which", ["small", "realtime"])
def test_noalloc_gram_matches_plan_gram_twice(which):
    import torch

    import paper_2405_11105_b300 as L
    from synth import REALTIME_256x128x100, SMALL_96x64x32, generate_packet
    if which == "small":
        rec, grid, mode = SMALL_96x64x32, (3, 3), L.LCF_T_FIXED
    else:
        rec, grid, mode = REALTIME_256x128x100, (8, 8), L.LCF_T_CURVATURE
    iq = generate_packet(rec, seed=2)
    cfg = L.lcf_config_default(rec.nz, rec.nx, rec.nt, grid[0], grid[1])
    cfg.thresh_mode = mode
    cfg.k_fixed = 3
    torch.cuda.set_device(0)
    d = torch.from_numpy(iq).cuda()
    plan = L.Plan(cfg)
    plan.filter(d)
    torch.cuda.synchronize()
    R_ref = plan.debug_gram()
    nd = grid[0] * grid[1]
    st = torch.cuda.current_stream().cuda_stream
    results = []
    for _ in range(2):
        R = torch.empty((nd, rec.nt, rec.nt, 2), dtype=torch.float64, device="cuda")
        R.fill_(float("nan"))                     # every entry must be written
        s = L.lcf_gram_noalloc(cfg, d.data_ptr(), R.data_ptr(), st)
        assert s == L.LCF_OK, L.lcf_status_string(s)
        torch.cuda.synchronize()
        Rh = R.cpu().numpy()
        results.append(Rh[..., 0] + 1j * Rh[..., 1])
    for Rn in results:
        assert np.all(np.isfinite(Rn))
        assert rel_fro(Rn, R_ref) <= GRAM_TOL
    assert rel_fro(results[1], results[0]) <= GRAM_TOL


def test_noalloc_rejects_oversize_problem():
    import torch

    import paper_2405_11105_b300 as L
    assert L.lcf_gram_noalloc_scratch_bytes() == 64 << 20
    cfg = L.lcf_config_default(512, 256, 100, 16, 16)
    d = torch.empty(8, dtype=torch.complex64, device="cuda")      # never read: rejected first
    R = torch.empty(8, dtype=torch.complex128, device="cuda")
    s = L.lcf_gram_noalloc(cfg, d.data_ptr(), R.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert s == L.LCF_ESCRATCH, L.lcf_status_string(s)
