"""Distributed (cluster) EVD for packets longer than 128 frames, with the CUDA-core
Gram and the long-packet projection, vs the FP64 oracle through the C ABI.

Same tolerances as the other GPU paths (eigenvalues in the 1e-6*lambda_1 band
<= 1e-4 relative, PD rel L2 <= 1e-3, cutoffs equal up to near-ties)."""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

from test_parity_evd_pair_gpu import check, pair_cfg  # noqa: E402
from test_parity_gpu import L, compare, rand_iq  # noqa: E402


@pytest.mark.parametrize("shape,grid,mode", [
    ((129, 33, 29), (2, 2), "LCF_T_MEDIAN"),      # shortest packet of the distributed EVD (4 CTAs)
    ((200, 40, 36), (2, 2), "LCF_T_CURVATURE"),   # the streaming workload's packet length
    ((201, 30, 26), (1, 2), "LCF_T_FIXED"),       # odd length: padded pair slot
    ((224, 24, 20), (1, 2), "LCF_T_SLOPE"),       # longest packet on 4 CTAs
    ((225, 24, 20), (2, 1), "LCF_T_CURVATURE"),   # shortest packet on 8 CTAs
    ((300, 36, 30), (2, 2), "LCF_T_CURVATURE"),   # the precision-stress workload's packet length
    ((320, 20, 20), (1, 1), "LCF_T_ADAPTIVE_SOFT"),  # longest packet of the library
])
def test_dist_shapes(shape, grid, mode):
    lib = L()
    nt, nz, nx = shape
    cfg, oc = pair_cfg(nz, nx, nt, grid[0], grid[1], thresh_mode=getattr(lib, mode), k_fixed=3, beta=1.0)
    check(compare(rand_iq(7, nt, nz, nx), cfg, oc, want_gram=False), soft=mode == "LCF_T_ADAPTIVE_SOFT")


def test_dist_zero_packet_is_degenerate():
    import torch
    lib = L()
    plan = lib.Plan.make(24, 20, 200, 2, 2, evd_path=lib.LCF_EVD_PAIR)
    pd = plan.filter(torch.zeros((200, 24, 20), dtype=torch.complex64, device="cuda"))
    st, flags = plan.status()
    assert st == lib.LCF_EDEGENERATE
    assert np.all(np.asarray(flags) & lib.LCF_WFLAG_DEGENERATE)
    assert float(pd.abs().max()) == 0.0


def test_long_packet_limits():
    lib = L()
    for kw, want in (({"nt": 321, "evd_path": lib.LCF_EVD_PAIR}, lib.LCF_EUNSUPPORTED),
                     ({"nt": 200, "evd_path": lib.LCF_EVD_PAIR, "project_path": lib.LCF_PATH_TC},
                      lib.LCF_EUNSUPPORTED),
                     ({"nt": 200, "evd_path": lib.LCF_EVD_PAIR, "thresh_mode": lib.LCF_T_LEARNED},
                      lib.LCF_EUNSUPPORTED),
                     ({"nt": 320, "evd_path": lib.LCF_EVD_PAIR}, lib.LCF_OK)):
        c = lib.lcf_config_default(24, 20, kw["nt"], 1, 1)
        for k, v in kw.items():
            setattr(c, k, v)
        try:
            lib.Plan(c).close()
            got = lib.LCF_OK
        except lib.LcfError as e:
            got = e.status
        assert got == want, (kw, got)
