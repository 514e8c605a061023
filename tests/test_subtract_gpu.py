"""The subtractive reconstruction (Eq. 5, lcf_config.project_form = LCF_PF_SUBTRACT) against
the FP64 oracle's literal Eq. 4 (the oracle pins Eq. 4 == Eq. 5 for hard weights).

Standard tolerances (PD rel L2 1e-3, alpha 1e-3; cutoffs as the other rules).  On the
precision-stress packet the subtractive form's double-float sums give PD and alpha within
1e-3 from the FP32 eigen-decomposition alone (no polish)."""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

from synth import REALTIME_256x128x100, SMALL_96x64x32, generate_packet  # noqa: E402
from test_parity_gpu import ALPHA_TOL, PD_TOL, L, assert_cutoffs, compare, configs, rand_iq  # noqa: E402


def fast(cfg):
    lib = L()
    cfg.gram_path, cfg.project_path, cfg.evd_path = lib.LCF_PATH_TC, lib.LCF_PATH_TC, lib.LCF_EVD_PAIR
    return cfg


@pytest.mark.parametrize("path,mode", [("plain", "LCF_T_FIXED"), ("fast", "LCF_T_FIXED"), ("fast", "LCF_T_CURVATURE"),
                                       ("fast", "LCF_T_MEDIAN"), ("fast", "LCF_T_NCC"), ("fast", "LCF_T_NONE")])
def test_subtract_small(path, mode):
    lib = L()
    iq = generate_packet(SMALL_96x64x32, seed=2)
    cfg, oc = configs(96, 64, 32, 3, 3, thresh_mode=getattr(lib, mode), k_fixed=3, beta=1.43,
                      project_form=lib.LCF_PF_SUBTRACT)
    if path == "fast":
        fast(cfg)
    r = compare(iq, cfg, oc, want_gram=False)
    print(path, mode, {k: r[k] for k in ("pd_err", "alpha_err")})
    assert r["status"] == lib.LCF_OK
    assert_cutoffs(r)
    assert r["pd_err"] <= PD_TOL and r["alpha_err"] <= ALPHA_TOL


def test_subtract_realtime_matches_identity_form():
    import torch
    lib = L()
    iq = generate_packet(REALTIME_256x128x100, seed=0)
    cfg, oc = configs(256, 128, 100, 8, 8, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0, project_form=lib.LCF_PF_SUBTRACT)
    r = compare(iq, fast(cfg), oc, want_gram=False)
    print({k: r[k] for k in ("pd_err", "alpha_err")})
    assert_cutoffs(r)
    assert r["pd_err"] <= PD_TOL and r["alpha_err"] <= ALPHA_TOL
    cfg2, _ = configs(256, 128, 100, 8, 8, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0)
    p2 = lib.Plan(fast(cfg2))
    pd2 = p2.filter(torch.from_numpy(iq).cuda()).cpu().numpy().astype(np.float64)
    assert np.linalg.norm(pd2 - r["pd"]) / np.linalg.norm(r["pd"]) <= PD_TOL


@pytest.mark.parametrize("shape,grid", [((200, 40, 36), (2, 2)), ((33, 40, 70), (2, 3)), ((2, 8, 8), (1, 1))])
def test_subtract_edge_shapes(shape, grid):
    lib = L()
    nt, nz, nx = shape
    cfg, oc = configs(nz, nx, nt, grid[0], grid[1], thresh_mode=lib.LCF_T_FIXED, k_fixed=1,
                      project_form=lib.LCF_PF_SUBTRACT)
    fast(cfg)
    r = compare(rand_iq(15, nt, nz, nx), cfg, oc, want_gram=False)
    print(shape, {k: r[k] for k in ("pd_err", "alpha_err")})
    assert r["pd_err"] <= PD_TOL and r["alpha_err"] <= ALPHA_TOL


def test_subtract_zero_packet_and_validation():
    import torch
    lib = L()
    plan = lib.Plan.make(12, 10, 16, 2, 2, thresh_mode=lib.LCF_T_FIXED, k_fixed=2, project_form=lib.LCF_PF_SUBTRACT)
    pd = plan.filter(torch.zeros((16, 12, 10), dtype=torch.complex64, device="cuda"))
    st, flags = plan.status()
    assert st == lib.LCF_EDEGENERATE and float(pd.abs().max()) == 0.0
    for mode in (lib.LCF_T_SIGMOID, lib.LCF_T_ADAPTIVE_SOFT):
        with pytest.raises(lib.LcfError) as e:
            lib.Plan.make(12, 10, 16, 2, 2, thresh_mode=mode, project_form=lib.LCF_PF_SUBTRACT)
        assert e.value.status == lib.LCF_EINVAL
