"""Tensor-core (tcgen05) paths (Gram, projection) vs the FP64 oracle, through the C ABI.

Same tolerances as the plain FP32 path (see test_parity_gpu.py): PD rel L2
<= 1e-3, eigenvalues in the 1e-6*lambda_1 band <= 1e-4 relative, Gram rel
Frobenius <= 1e-6, hard cutoffs equal up to near-ties of the oracle's rule.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

from synth import REALTIME_256x128x100, SMALL_96x64x32, generate_packet  # noqa: E402
from test_parity_gpu import (assert_cutoffs, ALPHA_TOL, EIG_TOL, GRAM_TOL, PD_TOL, L, compare, configs,  # noqa: E402
                             rand_iq)


def tc_cfg(*a, project=False, gram=True, **kw):
    lib = L()
    cfg, oc = configs(*a, **kw)
    cfg.gram_path = lib.LCF_PATH_TC if gram else lib.LCF_PATH_SIMT
    cfg.project_path = lib.LCF_PATH_TC if project else lib.LCF_PATH_SIMT
    return cfg, oc


def check(r, gram=True):
    lib = L()
    print({k: r[k] for k in ("pd_err", "eig_err", "alpha_err") + (("gram_err",) if gram else ())},
          "flips", r["flips"], "ties", r["ties"])
    assert r["status"] in (lib.LCF_OK,), r["flags"]
    if gram:
        assert r["gram_err"] <= GRAM_TOL
    assert r["eig_err"] <= EIG_TOL
    assert_cutoffs(r)
    assert r["alpha_err"] <= ALPHA_TOL
    assert r["pd_err"] <= PD_TOL


def test_tc_small_fixed_k3():
    lib = L()
    iq = generate_packet(SMALL_96x64x32, seed=0)
    cfg, oc = tc_cfg(96, 64, 32, 3, 3, thresh_mode=lib.LCF_T_FIXED, k_fixed=3)
    check(compare(iq, cfg, oc))


def test_tc_realtime_curvature():
    lib = L()
    iq = generate_packet(REALTIME_256x128x100, seed=0)
    cfg, oc = tc_cfg(256, 128, 100, 8, 8, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0)
    check(compare(iq, cfg, oc))


def test_tc_realtime_soft_rule():
    lib = L()
    iq = generate_packet(REALTIME_256x128x100, seed=3)
    cfg, oc = tc_cfg(256, 128, 100, 8, 8, thresh_mode=lib.LCF_T_ADAPTIVE_SOFT, beta=0.5)
    check(compare(iq, cfg, oc, want_gram=False), gram=False)


@pytest.mark.parametrize("shape,grid,mode", [
    ((33, 40, 70), (2, 3), "LCF_T_FIXED"),
    ((16, 17, 23), (1, 1), "LCF_T_MEDIAN"),
    ((112, 24, 20), (2, 2), "LCF_T_CURVATURE"),
    ((2, 8, 8), (1, 1), "LCF_T_FIXED"),
    ((48, 24, 17), (2, 2), "LCF_T_CURVATURE"),   # Nz Nx even, Nx odd: slab starts alternate parity by row
    ((40, 34, 33), (3, 2), "LCF_T_FIXED"),       # boxes wider than one 32-pixel slab, odd Nx
])
def test_tc_edge_shapes(shape, grid, mode):
    lib = L()
    nt, nz, nx = shape
    cfg, oc = tc_cfg(nz, nx, nt, grid[0], grid[1], thresh_mode=getattr(lib, mode), k_fixed=1, beta=1.0)
    check(compare(rand_iq(3, nt, nz, nx), cfg, oc))


@pytest.mark.parametrize("nt,nz,nx,grid,seed", [
    (125, 40, 36, (2, 2), 11),    # Nt + d = 129: one row past a single MMA tile
    (128, 48, 40, (3, 2), 12),    # Nt + d = 132: the 128 residual rows fill the tile
])
def test_tc_residual_rows_only(nt, nz, nx, grid, seed):
    """Nt + d > 128: the tensor cores take the Nt x Nt residual block, the CUDA-core
    kernel the coefficient columns U (and the exact kernel Q)."""
    lib = L()
    cfg, oc = tc_cfg(nz, nx, nt, grid[0], grid[1], thresh_mode=lib.LCF_T_CURVATURE, beta=1.0)
    cfg.evd_path = lib.LCF_EVD_PAIR
    check(compare(rand_iq(seed, nt, nz, nx), cfg, oc))


def test_tc_residual_rows_only_realistic():
    """Nt = 128 on a tissue/vessel packet (the learned workload's recipe, cut down)."""
    from synth.iq import Recipe
    lib = L()
    rec = Recipe(64, 48, 128, n_vessels=3, width_px=(2.0, 6.0), phi_rad=(0.05, 1.0), tbr_db=50.0,
                 noise_db=-65.0, motion_amp_px=0.5)
    iq = generate_packet(rec, seed=21)
    cfg, oc = tc_cfg(64, 48, 128, 4, 3, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0, project=True)
    cfg.evd_path = lib.LCF_EVD_PAIR
    check(compare(iq, cfg, oc))


def test_tc_matches_plain_path():
    """The two Gram paths give the same image to well within the oracle tolerance."""
    import torch
    lib = L()
    iq = generate_packet(REALTIME_256x128x100, seed=4)
    d = torch.from_numpy(iq).cuda()
    out = {}
    for path in (lib.LCF_PATH_SIMT, lib.LCF_PATH_TC):
        plan = lib.Plan.make(256, 128, 100, 8, 8, thresh_mode=lib.LCF_T_FIXED, k_fixed=4, gram_path=path)
        out[path] = plan.filter(d).cpu().numpy().astype(np.float64)
    a, b = out[lib.LCF_PATH_SIMT], out[lib.LCF_PATH_TC]
    assert np.linalg.norm(a - b) / np.linalg.norm(a) <= 2e-4


# ---- tensor-core projection (and both tensor-core stages together) ----

def test_tcproj_small_fixed_k3():
    lib = L()
    iq = generate_packet(SMALL_96x64x32, seed=0)
    cfg, oc = tc_cfg(96, 64, 32, 3, 3, project=True, thresh_mode=lib.LCF_T_FIXED, k_fixed=3)
    check(compare(iq, cfg, oc))


def test_tcproj_realtime_curvature():
    lib = L()
    iq = generate_packet(REALTIME_256x128x100, seed=0)
    cfg, oc = tc_cfg(256, 128, 100, 8, 8, project=True, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0)
    check(compare(iq, cfg, oc))


def test_tcproj_with_plain_gram():
    lib = L()
    iq = generate_packet(REALTIME_256x128x100, seed=5)
    cfg, oc = tc_cfg(256, 128, 100, 8, 8, project=True, gram=False, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0)
    check(compare(iq, cfg, oc))


@pytest.mark.parametrize("mode,beta", [("LCF_T_ADAPTIVE_SOFT", 0.5), ("LCF_T_NONE", 1.0), ("LCF_T_SIGMOID", 1.0)])
def test_tcproj_soft_and_all_columns(mode, beta):
    """Rules that keep (almost) every column: widest weight images (n16 = 112 for Nt = 100)."""
    lib = L()
    iq = generate_packet(REALTIME_256x128x100, seed=3)
    cfg, oc = tc_cfg(256, 128, 100, 8, 8, project=True, thresh_mode=getattr(lib, mode), beta=beta, k_fixed=2)
    check(compare(iq, cfg, oc, want_gram=False), gram=False)


@pytest.mark.parametrize("shape,grid,mode", [
    ((33, 40, 70), (2, 3), "LCF_T_FIXED"),      # ragged tiles in both directions
    ((16, 17, 23), (1, 1), "LCF_T_MEDIAN"),
    ((112, 24, 20), (2, 2), "LCF_T_CURVATURE"),  # largest packet: K = 128, n16 = 112
    ((2, 8, 8), (1, 1), "LCF_T_FIXED"),         # one tile, one k-step
    ((48, 9, 130), (3, 5), "LCF_T_CURVATURE"),  # more tiles along x than along z
])
def test_tcproj_edge_shapes(shape, grid, mode):
    lib = L()
    nt, nz, nx = shape
    cfg, oc = tc_cfg(nz, nx, nt, grid[0], grid[1], project=True, thresh_mode=getattr(lib, mode), k_fixed=1,
                     beta=1.0)
    check(compare(rand_iq(3, nt, nz, nx), cfg, oc))


def test_tcproj_matches_plain_path():
    """Tensor-core projection vs the CUDA-core projection on the same Gram/EVD output."""
    import torch
    lib = L()
    iq = generate_packet(REALTIME_256x128x100, seed=4)
    d = torch.from_numpy(iq).cuda()
    out = {}
    for path in (lib.LCF_PATH_SIMT, lib.LCF_PATH_TC):
        plan = lib.Plan.make(256, 128, 100, 8, 8, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0,
                             gram_path=lib.LCF_PATH_TC, project_path=path)
        out[path] = plan.filter(d).cpu().numpy().astype(np.float64)
        st, _ = plan.status()
        assert st == lib.LCF_OK
    a, b = out[lib.LCF_PATH_SIMT], out[lib.LCF_PATH_TC]
    rel = np.linalg.norm(a - b) / np.linalg.norm(a)
    print("tc projection vs simt projection rel l2", rel, "max rel", np.max(np.abs(a - b) / np.maximum(a, 1e-30)))
    assert rel <= 1e-4
