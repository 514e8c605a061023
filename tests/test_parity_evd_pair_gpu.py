"""CTA-pair (cluster) EVD vs the FP64 oracle and vs the one-CTA EVD, through the C ABI.

Same tolerances as the other GPU paths: eigenvalues in the 1e-6*lambda_1 band
<= 1e-4 relative, PD rel L2 <= 1e-3, hard cutoffs equal up to near-ties of
the oracle's rule, soft weights within 1e-3.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

from synth import REALTIME_256x128x100, SMALL_96x64x32, generate_packet  # noqa: E402
from test_parity_gpu import (assert_cutoffs, ALPHA_TOL, EIG_TOL, PD_TOL, L, compare, configs, rand_iq)  # noqa: E402


def pair_cfg(*a, tc=False, **kw):
    lib = L()
    cfg, oc = configs(*a, **kw)
    cfg.evd_path = lib.LCF_EVD_PAIR
    if tc:
        cfg.gram_path = lib.LCF_PATH_TC
        cfg.project_path = lib.LCF_PATH_TC
    return cfg, oc


def check(r, soft=False):
    lib = L()
    print({k: r[k] for k in ("pd_err", "eig_err", "alpha_err")}, "flips", r["flips"], "ties", r["ties"],
          "sweeps", sorted(set(((np.asarray(r["flags"]) >> 8) & 255).tolist())))
    assert r["status"] == lib.LCF_OK, r["flags"]
    assert r["eig_err"] <= EIG_TOL
    assert_cutoffs(r)
    assert r["alpha_err"] <= ALPHA_TOL
    assert r["pd_err"] <= PD_TOL
    if soft:
        assert np.max(np.abs(r["dbg"]["wt"] - r["ora"].wt)) <= 1e-3


def test_pair_small_fixed_k3():
    lib = L()
    iq = generate_packet(SMALL_96x64x32, seed=0)
    cfg, oc = pair_cfg(96, 64, 32, 3, 3, thresh_mode=lib.LCF_T_FIXED, k_fixed=3)
    check(compare(iq, cfg, oc, want_gram=False))


@pytest.mark.parametrize("tc", [False, True])
def test_pair_realtime_curvature(tc):
    lib = L()
    iq = generate_packet(REALTIME_256x128x100, seed=0)
    cfg, oc = pair_cfg(256, 128, 100, 8, 8, tc=tc, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0)
    check(compare(iq, cfg, oc, want_gram=False))


@pytest.mark.parametrize("mode,beta,extra", [
    ("LCF_T_SLOPE", 1.1, {}),
    ("LCF_T_MEDIAN", 1.43, {}),
    ("LCF_T_SIGMOID", 2.0, {"k_src": 0, "k_fixed": 4}),
    ("LCF_T_SIGMOID", 2.0, {"k_src": 3, "beta_src": 1.43}),
    ("LCF_T_ADAPTIVE_SOFT", 0.5, {}),
    ("LCF_T_CURVATURE", 1.5, {"curv_norm": 1}),
    ("LCF_T_NONE", 1.0, {}),
])
def test_pair_small_all_rules(mode, beta, extra):
    lib = L()
    iq = generate_packet(SMALL_96x64x32, seed=1)
    cfg, oc = pair_cfg(96, 64, 32, 3, 3, thresh_mode=getattr(lib, mode), beta=beta, **extra)
    check(compare(iq, cfg, oc, want_gram=False), soft=True)


@pytest.mark.parametrize("shape,grid,mode", [
    ((33, 40, 70), (2, 3), "LCF_T_FIXED"),       # odd Nt: padded pair slot
    ((16, 17, 23), (1, 1), "LCF_T_MEDIAN"),
    ((112, 24, 20), (2, 2), "LCF_T_CURVATURE"),   # largest Nt: 56 pairs, 13 V items per thread
    ((2, 8, 8), (1, 1), "LCF_T_FIXED"),          # one pair
    ((5, 12, 9), (2, 2), "LCF_T_CURVATURE"),     # head block = whole matrix (m = Nt)
    ((128, 40, 36), (2, 2), "LCF_T_CURVATURE"),   # largest Nt of the library: 64 pairs, 16 V items per thread
    ((127, 33, 29), (2, 3), "LCF_T_MEDIAN"),
])
def test_pair_edge_shapes(shape, grid, mode):
    lib = L()
    nt, nz, nx = shape
    cfg, oc = pair_cfg(nz, nx, nt, grid[0], grid[1], thresh_mode=getattr(lib, mode), k_fixed=1, beta=1.0)
    check(compare(rand_iq(3, nt, nz, nx), cfg, oc, want_gram=False))


@pytest.mark.parametrize("mode", ["LCF_T_CURVATURE", "LCF_T_ADAPTIVE_SOFT"])
def test_pair_nt128_with_tensor_core_projection(mode):
    """Nt = 128: plain Gram, CTA-pair EVD,
    tensor-core projection with one k-step per weight stage."""
    lib = L()
    nt, nz, nx = 128, 48, 40
    cfg, oc = pair_cfg(nz, nx, nt, 3, 2, thresh_mode=getattr(lib, mode), beta=1.0 if mode == "LCF_T_CURVATURE" else 0.5)
    cfg.project_path = lib.LCF_PATH_TC
    check(compare(rand_iq(5, nt, nz, nx), cfg, oc, want_gram=False), soft=mode != "LCF_T_CURVATURE")


def test_packet_length_limits():
    lib = L()
    for kw, want in (({"nt": 129, "gram_path": lib.LCF_PATH_TC, "evd_path": lib.LCF_EVD_PAIR}, lib.LCF_OK),
                     ({"nt": 128, "gram_path": lib.LCF_PATH_TC, "evd_path": lib.LCF_EVD_PAIR}, lib.LCF_OK),
                     ({"nt": 128, "evd_path": lib.LCF_EVD_CTA}, lib.LCF_EUNSUPPORTED),
                     ({"nt": 129, "evd_path": lib.LCF_EVD_PAIR}, lib.LCF_OK),          # distributed EVD
                     ({"nt": 129, "evd_path": lib.LCF_EVD_PAIR, "project_path": lib.LCF_PATH_TC}, lib.LCF_OK),
                     ({"nt": 124, "gram_path": lib.LCF_PATH_TC, "evd_path": lib.LCF_EVD_PAIR}, lib.LCF_OK)):
        c = lib.lcf_config_default(32, 32, kw["nt"], 2, 2)
        for k, v in kw.items():
            setattr(c, k, v)
        try:
            plan = lib.Plan(c)
            got = lib.LCF_OK
            plan.close()
        except lib.LcfError as e:
            got = e.status
        assert got == want, (kw, got)


def test_pair_zero_packet_is_degenerate():
    import torch
    lib = L()
    plan = lib.Plan.make(32, 32, 16, 2, 2, evd_path=lib.LCF_EVD_PAIR)
    pd = plan.filter(torch.zeros((16, 32, 32), dtype=torch.complex64, device="cuda"))
    st, flags = plan.status()
    assert st == lib.LCF_EDEGENERATE
    assert np.all(np.asarray(flags) & lib.LCF_WFLAG_DEGENERATE)
    assert float(pd.abs().max()) == 0.0


def test_pair_matches_one_cta_evd():
    """Eigenvalues and images of the two EVD kernels agree far inside the oracle tolerance."""
    import torch
    lib = L()
    iq = torch.from_numpy(generate_packet(REALTIME_256x128x100, seed=4)).cuda()
    res = {}
    for ev in (lib.LCF_EVD_CTA, lib.LCF_EVD_PAIR):
        plan = lib.Plan.make(256, 128, 100, 8, 8, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0, evd_path=ev)
        pd = plan.filter(iq).cpu().numpy().astype(np.float64)
        res[ev] = (pd, plan.debug()["lam"])
    (pa, la), (pb, lb) = res[lib.LCF_EVD_CTA], res[lib.LCF_EVD_PAIR]
    band = la >= 1e-6 * la[:, :1]
    rel = np.max(np.abs(la - lb)[band] / la[band])
    print("eigenvalue rel diff", rel, "pd rel", np.linalg.norm(pa - pb) / np.linalg.norm(pa))
    assert rel <= 2e-5
    assert np.linalg.norm(pa - pb) / np.linalg.norm(pa) <= 2e-4
