"""Method 4 (Eq. 8, the NCC of the tissue and blood images next to the cutoff) and
method 5 (Eq. 9) at method 4's cutoff, on the GPU vs the FP64 oracle, through the C ABI.

Tolerances as for the other rules: PD rel L2 <= 1e-3, eigenvalues in the 1e-6*lambda_1
band <= 1e-4, alpha <= 1e-3; cutoffs equal except where the oracle's own NCC curve has
its minimum within 1e-6 relative of the GPU's choice (counted and printed).
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

from synth import REALTIME_256x128x100, SMALL_96x64x32, generate_packet  # noqa: E402
from test_parity_gpu import (ALPHA_TOL, EIG_TOL, PD_TOL, L, assert_cutoffs, compare, configs,  # noqa: E402
                             rand_iq)


def fast(cfg):
    lib = L()
    cfg.gram_path, cfg.project_path, cfg.evd_path = lib.LCF_PATH_TC, lib.LCF_PATH_TC, lib.LCF_EVD_PAIR
    return cfg


def check(r):
    lib = L()
    print({k: r[k] for k in ("pd_err", "eig_err", "alpha_err")}, "k gpu", r["k_gpu"][:16].tolist())
    assert r["status"] == lib.LCF_OK, r["flags"]
    assert r["eig_err"] <= EIG_TOL
    assert_cutoffs(r)
    assert r["alpha_err"] <= ALPHA_TOL
    assert r["pd_err"] <= PD_TOL


@pytest.mark.parametrize("path", ["plain", "fast"])
def test_ncc_small(path):
    lib = L()
    iq = generate_packet(SMALL_96x64x32, seed=0)
    cfg, oc = configs(96, 64, 32, 3, 3, thresh_mode=lib.LCF_T_NCC)
    if path == "fast":
        fast(cfg)
    check(compare(iq, cfg, oc, want_gram=False))


def test_ncc_realtime_fast_path():
    lib = L()
    iq = generate_packet(REALTIME_256x128x100, seed=0)
    cfg, oc = configs(256, 128, 100, 8, 8, thresh_mode=lib.LCF_T_NCC)
    r = compare(iq, fast(cfg), oc, want_gram=False)
    check(r)
    # the rule is not a constant: the windows' cutoffs vary with their content
    assert len(set(r["k_gpu"].tolist())) > 1


@pytest.mark.parametrize("beta", [0.5, 2.0])
def test_sigmoid_at_ncc_cutoff(beta):
    """Method 5 with the cutoff of method 4, as the paper evaluates it."""
    lib = L()
    iq = generate_packet(SMALL_96x64x32, seed=1)
    cfg, oc = configs(96, 64, 32, 3, 3, thresh_mode=lib.LCF_T_SIGMOID, k_src=lib.LCF_T_NCC, beta=beta)
    r = compare(iq, fast(cfg), oc, want_gram=False)
    check(r)
    assert np.max(np.abs(r["dbg"]["wt"] - r["ora"].wt)) <= 1e-3


@pytest.mark.parametrize("shape,grid", [
    ((10, 24, 20), (1, 1)),       # fn = 5: one admissible cutoff (k = 5)
    ((7, 16, 12), (2, 2)),        # fn = 3: k in {3, 4}
    ((33, 40, 70), (2, 3)),       # odd Nt, ragged image
    ((128, 40, 36), (2, 2)),      # longest packet of the CTA-pair EVD
    ((200, 40, 36), (2, 2)),      # distributed EVD, band kernel over two column chunks
])
def test_ncc_edge_shapes(shape, grid):
    lib = L()
    nt, nz, nx = shape
    cfg, oc = configs(nz, nx, nt, grid[0], grid[1], thresh_mode=lib.LCF_T_NCC)
    fast(cfg)
    check(compare(rand_iq(12, nt, nz, nx), cfg, oc, want_gram=False))


def test_ncc_zero_packet_is_degenerate():
    import torch
    lib = L()
    cfg, _ = configs(12, 10, 16, 2, 2, thresh_mode=lib.LCF_T_NCC)
    plan = lib.Plan(fast(cfg))
    pd = plan.filter(torch.zeros((16, 12, 10), dtype=torch.complex64, device="cuda"))
    st, flags = plan.status()
    assert st == lib.LCF_EDEGENERATE
    assert np.all(np.asarray(flags) & lib.LCF_WFLAG_DEGENERATE)
    assert float(pd.abs().max()) == 0.0


def test_ncc_config_validation():
    lib = L()
    for kw, want in (({"thresh_mode": lib.LCF_T_SIGMOID, "k_src": lib.LCF_T_NCC}, lib.LCF_OK),
                     ({"thresh_mode": lib.LCF_T_SIGMOID, "k_src": lib.LCF_T_LEARNED}, lib.LCF_EINVAL),
                     ({"thresh_mode": lib.LCF_T_LEARNED, "k_src": lib.LCF_T_NCC}, lib.LCF_EINVAL),
                     ({"thresh_mode": 9}, lib.LCF_EINVAL)):
        c = lib.lcf_config_default(32, 32, 16, 2, 2)
        for k, v in kw.items():
            setattr(c, k, v)
        try:
            lib.Plan(c).close()
            got = lib.LCF_OK
        except lib.LcfError as e:
            got = e.status
        assert got == want, (kw, got)
