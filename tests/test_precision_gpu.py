"""Precision options against the FP64 oracle, through the C ABI: the tensor-core Gram's
product precisions (LCF_GP_*), the FP64-class eigenvalue polish (LCF_EP_FP64_POLISH)
and deeper deflation (lcf_config.deflate).

The default product mode (split fp16, three products) and every deflation depth and
polish setting are held to the standard tolerances (PD rel L2 1e-3, eigenvalues in the
1e-6*lambda_1 band 1e-4, Gram 1e-6, alpha 1e-3).  The narrower modes (bf16 x3, one-pass
fp16 = TF32's significand, one-pass bf16, E4M3) are the precision study: each reports its
errors for eigenvalues, filtered IQ and power Doppler, and the test checks that the Gram
error grows with the significand the mode keeps.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

import oracle as O  # noqa: E402
from synth import REALTIME_256x128x100, SMALL_96x64x32, generate_packet  # noqa: E402
from test_parity_gpu import (ALPHA_TOL, EIG_TOL, FILT_TOL, GRAM_TOL, PD_TOL, L, assert_cutoffs,  # noqa: E402
                             compare, configs, rand_iq)

MODES = ("LCF_GP_F16X3", "LCF_GP_BF16X3", "LCF_GP_F16", "LCF_GP_BF16", "LCF_GP_E4M3")


def fast(cfg, **kw):
    lib = L()
    cfg.gram_path, cfg.project_path, cfg.evd_path = lib.LCF_PATH_TC, lib.LCF_PATH_TC, lib.LCF_EVD_PAIR
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def filtered_iq_err(r, iq, oc, subset):
    import torch
    ora = O.filter(iq, oc, dbg_subset=subset)
    f = r["plan"].debug_filtered_iq(r["d_iq"], subset)
    torch.cuda.synchronize()
    f = f.cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(f - ora.filt) / np.linalg.norm(ora.filt))


@pytest.fixture(scope="module")
def realtime_study():
    """The real-time workload (256 x 128 x 100, 8 x 8 windows, method 1) in every product mode."""
    lib = L()
    iq = generate_packet(REALTIME_256x128x100, seed=0)
    rows = {}
    for m in MODES:
        cfg, oc = configs(256, 128, 100, 8, 8, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0)
        r = compare(iq, fast(cfg, gram_precision=getattr(lib, m)), oc, want_gram=True)
        r["filt_err"] = filtered_iq_err(r, iq, oc, 27)
        rows[m] = r
        print(m, {k: r[k] for k in ("gram_err", "eig_err", "alpha_err", "pd_err", "filt_err")},
              "cutoff flips", len(r["flips"]))
    return rows


def test_default_product_mode_meets_tolerances(realtime_study):
    r = realtime_study["LCF_GP_F16X3"]
    assert r["gram_err"] <= GRAM_TOL and r["eig_err"] <= EIG_TOL and r["alpha_err"] <= ALPHA_TOL
    assert r["pd_err"] <= PD_TOL and r["filt_err"] <= FILT_TOL
    assert_cutoffs(r)


def test_product_modes_error_follows_significand(realtime_study):
    """22 bits (fp16 x3) >= 16 (bf16 x3) >= 11 (fp16, TF32's significand) >= 8 (bf16) >= 4 (E4M3):
    a narrower operand never gives a smaller Gram error (the exact coefficient block and the FP32
    sums set a floor that hides the difference between the two three-product modes), and the
    one-pass modes' product errors show through it."""
    g = [realtime_study[m]["gram_err"] for m in MODES]
    print("Gram rel errors", dict(zip(MODES, g)))
    for a, b in zip(g, g[1:]):
        assert b >= 0.8 * a, g
    assert g[3] >= 4 * g[0] and g[4] >= 100 * g[0], g
    for m in MODES:
        assert np.all(np.isfinite(realtime_study[m]["pd"]))


@pytest.mark.parametrize("path", ["plain", "fast"])
def test_polish_small_and_realtime(path):
    """The Rayleigh-quotient polish leaves every tolerance met (and re-sorts nothing away)."""
    lib = L()
    for rec, grid, mode in ((SMALL_96x64x32, (3, 3), lib.LCF_T_FIXED), (REALTIME_256x128x100, (8, 8), lib.LCF_T_CURVATURE)):
        iq = generate_packet(rec, seed=0)
        cfg, oc = configs(rec.nz, rec.nx, rec.nt, grid[0], grid[1], thresh_mode=mode, k_fixed=3, beta=1.0,
                          evd_precision=lib.LCF_EP_FP64_POLISH)
        if path == "fast":
            fast(cfg)
        r = compare(iq, cfg, oc, want_gram=False)
        print(path, rec.nt, {k: r[k] for k in ("pd_err", "eig_err", "alpha_err")})
        assert r["status"] == lib.LCF_OK
        assert r["eig_err"] <= EIG_TOL and r["alpha_err"] <= ALPHA_TOL and r["pd_err"] <= PD_TOL
        assert_cutoffs(r)
        lam = r["dbg"]["lam"]
        assert np.all(np.diff(lam, axis=1) <= 0)   # descending after the re-sort


@pytest.mark.parametrize("shape,grid,deflate,path", [
    ((32, 96, 64), (3, 3), 8, "fast"),     # deeper than the one-tile exact-coefficient kernel
    ((100, 64, 48), (2, 2), 16, "fast"),
    ((112, 24, 20), (2, 2), 16, "fast"),   # Nt + d = 128
    ((100, 64, 48), (2, 2), 12, "plain"),
    ((200, 40, 36), (2, 2), 12, "fast"),   # long packet: tile pairs, CUDA-core U and Q
    ((300, 36, 30), (2, 2), 16, "plain"),
])
def test_deep_deflation(shape, grid, deflate, path):
    lib = L()
    nt, nz, nx = shape
    cfg, oc = configs(nz, nx, nt, grid[0], grid[1], thresh_mode=lib.LCF_T_CURVATURE, beta=1.0, deflate=deflate)
    if path == "fast":
        fast(cfg)
    else:
        cfg.evd_path = lib.LCF_EVD_PAIR if nt > 112 else lib.LCF_EVD_CTA
    r = compare(rand_iq(13, nt, nz, nx), cfg, oc, want_gram=True)
    print(shape, deflate, path, {k: r[k] for k in ("gram_err", "pd_err", "eig_err", "alpha_err")})
    assert r["status"] == lib.LCF_OK
    assert r["gram_err"] <= GRAM_TOL and r["eig_err"] <= EIG_TOL
    assert r["alpha_err"] <= ALPHA_TOL and r["pd_err"] <= PD_TOL
    assert_cutoffs(r)


def test_precision_config_validation():
    lib = L()
    for kw, want in (({"gram_precision": 5}, lib.LCF_EINVAL),
                     ({"gram_precision": lib.LCF_GP_BF16, "gram_path": lib.LCF_PATH_SIMT}, lib.LCF_EINVAL),
                     ({"evd_precision": 2}, lib.LCF_EINVAL),
                     ({"deflate": 17}, lib.LCF_EINVAL),
                     ({"deflate": 16}, lib.LCF_EINVAL),    # deflate must stay below Nt = 16
                     ({"deflate": 15}, lib.LCF_OK),
                     ({"thresh_mode": lib.LCF_T_LEARNED, "k_src": lib.LCF_T_CURVATURE,
                       "evd_precision": lib.LCF_EP_FP64_POLISH}, lib.LCF_EUNSUPPORTED)):
        c = lib.lcf_config_default(32, 32, 16, 2, 2)
        for k, v in kw.items():
            setattr(c, k, v)
        try:
            lib.Plan(c).close()
            got = lib.LCF_OK
        except lib.LcfError as e:
            got = e.status
        assert got == want, (kw, got)
