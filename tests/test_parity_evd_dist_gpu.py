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


@pytest.mark.parametrize("shape,grid,mode", [
    ((129, 33, 29), (2, 2), "LCF_T_MEDIAN"),       # shortest long packet: 128-row tiles, two column chunks
    ((200, 40, 36), (2, 2), "LCF_T_CURVATURE"),    # 96-row tiles, two chunks
    ((200, 40, 36), (2, 2), "LCF_T_ADAPTIVE_SOFT"),  # every column kept
    ((300, 36, 30), (2, 2), "LCF_T_CURVATURE"),    # 64-row tiles, three chunks
    ((320, 20, 20), (1, 1), "LCF_T_ADAPTIVE_SOFT"),  # longest packet, three chunks
])
def test_long_tensor_core_projection(shape, grid, mode):
    """Tensor-core projection of long packets (fewer resident tile rows, weight columns in
    chunks of 128) with the distributed EVD and the CUDA-core Gram."""
    lib = L()
    nt, nz, nx = shape
    cfg, oc = pair_cfg(nz, nx, nt, grid[0], grid[1], thresh_mode=getattr(lib, mode), k_fixed=3, beta=1.0)
    cfg.project_path = lib.LCF_PATH_TC
    check(compare(rand_iq(8, nt, nz, nx), cfg, oc, want_gram=False), soft=mode == "LCF_T_ADAPTIVE_SOFT")


@pytest.mark.parametrize("shape,grid,mode", [
    ((129, 33, 29), (2, 2), "LCF_T_MEDIAN"),        # two row tiles of 72 / 57 rows
    ((200, 40, 36), (2, 2), "LCF_T_CURVATURE"),     # two tiles of 104 / 96 rows (the streaming length)
    ((256, 24, 20), (1, 2), "LCF_T_SLOPE"),         # three tiles of 88 rows
    ((300, 36, 30), (2, 2), "LCF_T_ADAPTIVE_SOFT"), # three tiles of 104 / 104 / 92 rows
    ((320, 20, 20), (1, 1), "LCF_T_CURVATURE"),     # three tiles of 112 / 112 / 96 rows
])
def test_long_tensor_core_gram(shape, grid, mode):
    """Tensor-core Gram of long packets (tile pairs of at most 112 residual rows, both
    orders of each off-diagonal pair), with the tensor-core projection and the distributed EVD."""
    lib = L()
    nt, nz, nx = shape
    cfg, oc = pair_cfg(nz, nx, nt, grid[0], grid[1], thresh_mode=getattr(lib, mode), k_fixed=3, beta=1.0, tc=True)
    r = compare(rand_iq(9, nt, nz, nx), cfg, oc, want_gram=True)
    print("gram", r["gram_err"])
    assert r["gram_err"] <= 1e-6
    check(r, soft=mode == "LCF_T_ADAPTIVE_SOFT")


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
                     ({"nt": 200, "evd_path": lib.LCF_EVD_PAIR, "project_path": lib.LCF_PATH_TC}, lib.LCF_OK),
                     ({"nt": 320, "evd_path": lib.LCF_EVD_PAIR, "project_path": lib.LCF_PATH_TC}, lib.LCF_OK),
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


def test_stress_full_size_sampled():
    """The precision-stress workload at its full size (256 x 192 px, Nt = 300, 10 x 10
    windows, method 1): the whole packet through the library, then sampled outputs the
    oracle can compute one window at a time: the Gram, eigenvalues, cutoff and alpha of
    the nine windows that cover the image corner and of the centre window, and the power
    Doppler of three corner pixels (covered by those nine windows only), summed from the
    oracle's per-window EVD and weights (PD_k(p) = g_k(p)^2 / Nt sum_c wt_c^2 |s_p v_c|^2,
    alpha_k = Nz Nx Nt / sum_c wt_c^2 lambda_c, the identities the oracle pins).  The Gram
    and the eigenvalues in the 1e-6 lambda_1 band meet the standard tolerances; alpha and PD
    are held to the precision-stress bound below."""
    import oracle as O
    from synth import generate_packet
    from synth.iq import STRESS_256x192x300
    from test_parity_gpu import EIG_TOL, GRAM_TOL, configs, near_tie, run_gpu
    lib = L()
    nz, nx, nt, wz, wx = 256, 192, 300, 10, 10
    iq = generate_packet(STRESS_256x192x300, seed=0)
    cfg, oc = configs(nz, nx, nt, wz, wx, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0)
    cfg.evd_path = lib.LCF_EVD_PAIR
    pd, plan, _ = run_gpu(iq, cfg)
    st, flags = plan.status()
    assert st == lib.LCF_OK, flags
    dbg = plan.debug()
    Rg = plan.debug_gram()
    pix = [(0, 0), (1, 2), (3, 1)]
    corner = [iz * wx + ix for iz in range(3) for ix in range(3)]
    for (z, x) in pix:   # the corner windows are exactly the ones covering the sampled pixels
        cov = [k for k in range(wz * wx) if O.window_weights(oc, k)[z, x] > 0.0]
        assert sorted(cov) == corner, (z, x, cov)
    pd_ora = np.zeros(len(pix))
    pd_ora_ga = np.zeros(len(pix))   # with the GPU's alpha (separates the alpha and projection errors)
    s = iq.astype(np.complex128)
    errs = {"gram": 0.0, "eig": 0.0, "alpha": 0.0}
    for k in corner + [wz * wx // 2 + wx // 2]:
        R = O.gram(iq, oc, k)
        errs["gram"] = max(errs["gram"], np.linalg.norm(Rg[k] - R) / np.linalg.norm(R))
        lam, V, _ = O.eigh(R)
        m = lam >= 1e-6 * lam[0]
        errs["eig"] = max(errs["eig"], np.max(np.abs(dbg["lam"][k][m] - lam[m]) / lam[m]))
        wt, kk = O.weights(O.T_CURVATURE, lam, beta=1.0)
        kg = int(dbg["k"][k])
        if kg != kk:
            assert near_tie(oc, lam, dbg["lam"][k], kg, kk), (k, kg, kk)
            wt = (np.arange(nt) >= kg).astype(np.float64)   # the equally valid cutoff the GPU took
        alpha = nz * nx * nt / np.sum(wt ** 2 * lam)
        errs["alpha"] = max(errs["alpha"], abs(dbg["alpha"][k] - alpha) / alpha)
        print("window", k, "cutoff", kg, "kept eigenvalue sum / lambda_1", np.sum(wt ** 2 * lam) / lam[0],
              "alpha err", abs(dbg["alpha"][k] - alpha) / alpha)
        if k in corner:
            g = O.window_weights(oc, k)
            for i, (z, x) in enumerate(pix):
                proj = s[:, z, x] @ V   # s_p v_c over the columns c
                pd_ora[i] += alpha * g[z, x] ** 2 / nt * np.sum(wt ** 2 * np.abs(proj) ** 2)
                pd_ora_ga[i] += dbg["alpha"][k] * g[z, x] ** 2 / nt * np.sum(wt ** 2 * np.abs(proj) ** 2)
    pd_gpu = np.array([pd[z, x] for (z, x) in pix])
    errs["pd"] = float(np.max(np.abs(pd_gpu - pd_ora) / pd_ora))
    errs["pd_at_gpu_alpha"] = float(np.max(np.abs(pd_gpu - pd_ora_ga) / pd_ora_ga))
    print(errs)
    assert np.all(np.isfinite(pd)) and pd.min() >= 0.0
    assert errs["gram"] <= GRAM_TOL and errs["eig"] <= EIG_TOL
    # At this dynamic range (60 dB tissue-to-blood, -75 dB noise) the kept eigenvalue sum is
    # ~5e-8 of lambda_1, the FP32 unit roundoff: the FP32 eigen-decomposition resolves the
    # kept subspace and its energy only to ~u lambda_1, so alpha and PD carry errors of order
    # 1e-3 (measured 1.4e-3 and 2.6e-3). They are bounded here at 1e-2, ten times that floor.
    STRESS_TOL = 1e-2
    assert errs["alpha"] <= STRESS_TOL and errs["pd"] <= STRESS_TOL, errs
