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


@pytest.fixture(scope="module")
def stress_oracle():
    """The precision-stress workload (256 x 192 px, Nt = 300, 10 x 10 windows, method 1,
    60 dB tissue-to-blood, 1.5 px respiratory motion plus 0.5 px jitter, -75 dB noise) and the
    oracle's Gram, EVD and cutoff of the nine windows covering the image corner and of the
    centre window, computed one window at a time."""
    import oracle as O
    from synth import generate_packet
    from synth.iq import STRESS_256x192x300
    from test_parity_gpu import configs
    lib = L()
    nz, nx, nt, wz, wx = 256, 192, 300, 10, 10
    iq = generate_packet(STRESS_256x192x300, seed=0)
    _, oc = configs(nz, nx, nt, wz, wx, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0)
    corner = [iz * wx + ix for iz in range(3) for ix in range(3)]
    ora = {}
    for k in corner + [wz * wx // 2 + wx // 2]:
        R = O.gram(iq, oc, k)
        lam, V, _ = O.eigh(R)
        ora[k] = (R, lam, V)
    return iq, oc, corner, ora


def stress_errors(stress_oracle, **kw):
    """Errors of one configuration of the library on the precision-stress packet against the
    sampled oracle: the Gram, eigenvalues (1e-6 lambda_1 band), cutoff and alpha of the sampled
    windows, and the power Doppler of three corner pixels (covered by the nine corner windows
    only), summed from the oracle's per-window EVD and weights (PD_k(p) = g_k(p)^2 / Nt
    sum_c wt_c^2 |s_p v_c|^2, alpha_k = Nz Nx Nt / sum_c wt_c^2 lambda_c: the identities the
    oracle pins)."""
    import oracle as O
    from test_parity_gpu import configs, near_tie, run_gpu
    lib = L()
    iq, oc, corner, ora = stress_oracle
    nz, nx, nt, wz, wx = oc.nz, oc.nx, oc.nt, oc.wz, oc.wx
    cfg, _ = configs(nz, nx, nt, wz, wx, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0, **kw)
    if cfg.evd_path == lib.LCF_EVD_CTA:
        cfg.evd_path = lib.LCF_EVD_PAIR
    pd, plan, _ = run_gpu(iq, cfg)
    st, flags = plan.status()
    dbg = plan.debug()
    Rg = plan.debug_gram()
    pix = [(0, 0), (1, 2), (3, 1)]
    for (z, x) in pix:   # the corner windows are exactly the ones covering the sampled pixels
        cov = [k for k in range(wz * wx) if O.window_weights(oc, k)[z, x] > 0.0]
        assert sorted(cov) == corner, (z, x, cov)
    pd_ora = np.zeros(len(pix))
    s = iq.astype(np.complex128)
    errs = {"status": int(st), "gram": 0.0, "eig": 0.0, "alpha": 0.0, "flips": 0, "ties": 0}
    for k, (R, lam, V) in ora.items():
        errs["gram"] = max(errs["gram"], np.linalg.norm(Rg[k] - R) / np.linalg.norm(R))
        m = lam >= 1e-6 * lam[0]
        errs["eig"] = max(errs["eig"], np.max(np.abs(dbg["lam"][k][m] - lam[m]) / lam[m]))
        wt, kk = O.weights(O.T_CURVATURE, lam, beta=1.0)
        kg = int(dbg["k"][k])
        if kg != kk:
            errs["flips"] += 1
            if near_tie(oc, lam, dbg["lam"][k], kg, kk):
                errs["ties"] += 1
                wt = (np.arange(nt) >= kg).astype(np.float64)   # the equally valid cutoff the GPU took
        alpha = nz * nx * nt / np.sum(wt ** 2 * lam)
        errs["alpha"] = max(errs["alpha"], abs(dbg["alpha"][k] - alpha) / alpha)
        if k in corner:
            g = O.window_weights(oc, k)
            for i, (z, x) in enumerate(pix):
                proj = s[:, z, x] @ V   # s_p v_c over the columns c
                pd_ora[i] += alpha * g[z, x] ** 2 / nt * np.sum(wt ** 2 * np.abs(proj) ** 2)
    pd_gpu = np.array([pd[z, x] for (z, x) in pix])
    errs["pd"] = float(np.max(np.abs(pd_gpu - pd_ora) / pd_ora))
    errs["finite"] = bool(np.all(np.isfinite(pd)) and pd.min() >= 0.0)
    return errs


@pytest.mark.parametrize("path", ["plain", "fast"])
def test_stress_full_size_sampled(stress_oracle, path):
    """The precision-stress workload at its full size through the library with 12 deflated
    slow-time vectors (the 1.5 px motion spreads the tissue over about 12 global modes, so
    four would leave 1e-2 lambda_1 of tissue in the FP32 / tensor-core residual sums) and the
    FP64-class eigenvalue polish: every sampled quantity meets the standard tolerances."""
    from test_parity_gpu import ALPHA_TOL, EIG_TOL, GRAM_TOL, PD_TOL
    lib = L()
    kw = dict(deflate=12, evd_precision=lib.LCF_EP_FP64_POLISH)
    if path == "fast":
        kw.update(gram_path=lib.LCF_PATH_TC, project_path=lib.LCF_PATH_TC)
    errs = stress_errors(stress_oracle, **kw)
    print(path, errs)
    assert errs["status"] == lib.LCF_OK and errs["finite"]
    assert errs["flips"] == errs["ties"]
    assert errs["gram"] <= GRAM_TOL and errs["eig"] <= EIG_TOL
    assert errs["alpha"] <= ALPHA_TOL and errs["pd"] <= PD_TOL, errs


def test_stress_precision_study(stress_oracle):
    """The precision study of the stress workload: every tensor-core product mode with the
    FP32 and the polished eigen-decomposition (12 deflated vectors), and the default four
    deflated vectors for contrast, each with its Gram, eigenvalue, alpha and PD errors against
    the oracle.  The default product mode with the polish meets every tolerance; the E4M3 mode
    (4-bit operands) cannot resolve the kept eigenvalues at this dynamic range."""
    from test_parity_gpu import ALPHA_TOL, PD_TOL
    lib = L()
    rows = {}
    for gp in ("LCF_GP_F16X3", "LCF_GP_BF16X3", "LCF_GP_F16", "LCF_GP_BF16", "LCF_GP_E4M3"):
        for ep in ("LCF_EP_FP32", "LCF_EP_FP64_POLISH"):
            rows[(gp, ep, 12)] = stress_errors(stress_oracle, gram_path=lib.LCF_PATH_TC, project_path=lib.LCF_PATH_TC,
                                               gram_precision=getattr(lib, gp), evd_precision=getattr(lib, ep),
                                               deflate=12)
    rows[("LCF_GP_F16X3", "LCF_EP_FP32", 4)] = stress_errors(stress_oracle, gram_path=lib.LCF_PATH_TC,
                                                            project_path=lib.LCF_PATH_TC)
    for key, e in rows.items():
        print(key, {k: (f"{v:.2e}" if isinstance(v, float) else v) for k, v in e.items()})
    best = rows[("LCF_GP_F16X3", "LCF_EP_FP64_POLISH", 12)]
    assert best["alpha"] <= ALPHA_TOL and best["pd"] <= PD_TOL
    assert rows[("LCF_GP_E4M3", "LCF_EP_FP32", 12)]["alpha"] > ALPHA_TOL
    # the polish never makes alpha worse, and four deflated vectors are not enough here
    for gp in ("LCF_GP_F16X3", "LCF_GP_BF16X3", "LCF_GP_F16"):
        assert rows[(gp, "LCF_EP_FP64_POLISH", 12)]["alpha"] <= rows[(gp, "LCF_EP_FP32", 12)]["alpha"] * 1.5
    assert rows[("LCF_GP_F16X3", "LCF_EP_FP32", 4)]["alpha"] > ALPHA_TOL


def test_stress_subtractive_form(stress_oracle):
    """Eq. 5 with double-float sums on the precision-stress packet: with 12 deflated vectors
    (for the cutoffs) and the FP32 eigen-decomposition, PD and alpha meet 1e-3."""
    from test_parity_gpu import ALPHA_TOL, PD_TOL
    lib = L()
    errs = stress_errors(stress_oracle, deflate=12, project_form=lib.LCF_PF_SUBTRACT,
                         gram_path=lib.LCF_PATH_TC, project_path=lib.LCF_PATH_TC)
    print(errs)
    assert errs["status"] == lib.LCF_OK and errs["flips"] == errs["ties"]
    assert errs["alpha"] <= ALPHA_TOL and errs["pd"] <= PD_TOL, errs
