"""One-sided Jacobi EVD on the Cholesky factor (LCF_EVD_OS) vs the FP64 oracle and vs the
two-sided CTA-pair EVD, through the C ABI.

Same tolerances as the other GPU paths: eigenvalues in the 1e-6*lambda_1 band <= 1e-4
relative, PD rel L2 <= 1e-3, alpha <= 1e-3, hard cutoffs equal up to near-ties of the
oracle's rule, soft weights within 1e-3.  The rank-deficient cases (fewer pixels in a
window than frames) exercise the Cholesky stop and the Gram-Schmidt completion.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

from synth import REALTIME_256x128x100, SMALL_96x64x32, generate_packet  # noqa: E402
from test_parity_gpu import (ALPHA_TOL, EIG_TOL, PD_TOL, L, assert_cutoffs, compare, configs,  # noqa: E402
                             rand_iq)


def os_cfg(*a, tc=False, **kw):
    lib = L()
    cfg, oc = configs(*a, **kw)
    cfg.evd_path = lib.LCF_EVD_OS
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
    V = r["plan"].debug_eigvecs()
    for k in (0, V.shape[0] - 1):   # unitary eigenvectors
        G = V[k].conj().T.astype(np.complex128) @ V[k]
        assert np.max(np.abs(G - np.eye(G.shape[0]))) <= 1e-4


def test_os_small_fixed_k3():
    lib = L()
    iq = generate_packet(SMALL_96x64x32, seed=0)
    cfg, oc = os_cfg(96, 64, 32, 3, 3, thresh_mode=lib.LCF_T_FIXED, k_fixed=3)
    check(compare(iq, cfg, oc, want_gram=False))


@pytest.mark.parametrize("tc", [False, True])
def test_os_realtime_curvature(tc):
    lib = L()
    iq = generate_packet(REALTIME_256x128x100, seed=0)
    cfg, oc = os_cfg(256, 128, 100, 8, 8, tc=tc, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0)
    r = compare(iq, cfg, oc, want_gram=False)
    check(r)
    assert len(r["flips"]) == 0


@pytest.mark.parametrize("mode,beta,extra", [
    ("LCF_T_SLOPE", 1.1, {}),
    ("LCF_T_MEDIAN", 1.43, {}),
    ("LCF_T_SIGMOID", 2.0, {"k_src": 0, "k_fixed": 4}),
    ("LCF_T_SIGMOID", 2.0, {"k_src": 3, "beta_src": 1.43}),
    ("LCF_T_ADAPTIVE_SOFT", 0.5, {}),
    ("LCF_T_CURVATURE", 1.5, {"curv_norm": 1}),
    ("LCF_T_NONE", 1.0, {}),
    ("LCF_T_NCC", 1.0, {}),
])
def test_os_small_all_rules(mode, beta, extra):
    lib = L()
    iq = generate_packet(SMALL_96x64x32, seed=1)
    cfg, oc = os_cfg(96, 64, 32, 3, 3, tc=True, thresh_mode=getattr(lib, mode), beta=beta, **extra)
    check(compare(iq, cfg, oc, want_gram=False), soft=mode in ("LCF_T_SIGMOID", "LCF_T_ADAPTIVE_SOFT"))


@pytest.mark.parametrize("shape,grid,mode", [
    ((33, 40, 70), (2, 3), "LCF_T_FIXED"),       # odd Nt: five warps, seven zero columns
    ((16, 17, 23), (1, 1), "LCF_T_MEDIAN"),
    ((112, 24, 20), (2, 2), "LCF_T_CURVATURE"),
    ((2, 8, 8), (1, 1), "LCF_T_FIXED"),          # one warp, six zero columns, no block exchange
    ((4, 8, 8), (1, 1), "LCF_T_FIXED"),          # one warp, two columns per block
    ((5, 12, 9), (2, 2), "LCF_T_CURVATURE"),     # head block = whole matrix (m = Nt)
    ((17, 30, 22), (2, 2), "LCF_T_SLOPE"),       # three warps, the last holding one column
    ((128, 40, 36), (2, 2), "LCF_T_CURVATURE"),   # largest Nt: 16 warps, 32 blocks, no padding
    ((127, 33, 29), (2, 3), "LCF_T_MEDIAN"),
    ((9, 14, 12), (1, 1), "LCF_T_CURVATURE"),    # two warps: the smallest block exchange
    ((24, 16, 14), (1, 1), "LCF_T_MEDIAN"),      # three warps, no padding
    ((64, 28, 26), (2, 2), "LCF_T_CURVATURE"),   # 64 rows: the last one-row-pair layout
    ((65, 28, 26), (2, 2), "LCF_T_SLOPE"),       # 65: two row pairs, nine warps, seven zero columns
    ((3, 10, 9), (1, 2), "LCF_T_FIXED"),         # one warp, five zero columns
])
def test_os_edge_shapes(shape, grid, mode):
    lib = L()
    nt, nz, nx = shape
    cfg, oc = os_cfg(nz, nx, nt, grid[0], grid[1], tc=True, thresh_mode=getattr(lib, mode), k_fixed=1, beta=1.0)
    check(compare(rand_iq(3, nt, nz, nx), cfg, oc, want_gram=False))


@pytest.mark.parametrize("shape,mode", [
    ((32, 4, 4), "LCF_T_FIXED"),        # 16 pixels, 32 frames: rank 16
    ((40, 5, 3), "LCF_T_FIXED"),        # 15 pixels, 40 frames
    ((101, 9, 9), "LCF_T_NONE"),        # 81 pixels, odd Nt
])
def test_os_rank_deficient(shape, mode):
    """Fewer pixels than frames: the Gram has rank P < Nt, the Cholesky factor stops at the
    numerical rank and the vanished columns are completed to an orthonormal basis.  Rules
    that read the null eigenvalues (rounding noise here, ~1e-17 in the oracle) would decide
    from noise, so the cases use a fixed cutoff or none."""
    lib = L()
    nt, nz, nx = shape
    cfg, oc = os_cfg(nz, nx, nt, 1, 1, tc=False, thresh_mode=getattr(lib, mode), k_fixed=2, beta=1.0,
                     all_ones_window=1)
    r = compare(rand_iq(9, nt, nz, nx), cfg, oc, want_gram=False)
    check(r)


@pytest.mark.parametrize("mode", ["LCF_T_CURVATURE", "LCF_T_ADAPTIVE_SOFT"])
def test_os_nt128_with_tensor_core_paths(mode):
    lib = L()
    nt, nz, nx = 128, 48, 40
    cfg, oc = os_cfg(nz, nx, nt, 3, 2, tc=True, thresh_mode=getattr(lib, mode),
                     beta=1.0 if mode == "LCF_T_CURVATURE" else 0.5)
    check(compare(rand_iq(5, nt, nz, nx), cfg, oc, want_gram=False), soft=mode != "LCF_T_CURVATURE")


def test_os_polish_and_deflation():
    """The FP64-class polish and deeper deflation run on the one-sided eigenvectors too."""
    lib = L()
    iq = generate_packet(REALTIME_256x128x100, seed=2)
    cfg, oc = os_cfg(256, 128, 100, 8, 8, tc=True, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0,
                     evd_precision=lib.LCF_EP_FP64_POLISH, deflate=8)
    check(compare(iq, cfg, oc, want_gram=False))


def test_os_zero_packet_is_degenerate():
    import torch
    lib = L()
    plan = lib.Plan.make(32, 32, 16, 2, 2, evd_path=lib.LCF_EVD_OS)
    pd = plan.filter(torch.zeros((16, 32, 32), dtype=torch.complex64, device="cuda"))
    st, flags = plan.status()
    assert st == lib.LCF_EDEGENERATE
    assert np.all(np.asarray(flags) & lib.LCF_WFLAG_DEGENERATE)
    assert float(pd.abs().max()) == 0.0


def test_os_matches_pair_evd():
    """Eigenvalues and images of the one-sided and two-sided kernels agree far inside the
    oracle tolerance."""
    import torch
    lib = L()
    iq = torch.from_numpy(generate_packet(REALTIME_256x128x100, seed=4)).cuda()
    res = {}
    for ev in (lib.LCF_EVD_PAIR, lib.LCF_EVD_OS):
        plan = lib.Plan.make(256, 128, 100, 8, 8, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0, evd_path=ev)
        pd = plan.filter(iq).cpu().numpy().astype(np.float64)
        res[ev] = (pd, plan.debug()["lam"])
    (pa, la), (pb, lb) = res[lib.LCF_EVD_PAIR], res[lib.LCF_EVD_OS]
    band = la >= 1e-6 * la[:, :1]
    rel = np.max(np.abs(la - lb)[band] / la[band])
    print("eigenvalue rel diff", rel, "pd rel", np.linalg.norm(pa - pb) / np.linalg.norm(pa))
    assert rel <= 2e-5
    assert np.linalg.norm(pa - pb) / np.linalg.norm(pa) <= 2e-4


def test_os_learned_rule_is_refused():
    lib = L()
    c = lib.lcf_config_default(32, 32, 16, 2, 2)
    c.evd_path = lib.LCF_EVD_OS
    c.thresh_mode = lib.LCF_T_LEARNED
    c.k_src = lib.LCF_T_CURVATURE
    with pytest.raises(lib.LcfError) as e:
        lib.Plan(c).close()
    assert e.value.status == lib.LCF_EUNSUPPORTED


# ---- packets longer than 128 frames: Cholesky kernel + four-CTA cluster sweeps (Nt <= 224)
@pytest.mark.parametrize("shape,grid,mode,tc", [
    ((129, 33, 29), (2, 2), "LCF_T_MEDIAN", False),      # shortest: 9 warps, 144 columns, warp 0 idle in cross steps
    ((136, 20, 18), (1, 1), "LCF_T_FIXED", False),       # 144 columns, 8 padding: warp 0 idle
    ((182, 21, 17), (1, 1), "LCF_T_CURVATURE", True),    # 192 columns, 10 padding
    ((170, 20, 18), (1, 1), "LCF_T_MEDIAN", False),      # 176 columns, 6 padding: every warp works
    ((200, 40, 36), (2, 2), "LCF_T_CURVATURE", True),    # the streaming workload's packet length: 208 columns
    ((200, 40, 36), (2, 2), "LCF_T_ADAPTIVE_SOFT", True),
    ((201, 30, 26), (1, 2), "LCF_T_FIXED", False),       # odd length: 208 columns, 7 padding
    ((224, 24, 20), (1, 2), "LCF_T_SLOPE", True),        # longest on this path: 14 warps, no padding
    ((150, 22, 18), (1, 1), "LCF_T_NCC", True),          # method 4 after the cluster EVD
    ((200, 33, 29), (2, 2), "LCF_T_CURVATURE", True),    # odd pixel count: tile pairs without the tensor map
])
def test_os_long_packets(shape, grid, mode, tc):
    lib = L()
    nt, nz, nx = shape
    cfg, oc = os_cfg(nz, nx, nt, grid[0], grid[1], tc=tc, thresh_mode=getattr(lib, mode), k_fixed=3, beta=1.0)
    check(compare(rand_iq(7, nt, nz, nx), cfg, oc, want_gram=False), soft=mode == "LCF_T_ADAPTIVE_SOFT")


def test_os_long_rank_deficient():
    """144 pixels, 160 frames: the Cholesky kernel stops at the numerical rank and CTA 0 completes
    the vanished columns over the whole cluster's rows."""
    lib = L()
    cfg, oc = os_cfg(12, 12, 160, 1, 1, thresh_mode=lib.LCF_T_FIXED, k_fixed=2, all_ones_window=1)
    check(compare(rand_iq(10, 160, 12, 12), cfg, oc, want_gram=False))


def test_os_long_zero_packet_is_degenerate():
    import torch
    lib = L()
    plan = lib.Plan.make(24, 20, 200, 2, 2, evd_path=lib.LCF_EVD_OS)
    pd = plan.filter(torch.zeros((200, 24, 20), dtype=torch.complex64, device="cuda"))
    st, flags = plan.status()
    assert st == lib.LCF_EDEGENERATE
    assert np.all(np.asarray(flags) & lib.LCF_WFLAG_DEGENERATE)
    assert float(pd.abs().max()) == 0.0


def test_os_long_matches_distributed_evd():
    """The streaming length: eigenvalues and images of the one-sided cluster kernel and the
    two-sided distributed kernel agree far inside the oracle tolerance."""
    import torch
    lib = L()
    iq = torch.from_numpy(rand_iq(11, 200, 64, 48)).cuda()
    res = {}
    for ev in (lib.LCF_EVD_PAIR, lib.LCF_EVD_OS):
        plan = lib.Plan.make(64, 48, 200, 4, 4, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0, evd_path=ev)
        pd = plan.filter(iq).cpu().numpy().astype(np.float64)
        res[ev] = (pd, plan.debug()["lam"])
    (pa, la), (pb, lb) = res[lib.LCF_EVD_PAIR], res[lib.LCF_EVD_OS]
    band = la >= 1e-6 * la[:, :1]
    rel = np.max(np.abs(la - lb)[band] / la[band])
    print("eigenvalue rel diff", rel, "pd rel", np.linalg.norm(pa - pb) / np.linalg.norm(pa))
    assert rel <= 2e-5
    assert np.linalg.norm(pa - pb) / np.linalg.norm(pa) <= 2e-4


@pytest.mark.parametrize("nt,nz,nx,grid", [(32, 48, 40, (3, 3)), (200, 40, 36, (2, 2))])
def test_os_stream_graph_matches_packets(nt, nz, nx, grid):
    """lcf_filter_stream (all packets one CUDA graph, the cluster kernel launched with its cluster
    attribute inside the capture) gives every packet's lcf_filter image bit for bit."""
    import torch
    lib = L()
    stride = 8
    frames = torch.from_numpy(rand_iq(12, nt + 3 * stride, nz, nx)).cuda()
    plan = lib.Plan.make(nz, nx, nt, grid[0], grid[1], evd_path=lib.LCF_EVD_OS, thresh_mode=lib.LCF_T_CURVATURE,
                         beta=1.0)
    outs = plan.filter_stream(frames, stride)
    outs2 = plan.filter_stream(frames, stride, outs.clone())   # the captured graph again
    torch.cuda.synchronize()
    assert outs.shape[0] == 4 and torch.equal(outs, outs2)
    for i in range(4):
        one = plan.filter(frames[i * stride:i * stride + nt].contiguous())
        torch.cuda.synchronize()
        assert torch.equal(one, outs[i]), i


def test_os_long_packets_in_flight():
    """Lanes with the cluster EVD: images equal lcf_filter's bit for bit."""
    import torch
    lib = L()
    iq = torch.from_numpy(np.stack([rand_iq(20 + i, 200, 40, 36) for i in range(5)])).cuda()
    single = lib.Plan.make(40, 36, 200, 2, 2, evd_path=lib.LCF_EVD_OS)
    ref = torch.stack([single.filter(iq[p]) for p in range(5)])
    many = lib.Plan.make(40, 36, 200, 2, 2, evd_path=lib.LCF_EVD_OS, inflight=3)
    out = many.filter_many(iq)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
