"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test checks the oracle against something the paper or plain
mathematics fixes: closed forms, a different library routine (LAPACK eigh /
SVD through numpy), invariants, brute force on tiny inputs, hand-derived
fixtures in tests/golden/.  Chosen so that a dropped term, a wrong sign or
index, or a transposed operand anywhere in the oracle fails one of them.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from synth import SMALL_96x64x32, generate_packet

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_herm(rng, n, spread=None):
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    if spread is not None:        # PSD with eigenvalues spanning `spread` decades
        Q, _ = np.linalg.qr(A)
        lam = 10.0 ** (-spread * np.arange(n) / max(n - 1, 1))
        return (Q * lam) @ Q.conj().T
    return 0.5 * (A + A.conj().T)


# ---------------------------------------------------------------- Jacobi (Eq. 2)
def test_jacobi_2x2_closed_form():
    a, d, b = 3.0, -1.0, 1.5 - 2.0j
    A = np.array([[a, b], [np.conj(b), d]])
    lam, V, sw = O.eigh(A)
    r = np.sqrt(((a - d) / 2) ** 2 + abs(b) ** 2)
    np.testing.assert_allclose(lam, [(a + d) / 2 + r, (a + d) / 2 - r], rtol=0, atol=1e-14)
    # eigenvector equation and the phase convention (largest entry real > 0)
    np.testing.assert_allclose(A @ V, V * lam, atol=1e-13)
    for j in range(2):
        i = np.argmax(np.abs(V[:, j]))
        assert abs(V[i, j].imag) < 1e-15 and V[i, j].real > 0


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16])
def test_jacobi_vs_lapack(n):
    rng = np.random.default_rng(n)
    A = rand_herm(rng, n)
    lam, V, sw = O.eigh(A)
    ref = np.linalg.eigvalsh(A)[::-1]
    assert sw >= 0
    np.testing.assert_allclose(lam, ref, atol=1e-12 * np.abs(ref).max())
    assert np.all(np.diff(lam) <= 0)
    np.testing.assert_allclose(V.conj().T @ V, np.eye(n), atol=1e-12)
    assert np.linalg.norm(A @ V - V * lam) <= 1e-12 * np.linalg.norm(A)
    assert abs(np.trace(A).real - lam.sum()) <= 1e-12 * np.abs(A).sum()


def test_jacobi_graded_psd_small_eigenvalues():
    # eigenvalues 1 .. 1e-10: the FP64 solver must resolve the tail to ~1e-6 relative
    rng = np.random.default_rng(7)
    n = 24
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    lam_true = 10.0 ** (-10 * np.arange(n) / (n - 1))
    A = (Q * lam_true) @ Q.conj().T
    lam, V, _ = O.eigh(A)
    np.testing.assert_allclose(lam, lam_true, rtol=1e-5, atol=0)


def test_jacobi_sweep_cap_reports_nonconvergence():
    A = rand_herm(np.random.default_rng(3), 6)
    _, _, sw = O.eigh(A, max_sweeps=1)
    assert sw == -1


# ------------------------------------------------------------ windows (Eq. 11)
def test_window_geometry_totals():
    # support sizes follow from centres (i+1/2)*d - 1/2, sigma = d, |delta| <= 3 sigma
    cases = {(96, 64, 3, 3): (55296, (96, 64)), (256, 128, 8, 8): (778752, (192, 96)),
             (256, 192, 10, 10): (1277268, (154, 115))}
    for (nz, nx, wz, wx), (tot, big) in cases.items():
        cfg = O.OracleConfig(nz, nx, 8, wz, wx)
        sizes = []
        for k in range(wz * wx):
            (z0, z1, x0, x1), _ = O.window_box(cfg, k)
            sizes.append((z1 - z0, x1 - x0))
        assert sum(a * b for a, b in sizes) == tot
        assert max(sizes) == big


def test_window_weights_values():
    cfg = O.OracleConfig(256, 128, 8, 8, 8)
    (z0, z1, x0, x1), (cz, cx, sz, sx) = O.window_box(cfg, 9)     # iz = 1, ix = 1
    assert (cz, cx, sz, sx) == (47.5, 23.5, 32.0, 16.0)
    assert (z0, z1, x0, x1) == (0, 144, 0, 72)                   # 47.5+96 = 143.5, 23.5+48 = 71.5
    g = O.window_weights(cfg, 9)
    assert g[47, 23] == pytest.approx(np.exp(-0.5 * (0.5 / 32) ** 2 - 0.5 * (0.5 / 16) ** 2), rel=1e-15)
    assert g[143, 71] == pytest.approx(np.exp(-0.5 * (95.5 / 32) ** 2 - 0.5 * (47.5 / 16) ** 2), rel=1e-15)
    assert g[144, 0] == 0.0 and g[0, 72] == 0.0


# --------------------------------------------------------------- Gram (Eq. 12)
def small_iq(seed=0, nt=12, nz=10, nx=9):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((nt, nz, nx)) + 1j * rng.standard_normal((nt, nz, nx))).astype(np.complex64)


def test_gram_trace_hermitian_and_phase_invariance():
    iq = small_iq()
    cfg = O.OracleConfig(10, 9, 12, 2, 2, support_sigmas=1.0)
    for k in range(4):
        R = O.gram(iq, cfg, k)
        g = O.window_weights(cfg, k)
        s = iq.astype(np.complex128)
        tr = np.sum(g ** 2 * np.sum(np.abs(s) ** 2, axis=0))       # sum_p g^2 ||s_p||^2
        assert abs(np.trace(R).real - tr) <= 1e-13 * tr
        assert np.array_equal(R, R.conj().T)
        # a per-pixel phase e^{i phi_p} cancels in conj(s_p)^T s_p
        ph = np.exp(1j * np.random.default_rng(1).uniform(0, 6.28, (10, 9)))
        R2 = O.gram((iq * ph[None]).astype(np.complex64), cfg, k)
        # complex64 rounding of the rotated data limits this to ~1e-7
        np.testing.assert_allclose(R2, R, atol=1e-6 * np.abs(R).max())


def test_gram_orientation_against_matmul():
    # R[i, j] = sum_p conj(s_p(i)) s_p(j): catches a transposed operand
    iq = small_iq(2)
    cfg = O.OracleConfig(10, 9, 12, 1, 1, all_ones_window=1)
    R = O.gram(iq, cfg, 0)
    C = iq.reshape(12, -1).T.astype(np.complex128)               # Casorati: pixels x Nt
    np.testing.assert_allclose(R, C.conj().T @ C, atol=1e-12 * np.abs(R).max())
    assert not np.allclose(R, C.T @ C.conj())


# --------------------------------------- global-filter special cases (Eq. 3-5)
def global_cfg(iq, **kw):
    nt, nz, nx = iq.shape
    return O.OracleConfig(nz, nx, nt, 1, 1, all_ones_window=1, **kw)


def test_eigenvalues_are_squared_singular_values():
    iq = small_iq(3)
    cfg = global_cfg(iq, thresh_mode=O.T_FIXED, k_fixed=0)
    r = O.filter(iq, cfg)
    sv = np.linalg.svd(iq.reshape(12, -1).T.astype(np.complex128), compute_uv=False)
    np.testing.assert_allclose(r.lam[0], sv ** 2, rtol=1e-10)


@pytest.mark.parametrize("k", [1, 3, 6])
def test_global_filter_equals_svd_filter(k):
    # one all-ones window + fixed cutoff k == SVD filter removing k components
    iq = small_iq(4)
    cfg = global_cfg(iq, thresh_mode=O.T_FIXED, k_fixed=k, alpha_mode=1)
    r = O.filter(iq, cfg)
    C = iq.reshape(12, -1).T.astype(np.complex128)
    U, s, Vh = np.linalg.svd(C, full_matrices=False)
    Chat = (U[:, k:] * s[k:]) @ Vh[k:]                      # Eq. 5 form via LAPACK SVD
    pd = np.mean(np.abs(Chat) ** 2, axis=1).reshape(10, 9)
    np.testing.assert_allclose(r.pd, pd, rtol=1e-10, atol=1e-12 * pd.max())


def test_identity_weights_reproduce_input():
    iq = small_iq(5)
    cfg = global_cfg(iq, thresh_mode=O.T_NONE, alpha_mode=1)
    r = O.filter(iq, cfg, dbg_subset=0)
    np.testing.assert_allclose(r.filt, iq.astype(np.complex128), atol=1e-12)
    np.testing.assert_allclose(r.pd, np.mean(np.abs(iq.astype(np.complex128)) ** 2, axis=0), rtol=1e-12)


def test_rank_r_clutter_removed():
    rng = np.random.default_rng(6)
    nt, nz, nx, rnk = 16, 12, 10, 4
    # small-integer factors: C = A B^H is exactly representable in complex64,
    # so the packet really has rank r
    A = rng.integers(-3, 4, (nz * nx, rnk)) + 1j * rng.integers(-3, 4, (nz * nx, rnk))
    B = rng.integers(-3, 4, (nt, rnk)) + 1j * rng.integers(-3, 4, (nt, rnk))
    C = A @ B.conj().T
    assert np.array_equal(C.astype(np.complex64).astype(np.complex128), C)
    iq = C.T.reshape(nt, nz, nx).astype(np.complex64)
    cfg = global_cfg(iq, thresh_mode=O.T_FIXED, k_fixed=rnk, alpha_mode=1)
    r = O.filter(iq, cfg, dbg_subset=0)
    assert np.linalg.norm(r.filt) / np.linalg.norm(iq) <= 1e-10
    # eigenvalues beyond the rank vanish
    assert np.all(r.lam[0, rnk:] <= 1e-12 * r.lam[0, 0])


def test_eq4_equals_eq5_and_pd_identity_localized():
    # windowed subsets: C-hat = C_w V W V^H (Eq. 4) equals C_w (I - V W' V^H) (Eq. 5) for
    # hard k, and per pixel |C-hat|^2 summed over t equals sum_i wt_i^2 |(C_w V)_{p,i}|^2;
    # summed over pixels it equals sum_i wt_i^2 lambda_i (V unitary, R = C_w^H C_w).
    iq = small_iq(8, nt=10, nz=12, nx=11)
    cfg = O.OracleConfig(12, 11, 10, 2, 2, support_sigmas=1.5, thresh_mode=O.T_FIXED, k_fixed=2)
    for k in range(4):
        r = O.filter(iq, cfg, want_R=True, want_V=True, want_pdk=True, dbg_subset=k)
        V, wt, lam = r.V[k], r.wt[k], r.lam[k]
        g = O.window_weights(cfg, k)
        Cw = (g[None] * iq.astype(np.complex128)).reshape(10, -1).T
        keep_clutter = np.diag(1.0 - wt)
        Chat5 = Cw @ (np.eye(10) - V @ keep_clutter @ V.conj().T)
        np.testing.assert_allclose(r.filt.reshape(10, -1).T, Chat5, atol=1e-12 * np.abs(Cw).max())
        Y = Cw @ V
        pd_id = np.sum(wt ** 2 * np.abs(Y) ** 2, axis=1) / 10
        np.testing.assert_allclose(r.pdk[k].reshape(-1), pd_id, rtol=1e-10, atol=1e-14)
        assert np.sum(r.pdk[k]) == pytest.approx(np.sum(wt ** 2 * lam) / 10, rel=1e-10)
        assert np.allclose(r.R[k], Cw.conj().T @ Cw, atol=1e-12 * np.abs(r.R[k]).max())


# ----------------------------------------------------- blend (Eq. 13) and alpha
def test_alpha_normalises_each_subset_to_unit_mean():
    iq = generate_packet(SMALL_96x64x32, seed=0)
    cfg = O.OracleConfig(96, 64, 32, 3, 3, thresh_mode=O.T_FIXED, k_fixed=3)
    r = O.filter(iq, cfg, want_pdk=True)
    for k in range(9):
        assert np.mean(r.alpha[k] * r.pdk[k]) == pytest.approx(1.0, rel=1e-12)
    np.testing.assert_allclose(r.pd, np.tensordot(r.alpha, r.pdk, axes=1), rtol=1e-12)
    assert r.pd.mean() == pytest.approx(9.0, rel=1e-12)


def test_support_alpha_and_unit_alpha():
    iq = small_iq(9, nt=8, nz=14, nx=12)
    base = dict(support_sigmas=1.0, thresh_mode=O.T_FIXED, k_fixed=1)
    r1 = O.filter(iq, O.OracleConfig(14, 12, 8, 2, 2, alpha_mode=1, **base), want_pdk=True)
    np.testing.assert_allclose(r1.pd, r1.pdk.sum(0), rtol=1e-13)
    r2 = O.filter(iq, O.OracleConfig(14, 12, 8, 2, 2, alpha_mode=2, **base), want_pdk=True)
    cfg = O.OracleConfig(14, 12, 8, 2, 2, **base)
    for k in range(4):
        (z0, z1, x0, x1), _ = O.window_box(cfg, k)
        assert np.mean(r2.alpha[k] * r2.pdk[k][z0:z1, x0:x1]) == pytest.approx(1.0, rel=1e-12)


def test_zero_packet_is_degenerate():
    iq = np.zeros((8, 6, 5), np.complex64)
    r = O.filter(iq, O.OracleConfig(6, 5, 8, 1, 1, thresh_mode=O.T_FIXED, k_fixed=1))
    assert r.alpha[0] == 0.0 and (r.flags[0] & O.FLAG_DEGENERATE)
    assert np.all(r.pd == 0)


@pytest.mark.parametrize("mode", [O.T_FIXED, O.T_CURVATURE, O.T_MEDIAN, O.T_SIGMOID, O.T_ADAPTIVE_SOFT])
def test_scale_and_global_phase_invariance(mode):
    iq = generate_packet(SMALL_96x64x32, seed=1)
    cfg = O.OracleConfig(96, 64, 32, 3, 3, thresh_mode=mode, beta=1.5, k_fixed=3,
                         k_src=O.T_FIXED, beta_src=1.0)
    a = O.filter(iq, cfg).pd
    b = O.filter((iq * np.complex64(2.0 ** 5)).astype(np.complex64), cfg).pd     # exact scaling
    np.testing.assert_allclose(b, a, rtol=1e-9)
    c = O.filter((iq * np.complex64(1j)).astype(np.complex64), cfg).pd             # exact phase
    np.testing.assert_allclose(c, a, rtol=1e-9)


# ------------------------------------------------------- threshold rules
@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(GOLDEN, "threshold_closed_forms.json")) as f:
        return json.load(f)


def knee_spectrum(N, m):
    n = np.arange(1, N + 1)
    return 10.0 ** (-(np.minimum(n, m) - 1.0))


def test_curvature_knee(golden):
    for c in golden["knee_curvature"]:
        _, k = O.weights(O.T_CURVATURE, knee_spectrum(c["N"], c["m"]), beta=c["beta"])
        assert k == c["k"], c


def test_curvature_knee_literal_normalisation(golden):
    """curv_norm 1: the paper's literal beta*y(n)/y(1)*Nt curve (method 1, Eq. 6), on spectra
    whose cutoff follows by hand from the slope s = beta*N/|y(1)| (including y(1) < 0 and
    y(1) = 0)."""
    for c in golden["knee_curvature_literal"]:
        n = np.arange(1, c["N"] + 1)
        lam = 10.0 ** (c["a"] - (np.minimum(n, c["m"]) - 1.0))
        _, k = O.weights(O.T_CURVATURE, lam, beta=c["beta"], curv_norm=1)
        assert k == c["k"], c
        # the shifted curve of the same spectrum has slope s0 = beta*N/(m-1) whatever a is
        _, k0 = O.weights(O.T_CURVATURE, lam, beta=c["beta"], curv_norm=0)
        assert k0 == (c["m"] if c["beta"] * c["N"] / (c["m"] - 1) < 1.5328 else c["m"] + 1), c


def test_pd_sum_over_slow_time(golden):
    """pd_mode 1 (PD summed over slow time instead of averaged) on hand-derived packets:
    one all-ones window, a fixed cutoff or identity weights; alpha = 1 exposes the factor Nt,
    alpha by Eq. 13 cancels it."""
    for c in golden["pd_sum_over_time"]:
        rows = np.array(c["rows"], float)                     # [pixel][t][re, im]
        iq = (rows[..., 0] + 1j * rows[..., 1]).T.reshape(c["nt"], c["nz"], c["nx"]).astype(np.complex64)
        mode = O.T_FIXED if c["k"] >= 0 else O.T_NONE
        for pd_mode, alpha_mode, key in ((1, 1, "pd_sum_alpha1"), (0, 1, "pd_mean_alpha1"),
                                         (1, 0, "pd_alpha_eq13"), (0, 0, "pd_alpha_eq13")):
            cfg = O.OracleConfig(c["nz"], c["nx"], c["nt"], 1, 1, all_ones_window=1, thresh_mode=mode,
                                 k_fixed=max(c["k"], 0), pd_mode=pd_mode, alpha_mode=alpha_mode)
            pd = O.filter(iq, cfg).pd.ravel()
            np.testing.assert_allclose(pd, c[key], rtol=1e-14, atol=1e-14, err_msg=f"{key} pd_mode {pd_mode}")


def test_slope_knee(golden):
    for c in golden["knee_slope"]:
        wt, k = O.weights(O.T_SLOPE, knee_spectrum(c["N"], c["m"]), beta=c["beta"])
        assert k == c["k"], c
        assert np.all(wt[:k] == 0) and np.all(wt[k:] == 1)


def test_median_rule(golden):
    for c in golden["median"]:
        wt, k = O.weights(O.T_MEDIAN, np.array(c["lam"], float), beta=c["beta"])
        assert k == c["k"], c
        assert wt.sum() == len(c["lam"]) - k


def test_sigmoid_rule(golden):
    for c in golden["sigmoid"]:
        wt, k = O.weights(O.T_SIGMOID, np.ones(c["N"]), beta=c["beta"], k_fixed=c["k"],
                          k_src=O.T_FIXED)
        assert k == c["k"]
        np.testing.assert_allclose(wt[np.array(c["i"]) - 1], c["wt"], rtol=1e-15)


def test_adaptive_soft_rule(golden):
    c0, c1 = golden["adaptive_soft"]
    wt, k = O.weights(O.T_ADAPTIVE_SOFT, np.ones(c0["N"]), beta=c0["beta"])
    np.testing.assert_allclose(wt[np.array(c0["i"]) - 1], c0["wt"], rtol=1e-14)
    wt, _ = O.weights(O.T_ADAPTIVE_SOFT, np.array(c1["lam"]), beta=c1["beta"])
    np.testing.assert_allclose(wt, c1["wt"], rtol=1e-14)


def test_fixed_rule_bounds():
    lam = np.linspace(5, 1, 7)
    for kf, kexp in [(-1, 0), (0, 0), (3, 3), (9, 7)]:
        wt, k = O.weights(O.T_FIXED, lam, k_fixed=kf)
        assert k == kexp and wt.sum() == 7 - kexp


def test_rule_scores_agree_with_rules_and_override_equals_fixed():
    # the exported deciding quantities reproduce each rule's own choice
    lam = 10.0 ** (-(np.minimum(np.arange(1, 41), 7) - 1.0)) * (1 + 0.01 * np.arange(40))[::-1]
    lam = np.sort(lam)[::-1]
    sc = O.rule_scores(O.T_CURVATURE, lam, beta=1.0)
    _, k = O.weights(O.T_CURVATURE, lam, beta=1.0)
    assert int(np.argmax(sc)) + 1 == k
    sc = O.rule_scores(O.T_SLOPE, lam, beta=1.1)
    _, k = O.weights(O.T_SLOPE, lam, beta=1.1)
    assert np.all(sc[:k] > 1.1) and sc[k] <= 1.1
    sc = O.rule_scores(O.T_MEDIAN, lam, beta=1.43)
    _, k = O.weights(O.T_MEDIAN, lam, beta=1.43)
    assert np.sum(sc > 1.0) == k
    # a cutoff override gives exactly the fixed-k filter
    iq = generate_packet(SMALL_96x64x32, seed=3)
    a = O.filter(iq, O.OracleConfig(96, 64, 32, 3, 3, thresh_mode=O.T_CURVATURE),
                 k_override=np.full(9, 5, np.int32))
    b = O.filter(iq, O.OracleConfig(96, 64, 32, 3, 3, thresh_mode=O.T_FIXED, k_fixed=5))
    assert np.array_equal(a.pd, b.pd) and np.all(a.k == 5)


# ------------------------------------------------- method 4 (NCC, Eq. 8)
def ncc_from_left_vectors(absU, fn):
    """NCC(k) of Eq. 8 from the magnitudes of left singular vectors [pixels, Nt] (numpy)."""
    n = absU.shape[1]
    curve = np.full(n, np.nan)
    for k in range(fn, n - fn + 1):
        it = absU[:, k - fn:k].sum(axis=1)
        ib = absU[:, k:k + fn].sum(axis=1)
        curve[k - 1] = np.sum(it * ib) / (np.sqrt(np.sum(it * it)) * np.sqrt(np.sum(ib * ib)))
    return curve


@pytest.mark.parametrize("grid,win", [((1, 1), 0), ((2, 2), 3)])
def test_ncc_curve_matches_svd_of_windowed_casorati(grid, win):
    """The oracle's NCC curve (its Jacobi V, |C_w v_i| / sigma_i) against the same curve from
    LAPACK's SVD of the windowed Casorati matrix (|u_i| directly), on random data."""
    rng = np.random.default_rng(11)
    nt, nz, nx = 16, 12, 10
    iq = (rng.standard_normal((nt, nz, nx)) + 1j * rng.standard_normal((nt, nz, nx))).astype(np.complex64)
    cfg = O.OracleConfig(nz, nx, nt, grid[0], grid[1], all_ones_window=int(grid == (1, 1)))
    k, curve = O.ncc_curve(iq, cfg, win)
    g = O.window_weights(cfg, win).ravel()
    sup = g > 0
    C = iq.reshape(nt, -1).T.astype(np.complex128)[sup] * g[sup, None]       # C_w on the support
    U, sv, _ = np.linalg.svd(C, full_matrices=False)
    ref = ncc_from_left_vectors(np.abs(U), 5)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(curve))
    np.testing.assert_allclose(curve[fin], ref[fin], rtol=1e-10)
    assert k == int(np.nanargmin(ref)) + 1


def test_ncc_disjoint_supports_pick_the_split():
    """C = U D V^H whose first 9 left singular vectors live on one half of the image and the
    other 15 on the other half: at k = 9 the tissue and blood images do not overlap, so NCC(9)
    is 0 and every other cutoff mixes the halves (NCC > 0); methods 4 and 5 take k = 9."""
    rng = np.random.default_rng(5)
    nt, nz, nx, kst = 24, 12, 10, 9
    npx = nz * nx

    def orth(rows, cols):
        a = rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))
        return np.linalg.qr(a)[0]
    U = np.zeros((npx, nt), complex)
    U[:npx // 2, :kst] = orth(npx // 2, kst)
    U[npx // 2:, kst:] = orth(npx - npx // 2, nt - kst)
    sv = 2.0 ** (np.arange(nt, 0, -1) / 4.0)     # distinct, within 2^6 (little complex64 rounding leak)
    V = orth(nt, nt)
    C = (U * sv) @ V.conj().T
    iq = np.ascontiguousarray(C.T.reshape(nt, nz, nx)).astype(np.complex64)
    cfg = O.OracleConfig(nz, nx, nt, 1, 1, all_ones_window=1)
    k, curve = O.ncc_curve(iq, cfg, 0)
    assert k == kst
    assert curve[kst - 1] <= 1e-6   # zero up to the complex64 rounding of the packet
    others = np.delete(curve, kst - 1)
    assert np.nanmin(others) >= 0.05
    r = O.filter(iq, O.OracleConfig(nz, nx, nt, 1, 1, all_ones_window=1, thresh_mode=O.T_NCC))
    assert int(r.k[0]) == kst and np.all(r.wt[0][:kst] == 0) and np.all(r.wt[0][kst:] == 1)
    r = O.filter(iq, O.OracleConfig(nz, nx, nt, 1, 1, all_ones_window=1, thresh_mode=O.T_SIGMOID,
                                    k_src=O.T_NCC, beta=2.0))
    assert int(r.k[0]) == kst
    np.testing.assert_allclose(r.wt[0], 1.0 / (1.0 + np.exp(-2.0 * (np.arange(1, nt + 1) - kst))), rtol=1e-15)


@pytest.mark.parametrize("nt,ks", [(10, [5]), (7, [3, 4]), (6, [3]), (2, [1])])
def test_ncc_cutoff_range(nt, ks):
    """fn = min(5, Nt/2) neighbours on each side: the curve exists exactly for fn <= k <= Nt - fn."""
    rng = np.random.default_rng(nt)
    iq = (rng.standard_normal((nt, 8, 6)) + 1j * rng.standard_normal((nt, 8, 6))).astype(np.complex64)
    k, curve = O.ncc_curve(iq, O.OracleConfig(8, 6, nt, 1, 1, all_ones_window=1), 0)
    assert [i + 1 for i in np.nonzero(np.isfinite(curve))[0]] == ks
    assert k in ks
