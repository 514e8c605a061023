"""Learned cutoff rule: GPU training kernels against the FP64 reference (oracle/mlp.py),
then a network trained on the GPU replacing method 1 in a plan with a capped EVD.

Tolerances: loss 1e-5 relative; gradients 1e-4 relative per tensor (FP32 GEMMs vs
FP64); AdamW 1e-6 relative; learned PD vs the converged method-1 PD: mean |dB| over
pixels within 30 dB of the image maximum <= 0.5 dB.
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

from oracle import mlp as OM  # noqa: E402
from synth import Recipe, generate_packet  # noqa: E402
from test_parity_gpu import L  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("nt,hidden,batch", [(32, 64, 96), (100, 256, 257), (7, 33, 5)])
def test_loss_and_gradients_match_fp64(nt, hidden, batch):
    import torch
    lib = L()
    from paper_2405_11105_b300 import learned
    rng = np.random.default_rng(nt)
    net = lib.Mlp(nt, hidden=hidden, max_batch=512)
    flat = learned.init_params(nt + 2, hidden, nt, seed=nt)
    flat[net.nparams - nt:] = rng.standard_normal(nt).astype(np.float32) * 0.1   # nonzero output bias
    net.set_params(flat)
    X = rng.uniform(0, 1, (batch, nt + 2)).astype(np.float32)
    K = rng.integers(0, nt, batch).astype(np.int32)
    loss = net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(K).cuda())
    p = OM.unflatten(flat.astype(np.float64), nt + 2, hidden, nt)
    loss_o, g_o = OM.loss_and_grads(p, X.astype(np.float64), K)
    g = OM.unflatten(net.grads().astype(np.float64), nt + 2, hidden, nt)
    errs = {name: rel(g[name], g_o[name]) for name in g_o}
    print("loss", loss, loss_o, "grad rel errs", errs)
    assert abs(loss - loss_o) / loss_o <= 1e-5
    assert max(errs.values()) <= 1e-4
    logits = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    z_o, _ = OM.forward(p, X.astype(np.float64))
    assert rel(logits, z_o) <= 1e-5


def test_adamw_matches_fp64():
    import torch
    lib = L()
    from paper_2405_11105_b300 import learned
    nt, hidden, batch = 24, 48, 64
    rng = np.random.default_rng(5)
    net = lib.Mlp(nt, hidden=hidden, max_batch=batch)
    flat = learned.init_params(nt + 2, hidden, nt, seed=1)
    net.set_params(flat)
    X = torch.from_numpy(rng.uniform(0, 1, (batch, nt + 2)).astype(np.float32)).cuda()
    K = torch.from_numpy(rng.integers(0, nt, batch).astype(np.int32)).cuda()
    p = OM.unflatten(flat.astype(np.float64), nt + 2, hidden, nt)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    for t in (1, 2, 3):
        net.loss_grad(X, K)
        g = OM.unflatten(net.grads().astype(np.float64), nt + 2, hidden, nt)
        net.adamw(1e-3, wd=0.01)
        p, m, v = OM.adamw_step(p, g, m, v, t, 1e-3, wd=0.01)
        # continue the reference from the device's parameters so that only one step's rounding is compared
        got = OM.unflatten(net.params().astype(np.float64), nt + 2, hidden, nt)
        err = max(rel(got[n], p[n]) for n in p)
        assert err <= 1e-6, (t, err)
        p = got


def test_bad_label_gives_nan_loss_and_no_gradient():
    import torch
    lib = L()
    net = lib.Mlp(8, hidden=16, max_batch=4)
    from paper_2405_11105_b300 import learned
    net.set_params(learned.init_params(10, 16, 8, seed=2))
    X = torch.rand((2, 10), device="cuda")
    loss = net.loss_grad(X, torch.tensor([8, 8], dtype=torch.int32, device="cuda"))
    assert np.isnan(loss)
    assert np.all(net.grads() == 0)


SMALL = Recipe(64, 64, 32, n_vessels=(2, 6), width_px=(2.0, 8.0), phi_rad=(0.05, 1.0), tbr_db=(40.0, 55.0),
               noise_db=-60.0, motion_amp_px=(0.0, 1.0))


@pytest.fixture(scope="module")
def trained():
    from paper_2405_11105_b300 import learned
    full, fast = learned.make_plans(64, 64, 32, 4, 4, fast_sweeps=2)
    train_p = [generate_packet(SMALL, seed=100 + i) for i in range(160)]
    test_p = [generate_packet(SMALL, seed=900 + i) for i in range(12)]
    Xtr, Ktr = learned.collect(train_p, full, fast, 4, 4)
    Xte, Kte = learned.collect(test_p, full, fast, 4, 4)
    losses = []
    net = learned.train(Xtr, Ktr, 32, hidden=128, epochs=40, batch=256, lr=3e-3, log=lambda e, l: losses.append(l))
    return learned, net, (Xtr, Ktr, Xte, Kte), test_p, losses


def test_training_reduces_loss_and_learns_the_cutoff(trained):
    learned, net, (Xtr, Ktr, Xte, Kte), _, losses = trained
    acc_tr, _ = learned.accuracy(net, Xtr, Ktr)
    acc_te, pred = learned.accuracy(net, Xte, Kte)
    base = float(np.mean(Kte == np.bincount(Ktr).argmax()))
    near = float(np.mean(np.abs(pred - Kte) <= 1))
    print("loss first/last", losses[0], losses[-1], "train acc", acc_tr, "held-out acc", acc_te,
          "held-out within 1", near, "majority-class acc", base)
    assert losses[-1] < 0.5 * losses[0]
    assert acc_te >= base + 0.25
    assert near >= 0.75


def test_learned_plan_matches_converged_rule_in_db(trained):
    """The learned rule on a 2-sweep EVD against method 1 on the converged EVD: PD within
    0.5 dB on average, and what the cap saves in EVD time."""
    import torch
    learned, net, _, test_p, _ = trained
    lib = L()
    full, _ = learned.make_plans(64, 64, 32, 4, 4, fast_sweeps=2)
    lp = lib.Plan.make(64, 64, 32, 4, 4, thresh_mode=lib.LCF_T_LEARNED, k_src=lib.LCF_T_CURVATURE, beta_src=1.0,
                       gram_path=lib.LCF_PATH_TC, project_path=lib.LCF_PATH_TC, evd_path=lib.LCF_EVD_PAIR,
                       max_sweeps=2)
    lp.set_mlp(net, p_min=0.5)
    errs, agree, fb = [], [], 0
    for iq in test_p:
        d = torch.from_numpy(iq).cuda()
        a = full.filter(d).cpu().numpy().astype(np.float64)
        b = lp.filter(d).cpu().numpy().astype(np.float64)
        st, flags = lp.status()
        assert st in (lib.LCF_OK, lib.LCF_ENOCONV)      # the sweep cap is the point of the learned plan
        fb += int(np.sum(np.asarray(flags) & lib.LCF_WFLAG_FALLBACK != 0))
        agree.append(np.mean(full.debug()["k"] == lp.debug()["k"]))
        m = a >= a.max() * 1e-3
        errs.append(np.mean(np.abs(10 * np.log10(b[m] / a[m]))))
    # EVD stage time, converged rule vs learned rule with the cap
    d = torch.from_numpy(test_p[0]).cuda()
    t = {}
    for name, plan in (("full", full), ("learned", lp)):
        for _ in range(3):
            plan.filter(d)
        plan.profile(True)
        for _ in range(10):
            plan.filter(d)
        stg, n = plan.profile_read()
        plan.profile(False)
        t[name] = stg["evd"] / n
    print("mean |dB|", np.mean(errs), "max per packet", np.max(errs), "cutoff agreement", np.mean(agree),
          "fallback windows", fb, "EVD ms converged / learned", t)
    assert np.mean(errs) <= 0.5
    assert t["learned"] < t["full"]


def bf16_round(w):
    """FP32 -> nearest bf16 value (ties to even), as FP32: the plan stores its weights so."""
    u = np.ascontiguousarray(w, np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def test_in_kernel_inference_matches_fp64_forward(trained):
    """The learned rule inside the EVD kernel against the FP64 network of oracle/mlp.py on the
    same capped spectra: the kernel's features equal the reference features computed from the
    plan's eigenvalues (<= 1e-6), its logits equal the FP64 forward pass with the plan's bf16
    weights and FP32 biases (<= 1e-4 relative to the logit scale: FP32 accumulation), and every
    window's cutoff is the logits' argmax (or the fallback rule where the top softmax
    probability is below p_min), except at logit near-ties."""
    import torch
    learned, net, _, test_p, _ = trained
    lib = L()
    lp = lib.Plan.make(64, 64, 32, 4, 4, thresh_mode=lib.LCF_T_LEARNED, k_src=lib.LCF_T_CURVATURE, beta_src=1.0,
                       max_sweeps=2)
    lp.set_mlp(net, p_min=0.5)
    p = OM.unflatten(net.params().astype(np.float64), 34, net.hidden, 32)
    for name in ("W1", "W2", "W3", "W4"):
        p[name] = bf16_round(p[name]).astype(np.float64)
    pz, px = learned.window_centres(4, 4)
    worst_f, worst_z, checked, ties = 0.0, 0.0, 0, 0
    for iq in test_p[:6]:
        lp.filter(torch.from_numpy(iq).cuda())
        dbg = lp.debug()
        st, flags = lp.status()
        f_gpu, z_gpu = lp.debug_learned()
        X = np.stack([OM.features(dbg["lam"][w], pz[w], px[w]) for w in range(16)])
        worst_f = max(worst_f, float(np.max(np.abs(f_gpu - X))))
        z_ref, _ = OM.forward(p, X)
        scale = np.max(np.abs(z_ref), axis=1, keepdims=True)
        worst_z = max(worst_z, float(np.max(np.abs(z_gpu - z_ref) / scale)))
        for w in range(16):
            top2 = np.sort(z_ref[w])[-2:]
            if top2[1] - top2[0] <= 1e-4 * scale[w, 0]:
                ties += 1
                continue
            e = np.exp(z_ref[w] - z_ref[w].max())
            pmax = 1.0 / e.sum()
            fell_back = bool(flags[w] & lib.LCF_WFLAG_FALLBACK)
            if abs(pmax - 0.5) > 1e-4:
                assert fell_back == (pmax < 0.5), (w, pmax, flags[w])
            if not fell_back:
                assert int(dbg["k"][w]) == int(np.argmax(z_ref[w])), (w, dbg["k"][w], np.argmax(z_ref[w]))
            checked += 1
    print("feature max abs err", worst_f, "logit max rel err", worst_z, "windows checked", checked,
          "logit near-ties", ties)
    assert worst_f <= 1e-6
    assert worst_z <= 1e-4
    assert checked >= 80


def test_learned_rule_against_network_off(trained):
    """What the network buys: the same 2-sweep plan with the network switched off (p_min > 1,
    so every window takes method 1 on the capped spectrum) against the learned plan, both
    judged by method 1 on the converged EVD (mean |dB| over pixels within 30 dB of the
    maximum) and by cutoff agreement."""
    import torch
    learned, net, _, test_p, _ = trained
    lib = L()
    full, _ = learned.make_plans(64, 64, 32, 4, 4, fast_sweeps=2)
    arms = {}
    for name, pmin in (("learned", 0.5), ("network_off", 1.01)):
        lp = lib.Plan.make(64, 64, 32, 4, 4, thresh_mode=lib.LCF_T_LEARNED, k_src=lib.LCF_T_CURVATURE,
                           beta_src=1.0, max_sweeps=2)
        lp.set_mlp(net, p_min=pmin)
        errs, agree, fb = [], [], 0
        for iq in test_p:
            d = torch.from_numpy(iq).cuda()
            a = full.filter(d).cpu().numpy().astype(np.float64)
            kf = full.debug()["k"]
            b = lp.filter(d).cpu().numpy().astype(np.float64)
            st, flags = lp.status()
            fb += int(np.sum((np.asarray(flags) & lib.LCF_WFLAG_FALLBACK) != 0))
            agree.append(np.mean(kf == lp.debug()["k"]))
            m = a >= a.max() * 1e-3
            errs.append(np.mean(np.abs(10 * np.log10(b[m] / a[m]))))
        arms[name] = {"mean_db": float(np.mean(errs)), "worst_db": float(np.max(errs)),
                      "cutoff_agreement": float(np.mean(agree)), "fallback_windows": fb}
    print(arms)
    assert arms["network_off"]["fallback_windows"] == 16 * len(test_p)
    assert arms["learned"]["mean_db"] <= 0.5


def test_learned_rule_fallback_and_requirements(trained):
    import torch
    learned, net, _, test_p, _ = trained
    lib = L()
    d = torch.from_numpy(test_p[0]).cuda()
    mk = lambda **kw: lib.Plan.make(64, 64, 32, 4, 4, evd_path=lib.LCF_EVD_PAIR, max_sweeps=2, **kw)
    lp = mk(thresh_mode=lib.LCF_T_LEARNED, k_src=lib.LCF_T_MEDIAN, beta_src=1.43)
    with pytest.raises(lib.LcfError):
        lp.filter(d)                       # no network set yet
    lp.set_mlp(net, p_min=1.01)            # never confident: every window falls back to k_src
    a = lp.filter(d).cpu().numpy()
    st, flags = lp.status()
    assert np.all(np.asarray(flags) & lib.LCF_WFLAG_FALLBACK)
    ref = mk(thresh_mode=lib.LCF_T_MEDIAN, beta=1.43)
    b = ref.filter(d).cpu().numpy()
    assert np.array_equal(lp.debug()["k"], ref.debug()["k"])
    assert np.allclose(a, b, rtol=1e-6, atol=0)
    with pytest.raises(lib.LcfError):
        lib.Plan.make(64, 64, 32, 4, 4, thresh_mode=lib.LCF_T_LEARNED, evd_path=lib.LCF_EVD_CTA)
    other = lib.Mlp(16, hidden=32)
    with pytest.raises(lib.LcfError):
        lp.set_mlp(other)                  # wrong packet length
