"""Launch tuning (lcf_plan_get_tuning / lcf_plan_set_tuning / lcf_plan_autotune): every
tunable value keeps the results within the FP64 oracle's tolerances, the distributed EVD
runs on clusters of 4 and of 8 CTAs, and the autotuner's choice is cached by key."""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

from synth import SMALL_96x64x32, generate_packet  # noqa: E402
from test_parity_gpu import (ALPHA_TOL, EIG_TOL, PD_TOL, L, assert_cutoffs, configs, near_tie,  # noqa: E402
                             rand_iq, rel_l2, check_eigs)


def fast(cfg):
    lib = L()
    cfg.gram_path, cfg.project_path, cfg.evd_path = lib.LCF_PATH_TC, lib.LCF_PATH_TC, lib.LCF_EVD_PAIR
    return cfg


def run_with(plan, iq):
    import torch
    d = torch.from_numpy(iq).cuda()
    pd = plan.filter(d)
    torch.cuda.synchronize()
    return pd.cpu().numpy().astype(np.float64), plan.debug()


def check_against(ora, oc, pd, dbg, plan):
    lib = L()
    st, _ = plan.status()
    assert st == lib.LCF_OK
    flips = [int(k) for k in np.nonzero(dbg["k"] != ora.k)[0]]
    assert all(near_tie(oc, ora.lam[k], dbg["lam"][k], int(dbg["k"][k]), int(ora.k[k])) for k in flips), flips
    if not flips:
        assert rel_l2(pd, ora.pd) <= PD_TOL
    assert check_eigs(dbg["lam"], ora.lam) <= EIG_TOL
    assert float(np.max(np.abs(dbg["alpha"] - ora.alpha) / ora.alpha)) <= ALPHA_TOL


@pytest.mark.parametrize("path", ["plain", "fast"])
def test_every_split_value_within_tolerance(path):
    import oracle as O
    lib = L()
    iq = generate_packet(SMALL_96x64x32, seed=3)
    cfg, oc = configs(96, 64, 32, 3, 3, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0)
    if path == "fast":
        fast(cfg)
    ora = O.filter(iq, oc)
    plan = lib.Plan(cfg)
    for v in (1, 2, 7, 64):
        plan.set_tuning(gram_splits=v, simt_gram_splits=v, aug_splits=v, q_splits=v, basis_splits=v)
        pd, dbg = run_with(plan, iq)
        print(path, v, rel_l2(pd, ora.pd))
        check_against(ora, oc, pd, dbg, plan)


@pytest.mark.parametrize("nt", [200, 201, 213, 224])
def test_distributed_evd_cluster_sizes(nt):
    """Clusters of 4 and of 8 CTAs per window give the oracle's results where both are
    allowed (8 is what packets beyond 224 frames need)."""
    import oracle as O
    lib = L()
    nz, nx = 36, 30
    iq = rand_iq(14, nt, nz, nx)
    cfg, oc = configs(nz, nx, nt, 2, 2, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0)
    fast(cfg)
    ora = O.filter(iq, oc)
    plan = lib.Plan(cfg)
    assert plan.tuning().evd_cluster == 4
    for C in (4, 8):
        plan.set_tuning(evd_cluster=C)
        pd, dbg = run_with(plan, iq)
        print(nt, C, rel_l2(pd, ora.pd), check_eigs(dbg["lam"], ora.lam))
        check_against(ora, oc, pd, dbg, plan)


def test_invalid_tunings_rejected():
    lib = L()
    plan = lib.Plan.make(32, 32, 16, 2, 2)
    for kw in ({"gram_splits": 0}, {"aug_splits": 65}, {"evd_cluster": 5}, {"evd_cluster": 2}):
        with pytest.raises(lib.LcfError) as e:
            plan.set_tuning(**kw)
        assert e.value.status == lib.LCF_EINVAL
    long_plan = lib.Plan.make(20, 20, 300, 1, 1)
    with pytest.raises(lib.LcfError):
        long_plan.set_tuning(evd_cluster=4)      # 4 CTAs cannot hold a 300-frame window
    mid_plan = lib.Plan.make(20, 20, 129, 1, 1)
    with pytest.raises(lib.LcfError):
        mid_plan.set_tuning(evd_cluster=8)       # refused below 200 frames
    with pytest.raises(lib.LcfError):
        long_plan.set_tuning(gram_splits=2)      # tile pairs take whole windows


def test_autotune_and_cache(tmp_path):
    import torch
    import oracle as O
    lib = L()
    iq = generate_packet(SMALL_96x64x32, seed=4)
    cfg, oc = configs(96, 64, 32, 3, 3, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0)
    fast(cfg)
    cache = tmp_path / "tune.txt"
    d = torch.from_numpy(iq).cuda()
    a = lib.Plan(cfg)
    assert a.autotune(d, cache) is False
    ta = a.tuning().as_dict()
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].split()[0].split("|")[1:6] == ["96", "64", "32", "3", "3"]
    b = lib.Plan(cfg)
    assert b.autotune(d, cache) is True
    assert b.tuning().as_dict() == ta
    assert len(cache.read_text().splitlines()) == 1
    print("tuned", ta)
    ora = O.filter(iq, oc)
    pd, dbg = run_with(b, iq)
    check_against(ora, oc, pd, dbg, b)
