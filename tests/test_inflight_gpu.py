"""Several packets in flight (lcf_config.inflight, lcf_filter_many, rotating lcf_filter_host_async),
through the C ABI.

The lanes run the same kernels on their own workspaces, so every image must equal, bit for bit,
the one lcf_filter gives for the same packet; the first image is also checked against the FP64
oracle at the standard tolerance (PD rel L2 <= 1e-3).
"""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

import oracle as O  # noqa: E402
from synth import SMALL_96x64x32, generate_packet  # noqa: E402
from test_parity_gpu import PD_TOL, L, configs, rel_l2  # noqa: E402


def packets(npk, seed0=50):
    return np.stack([generate_packet(SMALL_96x64x32, seed=seed0 + i) for i in range(npk)])


@pytest.mark.parametrize("evd", ["LCF_EVD_PAIR", "LCF_EVD_OS"])
@pytest.mark.parametrize("inflight", [1, 2, 3, 4])
def test_filter_many_equals_filter(evd, inflight):
    import torch
    lib = L()
    iq = torch.from_numpy(packets(7)).cuda()
    single = lib.Plan.make(96, 64, 32, 3, 3, evd_path=getattr(lib, evd))
    ref = torch.stack([single.filter(iq[p]) for p in range(iq.shape[0])])
    many = lib.Plan.make(96, 64, 32, 3, 3, evd_path=getattr(lib, evd), inflight=inflight)
    out = many.filter_many(iq)
    out2 = many.filter_many(iq)   # the same buffers again
    torch.cuda.synchronize()
    assert torch.equal(out, ref) and torch.equal(out2, ref)
    assert many.workspace_bytes >= inflight * single.workspace_bytes * 0.99
    cfg, oc = configs(96, 64, 32, 3, 3, thresh_mode=lib.LCF_T_CURVATURE, beta=1.0)   # the defaults' rule
    assert (cfg.thresh_mode, cfg.beta) == (single.cfg.thresh_mode, single.cfg.beta)
    ora = O.filter(iq[0].cpu().numpy(), oc)
    assert rel_l2(out[0].cpu().numpy().astype(np.float64), ora.pd) <= PD_TOL


def test_filter_many_orders_against_the_stream():
    """Work queued on the caller's stream before the call is seen (the input written there),
    and work queued after it sees every image."""
    import torch
    lib = L()
    src = torch.from_numpy(packets(5, 80)).cuda()
    plan = lib.Plan.make(96, 64, 32, 3, 3, inflight=3)
    ref = torch.stack([plan.filter(src[p]) for p in range(5)])
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        iq = torch.zeros_like(src)
        torch.cuda._sleep(20_000_000)        # a long kernel ahead of the copy
        iq.copy_(src)
        out = plan.filter_many(iq, stream=s)
        total = out.sum(dim=(1, 2))
    s.synchronize()
    assert torch.equal(out, ref)
    assert torch.allclose(total, ref.sum(dim=(1, 2)))


def test_host_async_rotates_over_lanes():
    import torch
    lib = L()
    pk = packets(6, 90)
    plan = lib.Plan.make(96, 64, 32, 3, 3, evd_path=lib.LCF_EVD_OS, inflight=3)
    ref = [plan.filter(torch.from_numpy(pk[p]).cuda()).cpu().numpy() for p in range(6)]
    hin = [torch.from_numpy(pk[p]).pin_memory() for p in range(6)]
    hout = [torch.empty((96, 64), dtype=torch.float32).pin_memory() for _ in range(6)]
    for p in range(6):
        plan.filter_host_async(hin[p], hout[p])
    plan.sync()
    for p in range(6):
        assert np.array_equal(hout[p].numpy(), ref[p])


def test_inflight_validation():
    lib = L()
    for v, want in ((0, lib.LCF_OK), (4, lib.LCF_OK), (5, lib.LCF_EINVAL), (-1, lib.LCF_EINVAL)):
        c = lib.lcf_config_default(32, 32, 16, 2, 2)
        c.inflight = v
        try:
            lib.Plan(c).close()
            got = lib.LCF_OK
        except lib.LcfError as e:
            got = e.status
        assert got == want, (v, got)
