"""lcf_filter as one CUDA graph launch per packet (lcf_config.graph): every image equals
the stage-by-stage launch's bit for bit, for more (input, output) pairs than the plan keeps
graphs (the oldest are replaced), and a graph plan's launch count grows by the same number
of kernels per packet."""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

from synth import SMALL_96x64x32, generate_frames  # noqa: E402
from test_parity_gpu import L  # noqa: E402


@pytest.mark.parametrize("mode", ["LCF_T_CURVATURE", "LCF_T_NCC"])
def test_graph_plan_matches_stage_launches(mode):
    import torch
    lib = L()
    frames = generate_frames(SMALL_96x64x32, 32 + 19 * 4, seed=8)
    d = torch.from_numpy(frames).cuda()
    pk = [d[i * 4:i * 4 + 32].contiguous() for i in range(20)]
    kw = dict(thresh_mode=getattr(lib, mode), beta=1.0)
    ref = lib.Plan.make(96, 64, 32, 3, 3, **kw)
    gp = lib.Plan.make(96, 64, 32, 3, 3, graph=1, **kw)
    want = [ref.filter(p).cpu() for p in pk]
    outs = [torch.empty((96, 64), dtype=torch.float32, device="cuda") for _ in range(20)]
    for rnd in range(2):   # 20 pairs > 16 kept graphs: the second round recaptures some
        for i in range(20):
            gp.filter(pk[i], out=outs[i])
        torch.cuda.synchronize()
        for i in range(20):
            assert torch.equal(outs[i].cpu(), want[i]), (rnd, i)
    n0 = gp.launch_count()
    gp.filter(pk[3], out=outs[3])
    torch.cuda.synchronize()
    n1 = ref.launch_count()
    ref.filter(pk[3])
    torch.cuda.synchronize()
    assert gp.launch_count() - n0 == ref.launch_count() - n1 > 0
    st, _ = gp.status()
    assert st == lib.LCF_OK
