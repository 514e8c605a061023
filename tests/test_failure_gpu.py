"""Failure detection without a GPU fault: a bounded device-side wait that runs out
(on a flag nothing sets) reports LCF_ETIMEOUT, and the context stays usable."""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

from test_parity_gpu import L, rand_iq  # noqa: E402


def test_bounded_wait_times_out_and_context_survives():
    import torch
    lib = L()
    st, waited = lib.selftest_wait_timeout(0.05)
    assert st == lib.LCF_ETIMEOUT
    assert 0.04 <= waited <= 1.0
    # the context is still usable: a plan runs normally afterwards
    plan = lib.Plan.make(24, 20, 16, 2, 2, thresh_mode=lib.LCF_T_FIXED, k_fixed=1)
    pd = plan.filter(torch.from_numpy(rand_iq(1, 16, 24, 20)).cuda())
    assert plan.status()[0] == lib.LCF_OK
    assert np.isfinite(pd.cpu().numpy()).all()
    assert lib.selftest_wait_timeout(3.0)[0] == lib.LCF_EINVAL   # limits above 2 s are refused
