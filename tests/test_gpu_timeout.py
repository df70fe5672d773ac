"""Failure detection without a GPU fault: the entropy model's waits on its tensor-core work are
bounded.  The test hook withholds the first MMA commit, so that every wait genuinely runs out
(about a second); the kernel frees its Tensor Memory and ends, the blocking rate-distortion call
reports CC_ERR_TIMEOUT with a NaN loss, and the next call on the same context is correct again."""
import math

import pytest
import torch

from paper_2605_02726_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_recovers(cc):
    H, W = 24, 40
    img = torch.tensor(inputs.image(H, W, seed=1), device="cuda")
    lat, par = inputs.random_state(H, W, seed=2)
    gl, gp = torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda")
    ws = cc.workspace(H, W)
    hp = cc.hparams(lam=1e-2, seed=3)
    before = cc.rate_distortion(img, gl, gp, H=H, W=W, hp=hp, ws=ws)
    raw = cc.raw()
    assert raw.coolchic_test_inject_stall(1) == 0
    try:
        with pytest.raises(cc.CoolChicError) as err:
            cc.rate_distortion(img, gl, gp, H=H, W=W, hp=hp, ws=ws)
        assert "(-4)" in str(err.value) and "ran out" in str(err.value)
        # an asynchronous call: the loss record is NaN
        rd = torch.zeros(1, 3, dtype=torch.float64, device="cuda")
        st = cc.EncoderState(gl, gp)
        cc.timing_enable(cc.KERNEL_ARM, 4)  # eager launches (no replay of a graph captured earlier)
        try:
            cc.encode_step(img, st, 1, H=H, W=W, hp=hp, ws=ws, rd=rd)
            torch.cuda.synchronize()
        finally:
            cc.timing_disable()
        assert math.isnan(rd[0, 0].item())
    finally:
        raw.coolchic_test_inject_stall(0)
    after = cc.rate_distortion(img, gl, gp, H=H, W=W, hp=hp, ws=ws)
    assert after == before
