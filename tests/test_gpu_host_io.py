"""The host-buffer encoder entry point and the pipe-peak measurement, through the C ABI.

coolchic_encode_step_host copies a host image into its workspace, runs the iterations of
coolchic_encode_step and returns the last loss record: the state it leaves and the record it
returns are bitwise those of the device-pointer call on the same inputs."""
import numpy as np
import pytest
import torch

from paper_2605_02726_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_iters", [1, 3, 6])
def test_host_entry_point_is_bitwise_the_device_call(cc, n_iters):
    H, W = 72, 96
    img = inputs.image(H, W, seed=31)
    lat, par = inputs.random_state(H, W, seed=32)
    hp = cc.hparams(lam=1e-2, seed=5)
    dev_state = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"), step=4)
    host_state = dev_state.clone()
    rd = torch.zeros(n_iters, 3, dtype=torch.float64, device="cuda")
    cc.encode_step(torch.tensor(img, device="cuda"), dev_state, n_iters, H=H, W=W, hp=hp, ws=cc.workspace(H, W), rd=rd)
    host_img = torch.tensor(img).pin_memory()
    host_rd = torch.zeros(3, dtype=torch.float64).pin_memory()
    cc.encode_step_host(host_img, host_state, n_iters, H=H, W=W, hp=hp, ws=cc.workspace(H, W, host_io=True),
                        rd_host=host_rd)
    torch.cuda.synchronize()
    assert torch.equal(dev_state.latents, host_state.latents)
    assert torch.equal(dev_state.params, host_state.params)
    assert torch.equal(dev_state.v_lat, host_state.v_lat)
    assert int(host_state.step.item()) == 4 + n_iters
    np.testing.assert_array_equal(host_rd.numpy(), rd[-1].cpu().numpy())


@pytest.mark.parametrize("pinned", [True, False])
def test_host_entry_point_reads_the_image_of_each_call(cc, pinned):
    """Calls replayed from the library's graph (the image copy is a node of it, beside the first
    kernels) and calls from pageable memory (no graph: the copy cannot be captured; the record
    comes back by a copy instead of the kernel's direct write) read the host image as it is at
    each call: two calls with different contents in the same host buffer match the device path."""
    H, W = 40, 56
    lat, par = inputs.random_state(H, W, seed=41)
    hp = cc.hparams(lam=1e-2, seed=6)
    dev_state = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"))
    host_state = dev_state.clone()
    ws, ws_io = cc.workspace(H, W), cc.workspace(H, W, host_io=True)
    host_img = torch.zeros(3, H, W)
    host_rd = torch.zeros(3, dtype=torch.float64)
    if pinned:
        host_img, host_rd = host_img.pin_memory(), host_rd.pin_memory()
    rd = torch.zeros(1, 3, dtype=torch.float64, device="cuda")
    for call in range(3):
        img = inputs.image(H, W, seed=50 + call)
        cc.encode_step(torch.tensor(img, device="cuda"), dev_state, 1, H=H, W=W, hp=hp, ws=ws, rd=rd)
        host_img.copy_(torch.tensor(img))
        cc.encode_step_host(host_img, host_state, 1, H=H, W=W, hp=hp, ws=ws_io, rd_host=host_rd)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host_rd.numpy(), rd[0].cpu().numpy())
    assert torch.equal(dev_state.latents, host_state.latents)
    assert torch.equal(dev_state.params, host_state.params)


def test_host_entry_point_needs_the_host_io_workspace(cc):
    H, W = 16, 16
    lat, par = inputs.random_state(H, W, seed=1)
    st = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"))
    with pytest.raises(cc.CoolChicError, match="workspace too small"):
        cc.encode_step_host(torch.zeros(3, H, W), st, 1, H=H, W=W, hp=cc.hparams(), ws=cc.workspace(H, W))
    assert int(st.step.item()) == 0


@pytest.mark.parametrize("which", [0, 1])
def test_measured_pipe_peaks_are_plausible(cc, which):
    """The FP32 FMA ceiling lies between half and 105% of the unit-count figure (SMs x 128 lanes x
    2 FLOP at the 2070 MHz maximum SM clock); the TF32 mma.sync ceiling is positive and finite."""
    tf, ms = cc.measure_peak(which)
    assert ms >= 2.0 * 0.9 and np.isfinite(tf) and tf > 0
    if which == cc.PEAK_FP32_FMA:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        unit = sms * 128 * 2 * 2070e6 / 1e12
        assert 0.5 * unit < tf < 1.05 * unit, (tf, unit)
