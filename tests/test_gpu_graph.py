"""encode_step replays a CUDA graph of its first call when the same call comes again: the replayed
iterations must give the same bits as the same iterations launched eagerly (kernel timing forces
the eager path), for one- and multi-iteration calls, with and without loss records."""
import pytest
import torch

from paper_2605_02726_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(cc, H, W, n_calls, n_iters, eager, with_rd):
    img = torch.tensor(inputs.image(H, W, seed=5), device="cuda")
    lat, par = inputs.initial_state(H, W, seed=6)
    st = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"))
    ws = cc.workspace(H, W)
    hp = cc.hparams(lam=2e-3, seed=9)
    rd = torch.zeros(n_iters, 3, dtype=torch.float64, device="cuda") if with_rd else None
    recs = []
    if eager:
        cc.timing_enable(cc.KERNEL_ARM, 64)  # more launches than the calls make: every call eager
    try:
        for _ in range(n_calls):
            cc.encode_step(img, st, n_iters, H=H, W=W, hp=hp, ws=ws, rd=rd)
            if with_rd:
                recs.append(rd.clone())
        torch.cuda.synchronize()
    finally:
        if eager:
            cc.timing_disable()
    return st, recs


@pytest.mark.parametrize("n_iters,with_rd", [(1, False), (1, True), (3, True)])
def test_graph_replay_is_bitwise_the_eager_launches(cc, n_iters, with_rd):
    H, W = 40, 56
    a, ra = _run(cc, H, W, 4, n_iters, eager=True, with_rd=with_rd)
    b, rb = _run(cc, H, W, 4, n_iters, eager=False, with_rd=with_rd)
    for f in ("latents", "params", "m_lat", "v_lat", "m_par", "v_par", "step"):
        assert torch.equal(getattr(a, f), getattr(b, f)), f
    for x, y in zip(ra, rb):
        assert torch.equal(x, y)
