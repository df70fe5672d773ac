"""Batched encoder iterations: one set of launches for many images of different sizes.

Each job of a batch must follow the same trajectory as the single-image path: bitwise with the
default schedule (same CTA counts, hence the same summation order), within the loss tolerance
with another schedule (only the order of the parameter-gradient sums changes)."""
import numpy as np
import pytest
import torch

from paper_2605_02726_gb300 import inputs

pytestmark = pytest.mark.gpu

SIZES = [(64, 64), (37, 53), (96, 40), (8, 8), (130, 67)]


def _jobs(cc, seed0=300, lam=1e-2):
    jobs = []
    for j, (H, W) in enumerate(SIZES):
        img = torch.tensor(inputs.image(H, W, seed=seed0 + j), device="cuda")
        lat, par = inputs.random_state(H, W, seed=seed0 + 50 + j)
        st = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"), step=j)
        jobs.append((img, st, cc.hparams(lam=lam * (1 + j), seed=11 + j)))
    return jobs


def _single(cc, jobs, n):
    out = []
    for img, st, hp in jobs:
        s = st.clone()
        H, W = img.shape[1], img.shape[2]
        rd = torch.zeros(n, 3, dtype=torch.float64, device="cuda")
        cc.encode_step(img, s, n, H=H, W=W, hp=hp, ws=cc.workspace(H, W), rd=rd)
        out.append((s, rd))
    torch.cuda.synchronize()
    return out


def test_batch_default_schedule_is_bitwise_the_single_path(cc):
    jobs = _jobs(cc)
    n = 3
    ref = _single(cc, jobs, n)
    bjobs = [(img, st.clone(), hp) for img, st, hp in jobs]
    be = cc.BatchEncoder(bjobs, rd_capacity=n)
    be.step(n)
    torch.cuda.synchronize()
    rec = be.records().cpu().numpy()
    for j, ((_, st, _), (rs, rrd)) in enumerate(zip(bjobs, ref)):
        assert torch.equal(st.latents, rs.latents), j
        assert torch.equal(st.params, rs.params), j
        assert torch.equal(st.m_par, rs.m_par) and torch.equal(st.v_lat, rs.v_lat), j
        assert int(st.step.item()) == int(rs.step.item()) == j + n
        np.testing.assert_array_equal(rec[:, j, :], rrd.cpu().numpy())
    be.close()


def test_batch_other_schedule_and_graph_replay(cc):
    jobs = _jobs(cc, seed0=400)
    ref = _single(cc, jobs, 2)
    bjobs = [(img, st.clone(), hp) for img, st, hp in jobs]
    be = cc.BatchEncoder(bjobs, schedule=cc.Schedule(0.25, 0.5, 0.5, 0.5), rd_capacity=1)
    g = be.graph(1)
    recs = []
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        recs.append(be.records().cpu().numpy()[0].copy())
    for j, (rs, rrd) in enumerate(ref):
        r = rrd.cpu().numpy()
        for it in range(2):
            np.testing.assert_allclose(recs[it][j], r[it], rtol=1e-5, atol=0)
        assert int(bjobs[j][1].step.item()) == j + 2
    be.close()


def test_autotuner_returns_a_measured_candidate(cc):
    from paper_2605_02726_gb300 import autotune
    jobs = _jobs(cc, seed0=500)
    before = [st.latents.clone() for _, st, _ in jobs]
    sched, timings = autotune.tune(jobs, repeats=2)
    assert len(timings) == len(autotune.CANDIDATES) and all(t > 0 for t in timings.values())
    assert sched.as_tuple() == min(timings, key=timings.get)
    for (_, st, _), b in zip(jobs, before):  # tuning runs on clones
        assert torch.equal(st.latents, b)


def test_batch_with_the_largest_workload_sizes(cc):
    """A batch in the shape of the mixed-size workload: a 1536x1024 and a 1024x1024 job beside small
    ones.  One iteration: each job bitwise equal to the single-image path, and the largest job's
    loss record, forward and gradient against the FP64 oracle."""
    import oracle
    from tests.test_gpu_fullsize import _parity
    sizes = [(1536, 1024), (1024, 1024), (64, 64), (37, 53)]
    jobs = []
    for j, (H, W) in enumerate(sizes):
        img = torch.tensor(inputs.image(H, W, seed=700 + j, texture_sigma=0.02), device="cuda")
        lat, par = inputs.random_state(H, W, seed=750 + j)
        st = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"), step=2)
        jobs.append((img, st, cc.hparams(lam=1e-3, seed=77)))
    ref = _single(cc, jobs, 1)
    bjobs = [(img, st.clone(), hp) for img, st, hp in jobs]
    be = cc.BatchEncoder(bjobs, rd_capacity=1)
    be.step(1)
    torch.cuda.synchronize()
    rec = be.records().cpu().numpy()
    for j, ((_, st, _), (rs, rrd)) in enumerate(zip(bjobs, ref)):
        assert torch.equal(st.latents, rs.latents), j
        assert torch.equal(st.params, rs.params), j
        np.testing.assert_array_equal(rec[:, j, :], rrd.cpu().numpy())
    be.close()
    H, W = sizes[0]
    img = inputs.image(H, W, seed=700, texture_sigma=0.02)
    lat, par = inputs.random_state(H, W, seed=750)
    o = oracle.forward(img, lat, par, lam=1e-3, mode=oracle.MODE_NOISE, seed=77, step=2)
    assert abs(rec[0, 0, 0] - o["loss"]) <= 1e-4 * abs(o["loss"])
    assert abs(rec[0, 0, 1] - o["rate_bits"]) <= 1e-4 * abs(o["rate_bits"])
    _parity(cc, H, W, img, lat, par, step=2)
