"""Serving loop: admission by HBM budget, interleaved iterations of resident jobs, and each
result equal to the job run alone (bitwise: the batched kernels are the single-image kernels)."""
import math

import numpy as np
import pytest
import torch

from paper_2605_02726_gb300 import inputs

pytestmark = pytest.mark.gpu

SIZES = [(32, 48), (64, 64), (40, 24), (17, 29)]


def _requests(n_iters, offsets, sizes=SIZES):
    reqs = []
    for q, ((H, W), off) in enumerate(zip(sizes, offsets)):
        img = torch.tensor(inputs.image(H, W, seed=900 + q))
        reqs.append((off, img, 1e-3 * (q + 1), 70 + 5 * q, n_iters))
    return reqs


def _alone(cc, req):
    _, img, lam, seed, iters = req
    H, W = img.shape[1], img.shape[2]
    lat, par = inputs.initial_state(H, W, seed=seed + 1)
    st = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"))
    cc.encode_step(img.cuda(), st, iters, H=H, W=W, hp=cc.hparams(lam=lam, seed=seed), ws=cc.workspace(H, W))
    torch.cuda.synchronize()
    return st.latents.cpu(), st.params.cpu()


def test_each_result_is_the_same_alone_and_in_the_mix(cc):
    from paper_2605_02726_gb300.serve import EncodeServer
    reqs = _requests(20, [0.0, 0.0, 0.03, 0.06, 0.09], SIZES + [(512, 768)])  # ids follow arrival order
    srv = EncodeServer(hbm_budget=8 << 30, tick_iters=7)
    srv.run(reqs)
    assert len(srv.done) == len(reqs) and not srv.failed
    assert srv.ticks >= 3
    for rid, req in enumerate(reqs):
        lat, par = _alone(cc, req)
        got_lat, got_par = srv.done[rid].final
        assert torch.equal(got_lat, lat), rid
        assert torch.equal(got_par, par), rid


def test_small_budget_admits_one_job_at_a_time(cc):
    from paper_2605_02726_gb300.serve import EncodeServer, job_bytes
    sizes = [(48, 40)] * 4  # equal sizes: the budget holds exactly one job
    reqs = _requests(9, [0.0, 0.0, 0.0, 0.0], sizes)
    budget = job_bytes(48, 40) + 1024
    srv = EncodeServer(hbm_budget=budget, tick_iters=5)
    srv.run(reqs)
    assert len(srv.done) == len(reqs)
    assert srv.peak_in_use <= budget
    spans = sorted((j.admitted, j.finished) for j in srv.done.values())
    for (a0, f0), (a1, _) in zip(spans, spans[1:]):
        assert a1 >= f0 - 1e-3  # one at a time


def test_slots_bound_the_running_jobs_and_keep_arrival_order(cc):
    from paper_2605_02726_gb300.serve import EncodeServer
    reqs = _requests(12, [0.0] * 6, SIZES + [(24, 24), (33, 21)])
    srv = EncodeServer(hbm_budget=8 << 30, tick_iters=4, slots=2)
    seen = []
    orig = srv._launch

    def launch():
        n = orig()
        if n:
            seen.append(len(srv.inflight[-1].jobs))  # jobs in the tick just queued
        return n

    srv._launch = launch
    srv.run(reqs)
    assert len(srv.done) == len(reqs) and not srv.failed
    assert max(seen) <= 2
    admitted = [srv.done[rid].admitted for rid in range(len(reqs))]
    assert admitted == sorted(admitted)  # first come, first served
    for rid in (0, 5):  # the results are still each job's own
        lat, par = _alone(cc, reqs[rid])
        assert torch.equal(srv.done[rid].final[0], lat) and torch.equal(srv.done[rid].final[1], par)


def test_rejections_and_cancellation_leave_other_jobs_intact(cc):
    from paper_2605_02726_gb300.serve import EncodeServer
    reqs = _requests(12, [0.0, 0.0, 0.0, 0.0])
    srv = EncodeServer(hbm_budget=8 << 30, tick_iters=4)
    bad_lam = srv.submit(torch.zeros(3, 8, 8), float("nan"), 1, 5)
    bad_shape = srv.submit(torch.zeros(2, 8, 8), 1e-3, 1, 5)
    assert srv.failed[bad_lam] and srv.failed[bad_shape]
    ids = [srv.submit(img, lam, seed, iters) for _, img, lam, seed, iters in reqs]
    srv.tick(now=float("inf"))  # admit all, one tick
    assert srv.cancel(ids[1])
    while srv.active:
        srv.tick(now=float("inf"))
    assert srv.failed[ids[1]] == "cancelled" and ids[1] not in srv.done
    assert srv.in_use == 0
    for q in (0, 2, 3):
        lat, par = _alone(cc, reqs[q])
        assert torch.equal(srv.done[ids[q]].final[0], lat)
        assert torch.equal(srv.done[ids[q]].final[1], par)
