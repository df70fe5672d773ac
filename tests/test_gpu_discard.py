"""Encoder iterations drop the L2 lines of synthesis scratch (t, the kept dense latents, dt, dz) after
their last read with discard.global.L2.  A discarded line holds undefined data afterwards, so a
discard placed before a read would change results: the same encode, single-image (five iterations,
eagerly and from the library's graph) and batched, must come out bitwise the same in a process where
COOLCHIC_DISCARD=0 turns the discards off."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

_RUN = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2605_02726_gb300 import inputs, lib as cc
out = []
for H, W in [(72, 96), (37, 53)]:
    img = torch.tensor(inputs.image(H, W, seed=11), device="cuda")
    lat, par = inputs.random_state(H, W, seed=12)
    hp = cc.hparams(lam=1e-2, seed=4)
    ws = cc.workspace(H, W)
    st = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"))
    cc.encode_step(img, st, 5, H=H, W=W, hp=hp, ws=ws)        # eager (more than 4 iterations)
    for _ in range(3):
        cc.encode_step(img, st, 2, H=H, W=W, hp=hp, ws=ws)    # captured, then replayed
    out += [st.latents.cpu().numpy(), st.params.cpu().numpy()]
jobs = []
for q, (H, W) in enumerate([(48, 40), (64, 64)]):
    lat, par = inputs.random_state(H, W, seed=20 + q)
    jobs.append((torch.tensor(inputs.image(H, W, seed=30 + q), device="cuda"),
                 cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda")),
                 cc.hparams(lam=1e-3, seed=8 + q)))
be = cc.BatchEncoder(jobs, rd_capacity=4)
be.step(4)
torch.cuda.synchronize()
be.close()
for _, s, _ in jobs:
    out += [s.latents.cpu().numpy(), s.params.cpu().numpy()]
np.savez(sys.argv[2], *out)
"""


def _run(tmp_path, tag, discard):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, COOLCHIC_DISCARD="1" if discard else "0")
    path = str(tmp_path / f"{tag}.npz")
    r = subprocess.run([sys.executable, "-c", _RUN, root, path], capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    with np.load(path) as z:
        return [z[k] for k in sorted(z.files, key=lambda f: int(f.split("_")[1]))]


def test_discarding_dead_scratch_changes_no_result(tmp_path):
    on, off = _run(tmp_path, "on", True), _run(tmp_path, "off", False)
    assert len(on) == len(off) == 8
    for a, b in zip(on, off):
        np.testing.assert_array_equal(a, b)
