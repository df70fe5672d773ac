"""SOAP on the network parameters (Sec. IV-B), the CUDA path against the FP64 oracle.

SOAP's eigenbases are unique (up to signs, which its step does not see) only where the
preconditioners' eigenvalues are distinct, so parity is checked from states whose L and R have
well-separated spectra: one encoder iteration in the middle of a refresh period (the update, the
moments and the preconditioners), one at a refresh (the new eigenbases, canonical signs), and the
first call (L, R from the first gradient, the blocks not moved).  Gradients carry the path's FP32
error (1e-3 of each block's largest entry), so the step is compared on that scale."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_02726_gb300 import inputs

pytestmark = pytest.mark.gpu

LAM, SEED = 1e-2, 31


def _orth(rng, n):
    q, r = np.linalg.qr(rng.standard_normal((n, n)))
    return q * np.sign(np.diag(r))


def _soap_state(rng):
    """L, R with eigenvalues spread over two decades, their eigenbases as the oracle writes them."""
    S = []
    for _, m, n in oracle.soap_blocks():
        mats = {}
        for side, d in (("L", m), ("R", n)):
            U = _orth(rng, d)
            lam = np.logspace(0.0, -2.0, d) * (1.0 + 0.1 * rng.random())
            mats[side] = (U * lam) @ U.T
            mats["Q" + side], _ = oracle.sym_eig(mats[side])
        S += [mats["L"].ravel(), mats["R"].ravel(), mats["QL"].ravel(), mats["QR"].ravel()]
    return np.concatenate(S)


def _run(cc, step, seed, zero_state=False):
    H, W = 40, 48
    rng = np.random.default_rng(seed)
    img = inputs.image(H, W, seed=seed)
    lat, par = inputs.random_state(H, W, seed=seed + 1)
    NP = inputs.N_PARAMS
    if zero_state:
        M, V, S = np.zeros(NP), np.zeros(NP), np.zeros(oracle.soap_state_count())
    else:
        M = rng.standard_normal(NP) * 1e-3
        V = rng.uniform(1e-6, 1e-5, NP)
        S = _soap_state(rng)
    # CUDA path
    st = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"), step=step, soap=True)
    st.m_par.copy_(torch.tensor(M, dtype=torch.float32))
    st.v_par.copy_(torch.tensor(V, dtype=torch.float32))
    st.soap.copy_(torch.tensor(S, dtype=torch.float32))
    M32, V32, S32 = (st.m_par.double().cpu().numpy(), st.v_par.double().cpu().numpy(),
                     st.soap.double().cpu().numpy())
    cc.encode_step(torch.tensor(img, device="cuda"), st, 1, H=H, W=W, hp=cc.hparams(lam=LAM, seed=SEED, soap=True),
                   ws=cc.workspace(H, W))
    torch.cuda.synchronize()
    # oracle, from the same FP32 values
    P = par.astype(np.float64)
    g = oracle.loss_grad(img, lat, par, lam=LAM, mode=oracle.MODE_NOISE, seed=SEED, step=step)
    Mo, Vo, So = M32.copy(), V32.copy(), S32.copy()
    oracle.soap_params(P, g["grad_params"], Mo, Vo, So, step + 1, lr=1e-2)
    got = dict(P=st.params.double().cpu().numpy(), M=st.m_par.double().cpu().numpy(),
               V=st.v_par.double().cpu().numpy(), S=st.soap.double().cpu().numpy())
    ref = dict(P=P, M=Mo, V=Vo, S=So)
    assert int(st.step.item()) == step + 1
    return par.astype(np.float64), S32, got, ref


def _close(name, a, b, tol=1e-3, atol=0.0):
    scale = np.abs(b).max()
    err = np.abs(a - b).max()
    assert err <= tol * scale + atol, f"{name}: max err {err:.3e}, scale {scale:.3e}"


def _check_eigenbasis(name, L, Q):
    """The GPU eigenbasis Q of its own preconditioner L against the oracle's eigen-decomposition of
    that L, column by column, up to sign (the step does not see signs), within the FP32 Jacobi
    accuracy scaled by each eigenvalue's distance to the others (columns of near-repeated
    eigenvalues are not unique and are skipped)."""
    Qr, lam = oracle.sym_eig(L)
    d = L.shape[0]
    top = np.abs(lam).max()
    for j in range(d):
        gap = min([abs(lam[j] - lam[i]) for i in range(d) if i != j] or [top])
        if gap < 1e-4 * top:
            continue
        err = min(np.abs(Q[:, j] - Qr[:, j]).max(), np.abs(Q[:, j] + Qr[:, j]).max())
        assert err <= 1e-5 * top / gap + 1e-5, f"{name} column {j}: err {err:.2e}, gap {gap / top:.2e}"


def _state_slices():
    out, o = [], 0
    for off, m, n in oracle.soap_blocks():
        for nm, d in (("L", m * m), ("R", n * n), ("QL", m * m), ("QR", n * n)):
            out.append((off, m, n, nm, slice(o, o + d)))
            o += d
    return out


@pytest.mark.parametrize("step", [4, 10])
def test_soap_iteration_matches_oracle(cc, step):
    """A state that has taken `step` steps runs SOAP step `step`: 4 is inside a refresh period of
    10, 10 refreshes the eigenbases from the updated preconditioners."""
    P0, S0, got, ref = _run(cc, step, seed=50 + step)
    for off, m, n in oracle.soap_blocks():
        sl = slice(off, off + m * n)
        _close(f"dW {off}", got["P"][sl] - P0[sl], ref["P"][sl] - P0[sl])
        _close(f"M {off}", got["M"][sl], ref["M"][sl])
        _close(f"V {off}", got["V"][sl], ref["V"][sl])
    # the Adam-updated one-dimensional parameters as well
    mask = np.ones(inputs.N_PARAMS, bool)
    for off, m, n in oracle.soap_blocks():
        mask[off:off + m * n] = False
    _close("dW 1-D", got["P"][mask] - P0[mask], ref["P"][mask] - P0[mask])
    sl_of = {}
    for off, m, n, nm, sl in _state_slices():
        sl_of[(off, nm)] = (sl, m if nm in ("L", "QL") else n)
        if nm in ("L", "R"):
            _close(f"{nm} {off}", got["S"][sl], ref["S"][sl], tol=1e-4)
    refreshed = step % 10 == 0
    for off, m, n in oracle.soap_blocks():
        for side in ("L", "R"):
            (sl_q, d), (sl_l, _) = sl_of[(off, "Q" + side)], sl_of[(off, side)]
            if refreshed:  # the new eigenbasis of the new preconditioner
                _check_eigenbasis(f"Q{side} {off}", got["S"][sl_l].reshape(d, d), got["S"][sl_q].reshape(d, d))
            else:  # untouched between refreshes
                np.testing.assert_array_equal(got["S"][sl_q], S0[sl_q])


def test_soap_first_call_builds_preconditioners(cc):
    """SOAP step 0: L = (1 - b) G G^T, R = (1 - b) G^T G; the 2-D blocks do not move (the 1-D
    ones take their first Adam step); the eigenbases of the square blocks (full-rank L and R)
    match the oracle's."""
    P0, _, got, ref = _run(cc, 0, seed=70, zero_state=True)
    for off, m, n in oracle.soap_blocks():
        sl = slice(off, off + m * n)
        np.testing.assert_array_equal(got["P"][sl], P0[sl])
    sl_of = {}
    for off, m, n, nm, sl in _state_slices():
        sl_of[(off, nm)] = sl
        if nm in ("L", "R"):
            _close(f"{nm} {off}", got["S"][sl], ref["S"][sl], tol=2e-3)
    for off, m, n in oracle.soap_blocks():
        if m == n:
            _check_eigenbasis(f"QL {off}", got["S"][sl_of[(off, "L")]].reshape(m, m),
                              got["S"][sl_of[(off, "QL")]].reshape(m, m))
            _check_eigenbasis(f"QR {off}", got["S"][sl_of[(off, "R")]].reshape(n, n),
                              got["S"][sl_of[(off, "QR")]].reshape(n, n))


def test_soap_batch_equals_single_and_trains(cc):
    H, W = 32, 40
    img = torch.tensor(inputs.image(H, W, seed=3), device="cuda")
    lat, par = inputs.initial_state(H, W, seed=4)
    hp = cc.hparams(lam=1e-3, seed=5, soap=True)
    single = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"), soap=True)
    batched = single.clone()
    rd = torch.zeros(30, 3, dtype=torch.float64, device="cuda")
    cc.encode_step(img, single, 30, H=H, W=W, hp=hp, ws=cc.workspace(H, W), rd=rd)
    be = cc.BatchEncoder([(img, batched, hp)], rd_capacity=30)
    be.step(30)
    torch.cuda.synchronize()
    assert torch.equal(single.params, batched.params) and torch.equal(single.soap, batched.soap)
    be.close()
    loss = rd[:, 0].cpu().numpy()
    assert np.all(np.isfinite(loss)) and loss[-1] < loss[0]
