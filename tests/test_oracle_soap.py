"""Pins of the oracle's SOAP step for the network parameters (Sec. IV-B) against facts outside it:
the eigen-decomposition against numpy.linalg.eigh (a library routine), SOAP reducing to Adam when
the preconditioners are diagonal (its eigenbasis is then the identity), the closed form of the
first real step (N' = sign(G')), and equivariance under orthogonal changes of basis of a layer's
input and output spaces (which catches a transposed or swapped rotation)."""
import numpy as np
import pytest

import oracle
from paper_2605_02726_gb300 import inputs

NP = inputs.N_PARAMS


@pytest.mark.parametrize("n", [2, 5, 16, 27, 40])
def test_sym_eig_matches_numpy(n):
    rng = np.random.default_rng(n)
    for A in (rng.standard_normal((n, n)), rng.standard_normal((n, 3))):
        A = A @ A.T if A.shape[1] == n else A @ A.T + np.diag(np.arange(n) * 1e-3)
        Q, lam = oracle.sym_eig(A)
        w, U = np.linalg.eigh(A)
        scale = np.abs(w).max()
        np.testing.assert_allclose(lam, w[::-1], rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(Q.T @ Q, np.eye(n), rtol=0, atol=1e-12)
        np.testing.assert_allclose(A @ Q, Q * lam, rtol=0, atol=1e-11 * scale)
        # columns: numpy's, ordered by decreasing eigenvalue, entry of largest magnitude positive
        # (compared where the eigenvalue is well separated from its neighbours)
        U = U[:, ::-1]
        for j in range(n):
            gap = min([abs(lam[j] - lam[i]) for i in range(n) if i != j] or [scale])
            if gap < 1e-6 * scale:
                continue
            u = U[:, j] * np.sign(U[np.argmax(np.abs(U[:, j])), j])
            np.testing.assert_allclose(Q[:, j], u, rtol=0, atol=1e-9 * scale / gap)


def _diag_grad(rng, blocks, scale):
    """A gradient whose 2-D blocks are [D | 0] or [D ; 0] with D diagonal, entries of decreasing
    magnitude and random signs: every preconditioner stays diagonal in the same order."""
    g = rng.standard_normal(NP) * scale
    for off, m, n in blocks:
        B = np.zeros((m, n))
        k = min(m, n)
        mags = np.linspace(2.0, 1.0, k) * scale * (1.0 + 0.1 * rng.random())
        B[np.arange(k), np.arange(k)] = mags * rng.choice([-1.0, 1.0], k)
        g[off:off + m * n] = B.ravel()
    return g


def test_soap_with_diagonal_preconditioners_is_adam():
    rng = np.random.default_rng(7)
    blocks = oracle.soap_blocks()
    _, par = inputs.random_state(8, 8, seed=3)
    P = par.astype(np.float64)
    m, v, S = np.zeros(NP), np.zeros(NP), np.zeros(oracle.soap_state_count())
    Pa, ma, va = P.copy(), np.zeros(NP), np.zeros(NP)
    grads = [_diag_grad(rng, blocks, 1e-2) for _ in range(6)]
    for t, g in enumerate(grads, start=1):
        oracle.soap_params(P, g, m, v, S, t, lr=1e-2)
        if t >= 2:  # SOAP's step t - 1 is Adam's step t - 1 with SOAP's betas
            oracle.adam(Pa, g, ma, va, t - 1, lr=1e-2, b1=0.95, b2=0.95)
    for off, mm, nn in blocks:
        sl = slice(off, off + mm * nn)
        np.testing.assert_allclose(P[sl], Pa[sl], rtol=0, atol=1e-13)


def test_first_soap_step_closed_form():
    """Step 0 builds L = (1 - b) G0 G0^T and its eigenbasis; step 1 (zero moments) moves W by
    -lr Q_L sign(Q_L^T G1 Q_R) Q_R^T (up to eps), independent of the signs of the eigenvectors.
    Checked on the square blocks, whose L and R have full rank after one gradient: a non-square
    block's larger side has a null space, where the eigenbasis (and so SOAP's step) is not unique."""
    rng = np.random.default_rng(11)
    _, par = inputs.random_state(8, 8, seed=4)
    P = par.astype(np.float64)
    m, v, S = np.zeros(NP), np.zeros(NP), np.zeros(oracle.soap_state_count())
    g0, g1 = rng.standard_normal(NP) * 1e-2, rng.standard_normal(NP) * 1e-2
    oracle.soap_params(P, g0, m, v, S, 1, lr=1e-2)
    W0 = P.copy()
    oracle.soap_params(P, g1, m, v, S, 2, lr=1e-2)
    square = [(off, mm, nn) for off, mm, nn in oracle.soap_blocks() if mm == nn]
    assert len(square) == 2
    for off, mm, nn in square:
        G0 = g0[off:off + mm * nn].reshape(mm, nn)
        G1 = g1[off:off + mm * nn].reshape(mm, nn)
        _, QL = np.linalg.eigh(G0 @ G0.T)
        _, QR = np.linalg.eigh(G0.T @ G0)
        Gr = QL.T @ G1 @ QR
        step = QL @ (Gr / (np.abs(Gr) + 1e-8)) @ QR.T
        np.testing.assert_allclose(W0[off:off + mm * nn] - P[off:off + mm * nn], 1e-2 * step.ravel(),
                                   rtol=0, atol=1e-10)


def _orth(rng, n):
    q, r = np.linalg.qr(rng.standard_normal((n, n)))
    return q * np.sign(np.diag(r))


def test_soap_is_equivariant_under_orthogonal_changes_of_basis():
    """W -> U W V^T, G -> U G V^T (and so every preconditioner) gives the rotated trajectory.
    On a square block (ARM W2, 16 x 16), whose preconditioners have full rank from the first
    gradient on, so that every eigenbasis is unique up to signs, which the step does not see."""
    rng = np.random.default_rng(5)
    off, mm, nn = oracle.soap_blocks()[1]  # ARM W2, 16 x 16
    assert mm == nn == 16
    U, V = _orth(rng, mm), _orth(rng, nn)
    _, par = inputs.random_state(8, 8, seed=6)
    runs = []
    for rot in (False, True):
        P = par.astype(np.float64)
        if rot:
            P[off:off + mm * nn] = (U @ P[off:off + mm * nn].reshape(mm, nn) @ V.T).ravel()
        m, v, S = np.zeros(NP), np.zeros(NP), np.zeros(oracle.soap_state_count())
        grng = np.random.default_rng(9)
        for t in range(1, 15):  # through the eigenbasis refresh at SOAP step 10
            g = grng.standard_normal(NP) * 1e-2
            if rot:
                g[off:off + mm * nn] = (U @ g[off:off + mm * nn].reshape(mm, nn) @ V.T).ravel()
            oracle.soap_params(P, g, m, v, S, t, lr=1e-2)
        runs.append(P[off:off + mm * nn].reshape(mm, nn))
    np.testing.assert_allclose(U @ runs[0] @ V.T, runs[1], rtol=0, atol=1e-10)


def test_soap_encode_runs_and_trains():
    H, W = 16, 16
    img = inputs.image(H, W, seed=2)
    lat, par = inputs.initial_state(H, W, seed=3)
    st = oracle.State(lat, par)
    S = np.zeros(oracle.soap_state_count())
    loss = oracle.encode_soap(img, st, S, 25, lam=1e-3, seed=4)
    assert np.all(np.isfinite(loss)) and loss[-1] < loss[0] and st.step == 25
