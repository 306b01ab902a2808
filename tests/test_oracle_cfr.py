"""Pins of the CFR / Eq. 5 oracle (oracle/cfr.py) and of the oracle's
per-path complex derivatives: closed forms of one- and two-path responses,
Parseval's identity through numpy's FFT (the loss on the CIR equals the
loss on the CFR), and FP64 central differences of the oracle's own field."""
import numpy as np
import pytest

import oracle
from oracle import cfr
from paper_2507_04021_gb300 import inputs

RX = np.array([[4.0, 3.0, 1.2], [1.5, 3.2, 1.0]], np.float32)
F = cfr.freqs(28e9, 1.5e9, 129)


def test_frequency_grid():
    assert F.size == 129 and F[64] == 28e9
    assert F[0] == pytest.approx(28e9 - 0.75e9) and F[-1] == pytest.approx(28e9 + 0.75e9)
    assert np.allclose(np.diff(F), 1.5e9 / 128)


def test_one_and_two_path_closed_forms():
    a1, t1 = 3e-4 * np.exp(0.7j), 2.3e-8
    H = cfr.cfr([a1], [t1], [0], 1, F)[0]
    assert np.allclose(np.abs(H), abs(a1), rtol=1e-12)
    step = H[1:] / H[:-1]
    assert np.allclose(np.angle(step), np.angle(np.exp(-2j * np.pi * (F[1] - F[0]) * t1)), atol=1e-9)
    a2, t2 = 1e-4 * np.exp(-1.1j), 3.1e-8
    H2 = cfr.cfr([a1, a2], [t1, t2], [0, 0], 1, F)[0]
    want = (abs(a1) ** 2 + abs(a2) ** 2 + 2 * abs(a1) * abs(a2) *
            np.cos(np.angle(a1) - np.angle(a2) - 2 * np.pi * F * (t1 - t2)))
    assert np.allclose(np.abs(H2) ** 2, want, rtol=1e-10)


def test_cir_of_one_path_is_a_delayed_impulse():
    """One path whose delay is m0 / (N df) (df the grid step): its CFR is
    C exp(-j 2 pi n m0 / N) over the grid index n, so the inverse DFT is the
    impulse C delta[m - m0]: |h| = |a| at tap m0 and 0 elsewhere."""
    df = F[1] - F[0]
    a = 2e-4 * np.exp(0.3j)
    for m0 in (1, 5, 40):
        tau = m0 / (F.size * df)
        h = cfr.cir(cfr.cfr([a], [tau], [0], 1, F))[0]
        assert int(np.argmax(np.abs(h))) == m0
        assert abs(h[m0]) == pytest.approx(abs(a), rel=1e-9)
        assert np.abs(np.delete(h, m0)).max() < 1e-9 * abs(a)


def test_eq5_on_cfr_equals_eq5_on_cir():
    rng = np.random.default_rng(1)
    H = rng.standard_normal((3, 129)) + 1j * rng.standard_normal((3, 129))
    T = rng.standard_normal((3, 129)) + 1j * rng.standard_normal((3, 129))
    h, t = np.fft.ifft(H, axis=1), np.fft.ifft(T, axis=1)
    want = np.sum(np.abs(h - t) ** 2, axis=1) / np.sum(np.abs(t) ** 2, axis=1)
    assert np.allclose(cfr.eq5_loss(H, T), want, rtol=1e-12)


@pytest.fixture(scope="module")
def room_sim():
    room = inputs.room_scene()
    osc = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    p = oracle.SimParams(max_depth=2, capture=1, diffuse=1, n_rays=4000, rep_tries=8)
    return oracle.OracleSim(osc, room.tx, RX, p)


MATS = (np.array([5.3, 3.0]), np.array([0.03, 0.01]), np.array([0.3, 0.2]))


def _a(sim, mats):
    a, _ = sim.field(*mats)
    return a


def test_path_grads_match_central_differences(room_sim):
    G = room_sim.path_grads(*MATS)
    assert G.shape[1:] == (3, 2) and G.shape[0] > 5
    for t in range(3):
        for l in range(2):
            up = [m.copy() for m in MATS]
            dn = [m.copy() for m in MATS]
            h = 1e-6 * max(abs(MATS[t][l]), 1e-3)
            up[t][l] += h
            dn[t][l] -= h
            fd = (_a(room_sim, up) - _a(room_sim, dn)) / (2 * h)
            scale = np.abs(fd).max() + 1e-30
            assert np.allclose(G[:, t, l], fd, atol=1e-6 * scale, rtol=1e-5), (t, l)


def test_eq5_gradient_matches_central_differences(room_sim):
    P = room_sim.paths()
    hidden = (np.array([4.1, 2.4]), np.array([0.05, 0.002]), np.array([0.45, 0.1]))
    T = cfr.cfr(_a(room_sim, hidden), P["tau"], P["j"], 2, F)
    w = np.array([1.0, 0.5])

    def loss(m):
        return float(np.sum(w * cfr.eq5_loss(cfr.cfr(_a(room_sim, m), P["tau"], P["j"], 2, F), T)))

    H = cfr.cfr(_a(room_sim, MATS), P["tau"], P["j"], 2, F)
    g = cfr.eq5_grad(room_sim.path_grads(*MATS), P["tau"], P["j"], F, H, T, w)
    for t in range(3):
        for l in range(2):
            up = [m.copy() for m in MATS]
            dn = [m.copy() for m in MATS]
            h = 1e-6 * max(abs(MATS[t][l]), 1e-3)
            up[t][l] += h
            dn[t][l] -= h
            fd = (loss(up) - loss(dn)) / (2 * h)
            assert g[t, l] == pytest.approx(fd, rel=1e-5, abs=1e-9 * abs(g).max()), (t, l)
