"""Pins of the vector-polarisation reading (pol = 2) in the oracle: closed
forms that follow from the geometry alone (vertical polarisation lies in
the plane of incidence of a floor reflection and across that of a vertical
wall seen at constant height; normal incidence reflects any polarisation
by Gamma_TE because Gamma_TM = -Gamma_TE there), rotation invariance about
the polarisation axis, and FP64 central differences of its derivatives."""
import numpy as np
import pytest

import oracle
from paper_2507_04021_gb300 import inputs

ETA = (5.3, 0.03)


def _gammas(cos_t):
    te = oracle.fresnel(ETA[0], ETA[1], 28e9, cos_t, 0)
    tm = oracle.fresnel(ETA[0], ETA[1], 28e9, cos_t, 1)
    return te, tm


def test_los_is_unity():
    for rx in ([3.0, 1.0, 1.5], [1.0, 2.0, 4.0], [0.5, -2.0, 0.2]):
        assert oracle.jones_amplitude([0, 0, 1.5], rx, np.zeros((0, 3)), np.zeros((0, 2))) == pytest.approx(1.0)


def test_floor_reflection_is_tm():
    h, L = 1.2, 5.0
    cos_t = h / np.hypot(L / 2, h)
    te, tm = _gammas(cos_t)
    a = oracle.jones_amplitude([0, 0, h], [L, 0, h], [[L / 2, 0, 0]], [[0.9 * te, 0.9 * tm]])
    assert a == pytest.approx(0.9 * tm, rel=1e-12)


def test_vertical_wall_at_constant_height_is_te():
    W, L = 2.0, 6.0
    cos_t = W / np.hypot(L / 2, W)
    te, tm = _gammas(cos_t)
    a = oracle.jones_amplitude([0, 0, 1.0], [L, 0, 1.0], [[L / 2, W, 1.0]], [[te, tm]])
    assert a == pytest.approx(te, rel=1e-12)


def test_normal_incidence_any_polarisation():
    te, tm = _gammas(1.0)
    assert tm == pytest.approx(-te, rel=1e-12)
    for tx, rx, q in (([0, 0, 1], [0, 1, 1], [0, 3, 1]), ([1, 1, 0.5], [1, 1, 1.5], [1, 1, 3.0])):
        a = oracle.jones_amplitude(tx, rx, [q], [[te, tm]])
        # horizontal: theta^ = -z across the plane; vertical: the x^ convention
        assert abs(a) == pytest.approx(abs(te), rel=1e-12)


def test_rotation_about_z_leaves_the_amplitude():
    rng = np.random.default_rng(3)
    tx = np.array([0.3, -0.2, 1.1])
    rx = np.array([4.0, 2.5, 0.7])
    pts = rng.uniform(-3, 3, (3, 3)) + np.array([2, 1, 1.5])
    D = rng.standard_normal((3, 2)) + 1j * rng.standard_normal((3, 2))
    a0 = oracle.jones_amplitude(tx, rx, pts, D)
    for ang in (0.4, 1.9, -2.6):
        c, s = np.cos(ang), np.sin(ang)
        Rz = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
        a = oracle.jones_amplitude(Rz @ tx, Rz @ rx, pts @ Rz.T, D)
        assert a == pytest.approx(a0, rel=1e-10)


RX = np.array([[4.0, 3.0, 1.2], [1.5, 3.2, 1.0]], np.float32)
MATS = (np.array([5.3, 3.0]), np.array([0.03, 0.01]), np.array([0.3, 0.2]))


def test_vector_path_grads_match_central_differences():
    room = inputs.room_scene()
    osc = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    sim = oracle.OracleSim(osc, room.tx, RX, oracle.SimParams(max_depth=2, capture=1, diffuse=1,
                                                              n_rays=4000, rep_tries=8, pol=2))
    G = sim.path_grads(*MATS)
    assert G.shape[0] > 5
    for t in range(3):
        for l in range(2):
            up = [m.copy() for m in MATS]
            dn = [m.copy() for m in MATS]
            h = 1e-6 * max(abs(MATS[t][l]), 1e-3)
            up[t][l] += h
            dn[t][l] -= h
            fd = (sim.field(*up)[0] - sim.field(*dn)[0]) / (2 * h)
            scale = np.abs(fd).max() + 1e-30
            assert np.allclose(G[:, t, l], fd, atol=1e-6 * scale, rtol=1e-5), (t, l)
    # the vector model differs from the scalar TE model (polarisation matters)
    sim_te = oracle.OracleSim(osc, room.tx, RX, oracle.SimParams(max_depth=2, capture=1, diffuse=1,
                                                                 n_rays=4000, rep_tries=8, pol=0))
    assert not np.allclose(np.abs(sim.field(*MATS)[0]), np.abs(sim_te.field(*MATS)[0]))


def _theta(d):
    h = np.hypot(d[0], d[1])
    if h < 1e-12:
        return np.array([1.0, 0.0, 0.0])
    return np.array([d[2] * d[0] / h, d[2] * d[1] / h, -h])


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_perfect_conductor_chain_equals_vector_image_maps(k):
    """With Gamma_TE = -1 and Gamma_TM = +1 (a perfect conductor) every
    reflection maps the field vector by the image rule E -> -E + 2 (E.n) n
    (tangential part reversed, normal part kept); the 2x2 basis chain must
    equal that plain 3D computation on random multi-bounce geometry."""
    rng = np.random.default_rng(10 + k)
    for _ in range(20):
        tx = rng.uniform(-2, 2, 3)
        rx = rng.uniform(-2, 2, 3)
        pts = rng.uniform(-3, 3, (k, 3))
        chain = [tx] + list(pts) + [rx]
        d = [(chain[m + 1] - chain[m]) / np.linalg.norm(chain[m + 1] - chain[m])
             for m in range(k + 1)]
        E = _theta(d[0])
        for m in range(k):
            n = d[m + 1] - d[m]
            n /= np.linalg.norm(n)
            E = -E + 2.0 * (E @ n) * n
        want = E @ _theta(-d[k])
        got = oracle.jones_amplitude(tx, rx, pts, [[-1.0, 1.0]] * k)
        assert got == pytest.approx(want, abs=1e-10)
