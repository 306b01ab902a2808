"""Pins of the oracle's single-bounce edge diffraction (Sec. II-B-3) to things
other than itself: the transition function against SciPy's Fresnel
integrals; the diffraction point against a numerical minimisation of the
path length; the general-n wedge coefficient against the textbook
half-plane form (n = 2, perfect conductor); continuity of the total field
across the incident and reflection shadow boundaries (the diffracted field
jumps by exactly the LOS / reflected field there); the vector model against
the soft / hard coefficients where the polarisation is fixed by symmetry;
and finite differences of the path derivatives."""
import cmath
import math

import numpy as np
import pytest

import oracle
from paper_2507_04021_gb300 import inputs

scipy_special = pytest.importorskip("scipy.special")
scipy_optimize = pytest.importorskip("scipy.optimize")

F0 = 28e9
C0 = 299792458.0
K0 = 2 * math.pi * F0 / C0
LAM = C0 / F0
ETA = complex(5.3, -0.03 / (2 * math.pi * F0 * 8.8541878128e-12))
PEC = complex(1e14, -1e14)


def _F_scipy(x):
    """2j sqrt(x) e^{jx} int_{sqrt x}^inf e^{-j t^2} dt from C(z), S(z)."""
    u = math.sqrt(x)
    S, Cc = scipy_special.fresnel(u * math.sqrt(2 / math.pi))
    head = math.sqrt(math.pi / 2) * (Cc - 1j * S)
    tail = math.sqrt(math.pi / 2) * (1 - 1j) / 2 - head
    return 2j * u * cmath.exp(1j * x) * tail


@pytest.mark.parametrize("x", np.concatenate([np.logspace(-6, 4, 41), [59.9, 60.1, 0.5, 3.0]]))
def test_transition_function_matches_fresnel_integrals(x):
    assert oracle.utd_F(x) == pytest.approx(_F_scipy(x), rel=1e-9, abs=1e-12)


def test_transition_function_limits():
    # F -> 1 far from the boundaries; F ~ sqrt(pi x) e^{j pi/4} near them
    assert abs(oracle.utd_F(1e5) - 1.0) < 1e-5
    x = 1e-8
    assert oracle.utd_F(x) == pytest.approx(math.sqrt(math.pi * x) * cmath.exp(1j * math.pi / 4),
                                            rel=1e-3)


def _box_edge():
    """Edge along y through the origin: face 0 the top (normal +z, extending
    to -x), face n the side (normal +x, extending to -z); n = 3/2."""
    return dict(a=(0.0, -1.0, 0.0), b=(0.0, 1.0, 0.0), n0=(0.0, 0.0, 1.0), n1=(1.0, 0.0, 0.0))


def test_exterior_angle_closed_forms():
    """n pi is the exterior angle of the wedge, 2 pi minus the angle between
    its faces: a right-angled box edge gives n = 3/2, a thin half-plane
    n -> 2, a 60-degree wedge n = 5/3 and a 120-degree one n = 4/3."""
    tx, rx = (1.0, 0.3, 1.0), (0.8, -0.2, -1.2)
    a, b = (0.0, -1.0, 0.0), (0.0, 1.0, 0.0)
    for interior, want in [(90.0, 1.5), (1e-6, 2.0), (60.0, 5.0 / 3.0), (120.0, 4.0 / 3.0)]:
        g = math.radians(interior)
        # face 0 extends along -x with normal +z; face n is face 0 turned by the
        # interior angle about the edge (y axis), its normal pointing outwards
        n0 = (0.0, 0.0, 1.0)
        n1 = (math.sin(g), 0.0, -math.cos(g))
        ok, D, s_in, s_out, phi_in, phi_out, nw, sinb = oracle.diffraction_geometry(
            tx, rx, a, b, n0, n1)
        assert nw == pytest.approx(want, abs=1e-6), interior


def test_keller_point_minimises_the_path_length():
    rng = np.random.default_rng(11)
    E = inputs.room_edges(12)
    checked = 0
    for i in range(len(E)):
        for _ in range(16):
            tx = rng.uniform((0.3, 0.3, 0.3), (4.7, 3.7, 2.7))
            rx = rng.uniform((0.3, 0.3, 0.3), (4.7, 3.7, 2.7))
            a, b = E.a[i].astype(np.float64), E.b[i].astype(np.float64)
            ok, D, s_in, s_out, *_ = oracle.diffraction_geometry(tx, rx, a, b, E.n0[i], E.n1[i])
            if not ok:
                continue
            L = np.linalg.norm(b - a)
            e = (b - a) / L
            f = lambda t: np.linalg.norm(tx - a - t * e) + np.linalg.norm(a + t * e - rx)  # noqa
            r = scipy_optimize.minimize_scalar(f, bounds=(0.0, L), method="bounded",
                                               options={"xatol": 1e-12})
            assert np.linalg.norm(D - (a + r.x * e)) < 1e-5
            assert s_in + s_out == pytest.approx(r.fun, rel=1e-12)
            # Keller cone: equal angles with the edge on both sides
            assert np.dot((D - tx) / s_in, e) == pytest.approx(np.dot((rx - D) / s_out, e), abs=1e-9)
            checked += 1
    assert checked > 10


def test_no_path_outside_the_segment_or_inside_the_wedge():
    g = _box_edge()
    tx = np.array([-2.0, 0.0, 1.0])
    # the Keller point would lie beyond the end of the edge
    assert oracle.diffraction_amplitude(tx, [3.0, 5.0, -1.0], g["a"], g["b"], g["n0"], g["n1"],
                                        ETA, ETA) is None
    # RX inside the solid wedge (below the top, behind the side)
    assert oracle.diffraction_amplitude(tx, [-0.5, 0.0, -0.5], g["a"], g["b"], g["n0"], g["n1"],
                                        ETA, ETA) is None
    assert oracle.diffraction_amplitude(tx, [2.0, 0.0, -1.0], g["a"], g["b"], g["n0"], g["n1"],
                                        ETA, ETA) is not None


def _rx_at(phi, r, t0, n0, y=0.0):
    return r * (math.cos(phi) * np.asarray(t0) + math.sin(phi) * np.asarray(n0)) + np.array([0, y, 0])


def test_half_plane_pec_matches_the_textbook_form():
    """n -> 2 (a wedge of interior angle 1e-7 rad), perfect conductor:
    D_{s,h} = -e^{-j pi/4} / (2 sqrt(2 pi k) sin b0) [F(kL a(b-)) / cos(b-/2)
    -/+ F(kL a(b+)) / cos(b+/2)], a(b) = 2 cos^2(b / 2)."""
    alpha = 1e-7
    n0 = np.array([0.0, 0.0, 1.0])
    n1 = np.array([math.sin(alpha), 0.0, -math.cos(alpha)])
    a, b = (0.0, -2.0, 0.0), (0.0, 2.0, 0.0)
    t0 = np.array([-1.0, 0.0, 0.0])
    tx = _rx_at(0.7, 2.0, t0, n0) + np.array([0, -0.4, 0])
    for phi in (1.1, 2.0, 3.0, 4.4, 5.6):
        rx = _rx_at(phi, 3.0, t0, n0, y=0.5)
        ok, D, s_in, s_out, phi_in, phi_out, nw, sinb = oracle.diffraction_geometry(
            tx, rx, a, b, n0, n1)
        assert ok and nw == pytest.approx(2.0, abs=1e-7)
        L = s_in * s_out * sinb ** 2 / (s_in + s_out)
        geo = LAM / (4 * math.pi * math.sqrt(s_in * s_out * (s_in + s_out)))
        bm, bp = phi_out - phi_in, phi_out + phi_in
        Fm = _F_scipy(K0 * L * 2 * math.cos(bm / 2) ** 2) / math.cos(bm / 2)
        Fp = _F_scipy(K0 * L * 2 * math.cos(bp / 2) ** 2) / math.cos(bp / 2)
        Kf = -cmath.exp(-1j * math.pi / 4) / (2 * math.sqrt(2 * math.pi * K0) * sinb)
        for pol, sgn in ((0, -1.0), (1, +1.0)):
            want = geo * Kf * (Fm + sgn * Fp)
            got = oracle.diffraction_amplitude(tx, rx, a, b, n0, n1, PEC, PEC, F0, pol)
            assert got == pytest.approx(want, rel=2e-6), (phi, pol)


def _jump(tx, g, phi_b, pol, eta=ETA, eps=1e-7, r=3.0):
    t0, n0 = np.array([-1.0, 0.0, 0.0]), np.array(g["n0"])
    lo = oracle.diffraction_amplitude(tx, _rx_at(phi_b - eps, r, t0, n0), g["a"], g["b"], g["n0"],
                                      g["n1"], eta, eta, F0, pol)
    hi = oracle.diffraction_amplitude(tx, _rx_at(phi_b + eps, r, t0, n0), g["a"], g["b"], g["n0"],
                                      g["n1"], eta, eta, F0, pol)
    return lo, hi


@pytest.mark.parametrize("pol", [0, 1])
def test_incident_shadow_boundary_continuity(pol):
    """Across phi = pi + phi' the LOS disappears; the diffracted field jumps
    by the LOS field, lambda / (4 pi |RX - TX|), so the total is continuous."""
    g = _box_edge()
    tx = np.array([-2.0, 0.0, 1.0])
    phi_in = math.atan2(1.0, 2.0)
    lo, hi = _jump(tx, g, math.pi + phi_in, pol)
    d = math.hypot(2.0, 1.0) + 3.0
    a_los = LAM / (4 * math.pi * d)
    assert (hi - lo) == pytest.approx(a_los, rel=1e-5)
    assert abs(hi - lo - a_los) < 1e-5 * a_los


@pytest.mark.parametrize("pol", [0, 1])
def test_reflection_shadow_boundary_continuity(pol):
    """Across phi = pi - phi' the reflection off face 0 disappears; the
    diffracted field jumps by R0 lambda / (4 pi (s + s')), R0 the face's
    Fresnel coefficient at its incidence cosine (Luebbers' weighting)."""
    g = _box_edge()
    tx = np.array([-2.0, 0.0, 1.0])
    phi_in = math.atan2(1.0, 2.0)
    lo, hi = _jump(tx, g, math.pi - phi_in, pol)
    d = math.hypot(2.0, 1.0) + 3.0
    R0 = oracle.fresnel_eta(ETA, math.sin(phi_in), pol)
    assert (hi - lo) == pytest.approx(R0 * LAM / (4 * math.pi * d), rel=1e-5)


def test_vector_model_reduces_to_soft_and_hard():
    # vertical edge, TX and RX at one height: the field is along the edge (soft)
    a, b = (2.0, 2.0, 0.0), (2.0, 2.0, 3.0)
    n0, n1 = (0.0, -1.0, 0.0), (1.0, 0.0, 0.0)
    tx, rx = (0.5, 0.7, 1.4), (3.6, 3.1, 1.4)
    v = oracle.diffraction_amplitude(tx, rx, a, b, n0, n1, ETA, ETA, F0, 2)
    s = oracle.diffraction_amplitude(tx, rx, a, b, n0, n1, ETA, ETA, F0, 0)
    assert v is not None and v == pytest.approx(s, rel=1e-12)
    # horizontal edge along y, TX and RX in the plane y = 0: normal to the edge (hard)
    g = _box_edge()
    tx, rx = (-2.0, 0.0, 1.0), (2.0, 0.0, -1.3)
    v = oracle.diffraction_amplitude(tx, rx, g["a"], g["b"], g["n0"], g["n1"], ETA, ETA, F0, 2)
    h = oracle.diffraction_amplitude(tx, rx, g["a"], g["b"], g["n0"], g["n1"], ETA, ETA, F0, 1)
    assert v is not None and v == pytest.approx(h, rel=1e-12)


RX = np.array([[4.0, 3.0, 1.2], [1.5, 3.2, 1.0], [4.2, 0.8, 2.1], [2.5, 2.0, 0.5]], np.float32)
MATS = (np.array([5.3, 3.0]), np.array([0.03, 0.01]), np.array([0.3, 0.2]))


@pytest.mark.parametrize("pol", [0, 2])
def test_diffracted_path_derivatives_match_central_differences(pol):
    room = inputs.room_scene()
    E = inputs.room_edges()
    osc = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    sim = oracle.OracleSim(osc, room.tx, RX, oracle.SimParams(
        max_depth=1, capture=1, diffuse=0, n_rays=500, rep_tries=8, pol=pol, diffraction=1),
        edges=E)
    P = sim.paths()
    dif = P["type"] == 2
    assert dif.sum() > 10
    G = sim.path_grads(*MATS)
    for t in range(2):
        for l in range(2):
            up = [m.copy() for m in MATS]
            dn = [m.copy() for m in MATS]
            h = 1e-6 * max(abs(MATS[t][l]), 1e-3)
            up[t][l] += h
            dn[t][l] -= h
            fd = (sim.field(*up)[0] - sim.field(*dn)[0]) / (2 * h)
            scale = np.abs(fd[dif]).max() + 1e-30
            assert np.allclose(G[dif, t, l], fd[dif], atol=1e-6 * scale, rtol=1e-5), (t, l)
    assert np.all(G[dif, 2, :] == 0)  # no roughness dependence


def test_diffraction_point_must_see_tx_and_rx():
    """Sec. II-B-3: a diffracted path exists only when its diffraction point
    sees both the TX and the RX.  One free-standing box edge, and a plate of
    points placed across the TX -> D segment: without the plate the edge
    gives its path, with it (or with the plate across D -> RX) none."""
    g = _box_edge()
    E = inputs.Edges(a=np.array([g["a"]], np.float32), b=np.array([g["b"]], np.float32),
                     n0=np.array([g["n0"]], np.float32), n1=np.array([g["n1"]], np.float32),
                     m0=np.zeros(1, np.uint8), m1=np.ones(1, np.uint8))
    tx = np.array([-1.5, 0.2, 1.2])
    rx = np.array([[1.2, -0.1, -1.0]])
    ok, D, *_ = oracle.diffraction_geometry(tx, rx[0], g["a"], g["b"], g["n0"], g["n1"])
    assert ok

    def plate_across(p0, p1):
        """A 0.6 m square of points, 3 cm apart, across the segment's middle."""
        c = 0.5 * (p0 + p1)
        u = (p1 - p0) / np.linalg.norm(p1 - p0)
        e1 = np.cross(u, [0.0, 1.0, 0.0])
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(u, e1)
        s = np.arange(-0.3, 0.3 + 1e-9, 0.03)
        A, B = np.meshgrid(s, s, indexing="ij")
        pts = c + A.reshape(-1, 1) * e1 + B.reshape(-1, 1) * e2
        return pts, np.tile(u, (len(pts), 1))

    far = (np.array([[10.0, 10.0, 10.0]]), np.array([[0.0, 0.0, 1.0]]))  # nothing in the way
    counts = []
    for pts, nrm in (far, plate_across(tx, D), plate_across(D, rx[0])):
        n = len(pts)
        osc = oracle.OracleScene(pts.astype(np.float32), nrm.astype(np.float32),
                                 np.zeros(n, np.uint16), np.zeros(n, np.uint8), r_p=0.05)
        sim = oracle.OracleSim(osc, tx, rx, oracle.SimParams(max_depth=1, capture=1, diffuse=0,
                                                             n_rays=100, diffraction=1), edges=E)
        counts.append(int(np.sum(sim.paths()["type"] == 2)))
    assert counts == [1, 0, 0]


@pytest.mark.parametrize("pol", [0, 1])
def test_grazing_face_material_drops_out(pol):
    """Each face's reflection factor takes that face's own incidence cosine:
    sin(beta0) sin(phi') on face 0, sin(beta0) sin(n pi - phi) on face n.  A
    wave grazing a face (cosine -> 0) reflects with -1 from any material
    (TE and TM alike), so with the RX grazing face n the coefficient stops
    depending on face n's material, and with the TX grazing face 0 on face
    0's; away from grazing both materials matter."""
    g = _box_edge()
    t0, n0 = (-1.0, 0.0, 0.0), (0.0, 0.0, 1.0)
    A, B = ETA, complex(2.0, -0.5)
    eps = 1e-7
    edge = (g["a"], g["b"], g["n0"], g["n1"])

    def amp(tx, rx, e0, e1):
        a = oracle.diffraction_amplitude(tx, rx, *edge, e0, e1, F0, pol)
        assert a is not None
        return a

    for phi_in, y_tx, phi_out, y_rx in [(0.7, 0.2, 1.2 * math.pi, -0.1),
                                        (1.1, -0.3, 0.9 * math.pi, 0.4)]:
        tx = _rx_at(phi_in, 2.0, t0, n0, y_tx)
        rx = _rx_at(phi_out, 1.5, t0, n0, y_rx)
        rx_g = _rx_at(1.5 * math.pi - eps, 1.5, t0, n0, y_rx)  # grazing face n
        tx_g = _rx_at(eps, 2.0, t0, n0, y_tx)                  # grazing face 0
        a, b = amp(tx, rx_g, ETA, A), amp(tx, rx_g, ETA, B)
        assert abs(a - b) < 1e-5 * abs(a)
        a, b = amp(tx_g, rx, A, ETA), amp(tx_g, rx, B, ETA)
        assert abs(a - b) < 1e-5 * abs(a)
        a, b = amp(tx, rx, ETA, A), amp(tx, rx, ETA, B)
        assert abs(a - b) > 1e-3 * abs(a)
        a, b = amp(tx, rx, A, ETA), amp(tx, rx, B, ETA)
        assert abs(a - b) > 1e-3 * abs(a)


@pytest.mark.parametrize("pol", [0, 1])
def test_perfect_conductor_wedge_is_reciprocal(pol):
    """For a perfect conductor (R0 = Rn = -/+1) the wedge coefficient is
    symmetric in (phi, phi') and the spreading in (s, s'): exchanging TX and
    RX gives the same diffracted field, on random wedges and positions."""
    rng = np.random.default_rng(21 + pol)
    E = inputs.room_edges(16, seed=99)
    checked = 0
    for i in range(len(E)):
        for _ in range(6):
            tx = rng.uniform((0.3, 0.3, 0.3), (4.7, 3.7, 2.7))
            rx = rng.uniform((0.3, 0.3, 0.3), (4.7, 3.7, 2.7))
            # |eta| = 1e30: Gamma_TM departs from +1 by ~2 / (cos sqrt|eta|), so the
            # perfect-conductor limit holds to 1e-12 even at grazing incidence
            pec = complex(1e30, -1e30)
            args = (E.a[i], E.b[i], E.n0[i], E.n1[i], pec, pec, F0, pol)
            ab = oracle.diffraction_amplitude(tx, rx, *args)
            ba = oracle.diffraction_amplitude(rx, tx, *args)
            assert (ab is None) == (ba is None)
            if ab is None:
                continue
            assert ab == pytest.approx(ba, rel=1e-9)
            checked += 1
    assert checked > 10
