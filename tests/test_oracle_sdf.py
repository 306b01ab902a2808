"""Pins of the oracle's SDF intersection (Eq. 2, the prior work's model, kept
for the ablation against the disc model): on planar faces with exact normals
the weighted tangent-plane distance is the distance to the plane, so hits
land on the face; a single point gives the plane through it, where the
Gaussian defines the field; and a dense brute-force scan of the field along
each ray (numpy, from the points) finds the same first surface crossing."""
import numpy as np
import pytest

import oracle
from paper_2507_04021_gb300 import inputs

SIG = 0.1  # the room's points are ~14 cm apart: 2 sigma must bridge them
SIG_POINT = 0.025
SIG_OFFICE = 0.08  # 60,000 office points, ~11 cm apart


@pytest.fixture(scope="module")
def room_osc():
    room = inputs.room_scene()
    return room, oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)


def _rays(n, seed):
    rng = np.random.default_rng(seed)
    o = rng.uniform((0.8, 0.8, 0.6), (4.2, 3.2, 2.4), (n, 3))
    d = rng.normal(size=(n, 3))
    return o, d / np.linalg.norm(d, axis=1, keepdims=True)


def test_planar_faces_are_hit_exactly(room_osc):
    room, osc = room_osc
    L = np.array(room.extra["room"])
    o, d = _rays(200, 1)
    pts_dps = osc.point_dps()
    checked = 0
    for i in range(len(o)):
        h = osc.cast_sdf(o[i], d[i], SIG)
        assert h["hit"]
        labels = np.unique(room.surf[pts_dps == h["dps"]])
        if len(labels) != 1:
            continue  # a DPS at an edge of the room mixes two faces
        f = int(labels[0])
        axis, off = f // 2, (0.0 if f % 2 == 0 else L[f // 2])
        assert abs(h["q"][axis] - off) < 1e-6
        nrm = np.zeros(3)
        nrm[axis] = 1.0 if f % 2 == 0 else -1.0
        assert np.allclose(h["n"], nrm, atol=1e-9)
        checked += 1
    assert checked > 150


def test_single_point_gives_its_tangent_plane():
    p = np.array([[0.30, 0.20, 0.10]], np.float32)
    n = np.array([[0.0, 0.6, 0.8]], np.float32)
    osc = oracle.OracleScene(p, n, np.zeros(1, np.uint16), np.zeros(1, np.uint8), rho=0.0625,
                             r_p=0.05)
    o = np.array([0.31, 0.5, 0.5])  # crosses the plane 1 cm from the point
    d = np.array([0.0, -0.6, -0.8])
    h = osc.cast_sdf(o, d, SIG_POINT)
    pd = p[0].astype(np.float64)
    nd = n[0].astype(np.float64)
    t_plane = nd @ (pd - o) / (nd @ d)
    # within the final bisection interval (sigma / 2 halved 20 times)
    assert h["hit"] and h["t"] == pytest.approx(t_plane, abs=0.5 * SIG_POINT / 2 ** 20)
    # a ray whose plane crossing lies beyond 2 sigma of the point misses
    o2 = np.array([0.30 + 3 * SIG_POINT, 0.5, 0.5])
    assert not osc.cast_sdf(o2, d, SIG_POINT)["hit"]
    # one point's weight is exp(-r^2 / (2 sigma^2)), so the field is defined
    # (W >= e^-2) only within r <= 2 sigma of it: a ray along -n crossing the
    # plane at lateral offset 1.6 sigma hits, one at 2.4 sigma misses.  The
    # offset runs diagonally in the plane, so that every coordinate of the
    # crossing stays within 2 sigma of the point (inside the marched box).
    nu = nd / np.linalg.norm(nd)
    t1 = np.array([1.0, 0.0, 0.0])
    u = t1 + np.cross(nu, t1)
    u /= np.linalg.norm(u)
    for r, hit in [(1.6, True), (2.4, False)]:
        o3 = pd + r * SIG_POINT * u + 0.4 * nu
        assert np.all(np.abs(r * SIG_POINT * u) < 2 * SIG_POINT)
        assert osc.cast_sdf(o3, -nu, SIG_POINT)["hit"] == hit, r
    # a surface is entered from outside only: from behind, the field rises
    # through zero (- to +), which is no hit
    assert not osc.cast_sdf(pd - 0.4 * nu, nu, SIG_POINT)["hit"]


def test_label_is_the_nearest_points():
    """Two points of different labels in one DPS: the SDF hit takes the label
    of the point nearest to it."""
    p = np.array([[0.10, 0.10, 0.0], [0.14, 0.10, 0.0]], np.float32)
    n = np.array([[0, 0, 1.0], [0, 0, 1.0]], np.float32)
    surf = np.array([3, 7], np.uint16)
    osc = oracle.OracleScene(p, n, surf, np.zeros(2, np.uint8), rho=0.0625, r_p=0.05)
    assert osc.n_dps == 1
    for x, want in [(0.105, 3), (0.135, 7)]:
        h = osc.cast_sdf(np.array([x, 0.10, 0.3]), np.array([0, 0, -1.0]), SIG_POINT)
        assert h["hit"] and (h["labels"] & 0xFFFF) == want, x


def test_first_crossing_matches_a_dense_scan():
    office = inputs.office_scene(n_points=60000)
    osc = oracle.OracleScene(office.pos, office.nrm, office.surf, office.mat, rho=0.0625,
                             r_p=0.05)
    pts = office.pos.astype(np.float64)
    nrm = office.nrm.astype(np.float64)
    dps = osc.point_dps()
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(40):
        o = np.array([rng.uniform(1, 19), rng.uniform(1, 9), rng.uniform(0.5, 2.5)])
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        h = osc.cast_sdf(o, d, SIG_OFFICE, delta=1e-7)
        if not h["hit"] or h["amb"]:
            continue
        # dense scan of the hit DPS's field around the reported crossing
        P, N = pts[dps == h["dps"]], nrm[dps == h["dps"]]
        ts = h["t"] + np.linspace(-SIG_OFFICE / 2, SIG_OFFICE / 2, 4001)
        s = o[None] + ts[:, None] * d[None]
        v = s[:, None, :] - P[None]
        w = np.exp(-(v ** 2).sum(-1) / (2 * SIG_OFFICE ** 2))
        f = (w * (v * N[None]).sum(-1)).sum(1) / w.sum(1)
        cross = np.nonzero((f[:-1] > 0) & (f[1:] <= 0))[0]
        assert len(cross) >= 1
        tc = ts[cross[np.argmin(np.abs(ts[cross] - h["t"]))]]
        assert abs(tc - h["t"]) <= (ts[1] - ts[0]) * 1.01
        checked += 1
    assert checked > 20
