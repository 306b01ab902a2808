"""Pins for the oracle's path computation (Sec. II-B): specular refinement
against the textbook image-source enumeration of a rectangular room and
against a library minimisation of Eq. 1, dedup invariance, visibility and
diffuse validation, and the adjoint against FP64 finite differences.  CPU only."""
import itertools

import numpy as np
import pytest
from scipy.optimize import minimize

import oracle
from paper_2507_04021_gb300 import inputs

C0 = 299792458.0
ROOM = (5.0, 4.0, 3.0)


def dense_room(spacing=0.04):
    """Noise-free shoebox with a square lattice of discs on each face (r_p = spacing)."""
    pts, nrm, surf = [], [], []
    fid = 0
    for axis in range(3):
        u, v = [a for a in range(3) if a != axis]
        nu, nv = int(round(ROOM[u] / spacing)), int(round(ROOM[v] / spacing))
        gu = (np.arange(nu) + 0.5) * spacing
        gv = (np.arange(nv) + 0.5) * spacing
        U, V = np.meshgrid(gu, gv, indexing="ij")
        for off, sgn in ((0.0, 1.0), (ROOM[axis], -1.0)):
            p = np.zeros((U.size, 3))
            p[:, axis] = off
            p[:, u] = U.ravel()
            p[:, v] = V.ravel()
            n = np.zeros_like(p)
            n[:, axis] = sgn
            pts.append(p); nrm.append(n); surf.append(np.full(U.size, fid))
            fid += 1
    pos = np.concatenate(pts).astype(np.float32)
    return pos, np.concatenate(nrm).astype(np.float32), np.concatenate(surf).astype(np.uint16)


def image_source_paths(tx, rx, max_order=2):
    """Textbook image sources of a rectangular room: for a wall sequence, mirror
    the source through each wall in turn; the path length is |image - rx|.
    Returns {wall sequence: (length, reflection points)} for valid paths."""
    walls = [(0, 0.0), (0, ROOM[0]), (1, 0.0), (1, ROOM[1]), (2, 0.0), (2, ROOM[2])]
    out = {}
    for order in range(1, max_order + 1):
        for seq in itertools.product(range(6), repeat=order):
            if any(seq[i] == seq[i + 1] for i in range(order - 1)):
                continue
            imgs = [np.array(tx, float)]
            for w in seq:
                a, off = walls[w]
                im = imgs[-1].copy()
                im[a] = 2 * off - im[a]
                imgs.append(im)
            # back-trace from rx
            tgt = np.array(rx, float)
            pts = [None] * order
            ok = True
            for m in range(order - 1, -1, -1):
                a, off = walls[seq[m]]
                src = imgs[m + 1]
                s = (off - tgt[a]) / (src[a] - tgt[a])
                if not (0 < s < 1):
                    ok = False
                    break
                p = tgt + s * (src - tgt)
                if np.any(p < -1e-12) or np.any(p > np.array(ROOM) + 1e-12):
                    ok = False
                    break
                pts[m] = p
                tgt = p
            if ok:
                out[tuple(seq)] = (float(np.linalg.norm(imgs[-1] - np.array(rx, float))), pts)
    return out


def _decode_labels(hi, lo, k):
    lab = [int((int(lo) >> (16 * m)) & 0xFFFF) for m in range(4)] + [int(int(hi) & 0xFFFF)]
    return tuple(lab[:k])


@pytest.fixture(scope="module")
def shoebox():
    pos, nrm, surf = dense_room()
    mat = np.zeros(pos.shape[0], np.uint8)
    mat[surf == 4] = 1
    sc = oracle.OracleScene(pos, nrm, surf, mat, r_p=0.04, grid_cell=0.25)
    tx = np.array([1.0, 1.0, 1.5], np.float32)
    rx = np.array([[4.0, 3.0, 1.2]], np.float32)
    p = oracle.SimParams(max_depth=2, capture=1, diffuse=0, n_rays=20000, rep_tries=8)
    sim = oracle.OracleSim(sc, tx, rx, p)
    return sc, sim, tx, rx


def _edge_distance(pt, axis):
    d = []
    for a in range(3):
        if a == axis:
            continue
        d += [pt[a], ROOM[a] - pt[a]]
    return min(d)


def test_shoebox_image_sources(shoebox):
    """Valid refined specular keys of order <= 2 = the image-source enumeration,
    with identical delays."""
    sc, sim, tx, rx = shoebox
    expect = image_source_paths(tx.astype(float), rx[0].astype(float), 2)
    walls_axis = [0, 0, 1, 1, 2, 2]
    P = sim.paths()
    got = {}
    for i in range(len(P["hi"])):
        if P["k"][i] == 0:
            continue
        got[_decode_labels(P["hi"][i], P["lo"][i], P["k"][i])] = i
    # every image-source path away from face edges is found
    for seq, (length, pts) in expect.items():
        far = all(_edge_distance(p, walls_axis[w]) > 0.1 for p, w in zip(pts, seq))
        if far:
            assert seq in got, seq
    for seq, i in got.items():
        assert seq in expect, seq
        length, pts = expect[seq]
        assert P["tau"][i] * C0 == pytest.approx(length, rel=1e-12)
        for m, p in enumerate(pts):
            assert np.allclose(P["pts"][i, m], p, atol=1e-9)
    assert len(got) >= 20 and len(got) <= len(expect)


def test_refined_points_minimise_eq1(shoebox):
    """Eq. 1 minimised with a library optimiser over points on the same planes
    agrees with the refined interaction points."""
    sc, sim, tx, rx = shoebox
    walls = [(0, 0.0), (0, ROOM[0]), (1, 0.0), (1, ROOM[1]), (2, 0.0), (2, ROOM[2])]
    P = sim.paths()
    checked = 0
    for i in range(len(P["hi"])):
        k = int(P["k"][i])
        if k == 0:
            continue
        seq = _decode_labels(P["hi"][i], P["lo"][i], k)

        def unpack(x):
            pts = []
            for m, w in enumerate(seq):
                a, off = walls[w]
                p = np.zeros(3)
                p[a] = off
                others = [b for b in range(3) if b != a]
                p[others[0]], p[others[1]] = x[2 * m], x[2 * m + 1]
                pts.append(p)
            return pts

        def f_d(x):
            chain = [tx.astype(float)] + unpack(x) + [rx[0].astype(float)]
            return sum(np.linalg.norm(chain[j + 1] - chain[j]) for j in range(len(chain) - 1))

        x0 = np.full(2 * k, 1.0)
        res = minimize(f_d, x0, method="BFGS", options={"gtol": 1e-12, "maxiter": 2000})
        opt = unpack(res.x)
        for m in range(k):
            assert np.allclose(opt[m], P["pts"][i, m], atol=1e-5)
        assert res.fun == pytest.approx(P["tau"][i] * C0, rel=1e-9)
        checked += 1
    assert checked >= 20


def test_dedup_independent_of_processing_order(shoebox):
    sc, sim, tx, rx = shoebox
    p = sim.params
    ids = np.random.default_rng(5).permutation(p.n_rays)
    sim2 = oracle.OracleSim(sc, tx, rx, p, ray_ids=ids)
    k1, k2 = sim.keys(), sim2.keys()
    assert np.array_equal(k1["hi"], k2["hi"]) and np.array_equal(k1["lo"], k2["lo"])
    assert np.array_equal(k1["rep"], k2["rep"])
    assert np.array_equal(k1["valid"], k2["valid"])


def test_diffuse_in_convex_room_always_valid(shoebox):
    """In an empty convex room every diffuse candidate sees the RX in front of
    its wall and unobstructed, so every diffuse key validates with its first
    (lowest ray id) candidate."""
    sc, _, tx, rx = shoebox
    p = oracle.SimParams(max_depth=2, capture=1, diffuse=1, n_rays=2000, rep_tries=8)
    sim = oracle.OracleSim(sc, tx, rx, p)
    K = sim.keys()
    H = sim.hits()
    ray, _, _ = sim.tried()
    first = np.concatenate([[0], np.cumsum(K["n_tried"])])[:-1]
    diff = ((K["hi"] >> np.uint64(55)) & np.uint64(1)).astype(bool)
    kk = ((K["hi"] >> np.uint64(52)) & np.uint64(7)).astype(int)
    # scatter points near a room edge sit in DPS mixing two walls; leave them out
    q = H["q"][ray[first], kk - 1]
    lo = np.minimum(q, np.array(ROOM) - q)
    near_edges = (lo < 0.1).sum(axis=1) >= 2
    sel = diff & ~near_edges
    assert sel.sum() > 100
    assert K["valid"][sel].all()
    assert (K["n_tried"][sel] == 1).all()


def _plate(center, normal, half, spacing, surf_id):
    normal = np.asarray(normal, float)
    a = int(np.argmax(np.abs(normal)))
    u, v = [b for b in range(3) if b != a]
    g = np.arange(-half, half + 1e-9, spacing)
    U, V = np.meshgrid(g, g, indexing="ij")
    p = np.zeros((U.size, 3))
    p[:, a] = center[a]
    p[:, u] = center[u] + U.ravel()
    p[:, v] = center[v] + V.ravel()
    n = np.tile(normal, (U.size, 1))
    return p, n, np.full(U.size, surf_id)


def test_visibility_and_los_occlusion():
    """A plate between RX and a wall patch hides the patch's DPS from the RX
    and blocks LOS; without the plate both are clear."""
    wall = _plate([0.0, 0.0, 0.0], [1, 0, 0], 0.5, 0.02, 0)
    plate = _plate([1.0, 0.0, 0.0], [1, 0, 0], 0.2, 0.02, 1)
    rx = np.array([[2.0, 0.0, 0.0]])
    for with_plate in (False, True):
        parts = [wall] + ([plate] if with_plate else [])
        pos = np.concatenate([p[0] for p in parts]).astype(np.float32)
        nrm = np.concatenate([p[1] for p in parts]).astype(np.float32)
        surf = np.concatenate([p[2] for p in parts]).astype(np.uint16)
        sc = oracle.OracleScene(pos, nrm, surf, np.zeros(pos.shape[0], np.uint8), r_p=0.02)
        vox, cnt, recv = sc.dps()
        # DPS on the wall nearest to the x axis
        wall_dps = [d for d in range(len(cnt)) if abs(recv[d, 0]) < 1e-6]
        near = min(wall_dps, key=lambda d: np.hypot(recv[d, 1], recv[d, 2]))
        far = max(wall_dps, key=lambda d: np.hypot(recv[d, 1], recv[d, 2]))
        bit, amb = sc.vis_pairs(rx, [0, 0], [near, far])
        assert bit[0] == (not with_plate)
        assert bit[1]  # the plate does not cover the wall's corner
        h = sc.cast(rx[0], [-1.0, 0.0, 0.0], t_max=1.5, weighted=False)
        assert h["hit"] == with_plate


def test_rough_wall_fully_visible_from_the_front():
    """Nothing stands between a receiver and a single wall in front of it, so
    every DPS of the wall is visible (the visibility matrix of Sec. II-B-1),
    also when the wall is rough: the test cast toward a DPS ends short of
    its reception point by the DPS's own extent (half a voxel diagonal plus
    r_p), so the bumps of its neighbours around that point do not count."""
    rng = np.random.default_rng(11)
    pos, nrm, surf = _plate([0.0, 0.0, 0.0], [1, 0, 0], 0.5, 0.02, 0)
    pos[:, 0] += rng.uniform(-0.005, 0.005, pos.shape[0])  # +-5 mm of roughness
    sc = oracle.OracleScene(pos.astype(np.float32), nrm.astype(np.float32),
                            surf.astype(np.uint16), np.zeros(pos.shape[0], np.uint8), r_p=0.05)
    _, cnt, _ = sc.dps()
    rx = np.array([[1.5, 0.2, -0.1]])
    n = len(cnt)
    bit, amb = sc.vis_pairs(rx, np.zeros(n, np.int32), np.arange(n, dtype=np.int32), delta=1e-7)
    assert n > 200
    assert bit[~amb].all() and amb.mean() < 0.02
    # a receiver closer to a reception point than the DPS's extent sees it by
    # definition (the test cast would start inside the DPS)
    _, _, recv = sc.dps()
    rx2 = np.array([[0.05, 0.0, 0.0]])
    margin = np.sqrt(3.0) / 2.0 * 0.0625 + 0.05
    near = np.nonzero(np.linalg.norm(recv - rx2[0], axis=1) - margin <= 1e-3)[0]
    assert near.size >= 2
    bit2, _ = sc.vis_pairs(rx2, np.zeros(near.size, np.int32), near.astype(np.int32))
    assert bit2.all()


# axis-aligned rectangles: (axis of the normal, plane coordinate, outward
# normal sign, (lo, hi) of the other two coordinates in axis order)
# (gaps of at least 30 cm between them keep every DPS on one surface)
_RECTS = {
    0: (2, 0.0, +1, ((-2.0, 1.8), (-2.0, 2.0))),   # floor z = 0
    1: (0, 2.0, -1, ((-2.0, 2.0), (0.3, 2.5))),    # wall x = 2
    2: (1, 0.5, -1, ((-0.8, 0.4), (0.3, 1.6))),    # occluder y = 0.5
    3: (0, 1.0, -1, ((-1.2, 0.4), (0.4, 2.0))),    # screen x = 1, parallel to the wall
}


def _rect_points(label, spacing=0.04):
    ax, c, sgn, ((a0, a1), (b0, b1)) = _RECTS[label]
    u, v = [b for b in range(3) if b != ax]
    A, B = np.meshgrid(np.arange(a0, a1 + 1e-9, spacing), np.arange(b0, b1 + 1e-9, spacing),
                       indexing="ij")
    p = np.zeros((A.size, 3))
    p[:, ax], p[:, u], p[:, v] = c, A.ravel(), B.ravel()
    n = np.zeros((A.size, 3))
    n[:, ax] = sgn
    return p, n


def _crosses(p0, p1, label, margin, end_eps):
    """Whether the open segment p0 -> p1 passes through rectangle `label`
    (grown by `margin`, the disc radius) away from its end points."""
    ax, c, _, ((a0, a1), (b0, b1)) = _RECTS[label]
    u, v = [b for b in range(3) if b != ax]
    d = p1[ax] - p0[ax]
    if d == 0.0:
        return False
    t = (c - p0[ax]) / d
    L = np.linalg.norm(p1 - p0)
    if not (end_eps / L < t < 1.0 - end_eps / L):
        return False
    x = p0 + t * (p1 - p0)
    return a0 - margin <= x[u] <= a1 + margin and b0 - margin <= x[v] <= b1 + margin


def test_valid_paths_are_physical():
    """Every valid path of a scene with an occluder obeys the geometry that
    Sec. II-B-1 / II-B-2 validate, checked here analytically against the
    scene's rectangles: each interaction point lies on the surface its key
    names (within t_d), each specular interaction reflects (both legs on the
    same side of its surface), no leg passes through a surface, and the
    delay is the polyline's length over the speed of light.  The
    occluder blocks the floor's specular image path to the RX, and a screen
    in front of the wall blocks the wall's image path on its TX side, so
    those keys are rejected while the screen's own reflection is valid."""
    parts = [_rect_points(l) for l in _RECTS]
    pos = np.vstack([p for p, _ in parts]).astype(np.float32)
    nrm = np.vstack([n for _, n in parts]).astype(np.float32)
    surf = np.concatenate([np.full(len(p), l) for l, (p, _) in enumerate(parts)]).astype(np.uint16)
    osc = oracle.OracleScene(pos, nrm, surf, np.zeros(len(pos), np.uint8), rho=0.25, r_p=0.05,
                             grid_cell=0.25)
    tx = np.array([-1.0, -1.0, 1.2])
    rx = np.array([[-0.5, 1.2, 1.0]])
    t_d = 0.01
    p = oracle.SimParams(max_depth=2, capture=1, diffuse=1, n_rays=100000, t_d=t_d)
    sim = oracle.OracleSim(osc, tx, rx, p)
    P = sim.paths()
    K = sim.keys()
    n_checked = 0
    for i in range(len(P["type"])):
        k, ty = int(P["k"][i]), int(P["type"][i])
        if k == 0:
            continue
        pts = [tx] + [P["pts"][i, m] for m in range(k)] + [rx[0]]
        lo = int(P["lo"][i])
        labels = [(lo >> (16 * m)) & 0xFFFF for m in range(min(k, 4))]
        for m in range(1, k + 1):
            q = pts[m]
            if ty == 1 and m == k:  # the scatter point: on some surface
                on = [l for l in _RECTS if abs(q[_RECTS[l][0]] - _RECTS[l][1]) <= t_d]
                assert on, (i, q)
                continue
            ax, c, _, _ = _RECTS[labels[m - 1]]
            assert abs(q[ax] - c) <= t_d + 1e-9, (i, m, q)
            a = pts[m - 1][ax] - c
            b = pts[m + 1][ax] - c
            assert a * b > 0, (i, m)  # reflection, not transmission
        # the delay is the polyline's length over c (specular and diffuse)
        length = sum(np.linalg.norm(pts[m + 1] - pts[m]) for m in range(k + 1))
        assert P["length"][i] == pytest.approx(length, rel=1e-9)
        assert P["tau"][i] == pytest.approx(length / 299792458.0, rel=1e-9)
        # inside a rectangle of points 4 cm apart every spot is within 3 cm of
        # a disc centre (r_p = 5 cm): a leg through it is certainly blocked
        for m in range(k + 1):
            for l in _RECTS:
                assert not _crosses(pts[m], pts[m + 1], l, 0.0, 0.02), (i, m, l)
        n_checked += 1
    assert n_checked > 20
    # the floor's one-bounce specular image path is blocked by the occluder
    img = tx * np.array([1, 1, -1.0])
    t = img[2] / (img[2] - rx[0, 2])
    fp = img + t * (rx[0] - img)
    assert _crosses(fp, rx[0], 2, 0.0, 0.02)
    spec1 = (((K["hi"] >> np.uint64(52)) & np.uint64(7)) == 1) & \
        (((K["hi"] >> np.uint64(55)) & np.uint64(1)) == 0)
    for label, valid in ((0, False), (1, False), (3, True)):
        sel = spec1 & (K["lo"] == label)
        assert sel.sum() == 1 and bool(K["valid"][sel][0]) == valid, label


def test_refinement_converges_on_a_cylinder():
    """Sec. II-B-2 on a curved surface: a convex cylinder (R = 3 m) of points
    with radial normals.  A candidate's own hit gives only an approximate
    tangent plane, so the image-method point must be refined (the hit's plane
    replaces the solve's until the normal is within t_a and the hit within
    t_d).  At the valid single-bounce path's point the law of reflection
    must hold to within t_a (plus half a degree for the discs' normals): the
    two legs' unit vectors sum to a vector within 1.5 degrees of the radial
    normal there.  The point must also lie within 5 cm of the true specular
    point, found here by root finding on the cylinder angle.  Several TX/RX
    placements, and a wide capture sphere whose candidates start several
    degrees off.  A key must validate within its first 8 candidates (a cap):
    without a cap every candidate is refined, and some candidate may start
    within t_a already and prove nothing about the retries."""
    R = 3.0
    na = int(round(2 * np.pi * R / 0.02))
    th = np.arange(na) * (2 * np.pi / na)
    z = np.arange(0.0, 2.0 + 1e-9, 0.02)
    TH, Z = np.meshgrid(th, z, indexing="ij")
    pos = np.column_stack([R * np.cos(TH.ravel()), R * np.sin(TH.ravel()), Z.ravel()])
    nrm = np.column_stack([np.cos(TH.ravel()), np.sin(TH.ravel()), np.zeros(TH.size)])
    n = len(pos)
    osc = oracle.OracleScene(pos.astype(np.float32), nrm.astype(np.float32),
                             np.zeros(n, np.uint16), np.zeros(n, np.uint8), rho=0.0625,
                             r_p=0.05, grid_cell=0.25)
    brentq = pytest.importorskip("scipy.optimize").brentq

    def at(a, d):
        return np.array([(R + d) * np.cos(a), (R + d) * np.sin(a), 1.0])

    for a_tx, d_tx, a_rx, d_rx in [(0.2, 1.2, 1.3, 1.6), (3.5, 2.5, 4.3, 1.0), (2.0, 1.0, 2.5, 2.5)]:
        tx, rx = at(a_tx, d_tx), at(a_rx, d_rx)
        p = oracle.SimParams(max_depth=1, capture=0, diffuse=0, n_rays=200000, r_rx=0.4,
                             rep_tries=8)
        P = oracle.OracleSim(osc, tx, rx[None], p).paths()
        spec = (P["type"] == 0) & (P["k"] == 1)
        assert spec.sum() == 1, (a_tx, a_rx)
        q = P["pts"][spec][0, 0]

        def tangential(a):
            pt = np.array([R * np.cos(a), R * np.sin(a), 1.0])
            u = (tx - pt) / np.linalg.norm(tx - pt) + (rx - pt) / np.linalg.norm(rx - pt)
            return u @ np.array([-np.sin(a), np.cos(a), 0.0])
        a_star = brentq(tangential, a_tx, a_rx)
        want = np.array([R * np.cos(a_star), R * np.sin(a_star), 1.0])
        b = (tx - q) / np.linalg.norm(tx - q) + (rx - q) / np.linalg.norm(rx - q)
        nr = np.array([q[0], q[1], 0.0])
        ang = np.degrees(np.arccos(np.clip(b @ nr / (np.linalg.norm(b) * np.linalg.norm(nr)),
                                           -1.0, 1.0)))
        assert ang < 1.5, (a_tx, a_rx, ang)
        assert np.linalg.norm(q - want) < 0.05, (a_tx, a_rx, q, want)


def test_adjoint_matches_central_differences(office):
    """Analytic dP_j / d(eps_r, sigma, S)_l (one-hot dL/dP) and the gradient of
    the per-RX dB-gain MSE against FP64 central differences of the oracle's
    own forward, on an office sample with diffuse paths."""
    sc = oracle.OracleScene(office.pos, office.nrm, office.surf, office.mat, r_p=0.015,
                            grid_cell=0.1)
    p = oracle.SimParams(max_depth=3, capture=1, diffuse=1, n_rays=1_000_000, rep_tries=4)
    sim = oracle.OracleSim(sc, office.tx, office.rx, p, ray_ids=np.arange(0, 1_000_000, 2000))
    base = [office.eps_r.astype(float), office.sigma.astype(float), office.scat.astype(float)]
    M = office.rx.shape[0]
    _, P0 = sim.field(*base)
    checked = 0
    for j in (0, 5, 11):
        dL = np.zeros(M)
        dL[j] = 1.0
        grads = sim.backward(*base, dL)
        for which in range(3):
            for l in range(len(base[0])):
                x = base[which][l]
                h = 1e-4 * x
                up = [b.copy() for b in base]
                dn = [b.copy() for b in base]
                up[which][l] += h
                dn[which][l] -= h
                fd = (sim.field(*up)[1][j] - sim.field(*dn)[1][j]) / (2 * h)
                if abs(fd) * x < 1e-7 * P0[j]:
                    continue  # below the resolution of the difference
                assert grads[which][l] == pytest.approx(fd, rel=1e-3)
                checked += 1
    assert checked >= 30
    # the configured loss: MSE of per-RX path gain in dB
    target = np.linspace(-75, -65, M)
    G0 = 10 * np.log10(P0)
    dL_dP = 2 * (G0 - target) / M * 10 / (P0 * np.log(10))
    ge, gs, gc = sim.backward(*base, dL_dP)

    def loss(b):
        return np.mean((10 * np.log10(sim.field(*b)[1]) - target) ** 2)

    for which, g in ((0, ge), (2, gc)):
        for l in range(len(base[0])):
            h = 1e-5 * base[which][l]
            up = [b.copy() for b in base]
            dn = [b.copy() for b in base]
            up[which][l] += h
            dn[which][l] -= h
            fd = (loss(up) - loss(dn)) / (2 * h)
            assert g[l] == pytest.approx(fd, rel=1e-3, abs=1e-6)


def test_single_wall_amplitude_snell_form(shoebox):
    """First-order path: a = lambda/(4 pi d) * R * Gamma_TE(theta), with Gamma
    from the Snell-law form and theta from the image-source geometry (S = 0,
    so R = 1)."""
    import cmath
    sc, sim, tx, rx = shoebox
    eps = np.array([5.3, 3.0])
    sig = np.array([0.03, 0.01])
    a, _ = sim.field(eps, sig, np.zeros(2))
    P = sim.paths()
    expect = image_source_paths(tx.astype(float), rx[0].astype(float), 1)
    walls_axis = [0, 0, 1, 1, 2, 2]
    lam = C0 / 28e9
    n_checked = 0
    for i in range(len(P["hi"])):
        if P["k"][i] != 1:
            continue
        w = _decode_labels(P["hi"][i], P["lo"][i], 1)
        length, pts = expect[w]
        ax = walls_axis[w[0]]
        din = (pts[0] - tx.astype(float)) / np.linalg.norm(pts[0] - tx.astype(float))
        c = abs(din[ax])
        l = 1 if w[0] == 4 else 0
        eta = complex(eps[l], -sig[l] / (2 * np.pi * 28e9 * 8.8541878128e-12))
        n2 = cmath.sqrt(eta)
        ct = cmath.sqrt(1 - (1 - c * c) / eta)
        gam = (c - n2 * ct) / (c + n2 * ct)
        want = lam / (4 * np.pi * length) * gam
        assert abs(a[i] - want) < 1e-10 * abs(want)
        n_checked += 1
    assert n_checked == 6
