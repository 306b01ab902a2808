"""Pins for the oracle's geometry: voxelisation (Sec. II-A), the ray/disc
intersection and Eq. 3 / Eq. 4 weighted average (Sec. II-C), the Fibonacci
launch, and brute force vs the uniform grid.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2507_04021_gb300 import inputs


def _scene(points, normals, surf=None, mat=None, **kw):
    pos = np.asarray(points, np.float32).reshape(-1, 3)
    nrm = np.asarray(normals, np.float32).reshape(-1, 3)
    n = pos.shape[0]
    surf = np.zeros(n, np.uint16) if surf is None else np.asarray(surf, np.uint16)
    mat = np.zeros(n, np.uint8) if mat is None else np.asarray(mat, np.uint8)
    return oracle.OracleScene(pos, nrm, surf, mat, **kw)


def test_table1_defaults_match_paper():
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1_params.json")))
    p = oracle.SimParams()
    assert p.kappa == g["kappa"]
    assert p.t_a_deg == g["t_a"] and p.t_d == g["t_d"]
    sc = _scene([[0, 0, 0]], [[0, 0, 1]])
    assert sc.rho == g["rho"] and sc.r_p == g["r_p"] and sc.lambda_d == g["lambda_d"]


def test_voxelisation_matches_float32_floor(room):
    """DPS = distinct voxels floor((p - bmin)/rho) taken in float32; reception point = mean."""
    sc = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, r_p=0.05)
    bmin = room.pos.min(axis=0)
    v = np.floor((room.pos - bmin) / np.float32(0.0625)).astype(np.int64)
    uniq, inv, cnt = np.unique(v, axis=0, return_inverse=True, return_counts=True)
    vox, c, recv = sc.dps()
    assert np.array_equal(sc.bmin(), bmin)
    assert np.array_equal(vox, uniq)
    assert np.array_equal(c, cnt)
    mean = np.zeros((uniq.shape[0], 3))
    np.add.at(mean, inv.ravel(), room.pos.astype(np.float64))
    mean /= cnt[:, None]
    assert np.allclose(recv, mean, rtol=0, atol=1e-12)
    assert np.array_equal(sc.point_dps(), inv.ravel())


def test_voxel_membership_is_the_exact_floor_up_to_float32_rounding(office):
    """Sec. II-A's voxel of a point is floor((p - bmin) / rho).  The oracle
    takes that integer decision in float32, the kernel's precision (a
    reading); here it is pinned to the exact quotient evaluated in FP64:
    every point farther from a voxel face than the float32 rounding of the
    quotient gets exactly floor of the exact value, and the few that are
    nearer get it or a neighbour (counted: the points whose DPS depends on
    the precision)."""
    sc = oracle.OracleScene(office.pos, office.nrm, office.surf, office.mat, r_p=0.015,
                            grid_cell=0.1)
    vox, _, _ = sc.dps()
    v = vox[sc.point_dps()].astype(np.int64)
    bmin = sc.bmin().astype(np.float64)
    q = (office.pos.astype(np.float64) - bmin) / 0.0625  # rho = 0.0625 is exact in binary
    fl = np.floor(q)
    # float32 rounding of the difference and of the quotient: a few ulp of q
    band = 4.0 * np.spacing(np.abs(q).astype(np.float32)).astype(np.float64) + 1e-12
    near = (q - fl < band) | (fl + 1.0 - q < band)
    far = ~near
    assert np.array_equal(v[far], fl[far].astype(np.int64))
    assert np.all(np.abs(v[near] - fl[near]) <= 1)
    n_near = int(near.any(axis=1).sum())
    print("points within float32 rounding of a voxel face:", n_near, "of", len(v))
    assert n_near < 1e-3 * len(v)


def test_single_disc_hit_and_miss():
    sc = _scene([[0, 0, 0]], [[0, 0, 1]], r_p=0.05)
    h = sc.cast([0.01, 0.02, 1.0], [0, 0, -1])
    assert h["hit"] and h["idx"] == 0
    assert np.allclose(h["q"], [0.01, 0.02, 0.0], atol=1e-15)
    assert np.allclose(h["n"], [0, 0, 1]) and h["t"] == pytest.approx(1.0)
    # hit from behind: normal turned to face the ray
    h = sc.cast([0.01, 0.02, -1.0], [0, 0, 1])
    assert h["hit"] and np.allclose(h["n"], [0, 0, -1])
    # outside the disc (closed disc of radius r_p)
    assert not sc.cast([0.06, 0.0, 1.0], [0, 0, -1])["hit"]
    assert sc.cast([0.0499, 0.0, 1.0], [0, 0, -1])["hit"]
    # behind the origin / below t_min
    assert not sc.cast([0.0, 0.0, -1.0], [0, 0, -1])["hit"]
    assert not sc.cast([0.0, 0.0, 5e-5], [0, 0, -1])["hit"]


def test_depth_attenuation_closed_form():
    """Ray along the common normal through two parallel discs Delta apart in one
    voxel: r_i = 0, so Eq. 4 gives weights 1 and exp(-lambda_d Delta) and Eq. 3
    puts q at depth Delta e^{-l D} / (1 + e^{-l D}) behind the first disc."""
    for lam, D in [(100.0, 0.01), (50.0, 0.02), (400.0, 0.005)]:
        sc = _scene([[0, 0, 0], [0, 0, -D]], [[0, 0, 1], [0, 0, 1]], r_p=0.05, lambda_d=lam)
        assert sc.n_dps == 1
        h = sc.cast([0, 0, 1.0], [0, 0, -1])
        D32 = float(np.float32(D))  # the scene stores float32 positions
        w = np.exp(-lam * D32)
        assert h["idx"] == 0
        assert h["q"][2] == pytest.approx(-D32 * w / (1 + w), rel=1e-12)
    # a disc in another voxel is not averaged
    sc = _scene([[0, 0, 0], [0, 0, -0.1]], [[0, 0, 1], [0, 0, 1]], r_p=0.05)
    assert sc.n_dps == 2
    h = sc.cast([0, 0, 1.0], [0, 0, -1])
    assert h["q"][2] == 0.0
    # skipping the first DPS exposes the second disc
    h2 = sc.cast([0, 0, 1.0], [0, 0, -1], skip_dps=h["dps"])
    assert h2["idx"] == 1 and h2["q"][2] == pytest.approx(-0.1)


def test_gaussian_weight_symmetry_and_limit():
    """Two tilted discs mirror-symmetric about the plane x = 0, ray along -z in
    that plane: equal weights, so the averaged normal is the symmetric one."""
    a = np.deg2rad(10.0)
    n1 = [np.sin(a), 0, np.cos(a)]
    n2 = [-np.sin(a), 0, np.cos(a)]
    sc = _scene([[0.01, 0, 0], [-0.01, 0, 0]], [n1, n2], r_p=0.05)
    h = sc.cast([0, 0.003, 1.0], [0, 0, -1])
    assert h["hit"]
    assert abs(h["n"][0]) < 1e-12 and h["n"][2] > 0.98
    # large lambda_d: q -> q_min
    sc = _scene([[0, 0, 0], [0, 0, -0.01]], [[0, 0, 1], [0, 0, 1]], r_p=0.05, lambda_d=1e5)
    assert abs(sc.cast([0, 0, 1.0], [0, 0, -1])["q"][2]) < 1e-12
    # weights are invariant to a rigid motion of scene and ray
    rng = np.random.default_rng(0)
    P = rng.normal(0, 0.01, (5, 3)); P[:, 2] = rng.normal(0, 0.002, 5)
    N = np.tile([0, 0, 1.0], (5, 1)) + rng.normal(0, 0.05, (5, 3))
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    o, d = np.array([0.002, -0.001, 1.0]), np.array([0.01, 0.02, -1.0])
    d /= np.linalg.norm(d)
    from scipy.spatial.transform import Rotation
    R = Rotation.from_euler("xyz", [0.3, -0.2, 0.5]).as_matrix()
    sh = np.array([3.0, 2.0, 1.0])
    s1 = _scene(P, N, r_p=0.05)
    h1 = s1.cast(o, d)
    # keep everything in one voxel after the motion: scale up rho
    s1b = _scene(P, N, r_p=0.05, rho=10.0)
    s2 = _scene(P @ R.T + sh, N @ R.T, r_p=0.05, rho=10.0)
    h1b = s1b.cast(o, d)
    h2 = s2.cast(R @ o + sh, R @ d)
    assert h1["hit"] and h2["hit"] and h1b["idx"] == h2["idx"]
    assert np.allclose(R @ h1b["q"] + sh, h2["q"], atol=2e-6)
    assert np.allclose(R @ h1b["n"], h2["n"], atol=2e-6)


def test_gaussian_weight_closed_form():
    """Two discs whose planes both pass through the hit point X of a ray along
    -z: disc 1 tilted by alpha with its centre a from X, disc 2 level with its
    centre b from X.  Both meet the ray at X (q_i = q_min, so the Eq. 4 depth
    factors are 1) and the Eq. 3 normal leans from +z toward n_1 by theta with
    tan(theta) = w1 sin(alpha) / (w1 cos(alpha) + w2), where
    w1 / w2 = exp(-(a^2 - b^2) / (2 r_p^2)): the Gaussian's width in closed form."""
    rp = 0.05
    for alpha_deg, a, b in [(20.0, 0.03, 0.01), (35.0, 0.045, 0.02), (10.0, 0.0, 0.04)]:
        al = np.deg2rad(alpha_deg)
        n1 = np.array([np.sin(al), 0.0, np.cos(al)])
        p1 = a * np.array([np.cos(al), 0.0, -np.sin(al)])  # in plane 1, a from X = 0
        p2 = np.array([0.0, b, 0.0])
        # lambda_d near 0: the float32 rounding of disc 1 moves its plane hit by
        # ~1e-9 m, which must not enter through the depth factor
        sc = _scene([p1, p2], [n1, [0, 0, 1]], r_p=rp, rho=10.0, lambda_d=1e-9)
        assert sc.n_dps == 1
        h = sc.cast([0.0, 0.0, 1.0], [0, 0, -1])
        assert h["hit"]
        # the scene keeps float32 positions and normals, as given
        P = np.array([p1, p2], np.float32).astype(np.float64)
        N = np.array([n1, [0, 0, 1]], np.float32).astype(np.float64)
        X = [np.array([0.0, 0.0, np.dot(P[i], N[i]) / N[i, 2]]) for i in range(2)]
        ra = np.linalg.norm(X[0] - P[0])
        rb = np.linalg.norm(X[1] - P[1])
        w_ratio = np.exp(-(ra * ra - rb * rb) / (2.0 * rp * rp))
        v = w_ratio * N[0] + N[1]  # the weighted normal sum, up to the factor w2
        theta = np.arctan2(v[0], v[2])
        n_got = np.asarray(h["n"])
        assert abs(n_got[1]) < 1e-12
        assert np.arctan2(n_got[0], n_got[2]) == pytest.approx(theta, abs=1e-9)


def test_non_finite_rays_hit_nothing():
    """Test-API guard: a ray with a NaN or infinite component is a miss for
    both intersection models (it must not reach the grid walk)."""
    sc = _scene([[0, 0, 0]], [[0, 0, 1]], r_p=0.05, grid_cell=0.25)
    for o, d in [([np.nan, 0, 1.0], [0, 0, -1]), ([0, 0, 1.0], [0, np.nan, -1]),
                 ([0, 0, np.inf], [0, 0, -1]), ([0, 0, 1.0], [0, 0, 0])]:
        assert not sc.cast(o, d)["hit"]
        assert not sc.cast_sdf(np.array(o, float), np.array(d, float), 0.02)["hit"]


def test_tie_rule_smaller_index():
    """Coplanar discs covering the hit point tie exactly in t: q_min is the
    smaller point index."""
    sc = _scene([[0.01, 0, 0], [-0.01, 0, 0]], [[0, 0, 1], [0, 0, 1]], r_p=0.05)
    assert sc.cast([0, 0, 1.0], [0, 0, -1])["idx"] == 0
    sc = _scene([[-0.01, 0, 0], [0.01, 0, 0]], [[0, 0, 1], [0, 0, 1]], r_p=0.05)
    assert sc.cast([0, 0, 1.0], [0, 0, -1])["idx"] == 0


def test_ambiguity_flags_edges():
    sc = _scene([[0, 0, 0]], [[0, 0, 1]], r_p=0.05)
    assert sc.cast([0.04999, 0, 1.0], [0, 0, -1], delta=1e-4)["amb"]
    assert not sc.cast([0.02, 0, 1.0], [0, 0, -1], delta=1e-4)["amb"]
    # grazing incidence widens the band by 1/|d.n|
    d = np.array([1.0, 0, -0.01]); d /= np.linalg.norm(d)
    o = np.array([0.049 - 100 * 0.0, 0, 0]) - 1.0 * d
    assert sc.cast(o, d, delta=1e-5)["amb"]


def test_fibonacci_directions():
    N = 20000
    ids = np.arange(N)
    D = oracle.fib_dirs(N, ids)
    assert np.allclose(np.linalg.norm(D, axis=1), 1.0, atol=1e-14)
    assert np.linalg.norm(D.mean(axis=0)) < 2.0 / N
    # independent integer arithmetic for the golden angle (Python big ints)
    G = 0x61C8864680B583EB
    for i in (0, 1, 2, 7, 12345, 19999):
        u = (i * G) % (1 << 64)
        phi = 2 * np.pi * (u / 2.0 ** 64)
        z = 1 - (2 * i + 1) / N
        r = np.sqrt(1 - z * z)
        assert np.allclose(D[i], [r * np.cos(phi), r * np.sin(phi), z], atol=1e-12)
    assert G == round((2 - (1 + 5 ** 0.5) / 2) * 2 ** 64) or abs(G - (2 - (1 + 5 ** 0.5) / 2) * 2 ** 64) < 2 ** 12


def _compare_casts(sa, sb, rays, delta):
    for o, d in rays:
        ha = sa.cast(o, d, delta=delta)
        hb = sb.cast(o, d, delta=delta)
        assert ha["hit"] == hb["hit"]
        assert ha["amb"] == hb["amb"]
        if ha["hit"]:
            assert ha["idx"] == hb["idx"]
            assert np.array_equal(ha["q"], hb["q"]) or np.allclose(ha["q"], hb["q"], atol=1e-12)


def test_grid_equals_brute_force_room(room):
    bf = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, r_p=0.05)
    gr = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, r_p=0.05, grid_cell=0.25)
    rng = np.random.default_rng(1)
    rays = []
    for _ in range(400):
        o = rng.uniform([0.2, 0.2, 0.2], [4.8, 3.8, 2.8])
        d = rng.normal(size=3)
        rays.append((o, d / np.linalg.norm(d)))
    _compare_casts(bf, gr, rays, delta=1e-5 * room.diag)


def test_grid_equals_brute_force_office_subset(office):
    """Office scene restricted to a 3 m x 3 m corner so brute force stays cheap."""
    m = (office.pos[:, 0] < 3.0) & (office.pos[:, 1] < 3.0)
    pos, nrm, surf, mat = office.pos[m], office.nrm[m], office.surf[m], office.mat[m]
    bf = oracle.OracleScene(pos, nrm, surf, mat, r_p=0.015)
    gr = oracle.OracleScene(pos, nrm, surf, mat, r_p=0.015, grid_cell=0.1)
    rng = np.random.default_rng(2)
    rays = []
    for _ in range(150):
        o = rng.uniform([0.3, 0.3, 0.3], [2.7, 2.7, 2.7])
        d = rng.normal(size=3)
        rays.append((o, d / np.linalg.norm(d)))
    _compare_casts(bf, gr, rays, delta=1e-5 * office.diag)


def test_dps_directed_launch_hits_its_target_dps():
    """One ray per DPS (Sec. II-B), ray i toward the reception point of the
    i-th DPS in voxel Morton order: in the convex room a ray aimed at a
    reception point either hits that DPS or a neighbour sharing its wall
    (the reception point lies between discs) or leaves through a gap."""
    room = inputs.room_scene()
    osc = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    sim = oracle.OracleSim(osc, room.tx, np.array([[4.0, 3.0, 1.2]]), oracle.SimParams(
        max_depth=1, capture=0, diffuse=0, n_rays=0, launch=1, validate=0))
    H = sim.hits()
    vox, cnt, recv = osc.dps()
    def spread(x):
        r = np.zeros_like(x)
        for b in range(21):
            r |= ((x >> b) & 1) << (3 * b)
        return r
    v = vox.astype(np.int64)
    order = np.argsort(spread(v[:, 0]) | (spread(v[:, 1]) << 1) | (spread(v[:, 2]) << 2), kind="stable")
    target = order[np.arange(osc.n_dps)]
    first = H["dps"][:, 0]
    hit = first >= 0
    assert hit.mean() > 0.3
    same = first[hit] == target[hit]
    near = np.abs(v[first[hit]] - v[target[hit]]).max(axis=1) <= 1
    assert same.mean() > 0.5 and near.all()
