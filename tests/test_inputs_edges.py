"""The seeded edge inputs (office box edges, free-standing room wedges) are
valid wedges in the sense nrt_scene_set_edges checks -- unit face normals
normal to the edge, faces not coplanar -- and convex: each face's in-plane
direction away from the edge points against the other face's outward normal.
The office edges lie on the boxes' faces."""
import numpy as np

from paper_2507_04021_gb300 import inputs


def _check_wedges(E):
    a, b = E.a.astype(np.float64), E.b.astype(np.float64)
    n0, n1 = E.n0.astype(np.float64), E.n1.astype(np.float64)
    e = b - a
    L = np.linalg.norm(e, axis=1)
    assert np.all(L >= 1e-6)
    e /= L[:, None]
    for n in (n0, n1):
        assert np.allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-3)
        assert np.all(np.abs((n * e).sum(1)) <= 1e-3)
    assert np.all(np.abs((n0 * n1).sum(1)) <= 1 - 1e-6)
    # convex: with t0 in face 0 (normal to the edge, oriented against n1) and
    # t1 likewise, the interior angle acos(t0 . t1) lies in (0, pi)
    t0 = np.cross(n0, e)
    t0 *= np.where((t0 * n1).sum(1) > 0, -1.0, 1.0)[:, None]
    t1 = np.cross(n1, e)
    t1 *= np.where((t1 * n0).sum(1) > 0, -1.0, 1.0)[:, None]
    ang = np.arccos(np.clip((t0 * t1).sum(1), -1, 1))
    assert np.all((ang > 1e-3) & (ang < np.pi - 1e-3))
    return ang


def test_office_edges_are_convex_box_edges():
    o = inputs.office_scene(n_points=2000)
    E = inputs.office_edges(o.extra["boxes"])
    assert len(E) == 8 * len(o.extra["boxes"])
    ang = _check_wedges(E)
    assert np.allclose(ang, np.pi / 2, atol=1e-6)  # box edges: right angles
    for i, (x0, x1, y0, y1, h) in enumerate(o.extra["boxes"]):
        pts = np.concatenate([E.a[8 * i:8 * i + 8], E.b[8 * i:8 * i + 8]]).astype(np.float64)
        on_x = np.isclose(pts[:, 0], x0, atol=1e-5) | np.isclose(pts[:, 0], x1, atol=1e-5)
        on_y = np.isclose(pts[:, 1], y0, atol=1e-5) | np.isclose(pts[:, 1], y1, atol=1e-5)
        assert np.all(on_x | on_y)
        assert np.all((pts[:, 2] >= -1e-6) & (pts[:, 2] <= h + 1e-5))
        assert np.all(E.m0[8 * i:8 * i + 8] == 4 + i % 4)


def test_room_wedges_are_valid_and_seeded():
    E = inputs.room_edges()
    assert len(E) == 24
    ang = _check_wedges(E)
    assert ang.min() > np.deg2rad(29) and ang.max() < np.deg2rad(151)
    E2 = inputs.room_edges()
    assert np.array_equal(E.a, E2.a) and np.array_equal(E.n1, E2.n1)
