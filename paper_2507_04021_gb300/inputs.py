"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module only *draws inputs*: point clouds of oriented, labelled surface
samples, transmitter/receiver positions, material tables, trajectories and ray
budgets.  It holds none of the method's arithmetic (no voxelisation, no
intersection, no field formula); both the CUDA library and the FP64 oracle
consume the float32 arrays it returns.

The paper's own scenes (a corridor and the Replica "room 0" scan, Sec. III)
are not available, so two synthetic indoor scenes stand in for them:

* ``room_scene``  -- a 5 x 4 x 3 m box room, 5,000 points on its six inner
  faces, no noise (the small case the oracle brute-forces).
* ``office_scene`` -- a 20 x 10 x 3 m room with 40 axis-aligned boxes,
  2,000,000 points with 1 cm Gaussian position noise and 2 degree normal
  jitter, 8 material labels.

Each point carries the attributes of the paper's augmented point cloud
(Sec. II): position p_i, unit normal n, surface label l_s (one per planar
face) and material label l_m.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Scene",
    "room_scene",
    "office_scene",
    "office_receivers",
    "office_materials",
    "trajectory",
    "ray_budgets",
    "rng_for",
    "Edges",
    "office_edges",
    "room_edges",
]

# Seeds: one per input family.
SEED_ROOM = 1
SEED_OFFICE = 2
SEED_HIDDEN_MATERIALS = 3
SEED_TRAJECTORY = 4
SEED_BUDGETS = 5
SEED_MLP = 6
SEED_EDGES = 7


def rng_for(seed: int, stream: int = 0) -> np.random.Generator:
    """PCG64 generator for (seed, stream); streams keep input families apart."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, stream])))


@dataclass
class Scene:
    """An augmented point cloud plus the antenna layout and materials drawn with it."""

    pos: np.ndarray          # float32 [N,3]
    nrm: np.ndarray          # float32 [N,3], unit
    surf: np.ndarray         # uint16 [N]  surface label l_s
    mat: np.ndarray          # uint8  [N]  material label l_m
    tx: np.ndarray           # float32 [3]
    rx: np.ndarray           # float32 [M,3]
    eps_r: np.ndarray        # float32 [L]
    sigma: np.ndarray        # float32 [L]  S/m
    scat: np.ndarray         # float32 [L]  scattering coefficient S
    freq: float              # Hz
    extra: dict = field(default_factory=dict)

    @property
    def n_points(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_labels(self) -> int:
        return int(self.eps_r.shape[0])

    @property
    def diag(self) -> float:
        """Diagonal of the axis-aligned bounding box of the point positions."""
        lo = self.pos.astype(np.float64).min(axis=0)
        hi = self.pos.astype(np.float64).max(axis=0)
        return float(np.linalg.norm(hi - lo))


# ---------------------------------------------------------------------------
# Rectangular faces.  A face is (axis, offset, (lo_u, hi_u), (lo_v, hi_v),
# normal_sign) where u, v are the two other axes in increasing order.
# ---------------------------------------------------------------------------

def _face_points(rng, axis, offset, ur, vr, n):
    u_ax, v_ax = [a for a in range(3) if a != axis]
    pts = np.empty((n, 3), np.float64)
    pts[:, axis] = offset
    pts[:, u_ax] = rng.uniform(ur[0], ur[1], n)
    pts[:, v_ax] = rng.uniform(vr[0], vr[1], n)
    return pts


def _face_area(ur, vr):
    return (ur[1] - ur[0]) * (vr[1] - vr[0])


def _split_by_area(n_total, areas):
    """Largest-remainder split of n_total over faces in proportion to area."""
    areas = np.asarray(areas, np.float64)
    raw = n_total * areas / areas.sum()
    cnt = np.floor(raw).astype(np.int64)
    rem = n_total - int(cnt.sum())
    order = np.argsort(-(raw - cnt), kind="stable")
    cnt[order[:rem]] += 1
    return cnt


def room_scene(n_points: int = 5000, seed: int = SEED_ROOM) -> Scene:
    """Box room [0,5]x[0,4]x[0,3], points uniform on the 6 inner faces.

    Face ids (= surface labels): 0 x=0, 1 x=5, 2 y=0, 3 y=4, 4 floor z=0,
    5 ceiling z=3.  Normals point into the room; no position noise.
    Material 1 = floor (eps_r 3.0, sigma 0.01 S/m), material 0 = walls and
    ceiling (eps_r 5.3, sigma 0.03 S/m); scattering coefficient 0.
    """
    rng = rng_for(seed)
    L = (5.0, 4.0, 3.0)
    faces = []  # (axis, offset, ur, vr, normal sign)
    for axis in range(3):
        u_ax, v_ax = [a for a in range(3) if a != axis]
        ur, vr = (0.0, L[u_ax]), (0.0, L[v_ax])
        faces.append((axis, 0.0, ur, vr, +1.0))
        faces.append((axis, L[axis], ur, vr, -1.0))
    counts = _split_by_area(n_points, [_face_area(f[2], f[3]) for f in faces])
    pos, nrm, surf, mat = [], [], [], []
    for fid, (f, c) in enumerate(zip(faces, counts)):
        axis, off, ur, vr, sgn = f
        p = _face_points(rng, axis, off, ur, vr, int(c))
        n = np.zeros_like(p)
        n[:, axis] = sgn
        pos.append(p)
        nrm.append(n)
        surf.append(np.full(int(c), fid, np.uint16))
        mat.append(np.full(int(c), 1 if fid == 4 else 0, np.uint8))
    return Scene(
        pos=np.concatenate(pos).astype(np.float32),
        nrm=np.concatenate(nrm).astype(np.float32),
        surf=np.concatenate(surf),
        mat=np.concatenate(mat),
        tx=np.array([1.0, 1.0, 1.5], np.float32),
        rx=np.array([[4.0, 3.0, 1.2]], np.float32),
        eps_r=np.array([5.3, 3.0], np.float32),
        sigma=np.array([0.03, 0.01], np.float32),
        scat=np.array([0.0, 0.0], np.float32),
        freq=28e9,
        extra={"room": L, "r_p": 0.05, "rho": 0.0625, "lambda_d": 100.0,
               "r_rx": 0.1, "n_rays": 20000, "max_depth": 2},
    )


def office_receivers() -> np.ndarray:
    """16 receivers on x in {2.5, 7.5, 12.5, 17.5}, y in {2, 4, 6, 8}, z = 1.2."""
    rx = [(x, y, 1.2) for x in (2.5, 7.5, 12.5, 17.5) for y in (2.0, 4.0, 6.0, 8.0)]
    return np.array(rx, np.float32)


OFFICE_TX = (3.0, 5.0, 2.0)
TRAJ_START = (2.0, 2.0, 1.0)


def office_materials(seed: int = SEED_OFFICE, n_labels: int = 8):
    """eps_r ~ U[2,7], sigma ~ logU[1e-3, 1e-1] S/m, S ~ U[0.1, 0.5] per label."""
    rng = rng_for(seed, 1)
    eps = rng.uniform(2.0, 7.0, n_labels)
    sig = np.exp(rng.uniform(np.log(1e-3), np.log(1e-1), n_labels))
    sca = rng.uniform(0.1, 0.5, n_labels)
    return eps.astype(np.float32), sig.astype(np.float32), sca.astype(np.float32)


def _rect_dist(px, py, x0, x1, y0, y1):
    dx = max(x0 - px, 0.0, px - x1)
    dy = max(y0 - py, 0.0, py - y1)
    return float(np.hypot(dx, dy))


def _office_boxes(rng, n_boxes, clear_pts):
    boxes = []
    while len(boxes) < n_boxes:
        sx, sy = rng.uniform(0.4, 2.0, 2)
        h = rng.uniform(0.4, 2.0)
        x0 = rng.uniform(0.0, 20.0 - sx)
        y0 = rng.uniform(0.0, 10.0 - sy)
        x1, y1 = x0 + sx, y0 + sy
        if all(_rect_dist(px, py, x0, x1, y0, y1) >= 0.5 for px, py in clear_pts):
            boxes.append((x0, x1, y0, y1, h))
    return np.array(boxes, np.float64)


def _inside_any_box(p, boxes, own):
    """Strictly inside some box other than `own` (floor points under a box count)."""
    inside = np.zeros(p.shape[0], bool)
    for b, (x0, x1, y0, y1, h) in enumerate(boxes):
        m = (p[:, 0] > x0) & (p[:, 0] < x1) & (p[:, 1] > y0) & (p[:, 1] < y1) & \
            (p[:, 2] >= 0.0) & (p[:, 2] < h) & (own != b)
        inside |= m
    return inside


def office_scene(n_points: int = 2_000_000, seed: int = SEED_OFFICE, n_boxes: int = 40,
                 pos_noise: float = 0.01, nrm_jitter_deg: float = 2.0) -> Scene:
    """20x10x3 m office with 40 boxes; see the module docstring.

    Surface labels: 0 x=0, 1 x=20, 2 y=0, 3 y=10, 4 floor, 5 ceiling, and
    6 + 5*b + f for box b, f in (-x, +x, -y, +y, top).  Material labels:
    floor 0, ceiling 1, long walls (y=0, y=10) 2, short walls (x=0, x=20) 3,
    box b -> 4 + b % 4.  Boxes keep 0.5 m horizontal clearance from the
    transmitter, every receiver and the trajectory start.
    """
    rng = rng_for(seed)
    rx = office_receivers()
    clear = [OFFICE_TX[:2], TRAJ_START[:2]] + [tuple(r[:2]) for r in rx.astype(np.float64)]
    boxes = _office_boxes(rng, n_boxes, clear)

    # faces: (axis, offset, ur, vr, normal sign, surf, mat, own box)
    Lr = (20.0, 10.0, 3.0)
    faces = []
    room_mat = {0: 3, 1: 3, 2: 2, 3: 2, 4: 0, 5: 1}
    fid = 0
    for axis in range(3):
        u_ax, v_ax = [a for a in range(3) if a != axis]
        ur, vr = (0.0, Lr[u_ax]), (0.0, Lr[v_ax])
        faces.append((axis, 0.0, ur, vr, +1.0, fid, room_mat[fid], -1)); fid += 1
        faces.append((axis, Lr[axis], ur, vr, -1.0, fid, room_mat[fid], -1)); fid += 1
    for b, (x0, x1, y0, y1, h) in enumerate(boxes):
        m = 4 + b % 4
        s0 = 6 + 5 * b
        faces.append((0, x0, (y0, y1), (0.0, h), -1.0, s0 + 0, m, b))
        faces.append((0, x1, (y0, y1), (0.0, h), +1.0, s0 + 1, m, b))
        faces.append((1, y0, (x0, x1), (0.0, h), -1.0, s0 + 2, m, b))
        faces.append((1, y1, (x0, x1), (0.0, h), +1.0, s0 + 3, m, b))
        faces.append((2, h, (x0, x1), (y0, y1), +1.0, s0 + 4, m, b))
    areas = np.array([_face_area(f[2], f[3]) for f in faces])
    prob = areas / areas.sum()

    acc_p, acc_f = [], []
    need = n_points
    while need > 0:
        batch = int(need * 1.15) + 1024
        fsel = rng.choice(len(faces), size=batch, p=prob)
        p = np.empty((batch, 3), np.float64)
        for fi in np.unique(fsel):
            idx = np.nonzero(fsel == fi)[0]
            axis, off, ur, vr = faces[fi][:4]
            p[idx] = _face_points(rng, axis, off, ur, vr, idx.size)
        own = np.array([faces[f][7] for f in fsel])
        keep = ~_inside_any_box(p, boxes, own)
        p, fsel = p[keep][:need], fsel[keep][:need]
        acc_p.append(p)
        acc_f.append(fsel)
        need -= p.shape[0]
    p = np.concatenate(acc_p)
    fsel = np.concatenate(acc_f)

    axis = np.array([faces[f][0] for f in range(len(faces))])[fsel]
    sgn = np.array([faces[f][4] for f in range(len(faces))])[fsel]
    n0 = np.zeros_like(p)
    n0[np.arange(p.shape[0]), axis] = sgn
    # tangent basis per face axis
    t1 = np.zeros_like(p)
    t2 = np.zeros_like(p)
    t1[np.arange(p.shape[0]), (axis + 1) % 3] = 1.0
    t2[np.arange(p.shape[0]), (axis + 2) % 3] = 1.0
    beta = rng.uniform(0.0, 2.0 * np.pi, p.shape[0])
    ax = np.cos(beta)[:, None] * t1 + np.sin(beta)[:, None] * t2
    alpha = np.abs(rng.normal(0.0, np.deg2rad(nrm_jitter_deg), p.shape[0]))
    n = n0 * np.cos(alpha)[:, None] + np.cross(ax, n0) * np.sin(alpha)[:, None]
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    p = p + rng.normal(0.0, pos_noise, p.shape)

    surf = np.array([faces[f][5] for f in range(len(faces))], np.uint16)[fsel]
    mat = np.array([faces[f][6] for f in range(len(faces))], np.uint8)[fsel]
    eps, sig, sca = office_materials(seed)
    return Scene(
        pos=p.astype(np.float32), nrm=n.astype(np.float32), surf=surf, mat=mat,
        tx=np.array(OFFICE_TX, np.float32), rx=rx,
        eps_r=eps, sigma=sig, scat=sca, freq=28e9,
        extra={"room": Lr, "boxes": boxes, "r_p": 0.015, "rho": 0.0625,
               "lambda_d": 100.0, "n_rays": 1_000_000, "max_depth": 5},
    )


@dataclass
class Edges:
    """Edges of the augmented point cloud (Sec. II): segment ends a -> b, the
    outward normals n0, n1 of the two faces that meet there and their
    material labels.  The faces bound a convex wedge."""
    a: np.ndarray   # [n, 3] float32
    b: np.ndarray   # [n, 3] float32
    n0: np.ndarray  # [n, 3] float32
    n1: np.ndarray  # [n, 3] float32
    m0: np.ndarray  # [n] uint8
    m1: np.ndarray  # [n] uint8

    def __len__(self) -> int:
        return int(self.m0.shape[0])


def _edges(rows) -> Edges:
    a, b, n0, n1, m0, m1 = zip(*rows)
    f = lambda x: np.asarray(x, np.float32).reshape(-1, 3)  # noqa: E731
    return Edges(f(a), f(b), f(n0), f(n1), np.asarray(m0, np.uint8), np.asarray(m1, np.uint8))


def office_edges(boxes: np.ndarray) -> Edges:
    """The convex edges of the office boxes: 4 vertical edges (floor to top)
    and the 4 edges of the top face, 8 per box; both faces carry the box's
    material (4 + b % 4)."""
    rows = []
    for b, (x0, x1, y0, y1, h) in enumerate(boxes):
        m = 4 + b % 4
        for x, nx in ((x0, -1.0), (x1, 1.0)):
            for y, ny in ((y0, -1.0), (y1, 1.0)):
                rows.append(((x, y, 0.0), (x, y, h), (nx, 0, 0), (0, ny, 0), m, m))
        for y, ny in ((y0, -1.0), (y1, 1.0)):
            rows.append(((x0, y, h), (x1, y, h), (0, 0, 1.0), (0, ny, 0), m, m))
        for x, nx in ((x0, -1.0), (x1, 1.0)):
            rows.append(((x, y0, h), (x, y1, h), (0, 0, 1.0), (nx, 0, 0), m, m))
    return _edges(rows)


def room_edges(n_edges: int = 24, seed: int = SEED_EDGES) -> Edges:
    """Free-standing wedges inside the 5 x 4 x 3 m room (no points of their
    own): random centre in [1, 4] x [0.8, 3.2] x [0.5, 2.5], random direction,
    length U[0.5, 1.5], interior angle U[30, 150] degrees, random face
    orientation about the edge and face materials in {0, 1}."""
    rng = rng_for(seed)
    rows = []
    for _ in range(n_edges):
        c = rng.uniform((1.0, 0.8, 0.5), (4.0, 3.2, 2.5))
        e = rng.normal(size=3)
        e /= np.linalg.norm(e)
        L = rng.uniform(0.5, 1.5)
        u = np.cross(e, rng.normal(size=3))
        u /= np.linalg.norm(u)
        w = np.cross(e, u)
        alpha = np.deg2rad(rng.uniform(30.0, 150.0))
        t0, t1 = u, np.cos(alpha) * u + np.sin(alpha) * w
        n0 = np.cross(e, t0)
        n0 = -n0 if n0 @ t1 > 0 else n0
        n1 = np.cross(e, t1)
        n1 = -n1 if n1 @ t0 > 0 else n1
        m = rng.integers(0, 2, 2)
        rows.append((c - 0.5 * L * e, c + 0.5 * L * e, n0 / np.linalg.norm(n0),
                     n1 / np.linalg.norm(n1), m[0], m[1]))
    return _edges(rows)


def trajectory(boxes: np.ndarray, n_steps: int = 256, step: float = 0.2,
               seed: int = SEED_TRAJECTORY, margin: float = 0.3) -> np.ndarray:
    """Robot TX positions on a 0.2 m-step polyline at 1.0 m height.

    The heading turns by U[-30, 30] degrees per step; a step that would come
    within `margin` of a wall or a box footprint mirrors the heading (x, then
    y component), else reverses it, else the robot stays put.
    """
    rng = rng_for(seed)

    def ok(x, y):
        if x < margin or x > 20.0 - margin or y < margin or y > 10.0 - margin:
            return False
        for (x0, x1, y0, y1, _h) in boxes:
            if _rect_dist(x, y, x0, x1, y0, y1) < margin:
                return False
        return True

    x, y = TRAJ_START[0], TRAJ_START[1]
    hd = rng.uniform(0.0, 2.0 * np.pi)
    out = np.empty((n_steps, 3), np.float64)
    for i in range(n_steps):
        out[i] = (x, y, TRAJ_START[2])
        hd += np.deg2rad(rng.uniform(-30.0, 30.0))
        moved = False
        for cand in (hd, np.pi - hd, -hd, hd + np.pi):
            nx, ny = x + step * np.cos(cand), y + step * np.sin(cand)
            if ok(nx, ny):
                x, y, hd, moved = nx, ny, cand, True
                break
        if not moved:
            pass
    return out.astype(np.float32)


def ray_budgets(n_pairs: int = 256, lo: int = 100_000, hi: int = 1_000_000,
                seed: int = SEED_BUDGETS) -> np.ndarray:
    """Per-pair ray budgets, integer U[lo, hi]."""
    return rng_for(seed).integers(lo, hi + 1, size=n_pairs).astype(np.int64)


def hidden_materials(n_labels: int = 8, seed: int = SEED_HIDDEN_MATERIALS):
    """Ground-truth materials for the material-learning workload."""
    return office_materials(seed, n_labels)


# ---------------------------------------------------------------- learned proposal
MLP_IN = 96       # Fourier features: 6 coordinates x 8 octaves x (sin, cos)
MLP_HIDDEN = 128  # three hidden layers


def mlp_param_count(n_in: int = MLP_IN, h: int = MLP_HIDDEN) -> int:
    return h * n_in + h + 2 * (h * h + h) + h + 1


def mlp_init(seed: int = SEED_MLP, n_in: int = MLP_IN, h: int = MLP_HIDDEN) -> np.ndarray:
    """Initial parameters of the proposal network, packed float32:
    W1[h][n_in], b1[h], W2[h][h], b2[h], W3[h][h], b3[h], w4[h], b4.
    Weights uniform in +-sqrt(6 / fan_in) (He-uniform for ReLU layers),
    biases zero."""
    rng = rng_for(seed)
    parts = []
    for fan_in, fan_out in ((n_in, h), (h, h), (h, h), (h, 1)):
        a = np.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-a, a, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def mlp_samples(n: int, n_tx: int, n_rays: int, pos_rate: float = 0.05, seed: int = SEED_MLP):
    """Synthetic training samples for the proposal network's parity tests:
    (tx index [n] int32, ray id [n] uint32, label [n] float32 in {0, 1})."""
    rng = rng_for(seed, 1)
    return (rng.integers(0, n_tx, n).astype(np.int32),
            rng.integers(0, n_rays, n).astype(np.uint32),
            (rng.random(n) < pos_rate).astype(np.float32))


def mlp_logits(n: int, seed: int = SEED_MLP) -> np.ndarray:
    """Synthetic logits for the launch-selection parity tests: a smooth
    profile over the index (as a trained network gives over neighbouring
    directions) plus noise, float32."""
    rng = rng_for(seed, 2)
    i = np.arange(n)
    return (3.0 * np.sin(i * 2e-4) - 2.0 + 0.5 * rng.standard_normal(n)).astype(np.float32)
