"""nrt_cast on a GPU, through the C ABI: closest hits of arbitrary rays under
the paper's disc model (Sec. II-C, Eq. 3 / Eq. 4) and under the SDF model of
its prior work (Eq. 2, the ablation), each against the FP64 oracle's cast on
the same rays.  Rays whose decisions the oracle marks ambiguous (within
delta = 1e-5 x scene diagonal of a threshold) are skipped."""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_04021_gb300 import inputs, nrt

pytestmark = pytest.mark.gpu


def _rays(n, lo, hi, seed):
    rng = np.random.default_rng(seed)
    o = rng.uniform(lo, hi, (n, 3)).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    return o, d


def _gpu_cast(sc, o, d, **kw):
    out = sc.cast(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), **kw)
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.fixture(scope="module")
def room_pair(room):
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    osc = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    return sc, osc


def test_disc_model_matches_oracle(room, room_pair):
    sc, osc = room_pair
    o, d = _rays(600, (0.8, 0.8, 0.6), (4.2, 3.2, 2.4), 1)
    g = _gpu_cast(sc, o, d, model=nrt.ISECT_DISC)
    delta = 1e-5 * room.diag
    checked = 0
    for i in range(len(o)):
        h = osc.cast(o[i].astype(np.float64), d[i].astype(np.float64), delta=delta)
        if h["amb"]:
            continue
        assert (g["dps"][i] >= 0) == h["hit"]
        if not h["hit"]:
            continue
        q = o[i].astype(np.float64) + float(g["t"][i]) * d[i].astype(np.float64)
        assert np.abs(q - h["q"]).max() < 2e-5
        assert np.abs(g["normal"][i] - h["n"]).max() < 1e-4
        checked += 1
    assert checked > 150  # the room's discs leave gaps: about a third of the rays hit


def _dps_root(scene, mask, o, d, sigma):
    """Root of one DPS's field along the ray (float64 numpy restatement of the
    per-DPS marching: sigma/2 steps over the points' box grown by 2 sigma,
    first outside-to-inside bracket, 20 bisections)."""
    P, N = scene.pos[mask].astype(np.float64), scene.nrm[mask].astype(np.float64)
    o = o.astype(np.float64)
    d = d.astype(np.float64) / np.linalg.norm(d.astype(np.float64))
    lo, hi = P.min(0) - 2 * sigma, P.max(0) + 2 * sigma
    t0, t1 = 1e-3, np.inf
    for a in range(3):
        if d[a] == 0:
            continue
        ta, tb = sorted(((lo[a] - o[a]) / d[a], (hi[a] - o[a]) / d[a]))
        t0, t1 = max(t0, ta), min(t1, tb)

    def f(t):
        v = o + t * d - P
        w = np.exp(-(v * v).sum(1) / (2 * sigma ** 2))
        return (w * (v * N).sum(1)).sum() / max(w.sum(), 1e-300), w.sum()

    h = sigma / 2
    fa, Wa = f(t0)
    for k in range(int(np.floor((t1 - t0) / h))):
        fb, Wb = f(t0 + (k + 1) * h)
        if min(Wa, Wb) >= np.exp(-2) and fa > 0 >= fb:
            lo_t, hi_t = t0 + k * h, t0 + (k + 1) * h
            for _ in range(20):
                m = 0.5 * (lo_t + hi_t)
                lo_t, hi_t = (m, hi_t) if f(m)[0] > 0 else (lo_t, m)
            return 0.5 * (lo_t + hi_t)
        fa, Wa = fb, Wb
    return np.inf


@pytest.mark.parametrize("scene_name,sigma", [("room", 0.1), ("office60k", 0.08)])
def test_sdf_model_matches_oracle(room, scene_name, sigma):
    if scene_name == "room":
        sc_in, lo, hi = room, (0.8, 0.8, 0.6), (4.2, 3.2, 2.4)
        r_p = 0.05
    else:
        sc_in, lo, hi = inputs.office_scene(n_points=60000), (1, 1, 0.5), (19, 9, 2.5)
        r_p = 0.05
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, sc_in.pos, sc_in.nrm, sc_in.surf, sc_in.mat, rho=0.0625, r_p=r_p)
    osc = oracle.OracleScene(sc_in.pos, sc_in.nrm, sc_in.surf, sc_in.mat, rho=0.0625, r_p=r_p)
    # the room's exact planes make many rays ambiguous (equal roots in
    # neighbouring DPS within the tie band): more rays there
    o, d = _rays(900 if scene_name == "room" else 300, lo, hi, 2)
    g = _gpu_cast(sc, o, d, model=nrt.ISECT_SDF, sigma=sigma)
    gv, _, _ = sc.dps()
    ov, _, _ = osc.dps()
    omap = {tuple(v): i for i, v in enumerate(ov)}
    delta = 1e-5 * sc_in.diag
    pdps = osc.point_dps()
    checked = ties = 0
    for i in range(len(o)):
        h = osc.cast_sdf(o[i].astype(np.float64), d[i].astype(np.float64), sigma, delta=delta)
        if h["amb"]:
            continue
        assert (g["dps"][i] >= 0) == h["hit"], i
        if not h["hit"]:
            continue
        assert abs(float(g["t"][i]) - h["t"]) < 1e-4
        assert np.abs(g["normal"][i] - h["n"]).max() < 1e-3
        D = omap[tuple(gv[g["dps"][i]])]
        if D == h["dps"]:
            assert int(g["labels"][i]) == h["labels"]
        else:
            # several DPS can carry the same surface (the room's exact planes):
            # the hit is unique, its DPS is not -- the GPU's DPS must have its
            # own root there
            t_own = _dps_root(sc_in, pdps == D, o[i], d[i], sigma)
            assert abs(t_own - h["t"]) < 1e-4
            ties += 1
        checked += 1
    print(scene_name, "checked", checked, "ties", ties)
    assert checked > 150


def test_cast_input_checks(room_pair):
    sc, _ = room_pair
    o = torch.zeros((4, 3), device="cuda")
    d = torch.ones((4, 3), device="cuda")
    with pytest.raises(nrt.NrtError):
        sc.cast(o, d, model=nrt.ISECT_SDF, sigma=0.0)
    with pytest.raises(nrt.NrtError):
        sc.cast(o, d, model=7)
