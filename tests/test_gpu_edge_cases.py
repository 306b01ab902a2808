"""Edge cases on a GPU, through the C ABI, against the FP64 oracle: a scene of
one DPS (the BVH root is itself a leaf) for the tracer and both intersection
models; ragged ray subsets (1, 31, 33 and 4097 rays: partial warps and
tiles); the maximum of 256 receivers; a scene that almost every ray escapes;
and the argument checks of nrt_trace."""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_04021_gb300 import inputs, nrt

from parity import compare_hits, compare_paths

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return nrt.Context(0)


def _patch(n=7, seed=3):
    """n points on a 4 cm floor patch inside one 6.25 cm voxel, normals +z."""
    rng = np.random.default_rng(seed)
    pos = np.column_stack([1.005 + rng.uniform(0, 0.04, n), 1.005 + rng.uniform(0, 0.04, n),
                           np.zeros(n)]).astype(np.float32)
    nrm = np.tile(np.array([0, 0, 1], np.float32), (n, 1))
    return pos, nrm, np.zeros(n, np.uint16), np.zeros(n, np.uint8)


def test_one_dps_scene_trace_and_casts(ctx):
    pos, nrm, surf, mat = _patch()
    sc = nrt.Scene(ctx, pos, nrm, surf, mat, rho=0.0625, r_p=0.05)
    assert sc.info()["n_dps"] == 1
    sc.set_materials(np.array([5.0], np.float32), np.array([0.01], np.float32),
                     np.array([0.0], np.float32))
    tx = np.array([1.0, 1.0, 1.0], np.float32)
    rx = np.array([[1.2, 1.1, 0.8]], np.float32)
    kp = dict(max_depth=2, capture=nrt.CAPTURE_SPHERE, diffuse=0, n_rays=200000, r_rx=0.3,
              rep_tries=8)
    res = sc.trace(tx, rx, nrt.default_trace_params(**kp))
    osc = oracle.OracleScene(pos, nrm, surf, mat, rho=0.0625, r_p=0.05)
    osim = oracle.OracleSim(osc, tx, rx, oracle.SimParams(delta=1e-6, **kp))
    h = compare_hits(res.hits(), osim.hits(), 1e-6)
    assert h["mismatch"] == 0 and h["checked"] > 1000, h
    hit_rows = (res.hits()["idx"][:, 0] >= 0).sum()
    assert hit_rows > 10  # some of the launch reaches the patch
    compare_paths(res.paths(), osim, np.array([5.0]), np.array([0.01]), np.array([0.0]), strict=("los", "specular"))
    # nrt_cast on the one-leaf tree, both models, against the oracle's casts
    rng = np.random.default_rng(4)
    o = np.tile(tx, (64, 1)).astype(np.float32)
    tgt = np.column_stack([1.005 + rng.uniform(-0.02, 0.06, 64), 1.005 + rng.uniform(-0.02, 0.06, 64),
                           np.zeros(64)])
    d = (tgt - o).astype(np.float32)
    for model, sigma in ((nrt.ISECT_DISC, 0.0), (nrt.ISECT_SDF, 0.02)):
        g = {k: v.cpu().numpy() for k, v in sc.cast(torch.from_numpy(o).cuda(),
                                                     torch.from_numpy(d).cuda(), model=model,
                                                     sigma=sigma).items()}
        n_hit = 0
        for i in range(64):
            dd = d[i].astype(np.float64) / np.linalg.norm(d[i].astype(np.float64))
            if model == nrt.ISECT_DISC:
                oh = osc.cast(o[i].astype(np.float64), dd, delta=1e-6)
                if oh["amb"]:
                    continue
                assert (g["dps"][i] >= 0) == oh["hit"]
                if oh["hit"]:
                    q = o[i] + g["t"][i] * dd
                    assert np.abs(q - oh["q"]).max() < 1e-5
            else:
                oh = osc.cast_sdf(o[i].astype(np.float64), dd, sigma, delta=1e-6)
                if oh["amb"]:
                    continue
                assert (g["dps"][i] >= 0) == oh["hit"]
                if oh["hit"]:
                    assert abs(float(g["t"][i]) - oh["t"]) < 1e-5
            n_hit += int(g["dps"][i] >= 0)
        assert n_hit > 10, model


@pytest.mark.parametrize("n_sub", [1, 31, 33, 4097])
def test_ragged_ray_subsets(ctx, room, n_sub):
    sc = nrt.Scene(ctx, room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    sc.set_materials(room.eps_r, room.sigma, room.scat)
    rng = np.random.default_rng(n_sub)
    ids = np.sort(rng.choice(20000, n_sub, replace=False)).astype(np.uint32)
    kp = dict(max_depth=2, capture=nrt.CAPTURE_SPHERE, diffuse=0, n_rays=20000, r_rx=0.3,
              rep_tries=8)
    res = sc.trace(room.tx, room.rx, nrt.default_trace_params(**kp), ray_subset=ids)
    delta = 1e-5 * room.diag
    osc = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    osim = oracle.OracleSim(osc, room.tx, room.rx, oracle.SimParams(delta=delta, **kp),
                            ray_ids=ids.astype(np.int64))
    g = res.hits()
    assert g["idx"].shape[0] == n_sub
    h = compare_hits(g, osim.hits(), delta)
    assert h["mismatch"] == 0, h
    compare_paths(res.paths(), osim, room.eps_r, room.sigma, room.scat, strict=("los", "specular"))


def test_256_receivers(ctx, room):
    sc = nrt.Scene(ctx, room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    sc.set_materials(room.eps_r, room.sigma, room.scat)
    gx, gy, gz = np.meshgrid(np.linspace(0.6, 4.4, 8), np.linspace(0.6, 3.4, 8),
                             np.linspace(0.5, 2.5, 4), indexing="ij")
    rx = np.column_stack([gx.ravel(), gy.ravel(), gz.ravel()]).astype(np.float32)
    assert rx.shape[0] == 256
    kp = dict(max_depth=1, capture=nrt.CAPTURE_SPHERE, diffuse=0, n_rays=8000, r_rx=0.25,
              rep_tries=8)
    res = sc.trace(room.tx, rx, nrt.default_trace_params(**kp))
    osc = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    osim = oracle.OracleSim(osc, room.tx, rx, oracle.SimParams(delta=1e-5 * room.diag, **kp))
    s = compare_paths(res.paths(), osim, room.eps_r, room.sigma, room.scat, strict=("los", "specular"))
    per_rx, c = res.counts()
    assert per_rx.shape == (256,) and per_rx.sum() == c["paths"]
    assert np.all(per_rx >= 1)  # every receiver at least sees the TX
    assert s["matched"] > 256
    with pytest.raises(nrt.NrtError):
        sc.trace(room.tx, np.vstack([rx, rx[:1]]), nrt.default_trace_params(**kp))


def test_nearly_every_ray_escapes(ctx):
    pos, nrm, surf, mat = _patch(n=3)
    sc = nrt.Scene(ctx, pos, nrm, surf, mat, rho=0.0625, r_p=0.01)
    sc.set_materials(np.array([5.0], np.float32), np.array([0.01], np.float32),
                     np.array([0.0], np.float32))
    rx = np.array([[3.0, 3.0, 1.0]], np.float32)
    res = sc.trace(np.array([0.0, 0.0, 1.0], np.float32), rx, nrt.default_trace_params(
        max_depth=5, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=100000, rep_tries=8))
    per_rx, c = res.counts()
    assert c["segments"] < 100000 + 100  # one segment per ray, a few hits at most
    assert c["paths"] >= 1 and per_rx[0] == c["paths"]  # the LOS path at least
    assert np.isfinite(res.power()).all()


def test_trace_argument_checks(ctx, room):
    sc = nrt.Scene(ctx, room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    sc.set_materials(room.eps_r, room.sigma, room.scat)
    ok = dict(max_depth=2, capture=nrt.CAPTURE_SPHERE, diffuse=0, n_rays=1000, r_rx=0.1)
    bad = [dict(ok, max_depth=0), dict(ok, max_depth=6), dict(ok, n_rays=0),
           dict(ok, rep_tries=-1), dict(ok, pol=3), dict(ok, diffuse=1),  # diffuse needs VIS
           dict(ok, diffraction=2)]
    for kp in bad:
        with pytest.raises(nrt.NrtError):
            sc.trace(room.tx, room.rx, nrt.default_trace_params(**kp))
    with pytest.raises(nrt.NrtError):
        sc.trace(np.array([np.nan, 1, 1], np.float32), room.rx, nrt.default_trace_params(**ok))
    with pytest.raises(nrt.NrtError):  # ray ids beyond the launch
        sc.trace(room.tx, room.rx, nrt.default_trace_params(**ok),
                 ray_subset=np.array([5, 2000], np.uint32))
    with pytest.raises(nrt.NrtError):
        sc.trace(room.tx, room.rx, nrt.default_trace_params(key_capacity=3000, **ok))
    # a valid call still works afterwards on the same context
    sc.trace(room.tx, room.rx, nrt.default_trace_params(**ok)).close()


def _same_paths(a, b):
    for k in ("key_hi", "key_lo", "rep", "rx", "a", "tau"):
        assert np.array_equal(a[k], b[k]), k


def test_capacity_hints_give_the_exact_result(office):
    """A context sizes the first simulation of a shape exactly (one host
    round trip) and later ones from that run's counts + 25%, without waiting
    for the host.  A hinted run, and a run that outgrows its hint (TX far
    above the office first, so the hint is small) and is redone with exact
    sizes, both equal a fresh context's exact run bit for bit."""
    kp = dict(max_depth=5, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=60000, rep_tries=0)
    p = nrt.default_trace_params(**kp)
    ctx_a = nrt.Context(0)
    sa = nrt.Scene(ctx_a, office.pos, office.nrm, office.surf, office.mat, r_p=0.015)
    sa.set_materials(office.eps_r, office.sigma, office.scat)
    far = sa.trace(np.array([10.0, 5.0, 200.0], np.float32), office.rx, p)
    far_cand = far.counts()[1]["candidates"]
    far.close()
    grown = sa.trace(office.tx, office.rx, p)  # outgrows the hint: redone exactly
    hinted = sa.trace(office.tx, office.rx, p)  # sized from the previous run
    assert hinted.times()["sizing_wait"] < 0.05
    ctx_b = nrt.Context(0)
    sb = nrt.Scene(ctx_b, office.pos, office.nrm, office.surf, office.mat, r_p=0.015)
    sb.set_materials(office.eps_r, office.sigma, office.scat)
    ref = sb.trace(office.tx, office.rx, p)
    R = ref.paths()
    assert len(R["rep"]) > 1000
    # the far run's hint (its count + 25% + 1024) is too small for the office TX
    assert far_cand + far_cand // 4 + 1024 < ref.counts()[1]["candidates"]
    for r in (grown, hinted):
        _same_paths(r.paths(), R)
        np.testing.assert_array_equal(r.power(), ref.power())
        c, cr = r.counts()[1], ref.counts()[1]
        for k in ("candidates", "keys", "paths", "segments"):
            assert c[k] == cr[k], k
