"""Single-bounce edge diffraction (Sec. II-B-3) on a GPU, through the C ABI,
against the FP64 oracle (itself pinned to SciPy's Fresnel integrals, a
numerical path-length minimisation, the half-plane coefficient and the
shadow-boundary continuity of the total field).

Room: 24 free-standing wedges of random orientation and angle in the empty
5 x 4 x 3 m room (every geometric branch of the coefficient).  Office: the
320 convex edges of its 40 boxes, whose faces are in the point cloud (the
visibility casts meet real geometry).  Paths are compared under the
per-path contract of the other path types: same keys and representatives
unless the oracle flags the decision ambiguous, coefficients within 1e-4
relative widened by the oracle's own sensitivity, delays within 1e-6."""
import numpy as np
import pytest

import oracle
from paper_2507_04021_gb300 import inputs, nrt

from parity import compare_paths

pytestmark = pytest.mark.gpu

RX4 = np.array([[4.0, 3.0, 1.2], [1.5, 3.2, 1.0], [4.2, 0.8, 2.1], [2.5, 2.0, 0.5]], np.float32)
MATS = (np.array([5.3, 3.0]), np.array([0.03, 0.01]), np.array([0.3, 0.2]))


@pytest.fixture(scope="module")
def ctx():
    return nrt.Context(0)


@pytest.fixture(scope="module")
def room_edges():
    return inputs.room_edges()


@pytest.fixture(scope="module")
def room_orc(room):
    return oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)


def _room_scene(ctx, room, edges, mats=None):
    sc = nrt.Scene(ctx, room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    sc.set_materials(*(mats if mats is not None else (room.eps_r, room.sigma, room.scat)))
    sc.set_edges(edges)
    return sc


def _check_diffracted(gp, osim):
    """Diffracted paths on both sides: the diffraction point (1e-5 m), face
    materials and incidence cosines (1e-5)."""
    O = osim.paths()
    where = {(int(h), int(l)): i for i, (h, l) in enumerate(zip(O["hi"], O["lo"]))}
    n = 0
    for i in np.nonzero(gp["type"] == 2)[0]:
        oi = where.get((int(gp["key_hi"][i]), int(gp["key_lo"][i])))
        if oi is None:
            continue
        assert O["type"][oi] == 2 and int(O["rep"][oi]) == int(gp["rep"][i])
        assert np.abs(gp["pts"][i, 0].astype(np.float64) - O["pts"][oi, 0]).max() < 1e-5
        assert np.array_equal(gp["mats"][i, :2], O["mats"][oi, :2])
        assert np.abs(gp["cos_theta"][i, :2] - O["cos"][oi, :2]).max() < 1e-5
        n += 1
    return n


@pytest.mark.parametrize("pol", [nrt.POL_TE, nrt.POL_TM, nrt.POL_VECTOR])
def test_room_wedges_match_oracle(ctx, room, room_orc, room_edges, pol):
    sc = _room_scene(ctx, room, room_edges)
    kp = dict(max_depth=2, capture=nrt.CAPTURE_VIS, diffuse=0, n_rays=4000, rep_tries=8, pol=pol,
              diffraction=1)
    res = sc.trace(room.tx, RX4, nrt.default_trace_params(**kp))
    osim = oracle.OracleSim(room_orc, room.tx, RX4, oracle.SimParams(delta=1e-5 * room.diag, **kp),
                            edges=room_edges)
    gp = res.paths()
    s = compare_paths(gp, osim, room.eps_r, room.sigma, room.scat, strict=("los", "specular", "diffracted"))
    nd = _check_diffracted(gp, osim)
    print("room wedges, pol", pol, s, "diffracted compared", nd,
          "casts", res.counts()[1]["diffraction_casts"])
    assert nd >= 10
    assert (gp["type"] == 2).sum() == (osim.paths()["type"] == 2).sum()
    res.close()


def test_office_box_edges_match_oracle(office):
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, office.pos, office.nrm, office.surf, office.mat, r_p=0.015)
    sc.set_materials(office.eps_r, office.sigma, office.scat)
    edges = inputs.office_edges(office.extra["boxes"])
    sc.set_edges(edges)
    ids = np.arange(0, 1_000_000, 250, dtype=np.uint32)
    kp = dict(max_depth=3, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=1_000_000, rep_tries=8,
              diffraction=1)
    res = sc.trace(office.tx, office.rx, nrt.default_trace_params(**kp), ray_subset=ids)
    osc = oracle.OracleScene(office.pos, office.nrm, office.surf, office.mat, r_p=0.015,
                             grid_cell=0.1)
    osim = oracle.OracleSim(osc, office.tx, office.rx,
                            oracle.SimParams(delta=1e-5 * office.diag, **kp),
                            ray_ids=ids.astype(np.int64), edges=edges)
    gp = res.paths()
    s = compare_paths(gp, osim, office.eps_r, office.sigma, office.scat, strict=("los", "specular", "diffracted"))
    nd = _check_diffracted(gp, osim)
    n_g, n_o = int((gp["type"] == 2).sum()), int((osim.paths()["type"] == 2).sum())
    print("office box edges:", s, "diffracted gpu", n_g, "oracle", n_o, "compared", nd)
    assert nd > 100
    assert s["max_dP_common"] < 1e-4


@pytest.mark.parametrize("pol", [nrt.POL_TE, nrt.POL_VECTOR])
def test_backward_with_diffraction_matches_oracle(ctx, room, room_orc, room_edges, pol):
    sc = _room_scene(ctx, room, room_edges, tuple(m.astype(np.float32) for m in MATS))
    kp = dict(max_depth=2, capture=nrt.CAPTURE_VIS, diffuse=0, n_rays=4000, rep_tries=8, pol=pol,
              diffraction=1)
    res = sc.trace(room.tx, RX4, nrt.default_trace_params(**kp))
    osim = oracle.OracleSim(room_orc, room.tx, RX4, oracle.SimParams(**kp), edges=room_edges)
    _, Po = osim.field(*MATS)
    dLdP = (1.0 / Po) * np.array([1.0, -0.5, 0.25, 2.0])
    g = res.backward(dLdP.astype(np.float32))
    want = osim.backward(*MATS, dLdP)
    for name, gi, wi in zip(("eps", "sigma", "S"), g, want):
        rel = np.abs(gi - wi) / np.maximum(np.abs(wi), 1e-3 * np.abs(wi).max())
        print(name, "max rel diff", float(rel.max()))
        assert rel.max() < 2e-3, (name, gi, wi)
    res.close()


def test_diffraction_off_leaves_the_other_paths(ctx, room, room_edges):
    sc = _room_scene(ctx, room, room_edges)
    kp = dict(max_depth=2, capture=nrt.CAPTURE_VIS, diffuse=0, n_rays=4000, rep_tries=8)
    on = sc.trace(room.tx, RX4, nrt.default_trace_params(diffraction=1, **kp)).paths()
    off = sc.trace(room.tx, RX4, nrt.default_trace_params(**kp)).paths()
    keep = on["type"] != 2
    for k in ("key_hi", "key_lo", "rep", "a", "tau"):
        assert np.array_equal(on[k][keep], off[k]), k
    assert (on["type"] == 2).sum() > 0


def test_batch_pairs_with_diffraction_equal_single_runs(office):
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, office.pos, office.nrm, office.surf, office.mat, r_p=0.015)
    sc.set_materials(office.eps_r, office.sigma, office.scat)
    sc.set_edges(inputs.office_edges(office.extra["boxes"]))
    traj = inputs.trajectory(office.extra["boxes"])
    rxf = np.array([17.5, 8.0, 1.2], np.float32)
    budgets = np.array([3000, 7000, 1500], np.int64)
    tx = traj[[0, 60, 120]]
    prm = lambda n: nrt.default_trace_params(max_depth=3, capture=nrt.CAPTURE_VIS, diffuse=1,  # noqa
                                             rep_tries=8, n_rays=n, diffraction=1)
    b = sc.trace_batch(tx, rxf, budgets, prm(1))
    B = b.paths()
    mask = np.uint64(0x00FFFFFFFFFFFFFF)
    n_dif = 0
    for j in range(len(budgets)):
        S = sc.trace(tx[j], rxf[None], prm(int(budgets[j]))).paths()
        mine = B["rx"] == j
        kb = {(int(h & mask), int(l)): i for i, (h, l) in
              enumerate(zip(B["key_hi"][mine], B["key_lo"][mine]))}
        ks = {(int(h & mask), int(l)): i for i, (h, l) in enumerate(zip(S["key_hi"], S["key_lo"]))}
        assert kb.keys() == ks.keys()
        dif = [key for key, i in ks.items() if S["type"][i] == 2]
        n_dif += len(dif)
        for key in dif:
            assert np.array_equal(B["a"][mine][kb[key]], S["a"][ks[key]])
    assert n_dif > 0


def test_edge_input_checks(ctx, room):
    sc = nrt.Scene(ctx, room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    e = inputs.room_edges(3)
    bad = inputs.Edges(e.a, e.b, 2.0 * e.n0, e.n1, e.m0, e.m1)  # normals not unit
    with pytest.raises(nrt.NrtError):
        sc.set_edges(bad)
    flat = inputs.Edges(e.a, e.b, e.n0, e.n0, e.m0, e.m1)  # both faces in one plane
    with pytest.raises(nrt.NrtError):
        sc.set_edges(flat)
    sc.set_materials(room.eps_r, room.sigma, room.scat)
    sc.set_edges(e)
    res = sc.trace(room.tx, RX4, nrt.default_trace_params(
        max_depth=1, capture=nrt.CAPTURE_VIS, n_rays=1000, diffraction=1))
    with pytest.raises(nrt.NrtError):  # a live result holds the scene
        sc.set_edges(e)
    import torch

    dldp = torch.ones(RX4.shape[0], dtype=torch.float32, device="cuda")
    grad = torch.zeros(3 * sc.n_labels, dtype=torch.float32, device="cuda")
    with pytest.raises(nrt.NrtError):  # the allocation-free backward is scalar-only
        res.backward_noalloc(dldp, grad)
    res.close()
    sc.set_edges(None)


def test_cfr_and_eq5_gradient_with_diffraction(ctx, room, room_orc, room_edges):
    """The CFR and the Eq. 5 gradient include the diffracted paths (room
    wedges, vector model) and match the oracle's under the same bound as the
    other path types: per frequency |dH| <= sum_p |a_p| (1e-4 + 2 pi f tau_p
    1e-6)."""
    from oracle import cfr

    sc = _room_scene(ctx, room, room_edges, tuple(m.astype(np.float32) for m in MATS))
    kp = dict(max_depth=2, capture=nrt.CAPTURE_VIS, diffuse=0, n_rays=4000, rep_tries=8,
              pol=nrt.POL_VECTOR, diffraction=1)
    res = sc.trace(room.tx, RX4, nrt.default_trace_params(**kp))
    osim = oracle.OracleSim(room_orc, room.tx, RX4, oracle.SimParams(**kp), edges=room_edges)
    BW, NF = 1.5e9, 129
    f = cfr.freqs(28e9, BW, NF)
    P = osim.paths()
    assert (P["type"] == 2).sum() > 10
    a, _ = osim.field(*MATS)
    Ho = cfr.cfr(a, P["tau"], P["j"], RX4.shape[0], f)
    H = res.cfr(BW, NF)
    amp = np.abs(a)
    bound = np.stack([(amp[P["j"] == j, None] * (1e-4 + 2 * np.pi * f[None, :] *
                                                  P["tau"][P["j"] == j, None] * 1e-6)).sum(0)
                      for j in range(RX4.shape[0])])
    assert np.all(np.abs(H - Ho) <= bound)
    hidden = (np.array([4.1, 2.4]), np.array([0.05, 0.002]), np.array([0.45, 0.1]))
    a_h, _ = osim.field(*hidden)
    T = cfr.cfr(a_h, P["tau"], P["j"], RX4.shape[0], f)
    w = np.array([1.0, 0.5, 0.25, 2.0])
    loss, g = res.cfr_backward(T, w, BW)
    go = cfr.eq5_grad(osim.path_grads(*MATS), P["tau"], P["j"], f, Ho, T, w)
    assert np.allclose(loss, cfr.eq5_loss(Ho, T), rtol=1e-2, atol=1e-4)
    for t in range(2):  # eps_r, sigma (S does not enter diffraction; it does the reflections)
        rel = np.abs(g[t] - go[t]) / np.maximum(np.abs(go[t]), 1e-2 * np.abs(go).max())
        assert rel.max() < 2e-2, t
    res.close()
