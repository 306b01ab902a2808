"""The vector polarisation model (pol = NRT_POL_VECTOR) on a GPU, through the
C ABI, against the FP64 oracle's vector model (itself pinned to closed forms
and finite differences): path coefficients under the per-path contract
(1e-4 relative, widened by the oracle's own geometric sensitivity), the
diffuse scatter normals it uses, per-label gradients of the power loss and
of the Eq. 5 CIR loss, and the scalar-only guard of the allocation-free
backward."""
import numpy as np
import pytest

import oracle
from oracle import cfr
from paper_2507_04021_gb300 import nrt

from parity import compare_paths

pytestmark = pytest.mark.gpu

RX4 = np.array([[4.0, 3.0, 1.2], [1.5, 3.2, 1.0], [4.2, 0.8, 2.1], [2.5, 2.0, 0.5]], np.float32)
MATS = (np.array([5.3, 3.0]), np.array([0.03, 0.01]), np.array([0.3, 0.2]))
HIDDEN = (np.array([4.1, 2.4]), np.array([0.05, 0.002]), np.array([0.45, 0.1]))
VEC = nrt.POL_VECTOR


@pytest.fixture(scope="module")
def ctx():
    return nrt.Context(0)


@pytest.fixture(scope="module")
def room_gpu(ctx, room):
    sc = nrt.Scene(ctx, room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    sc.set_materials(room.eps_r, room.sigma, room.scat)
    return sc


@pytest.fixture(scope="module")
def room_orc(room):
    return oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)


def _compare_normals(gp, osim):
    """Diffuse paths found by both sides with the same representative: the
    scatter normal (both face the incoming ray) under the hit contract --
    compared where the oracle marks every hit of the representative up to
    the scatter point certain, within 1e-4 widened where its shadow trace
    shows the bounce sequence amplifying rounding (twice its normal
    divergence at that bounce)."""
    O = osim.paths()
    ond = osim.path_normals()
    _, dn = osim.hit_sens()
    excl = osim.hits()["excl"]
    row_of = {int(r): i for i, r in enumerate(osim.ray_ids)}
    where = {(int(h), int(l)): i for i, (h, l) in enumerate(zip(O["hi"], O["lo"]))}
    n = 0
    for i in np.nonzero(gp["type"] == 1)[0]:
        oi = where.get((int(gp["key_hi"][i]), int(gp["key_lo"][i])))
        if oi is None or int(O["rep"][oi]) != int(gp["rep"][i]):
            continue
        row, k = row_of[int(gp["rep"][i])], int(gp["k"][i])
        if not k < excl[row]:
            continue
        tol = max(1e-4, 2.0 * dn[row, k - 1])
        assert np.abs(gp["normal"][i].astype(np.float64) - ond[oi]).max() <= tol
        n += 1
    assert np.all(gp["normal"][gp["type"] == 0] == 0.0)
    return n


def test_room_sphere_capture_vector(room, room_gpu, room_orc):
    kp = dict(max_depth=2, capture=nrt.CAPTURE_SPHERE, diffuse=0, n_rays=20000, r_rx=0.1,
              rep_tries=8, pol=VEC)
    res = room_gpu.trace(room.tx, room.rx, nrt.default_trace_params(**kp))
    osim = oracle.OracleSim(room_orc, room.tx, room.rx,
                            oracle.SimParams(delta=1e-5 * room.diag, **kp))
    s = compare_paths(res.paths(), osim, room.eps_r, room.sigma, room.scat, strict=("los", "specular"))
    print("room sphere, vector:", s)
    assert s["matched"] >= 1 and s["field_checked"] >= 1


def test_room_visibility_diffuse_vector(room, room_gpu, room_orc):
    kp = dict(max_depth=2, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=4000, rep_tries=8, pol=VEC)
    res = room_gpu.trace(room.tx, room.rx, nrt.default_trace_params(**kp))
    osim = oracle.OracleSim(room_orc, room.tx, room.rx,
                            oracle.SimParams(delta=1e-5 * room.diag, **kp))
    gp = res.paths()
    s = compare_paths(gp, osim, room.eps_r, room.sigma, room.scat, strict=("los", "specular"))
    nn = _compare_normals(gp, osim)
    print("room vis+diffuse, vector:", s, "normals compared", nn)
    assert s["matched"] > 100, s
    assert nn > 20


def test_vector_differs_from_scalar_and_los_is_scalar(room, room_gpu):
    """LOS paths carry theta^(u) . theta^(-u) = 1 (the scalar value); reflected
    paths change with the polarisation model."""
    kp = dict(max_depth=2, capture=nrt.CAPTURE_VIS, diffuse=0, n_rays=4000, rep_tries=8)
    a = {}
    for pol in (nrt.POL_TE, VEC):
        P = room_gpu.trace(room.tx, room.rx, nrt.default_trace_params(pol=pol, **kp)).paths()
        a[pol] = {(int(h), int(l)): (int(k), complex(x[0], x[1]))
                  for h, l, k, x in zip(P["key_hi"], P["key_lo"], P["k"], P["a"])}
    common = set(a[nrt.POL_TE]) & set(a[VEC])
    los = [key for key in common if a[VEC][key][0] == 0]
    refl = [key for key in common if a[VEC][key][0] > 0]
    assert los and refl
    for key in los:
        assert a[VEC][key][1] == pytest.approx(a[nrt.POL_TE][key][1], rel=1e-6)
    assert any(abs(a[VEC][key][1] - a[nrt.POL_TE][key][1]) > 1e-3 * abs(a[nrt.POL_TE][key][1])
               for key in refl)


def test_office_subset_vector(office):
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, office.pos, office.nrm, office.surf, office.mat, r_p=0.015)
    sc.set_materials(office.eps_r, office.sigma, office.scat)
    ids = np.arange(0, 1_000_000, 250, dtype=np.uint32)
    kp = dict(max_depth=5, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=1_000_000, rep_tries=8,
              pol=VEC)
    res = sc.trace(office.tx, office.rx, nrt.default_trace_params(**kp), ray_subset=ids)
    osc = oracle.OracleScene(office.pos, office.nrm, office.surf, office.mat, r_p=0.015,
                             grid_cell=0.1)
    osim = oracle.OracleSim(osc, office.tx, office.rx,
                            oracle.SimParams(delta=1e-5 * office.diag, **kp),
                            ray_ids=ids.astype(np.int64))
    gp = res.paths()
    s = compare_paths(gp, osim, office.eps_r, office.sigma, office.scat, strict=("los", "specular"))
    nn = _compare_normals(gp, osim)
    print("office subset, vector:", s, "normals compared", nn)
    assert s["matched"] > 0.8 * s["keys"], s
    assert s["max_dP_common"] < 1e-4
    assert nn > 100


@pytest.fixture(scope="module")
def room_pair_vector(room):
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    sc.set_materials(*(m.astype(np.float32) for m in MATS))
    kp = dict(max_depth=2, capture=nrt.CAPTURE_VIS, diffuse=0, n_rays=4000, rep_tries=8, pol=VEC)
    res = sc.trace(room.tx, RX4, nrt.default_trace_params(**kp))
    osc = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    osim = oracle.OracleSim(osc, room.tx, RX4, oracle.SimParams(**kp))
    return sc, res, osim


def test_backward_vector_matches_oracle(room_pair_vector):
    sc, res, osim = room_pair_vector
    _, Po = osim.field(*MATS)
    dLdP = (1.0 / Po) * np.array([1.0, -0.5, 0.25, 2.0])
    g = res.backward(dLdP.astype(np.float32))
    want = osim.backward(*MATS, dLdP)
    for name, gi, wi in zip(("eps", "sigma", "S"), g, want):
        rel = np.abs(gi - wi) / np.maximum(np.abs(wi), 1e-3 * np.abs(wi).max())
        print(name, "max rel diff", float(rel.max()))
        assert rel.max() < 2e-3, (name, gi, wi)


def test_backward_vector_diffuse_office_subset(office):
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, office.pos, office.nrm, office.surf, office.mat, r_p=0.015)
    sc.set_materials(office.eps_r, office.sigma, office.scat)
    ids = np.arange(0, 1_000_000, 250, dtype=np.uint32)
    kp = dict(max_depth=3, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=1_000_000, rep_tries=8,
              pol=VEC)
    res = sc.trace(office.tx, office.rx, nrt.default_trace_params(**kp), ray_subset=ids)
    osc = oracle.OracleScene(office.pos, office.nrm, office.surf, office.mat, r_p=0.015,
                             grid_cell=0.1)
    osim = oracle.OracleSim(osc, office.tx, office.rx,
                            oracle.SimParams(delta=1e-5 * office.diag, **kp),
                            ray_ids=ids.astype(np.int64))
    mats = tuple(m.astype(np.float64) for m in (office.eps_r, office.sigma, office.scat))
    _, Po = osim.field(*mats)
    dLdP = 1.0 / Po
    g = res.backward(dLdP.astype(np.float32))
    want = osim.backward(*mats, dLdP)
    for name, gi, wi in zip(("eps", "sigma", "S"), g, want):
        rel = np.abs(gi - wi) / np.maximum(np.abs(wi), 1e-3 * np.abs(wi).max())
        print(name, "max rel diff", float(rel.max()))
        assert rel.max() < 5e-3, (name, gi, wi)


def test_eq5_gradient_vector_matches_oracle(room_pair_vector):
    sc, res, osim = room_pair_vector
    BW, NF = 1.5e9, 129
    f = cfr.freqs(28e9, BW, NF)
    P = osim.paths()
    a_hidden, _ = osim.field(*HIDDEN)
    T = cfr.cfr(a_hidden, P["tau"], P["j"], RX4.shape[0], f)
    w = np.array([1.0, 0.5, 0.25, 2.0])
    loss, g = res.cfr_backward(T, w, BW)
    a, _ = osim.field(*MATS)
    Ho = cfr.cfr(a, P["tau"], P["j"], RX4.shape[0], f)
    lo = cfr.eq5_loss(Ho, T)
    go = cfr.eq5_grad(osim.path_grads(*MATS), P["tau"], P["j"], f, Ho, T, w)
    print("loss", loss, lo)
    assert np.allclose(loss, lo, rtol=1e-2, atol=1e-4)
    for t, name in enumerate(("eps", "sigma", "S")):
        rel = np.abs(g[t] - go[t]) / np.maximum(np.abs(go[t]), 1e-2 * np.abs(go).max())
        print(name, "gpu", g[t], "oracle", go[t], "max rel", float(rel.max()))
        assert rel.max() < 2e-2, name


def test_noalloc_backward_rejects_the_vector_model(room_pair_vector):
    import torch

    sc, res, _ = room_pair_vector
    dldp = torch.ones(RX4.shape[0], dtype=torch.float32, device="cuda")
    grad = torch.zeros(3 * sc.n_labels, dtype=torch.float32, device="cuda")
    with pytest.raises(nrt.NrtError):
        res.backward_noalloc(dldp, grad)
