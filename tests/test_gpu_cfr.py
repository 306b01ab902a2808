"""Channel frequency response and the Eq. 5 loss on a GPU (nrt_cfr,
nrt_cfr_backward) against the FP64 oracle (oracle/cfr.py).

Tolerance, derived from the per-path contract: |a| within 1e-4 and tau within
1e-6 relative give, per frequency, |dH_j(f)| <= sum_p |a_p| (1e-4 +
2 pi f tau_p 1e-6) (the phase error of a delay error); keys present on one
side only (ambiguous, flagged by the oracle) add their |a_p|."""
import numpy as np
import pytest

import oracle
from oracle import cfr
from paper_2507_04021_gb300 import inputs, nrt

pytestmark = pytest.mark.gpu

RX4 = np.array([[4.0, 3.0, 1.2], [1.5, 3.2, 1.0], [4.2, 0.8, 2.1], [2.5, 2.0, 0.5]], np.float32)
MATS = (np.array([5.3, 3.0]), np.array([0.03, 0.01]), np.array([0.3, 0.2]))
HIDDEN = (np.array([4.1, 2.4]), np.array([0.05, 0.002]), np.array([0.45, 0.1]))
BW, NF = 1.5e9, 129


@pytest.fixture(scope="module")
def room_pair(room):
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    sc.set_materials(*(m.astype(np.float32) for m in MATS))
    kp = dict(max_depth=2, capture=nrt.CAPTURE_VIS, diffuse=0, n_rays=4000, rep_tries=8)
    res = sc.trace(room.tx, RX4, nrt.default_trace_params(**kp))
    osc = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    osim = oracle.OracleSim(osc, room.tx, RX4, oracle.SimParams(**kp))
    return sc, res, osim


def _bound(P, a, f, unmatched):
    tau = P["tau"]
    amp = np.abs(a)
    b = np.zeros((RX4.shape[0], f.size))
    for j in range(RX4.shape[0]):
        m = P["j"] == j
        b[j] = (amp[m, None] * (1e-4 + 2 * np.pi * f[None, :] * tau[m, None] * 1e-6)).sum(0)
        b[j] += amp[m & unmatched].sum()
    return b


def test_cfr_matches_oracle(room_pair):
    sc, res, osim = room_pair
    f = cfr.freqs(28e9, BW, NF)
    H = res.cfr(BW, NF)
    P = osim.paths()
    a, _ = osim.field(*MATS)
    Ho = cfr.cfr(a, P["tau"], P["j"], RX4.shape[0], f)
    gp = res.paths()
    gk = set(zip(gp["key_hi"].tolist(), gp["key_lo"].tolist()))
    unmatched = np.array([(int(h), int(l)) not in gk for h, l in zip(P["hi"], P["lo"])])
    err = np.abs(H - Ho)
    bound = _bound(P, a, f, unmatched)
    print("CFR max |dH| / bound", float((err / bound).max()), "max |H|", float(np.abs(Ho).max()))
    assert np.all(err <= bound)


def test_eq5_loss_and_gradient_match_oracle(room_pair):
    sc, res, osim = room_pair
    f = cfr.freqs(28e9, BW, NF)
    P = osim.paths()
    a_hidden, _ = osim.field(*HIDDEN)
    T = cfr.cfr(a_hidden, P["tau"], P["j"], RX4.shape[0], f)  # target from the oracle
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


def test_office_cfr_matches_oracle(office):
    """Office ray subset with diffuse paths (16 RX)."""
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, office.pos, office.nrm, office.surf, office.mat, r_p=0.015)
    sc.set_materials(office.eps_r, office.sigma, office.scat)
    ids = np.arange(0, 1_000_000, 250, dtype=np.uint32)
    kp = dict(max_depth=3, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=1_000_000, rep_tries=8)
    res = sc.trace(office.tx, office.rx, nrt.default_trace_params(**kp), ray_subset=ids)
    H = res.cfr(BW, NF)
    osc = oracle.OracleScene(office.pos, office.nrm, office.surf, office.mat, r_p=0.015, grid_cell=0.1)
    osim = oracle.OracleSim(osc, office.tx, office.rx, oracle.SimParams(delta=1e-5 * office.diag, **kp),
                            ray_ids=ids.astype(np.int64))
    P = osim.paths()
    a, _ = osim.field(*(m.astype(np.float64) for m in (office.eps_r, office.sigma, office.scat)))
    f = cfr.freqs(float(np.float32(28e9)), BW, NF)
    Ho = cfr.cfr(a, P["tau"], P["j"], office.rx.shape[0], f)
    gp = res.paths()
    gk = set(zip(gp["key_hi"].tolist(), gp["key_lo"].tolist()))
    ok_keys = set(zip(P["hi"].tolist(), P["lo"].tolist()))
    unmatched = np.array([(int(h), int(l)) not in gk for h, l in zip(P["hi"], P["lo"])])
    # GPU-only keys: their |a| joins the bound
    ga = np.abs(gp["a"][:, 0] + 1j * gp["a"][:, 1])
    extra = np.zeros(office.rx.shape[0])
    for h, l, j, x in zip(gp["key_hi"], gp["key_lo"], gp["rx"], ga):
        if (int(h), int(l)) not in ok_keys:
            extra[j] += x
    amp = np.abs(a)
    bound = np.zeros_like(np.abs(H))
    for j in range(office.rx.shape[0]):
        m = P["j"] == j
        bound[j] = (amp[m, None] * (1e-4 + 2 * np.pi * f[None, :] * P["tau"][m, None] * 1e-6)).sum(0)
        bound[j] += amp[m & unmatched].sum() + extra[j]
    err = np.abs(H - Ho)
    print("office CFR: paths", len(P["tau"]), "unmatched", int(unmatched.sum()),
          "max |dH|/bound", float((err / bound).max()))
    assert np.all(err <= bound)


def test_recover_materials_with_the_cir_loss(office):
    """The Eq. 5 learning workload: office, 4 TX positions x 16 RX, CFR
    targets at hidden materials (seed 3), 200 Adam steps from eps_r 4,
    sigma 0.01, S 0.3.  eps_r and S within 5 %; sigma reported."""
    from paper_2507_04021_gb300 import learn
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, office.pos, office.nrm, office.surf, office.mat, r_p=0.015)
    traj = inputs.trajectory(office.extra["boxes"])
    txs = [office.tx] + [traj[i] for i in (0, 96, 192)]
    p = nrt.default_trace_params(max_depth=3, capture=nrt.CAPTURE_VIS, diffuse=1,
                                 n_rays=1_000_000, rep_tries=4)
    sc.set_materials(office.eps_r, office.sigma, office.scat)
    results = [sc.trace(tx, office.rx, p) for tx in txs]
    he, hs, hc = (x.astype(np.float64) for x in inputs.hidden_materials())
    T = learn.cfr_targets(sc, results, he, hs, hc)
    backend = learn.LibnrtCfrBackend(sc, results, T)
    L = len(he)
    fit = learn.recover_materials_cfr(backend, (np.full(L, 4.0), np.full(L, 0.01), np.full(L, 0.3)),
                                      steps=200, lr=0.05)
    print("CIR-loss recovery: loss", fit.loss[0], "->", fit.loss[-1])
    print(" eps rel err", np.round(np.abs(fit.eps - he) / he, 4))
    print(" S   rel err", np.round(np.abs(fit.scat - hc) / hc, 4))
    print(" sig rel err", np.round(np.abs(fit.sigma - hs) / hs, 3))
    assert fit.loss[-1] < 1e-2 * fit.loss[0]
    assert np.all(np.abs(fit.eps - he) / he < 0.05)
    assert np.all(np.abs(fit.scat - hc) / hc < 0.05)
