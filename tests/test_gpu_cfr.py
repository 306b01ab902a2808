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
