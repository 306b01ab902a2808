"""Material learning loop (Sec. III-B analogue) with the FP64 oracle as the
field/adjoint backend: checks the autograd wiring, the activations and the
recovery of hidden materials from per-RX path gains.  CPU only.

Identifiability (recorded): from received power alone at 28 GHz the
conductivity is weakly observable (Im eta = sigma / (2 pi f eps0) ~ 0.64
sigma, small against eps_r), so only eps_r and S are required to recover.
"""
import numpy as np
import pytest

import oracle
from paper_2507_04021_gb300 import inputs, learn


class OracleBackend:
    def __init__(self, sims):
        self.sims = sims

    def forward(self, e, s, c):
        return np.stack([sm.field(e, s, c)[1] for sm in self.sims])

    def backward(self, e, s, c, g):
        out = [np.zeros(len(e)) for _ in range(3)]
        for sm, gg in zip(self.sims, g):
            for k, a in enumerate(sm.backward(e, s, c, gg)):
                out[k] += a
        return out


def test_powerfn_gradient_matches_finite_differences(office):
    sc = oracle.OracleScene(office.pos, office.nrm, office.surf, office.mat, r_p=0.015,
                            grid_cell=0.1)
    sims = [oracle.OracleSim(sc, office.tx, office.rx,
                             oracle.SimParams(max_depth=2, capture=1, diffuse=1,
                                              n_rays=1_000_000, rep_tries=4),
                             ray_ids=np.arange(0, 1_000_000, 4000))]
    b = OracleBackend(sims)
    import torch
    u0, v0, w0 = learn.to_params(office.eps_r, office.sigma, office.scat)
    u = torch.tensor(u0, requires_grad=True)
    v = torch.tensor(v0, requires_grad=True)
    w = torch.tensor(w0, requires_grad=True)
    tgt = torch.linspace(-80, -60, office.rx.shape[0], dtype=torch.float64)[None]

    def loss_of(u, v, w):
        e, s, c = learn.from_params(u, v, w)
        P = learn.PowerFn.apply(e, s, c, b)
        return torch.mean((10 * torch.log10(P) - tgt) ** 2)

    L = loss_of(u, v, w)
    L.backward()
    for p, g in ((u, u.grad), (w, w.grad)):
        for l in range(len(p)):
            h = 1e-6
            d = torch.zeros_like(p)
            d[l] = h
            with torch.no_grad():
                args_p = [q + d if q is p else q for q in (u, v, w)]
                args_m = [q - d if q is p else q for q in (u, v, w)]
                fd = (loss_of(*args_p) - loss_of(*args_m)) / (2 * h)
            assert float(g[l]) == pytest.approx(float(fd), rel=1e-4, abs=1e-7)


def test_recover_hidden_materials(office):
    sc = oracle.OracleScene(office.pos, office.nrm, office.surf, office.mat, r_p=0.015,
                            grid_cell=0.1)
    traj = inputs.trajectory(office.extra["boxes"])
    txs = [office.tx] + [traj[i] for i in (0, 32, 64, 96, 128, 160, 192)]
    ids = np.arange(0, 1_000_000, 500)
    sims = [oracle.OracleSim(sc, tx, office.rx,
                             oracle.SimParams(max_depth=3, capture=1, diffuse=1,
                                              n_rays=1_000_000, rep_tries=4), ray_ids=ids)
            for tx in txs]
    b = OracleBackend(sims)
    he, hs, hc = (a.astype(np.float64) for a in inputs.hidden_materials())
    target = 10 * np.log10(b.forward(he, hs, hc))
    L = len(he)
    fit = learn.recover_materials(b, target, (np.full(L, 4.0), np.full(L, 0.01), np.full(L, 0.3)),
                                  steps=200, lr=0.1)
    assert fit.loss[-1] < 1e-3 * fit.loss[0]
    assert np.all(np.abs(fit.eps - he) / he < 0.05), fit.eps
    assert np.all(np.abs(fit.scat - hc) / hc < 0.05), fit.scat
