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


class _SmoothBackend:
    """A closed-form stand-in for the field (power = sum over labels of a
    smooth function of the materials per receiver) with its exact gradient:
    enough to exercise the optimiser's bookkeeping on the CPU."""

    def __init__(self, L=3, M=5):
        rng = np.random.default_rng(0)
        self.A = rng.uniform(0.5, 1.5, (1, M, L))

    def forward(self, e, s, c):
        return np.sum(self.A * (e / (1 + e) + 0.3 * np.tanh(10 * s) + c ** 2), axis=2) + 1e-3

    def backward(self, e, s, c, g):
        G = g[:, :, None] * self.A
        return (np.sum(G / (1 + e) ** 2, axis=(0, 1)),
                np.sum(G * 3.0 / np.cosh(10 * s) ** 2, axis=(0, 1)),
                np.sum(G * 2 * c, axis=(0, 1)))


def test_material_optimiser_checkpoint_resume(tmp_path):
    """Resuming from a checkpoint (parameters, Adam moments and step counts,
    loss history) reproduces the uninterrupted run exactly; resuming with
    fresh Adam state does not."""
    b = _SmoothBackend()
    tgt = 10 * np.log10(b.forward(np.array([3.0, 5.0, 2.0]), np.array([0.02, 0.05, 0.01]),
                                  np.array([0.2, 0.4, 0.3])))
    init = (np.full(3, 4.0), np.full(3, 0.01), np.full(3, 0.3))
    full = learn.recover_materials(b, tgt, init, steps=40, lr=0.05)
    ck = str(tmp_path / "mat.pt")
    learn.recover_materials(b, tgt, init, steps=15, lr=0.05, checkpoint=ck, checkpoint_every=5)
    res = learn.recover_materials(b, tgt, init, steps=40, lr=0.05, resume=ck)
    assert res.loss == full.loss
    assert np.array_equal(res.eps, full.eps) and np.array_equal(res.scat, full.scat)
    # the same parameters with a fresh optimiser take a different path
    part = learn.recover_materials(b, tgt, init, steps=15, lr=0.05)
    fresh = learn.recover_materials(b, tgt, (part.eps, part.sigma, part.scat), steps=25, lr=0.05)
    assert not np.allclose(fresh.eps, full.eps, rtol=1e-9, atol=0)
