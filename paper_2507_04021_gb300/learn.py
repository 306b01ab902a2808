"""Learning per-label materials through the hand-written adjoint (Sec. III-B).

The paper learns relative permittivity, conductivity and scattering
coefficient per material label with Adam and activations that keep them in
their valid ranges.  Here the forward is the library's field of stored paths
(``nrt_field``: path geometry does not depend on the materials, so nothing is
re-traced) and the backward is ``nrt_backward``.  The loss is the mean squared
error of the per-receiver path gain in dB over one or more simulations.

Activations (a reading of "appropriate activation functions"):
eps_r = 1 + softplus(u), sigma = exp(v), S = sigmoid(w).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch


class PowerFn(torch.autograd.Function):
    """P[r, j] = received power of simulation r at receiver j, as a function of
    per-label (eps_r, sigma, S).  ``backend`` provides two callables:
    ``forward(eps, sigma, scat) -> np.ndarray [R, M]`` and
    ``backward(eps, sigma, scat, dL_dP [R, M]) -> (g_eps, g_sigma, g_scat)``."""

    @staticmethod
    def forward(ctx, eps, sig, sca, backend):
        e = eps.detach().cpu().numpy().astype(np.float64)
        s = sig.detach().cpu().numpy().astype(np.float64)
        c = sca.detach().cpu().numpy().astype(np.float64)
        P = backend.forward(e, s, c)
        ctx.backend = backend
        ctx.mats = (e, s, c)
        ctx.dev = eps.device
        return torch.as_tensor(np.asarray(P, np.float64), device=eps.device)

    @staticmethod
    def backward(ctx, gP):
        e, s, c = ctx.mats
        ge, gs, gc = ctx.backend.backward(e, s, c, gP.detach().cpu().numpy().astype(np.float64))
        t = lambda a: torch.as_tensor(np.asarray(a, np.float64), device=ctx.dev)  # noqa: E731
        return t(ge), t(gs), t(gc), None


class LibnrtBackend:
    """Field and adjoint of stored paths through libnrt (one scene, R results)."""

    def __init__(self, scene, results):
        self.scene = scene
        self.results = list(results)

    def forward(self, eps, sig, sca):
        self.scene.set_materials(eps.astype(np.float32), sig.astype(np.float32),
                                 sca.astype(np.float32))
        out = []
        for r in self.results:
            r.field()
            out.append(r.power().astype(np.float64))
        return np.stack(out)

    def backward(self, eps, sig, sca, dL_dP):
        ge = np.zeros(len(eps))
        gs = np.zeros(len(eps))
        gc = np.zeros(len(eps))
        for r, g in zip(self.results, dL_dP):
            a, b, c = r.backward(g.astype(np.float32))
            ge += a
            gs += b
            gc += c
        return ge, gs, gc


def to_params(eps, sig, sca):
    """Unconstrained parameters (u, v, w) for given materials."""
    eps = np.asarray(eps, np.float64)
    return (np.log(np.expm1(eps - 1.0)), np.log(np.asarray(sig, np.float64)),
            np.log(np.asarray(sca, np.float64) / (1.0 - np.asarray(sca, np.float64))))


def from_params(u, v, w):
    return 1.0 + torch.nn.functional.softplus(u), torch.exp(v), torch.sigmoid(w)


@dataclass
class Fit:
    eps: np.ndarray
    sigma: np.ndarray
    scat: np.ndarray
    loss: list = field(default_factory=list)


def save_checkpoint(path, params, opt, hist):
    """Material optimiser state: the unconstrained parameters (u, v, w), Adam's
    moments and step counts, and the loss history."""
    torch.save({"params": [p.detach().clone() for p in params], "opt": opt.state_dict(),
                "loss": list(hist)}, path)


def recover_materials(backend, target_db, init, steps=200, lr=0.05, checkpoint=None,
                      checkpoint_every=0, resume=None) -> Fit:
    """Adam on the per-RX dB-gain MSE; target_db [R, M]; init = (eps, sigma, S).
    checkpoint / checkpoint_every: write the optimiser state to that path
    every so many steps (and after the last); resume: continue from such a
    checkpoint (its steps count toward `steps`)."""
    u0, v0, w0 = to_params(*init)
    u = torch.tensor(u0, requires_grad=True)
    v = torch.tensor(v0, requires_grad=True)
    w = torch.tensor(w0, requires_grad=True)
    tgt = torch.as_tensor(np.asarray(target_db, np.float64))
    opt = torch.optim.Adam([u, v, w], lr=lr)
    hist = []
    if resume is not None:
        st = torch.load(resume, weights_only=False)
        with torch.no_grad():
            for p, q in zip((u, v, w), st["params"]):
                p.copy_(q)
        opt.load_state_dict(st["opt"])
        hist = list(st["loss"])
    for it in range(len(hist), steps):
        opt.zero_grad()
        eps, sig, sca = from_params(u, v, w)
        P = PowerFn.apply(eps, sig, sca, backend)
        G = 10.0 * torch.log10(P)
        loss = torch.mean((G - tgt) ** 2)
        loss.backward()
        opt.step()
        hist.append(float(loss.detach()))
        if checkpoint and ((checkpoint_every and (it + 1) % checkpoint_every == 0) or it + 1 == steps):
            save_checkpoint(checkpoint, (u, v, w), opt, hist)
    with torch.no_grad():
        eps, sig, sca = from_params(u, v, w)
    return Fit(eps.numpy(), sig.numpy(), sca.numpy(), hist)


# ---------------------------------------------------------------- Eq. 5 (CIR) loss
class CfrLossFn(torch.autograd.Function):
    """Eq. 5 loss |h - h^|^2 / |h^|^2 on the CIR (equal on the CFR), weighted
    over receivers and summed over simulations, as a function of per-label
    (eps_r, sigma, S).  ``backend.loss_and_grads(eps, sigma, scat)`` returns
    (loss, (g_eps, g_sigma, g_scat)) from nrt_cfr_backward."""

    @staticmethod
    def forward(ctx, eps, sig, sca, backend):
        e = eps.detach().cpu().numpy().astype(np.float64)
        s = sig.detach().cpu().numpy().astype(np.float64)
        c = sca.detach().cpu().numpy().astype(np.float64)
        loss, g = backend.loss_and_grads(e, s, c)
        ctx.g = [torch.as_tensor(np.asarray(x, np.float64), device=eps.device) for x in g]
        return torch.as_tensor(loss, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, gL):
        return gL * ctx.g[0], gL * ctx.g[1], gL * ctx.g[2], None


class LibnrtCfrBackend:
    """CFR targets of R simulations (stored paths re-weighted by the field;
    nothing is re-traced) and the Eq. 5 loss with receivers weighted 1/M."""

    def __init__(self, scene, results, targets, bandwidth=1.5e9):
        self.scene = scene
        self.results = list(results)
        self.targets = [np.asarray(t) for t in targets]
        self.bandwidth = bandwidth

    def loss_and_grads(self, eps, sig, sca):
        self.scene.set_materials(eps.astype(np.float32), sig.astype(np.float32),
                                 sca.astype(np.float32))
        total = 0.0
        g = [np.zeros(len(eps)) for _ in range(3)]
        for r, T in zip(self.results, self.targets):
            r.field()
            w = np.full(r.n_rx, 1.0 / r.n_rx)
            loss, gr = r.cfr_backward(T, w, self.bandwidth)
            total += float(np.sum(w * loss))
            for i in range(3):
                g[i] += gr[i]
        return total, g


def cfr_targets(scene, results, eps, sig, sca, bandwidth=1.5e9, n_freq=129):
    """Target CFRs of the results at given materials (the ground truth)."""
    scene.set_materials(np.asarray(eps, np.float32), np.asarray(sig, np.float32),
                        np.asarray(sca, np.float32))
    out = []
    for r in results:
        r.field()
        out.append(r.cfr(bandwidth, n_freq))
    return out


def recover_materials_cfr(backend, init, steps=200, lr=0.05) -> Fit:
    """Adam on the Eq. 5 loss; init = (eps, sigma, S)."""
    u0, v0, w0 = to_params(*init)
    u = torch.tensor(u0, requires_grad=True)
    v = torch.tensor(v0, requires_grad=True)
    w = torch.tensor(w0, requires_grad=True)
    opt = torch.optim.Adam([u, v, w], lr=lr)
    hist = []
    for _ in range(steps):
        opt.zero_grad()
        eps, sig, sca = from_params(u, v, w)
        loss = CfrLossFn.apply(eps, sig, sca, backend)
        loss.backward()
        opt.step()
        hist.append(float(loss.detach()))
    with torch.no_grad():
        eps, sig, sca = from_params(u, v, w)
    return Fit(eps.numpy(), sig.numpy(), sca.numpy(), hist)
