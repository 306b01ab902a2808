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


class DevicePowerFn(torch.autograd.Function):
    """The same P[r, j] with every tensor on the GPU: the materials reach the
    library through nrt_set_materials_device, the power comes back through
    nrt_field_read_device and dL/dP goes to nrt_backward_noalloc, so a
    learning step copies nothing through the host.  ``backend`` is a
    LibnrtDeviceBackend."""

    @staticmethod
    def forward(ctx, eps, sig, sca, backend):
        ctx.backend = backend
        return backend.forward(eps, sig, sca)

    @staticmethod
    def backward(ctx, gP):
        ge, gs, gc = ctx.backend.backward(gP)
        return ge, gs, gc, None


class LibnrtDeviceBackend:
    """Field and adjoint of stored paths through libnrt with device buffers
    (one scene, R results with the same receivers; scalar polarisation models
    without diffraction, the cases nrt_backward_noalloc serves).  The
    library's work runs on the context stream, ordered after the caller's
    current stream and before its next work by stream waits."""

    on_device = True

    def __init__(self, scene, results):
        self.scene = scene
        self.results = list(results)
        self.device = torch.device("cuda", scene.ctx.device)
        self._stream = torch.cuda.ExternalStream(scene.ctx.stream_handle(), device=self.device)

    def _enter(self):
        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self._stream.cuda_stream:
            self._stream.wait_stream(cur)
        return cur

    def _leave(self, cur):
        if cur.cuda_stream != self._stream.cuda_stream:
            cur.wait_stream(self._stream)

    def forward(self, eps, sig, sca):
        mat = torch.stack([eps.detach(), sig.detach(), sca.detach()]).to(torch.float32).contiguous()
        P = torch.empty((len(self.results), self.results[0].n_rx), dtype=torch.float64,
                        device=self.device)
        cur = self._enter()
        self.scene.set_materials_device(mat)
        for i, r in enumerate(self.results):
            r.field()
            r.power_device(P[i])
        self._leave(cur)
        return P

    def backward(self, gP):
        L = self.scene.n_labels
        g = gP.detach().to(torch.float32).contiguous()
        grads = torch.empty((len(self.results), 3 * L), dtype=torch.float32, device=self.device)
        cur = self._enter()
        for i, r in enumerate(self.results):
            r.backward_noalloc(g[i], grads[i])
        self._leave(cur)
        tot = grads.to(torch.float64).sum(0).view(3, L)
        return tot[0], tot[1], tot[2]


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
    checkpoint (its steps count toward `steps`).  A backend with
    ``on_device`` (LibnrtDeviceBackend) keeps the parameters, the optimiser
    and the loss on its GPU; the loss history is read back only at
    checkpoints and at the end."""
    dev = backend.device if getattr(backend, "on_device", False) else None
    fn = DevicePowerFn if dev is not None else PowerFn
    u0, v0, w0 = to_params(*init)
    u = torch.tensor(u0, requires_grad=True, device=dev)
    v = torch.tensor(v0, requires_grad=True, device=dev)
    w = torch.tensor(w0, requires_grad=True, device=dev)
    tgt = torch.as_tensor(np.asarray(target_db, np.float64), device=dev)
    opt = torch.optim.Adam([u, v, w], lr=lr)
    hist = []
    pending = []

    def flush():
        if pending:
            hist.extend(torch.stack(pending).cpu().tolist())
            pending.clear()

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
        P = fn.apply(eps, sig, sca, backend)
        G = 10.0 * torch.log10(P)
        loss = torch.mean((G - tgt) ** 2)
        loss.backward()
        opt.step()
        pending.append(loss.detach())
        if checkpoint and ((checkpoint_every and (it + 1) % checkpoint_every == 0) or it + 1 == steps):
            flush()
            save_checkpoint(checkpoint, (u, v, w), opt, hist)
    flush()
    with torch.no_grad():
        eps, sig, sca = from_params(u, v, w)
    return Fit(eps.cpu().numpy(), sig.cpu().numpy(), sca.cpu().numpy(), hist)


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
