"""Learned launch proposal workflow (marshalling only: every step runs in
libnrt's kernels).

The paper traces a fixed Fibonacci launch (Sec. II-B).  The proposal adds a
small network that scores the launch's directions for a transmitter
position; a Gumbel-top-k draw over its logits (plus a stratified uniform
share) picks a ray subset of the same launch, traced like any subset.
Received power is computed from each key's refined geometry (Sec. II-B-2),
so a key found by any of its member rays gives the same path: the proposal
only has to find the keys that carry the power.

Workload (defaults): the office scene, RX-sphere capture (r = 0.1 m) at the
16 receivers, up to 5 specular interactions, no diffuse paths; training
rays = 20,000 launch rays for each of 250 trajectory positions (5M labelled
rays, label 1 = member of a valid specular key); evaluation at the other
trajectory positions, 1e5 proposed rays (90% Gumbel-top-k, 10% stratified)
against the uniform 1M launch.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np
import torch

from . import inputs, nrt

N_LAUNCH = 1_000_000


def sphere_params(n_rays: int = N_LAUNCH, labels: bool = False, max_depth: int = 5):
    return nrt.default_trace_params(max_depth=max_depth, capture=nrt.CAPTURE_SPHERE, diffuse=0,
                                    n_rays=n_rays, rep_tries=0, r_rx=0.1,
                                    ray_labels=int(labels))


@dataclass
class TrainingSet:
    tx_table: torch.Tensor   # [n_tx, 3] float32
    tx_index: torch.Tensor   # [n] int32
    ray_id: torch.Tensor     # [n] int32 (uint32 ids)
    label: torch.Tensor      # [n] float32
    positive_rate: float
    trace_s: float


def make_training_set(scene: nrt.Scene, txs: np.ndarray, rx: np.ndarray, rays_per_tx: int = 20000,
                      n_rays: int = N_LAUNCH, seed: int = inputs.SEED_MLP,
                      max_depth: int = 5) -> TrainingSet:
    """Trace a random ray subset of the launch from each TX with per-ray
    labels (the tracer's own validated specular keys)."""
    rng = inputs.rng_for(seed, 3)
    p = sphere_params(n_rays, labels=True, max_depth=max_depth)
    ids_all, lab_all, txi_all = [], [], []
    t0 = time.perf_counter()
    for t, tx in enumerate(txs):
        ids = np.sort(rng.choice(n_rays, rays_per_tx, replace=False)).astype(np.uint32)
        r = scene.trace(tx, rx, p, ray_subset=ids)
        ids_all.append(ids)
        lab_all.append(r.ray_labels())
        txi_all.append(np.full(ids.size, t, np.int32))
        r.close()
    dt = time.perf_counter() - t0
    lab = np.concatenate(lab_all).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    return TrainingSet(dev(np.asarray(txs, np.float32)), dev(np.concatenate(txi_all)),
                       dev(np.concatenate(ids_all).view(np.int32)), dev(lab),
                       float(lab.mean()), dt)


DEFAULT_SCHEDULE = ((2e-3, 10),)  # (learning rate, epochs) phases


def train(mlp: nrt.Mlp, data: TrainingSet, schedule=DEFAULT_SCHEDULE, batch: int = 8192,
          seed: int = inputs.SEED_MLP):
    """Adam over shuffled epochs; positives weighted by sqrt(negatives / positives)."""
    n = int(data.ray_id.shape[0])
    steps = n // batch
    pr = max(data.positive_rate, 1e-6)
    wp = float(np.sqrt((1.0 - pr) / pr))
    rng = inputs.rng_for(seed, 4)
    losses = []
    t0 = time.perf_counter()
    for lr, epochs in schedule:
        for _ in range(epochs):
            order = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
            losses.append(mlp.train(data.tx_table, data.tx_index, data.ray_id, data.label,
                                    order_dev=order, start=0, steps=steps, lr=lr, batch=batch,
                                    pos_weight=wp))
    return np.concatenate(losses), time.perf_counter() - t0, wp


@dataclass
class Evaluation:
    p_uniform: np.ndarray    # per-RX power, uniform launch
    p_proposal: np.ndarray   # per-RX power, proposed subset
    db_err: np.ndarray       # 10 log10(P_prop / P_unif)
    n_proposed: int
    ms_uniform: float
    ms_proposal: float       # scoring + selection + subset trace
    ms_score: float
    fallback: bool           # an RX had no path under the proposal
    power_recall: np.ndarray  # per RX: share of the uniform launch's path power whose keys
                              # the proposal also found (nan where the uniform launch has none)


def key_power(paths) -> dict:
    """key -> (rx, |a|^2) of a result's paths."""
    a = paths["a"].astype(np.float64)
    w = (a * a).sum(1)
    return {(int(h), int(l)): (int(j), float(x))
            for h, l, j, x in zip(paths["key_hi"], paths["key_lo"], paths["rx"], w)}


def power_recall(ref: dict, found: dict, n_rx: int) -> np.ndarray:
    tot = np.zeros(n_rx)
    got = np.zeros(n_rx)
    for k, (j, w) in ref.items():
        tot[j] += w
        if k in found:
            got[j] += w
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(tot > 0, got / tot, np.nan)


def evaluate(scene: nrt.Scene, mlp: nrt.Mlp, tx, rx, n_rays: int = N_LAUNCH, k_total: int = 100_000,
             top_frac: float = 0.9, seed: int = 1, max_depth: int = 5) -> Evaluation:
    """Uniform n_rays launch against the proposal's k_total rays (CUDA-event
    timing on the library's stream; both include their own readback)."""
    p = sphere_params(n_rays, max_depth=max_depth)
    st = torch.cuda.ExternalStream(scene.ctx.stream_handle())
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    torch.cuda.synchronize()
    ev[0].record(st)
    ru = scene.trace(tx, rx, p)
    ev[1].record(st)
    pu = ru.power().astype(np.float64)
    ku = key_power(ru.paths())
    ru.close()
    logits = torch.empty(n_rays, dtype=torch.float32, device="cuda")
    ids = torch.empty(k_total, dtype=torch.int32, device="cuda")
    k_top = int(round(top_frac * k_total))
    torch.cuda.synchronize()
    ev[2].record(st)
    mlp.score(tx, None, n_rays, logits, sync=False)
    ev[3].record(st)
    m = nrt.propose(scene.ctx, logits, k_top, k_total - k_top, seed, ids)
    rp = scene.trace(tx, rx, p, ray_subset=ids[:m])
    ev[4].record(st)
    pp = rp.power().astype(np.float64)
    per_rx, _ = rp.counts()
    kp = key_power(rp.paths())
    rp.close()
    torch.cuda.synchronize()
    with np.errstate(divide="ignore", invalid="ignore"):
        db = 10.0 * np.log10(pp / pu)
    return Evaluation(pu, pp, db, m, ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[4]),
                      ev[2].elapsed_time(ev[3]), bool(np.any(per_rx == 0)),
                      power_recall(ku, kp, len(pu)))


def uniform_subset(scene: nrt.Scene, tx, rx, k: int, n_rays: int = N_LAUNCH, seed: int = 0,
                   max_depth: int = 5):
    """(per-RX power, key -> (rx, |a|^2)) from k launch rays drawn uniformly at
    random: the method without the network, at the proposal's ray count."""
    ids = np.sort(inputs.rng_for(seed, 5).choice(n_rays, k, replace=False)).astype(np.uint32)
    r = scene.trace(tx, rx, sphere_params(n_rays, max_depth=max_depth), ray_subset=ids)
    p = r.power().astype(np.float64)
    kp = key_power(r.paths())
    r.close()
    return p, kp


def reference_keys(scene: nrt.Scene, tx, rx, n_rays: int = N_LAUNCH, max_depth: int = 5) -> dict:
    r = scene.trace(tx, rx, sphere_params(n_rays, max_depth=max_depth))
    k = key_power(r.paths())
    r.close()
    return k

