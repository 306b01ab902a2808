"""Benchmark: one full 5-interaction simulation of the office workload per step.

Workload: 20 x 10 x 3 m office, 2,000,000 oriented labelled points (40 boxes,
1 cm position noise, 2 degree normal jitter), 16 receivers, one TX, a
1,000,000-ray Fibonacci launch, up to 5 interactions, visibility-matrix
capture with diffuse last interactions, dedup, refinement and field.
A step is one call of the simulation (visibility matrix, trace, candidates,
dedup, diffuse validation, specular refinement and validation, field).
The scene build is setup and reported separately.

value     = ray segments cast per second (trace segments + visibility casts +
            LOS casts + validation casts), device-timed with CUDA events on the
            library's stream, the L2 flushed between steps.
ms_per_step = device time of one simulation.
e2e       = the same metric through the C ABI with host buffers: TX/RX copied
            in, all paths and the per-RX power read back, every step.
roofline  = the dominant work, the validation phase (every candidate of a key
            refined, the paper's rule): algorithmic bytes of its casts
            (oracle-counted disc reads per diffuse shadow cast; the
            trace-segment figure for specular refinement legs, tests/golden)
            over its CUDA-event duration, against the measured HBM copy
            bandwidth; roofline_other: the trace and visibility kernels.

batch     = the robot-trajectory workload: 256 TX-RX pairs with budgets
            U[1e5, 1e6], packet/schedule autotuned, the whole batch replayed
            from a CUDA graph; per-pair trace completion p50/p99 from device
            timestamps and pairs/s.

proposal  = the learned launch proposal: training on the GPU, then the
            uniform 1M launch against 1e5 proposed rays at held-out TX
            positions (speedup, receivers within 0.5 dB, power recall).

--impl reference times the FP64 CPU oracle on a bounded ray sample of the
same workload on the host cores (the reference arm of this tier).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms per 5-bounce sim & ray-segments/s; proposal vs uniform speedup @0.5 dB"
WORKLOAD = ("office 20x10x3 m + 40 boxes, 2M points, 16 RX, 1M Fibonacci rays, "
            "5 interactions, visibility capture + diffuse, dedup + refinement + field")
N_RAYS = 1_000_000


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# The ncu counters in profiles/office_sim_top_kernels.md hold while the
# sources they were taken from are unchanged: the validation phase's against
# the whole of csrc/sim.cu + csrc/nrt_device.cuh, the trace and visibility
# kernels' against the part of sim.cu before the validation code (which
# holds them and everything they call) + nrt_device.cuh.
_VALIDATION_MARK = "// Diffuse: the candidate's own interaction points"


def _source_hash(kernel):
    import hashlib
    sim = open(os.path.join(ROOT, "paper_2507_04021_gb300", "csrc", "sim.cu"), "rb").read()
    dev = open(os.path.join(ROOT, "paper_2507_04021_gb300", "csrc", "nrt_device.cuh"), "rb").read()
    if kernel in ("trace_kernel", "vis_kernel"):
        i = sim.find(_VALIDATION_MARK.encode())
        if i < 0:
            return None
        sim = sim[:i]
    return hashlib.sha256(sim + dev).hexdigest()


def _profile_value(key, kernel):
    """The committed summary's `key` figure for `kernel`, or None once the
    kernel's sources have changed since the capture."""
    path = os.path.join(ROOT, "profiles", "office_sim_top_kernels.md")
    if not os.path.exists(path):
        return None
    val = None
    sha = {}
    for ln in open(path):
        f = ln.split()
        if len(f) == 3 and f[0] == key and f[1] == kernel:
            val = float(f[2])
        if len(f) == 2 and f[0] in ("source_sha256", "source_sha256_traversal"):
            sha[f[0]] = f[1]
    want = sha.get("source_sha256_traversal" if kernel in ("trace_kernel", "vis_kernel")
                   else "source_sha256")
    return val if (val is not None and want is not None and want == _source_hash(kernel)) else None


def _traffic(kernel):
    """DRAM bytes per launch of `kernel` (per simulation for the validation
    phase) from the committed ncu summary, or None once its sources changed."""
    return _profile_value("traffic_bytes_per_launch", kernel)


def _l2_bytes(kernel):
    """L2 bytes per unit (lts__t_bytes per cast, from an ncu capture of the
    small case) of `kernel` from the committed summary, or None once its
    sources changed."""
    return _profile_value("l2_bytes_per_unit", kernel)


def _alg_bytes():
    d = json.load(open(os.path.join(ROOT, "tests", "golden", "office_algorithmic_bytes.json")))
    return d


_ORACLE_SCENE = {}


def run_oracle_sample(n_sample: int, threads: int = 0):
    """Time the FP64 oracle on a ray sample of the workload; returns casts/s info.
    The oracle's scene (voxels and its uniform grid) is built once, untimed."""
    import oracle
    from paper_2507_04021_gb300 import inputs
    if not _ORACLE_SCENE:
        o = inputs.office_scene()
        _ORACLE_SCENE["o"] = o
        _ORACLE_SCENE["sc"] = oracle.OracleScene(o.pos, o.nrm, o.surf, o.mat, r_p=0.015,
                                                 grid_cell=0.1)
    o, sc = _ORACLE_SCENE["o"], _ORACLE_SCENE["sc"]
    stride = max(1, N_RAYS // n_sample)
    ids = np.arange(0, N_RAYS, stride, dtype=np.int64)[:n_sample]
    p = oracle.SimParams(max_depth=5, capture=1, diffuse=1, n_rays=N_RAYS, rep_tries=0,
                         n_threads=threads)
    t0 = time.perf_counter()
    sim = oracle.OracleSim(sc, o.tx, o.rx, p, ray_ids=ids)
    sim.field(o.eps_r, o.sigma, o.scat)
    dt = time.perf_counter() - t0
    c = sim.cast_counts()
    casts = sum(c.values())
    return {"seconds": dt, "casts": casts, "rays": int(ids.size), "counts": c,
            "cores": oracle.max_threads() if threads <= 0 else threads}


def reference_arm(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    n_sample = _env_int("NRT_REF_SAMPLE", 10000)
    times, rates = [], []
    info = None
    for i in range(args.warmup + args.steps):
        info = run_oracle_sample(n_sample)
        if i >= args.warmup:
            times.append(info["seconds"])
            rates.append(info["casts"] / info["seconds"])
    value = float(np.sum([info["casts"]] * len(times)) / np.sum(times))
    sample = (f"{info['rays']} of the {N_RAYS} launch rays (every {N_RAYS // info['rays']}th), "
              f"full pipeline, {info['casts']} casts per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ray-segments/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.mean(times) * 1000.0), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_rays": info["rays"]},
        "cpu_baseline": {"value": value, "unit": "ray-segments/s", "cores": info["cores"],
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "ray-segments/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_bench(args, scene, o, rank, stream, flush):
    """Robot-trajectory batch: pairs along the seeded trajectory, one fixed RX,
    per-pair budgets U[1e5, 1e6]; autotuned packet/schedule; the whole batch
    replayed from a CUDA graph.  Each rank runs its own pairs (independent
    problems, weak scaling)."""
    import torch
    from paper_2507_04021_gb300 import inputs, nrt

    n = args.batch_pairs
    traj = inputs.trajectory(o.extra["boxes"])
    budgets = inputs.ray_budgets()[:n]
    tx = np.roll(traj, -rank * n, axis=0)[:n] if rank else traj[:n]
    rx = np.array([17.5, 8.0, 1.2], np.float32)
    p = nrt.default_trace_params(max_depth=5, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=1,
                                 rep_tries=0)
    cfgs = [(32, 1), (64, 1), (128, 1), (64, 0)]
    cal = scene.trace_batch(tx, rx, budgets, p, packet=64, schedule=1)
    tune_ms, best = cal.autotune(cfgs, repeats=1)
    cal.close()
    packet, schedule = cfgs[best]
    g = scene.trace_batch(tx, rx, budgets, p, packet=packet, schedule=schedule, use_graph=True)
    for _ in range(max(1, args.warmup)):
        g.replay()
    torch.cuda.synchronize()
    steps = max(1, args.batch_steps)
    tot, pair_ms, pair_paths_ms, launches, segs = [], [], [], 0, 0
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        tot.append(e0.elapsed_time(e1))
        pm, _, pv = g.batch_times(paths=True)
        pair_ms.append(pm)
        pair_paths_ms.append(pv)
        _, c = g.counts()
        launches += c["kernel_launches"] + 1
        segs += c["segments"] + c["vis_casts"] + c["los_casts"] + c["validation_casts"]
    _, c = g.counts()
    g.close()
    pm = np.concatenate(pair_ms)
    pv = np.concatenate(pair_paths_ms)
    ms = float(np.mean(tot))
    grouped = batch_groups(args, scene, tx, rx, budgets, p, packet, schedule, stream, flush)
    return {
        "workload": (f"{n} TX-RX pairs on the robot trajectory, RX (17.5, 8, 1.2), budgets "
                     f"U[1e5, 1e6] ({int(budgets.sum())} rays), 5 interactions, VIS + diffuse"),
        "pairs": n, "rays": int(budgets.sum()), "steps": steps,
        "ms_per_batch": ms, "pairs_per_s": n / (ms / 1000.0),
        "ray_segments_per_s": segs / (sum(tot) / 1000.0),
        "pair_trace_done_ms": {"p50": float(np.percentile(pm, 50)),
                               "p99": float(np.percentile(pm, 99))},
        "pair_paths_validated_ms": {"p50": float(np.percentile(pv, 50)),
                                    "p99": float(np.percentile(pv, 99))},
        "latency_note": "per-pair device timestamps from the start of the trace: the pair's last "
                        "traced ray, and its last path key validated (its path set known); the "
                        "field of all pairs follows in one pass, done at ms_per_batch",
        "autotune": {"configs": [list(c_) for c_ in cfgs], "trace_ms": [float(x) for x in tune_ms],
                     "chosen": {"packet": packet, "schedule": ["static", "persistent"][schedule]}},
        "graph": True, "gpu_launches": int(launches),
        "counts": {k: c[k] for k in ("segments", "vis_casts", "validation_casts", "candidates",
                                     "keys", "paths")},
        "grouped": grouped,
    }


def batch_groups(args, scene, tx, rx, budgets, p, packet, schedule, stream, flush, groups=4):
    """The same pairs as `groups` consecutive sub-batches (each its own graph),
    replayed back to back: a pair's path set is known when its group's
    validation is done, so latency falls at some cost in throughput.  Per-pair
    times are measured from the start of the first group: the group's start
    (CUDA events on the same stream) plus the pair's device stamp inside it."""
    import torch

    n = len(budgets)
    groups = max(1, min(groups, n))  # no empty group for small batches
    bounds = np.linspace(0, n, groups + 1).astype(int)
    plans = [scene.trace_batch(tx[a:b], rx, budgets[a:b], p, packet=packet, schedule=schedule,
                               use_graph=True) for a, b in zip(bounds[:-1], bounds[1:])]
    for g in plans:
        for _ in range(max(1, args.warmup)):
            g.replay()
    torch.cuda.synchronize()
    tot, pv_all, pm_all = [], [], []
    for _ in range(max(1, args.batch_steps)):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(groups + 1)]
        ev[0].record(stream)
        stamps = []
        for gi, g in enumerate(plans):
            g.replay()  # (synchronises: the stamps are read back per group)
            pm, _, pv = g.batch_times(paths=True)
            stamps.append((pm, pv))
            ev[gi + 1].record(stream)
        torch.cuda.synchronize()
        tot.append(ev[0].elapsed_time(ev[groups]))
        for gi, (pm, pv) in enumerate(stamps):
            start = ev[0].elapsed_time(ev[gi]) if gi else 0.0
            pm_all.append(start + pm)
            pv_all.append(start + pv)
    for g in plans:
        g.close()
    pm = np.concatenate(pm_all)
    pv = np.concatenate(pv_all)
    ms = float(np.mean(tot))
    return {"groups": groups, "ms_per_batch": ms, "pairs_per_s": n / (ms / 1000.0),
            "pair_trace_done_ms": {"p50": float(np.percentile(pm, 50)),
                                   "p99": float(np.percentile(pm, 99))},
            "pair_paths_validated_ms": {"p50": float(np.percentile(pv, 50)),
                                        "p99": float(np.percentile(pv, 99))},
            "note": "consecutive sub-batches of the trajectory, each a recorded graph; a group's "
                    "start is the previous group's end (host round trip between groups included)"}


def launch_bench(scene, o, tx, stream):
    """The paper's launch (one ray per DPS toward its reception point) against
    the Fibonacci sphere with the same number of rays: device time, paths
    and received power per receiver (office, 16 RX, 5 interactions, VIS +
    diffuse)."""
    import torch
    from paper_2507_04021_gb300 import nrt

    n_dps = int(scene.info()["n_dps"])
    out = {}
    for name, launch in (("dps", nrt.LAUNCH_DPS), ("fibonacci", nrt.LAUNCH_FIB)):
        p = nrt.default_trace_params(max_depth=5, capture=nrt.CAPTURE_VIS, diffuse=1,
                                     n_rays=n_dps, rep_tries=0)
        p.launch = launch
        scene.trace(tx, o.rx, p).close()  # warm-up
        ms = []
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = scene.trace(tx, o.rx, p)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            _, c = r.counts()
            pw = r.power().astype(np.float64)
            r.close()
        out[name] = {"rays": n_dps, "ms": float(np.median(ms)), "paths": c["paths"],
                     "keys": c["keys"],
                     "power_db": [round(float(10 * np.log10(x)), 3) if x > 0 else None for x in pw]}
    return out


def diffraction_bench(ctx, o, tx, stream, rays):
    """Single-bounce edge diffraction (Sec. II-B-3) on the 320 convex box edges
    of the office: the full simulation (1M rays, 16 RX, 5 interactions, VIS +
    diffuse) with and without diffraction, device-timed (median of 3), and the
    diffracted paths and edge visibility casts it adds."""
    import torch
    from paper_2507_04021_gb300 import inputs, nrt

    sc = nrt.Scene(ctx, o.pos, o.nrm, o.surf, o.mat, rho=0.0625, r_p=0.015, lambda_d=100.0)
    sc.set_materials(o.eps_r, o.sigma, o.scat)
    edges = inputs.office_edges(o.extra["boxes"])
    sc.set_edges(edges)
    out = {"edges": len(edges)}
    for name, flag in (("off", 0), ("on", 1)):
        p = nrt.default_trace_params(max_depth=5, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=rays,
                                     rep_tries=0, diffraction=flag)
        sc.trace(tx, o.rx, p).close()  # warm-up
        ms = []
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = sc.trace(tx, o.rx, p)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            _, c = r.counts()
            r.close()
        out[name] = {"ms": float(np.median(ms)), "paths": c["paths"],
                     "diffraction_casts": c["diffraction_casts"]}
    out["diffracted_paths"] = out["on"]["paths"] - out["off"]["paths"]
    return out


def rp_variant_bench(ctx, o, tx, stream, rays, r_p=0.025):
    """The office simulation with the larger disc radius r_p = 0.025 m (the
    second radius of the office configuration): device time (median of 3
    after a warm-up), counts and ray segments per second."""
    import torch
    from paper_2507_04021_gb300 import nrt

    sc = nrt.Scene(ctx, o.pos, o.nrm, o.surf, o.mat, rho=0.0625, r_p=r_p, lambda_d=100.0)
    sc.set_materials(o.eps_r, o.sigma, o.scat)
    p = nrt.default_trace_params(max_depth=5, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=rays,
                                 rep_tries=0)
    sc.trace(tx, o.rx, p).close()
    ms = []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = sc.trace(tx, o.rx, p)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        _, c = r.counts()
        r.close()
    t = float(np.median(ms))
    casts = c["segments"] + c["vis_casts"] + c["los_casts"] + c["validation_casts"]
    return {"r_p": r_p, "ms": t, "ray_segments_per_s": casts / (t / 1e3),
            "counts": {k: c[k] for k in ("segments", "vis_casts", "validation_casts", "keys",
                                         "paths")}}


def _face_plane(surf, boxes, room=(20.0, 10.0, 3.0)):
    """(axis, offset) of the office's planar face with surface label surf."""
    if surf < 6:
        return surf // 2, 0.0 if surf % 2 == 0 else room[surf // 2]
    b, f = divmod(surf - 6, 5)
    x0, x1, y0, y1, h = boxes[b]
    return [(0, x0), (0, x1), (1, y0), (1, y1), (2, h)][f]


def isect_bench(scene, o, stream, n=1_000_000):
    """Intersection-model ablation (Sec. II-C against the prior work's SDF,
    Eq. 2): the first hit of n seeded random directions from the office TX
    under each model (nrt_cast), device-timed (median of 3 after a warm-up),
    the share of rays that hit, and the distance of each hit from the true
    face plane of its surface label (the points carry 1 cm noise)."""
    import torch
    from paper_2507_04021_gb300 import inputs, nrt

    rng = inputs.rng_for(inputs.SEED_EDGES, 9)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    dd = torch.from_numpy(d.astype(np.float32)).cuda()
    oo = torch.from_numpy(np.tile(np.asarray(o.tx, np.float32), (n, 1))).cuda()
    torch.cuda.synchronize()  # the casts run on the library's stream
    boxes = o.extra["boxes"]
    out = {"rays": n}
    for name, model, sigma in (("disc", nrt.ISECT_DISC, 0.0), ("sdf", nrt.ISECT_SDF, 0.015)):
        scene.cast(oo, dd, model=model, sigma=sigma)
        ms = []
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = scene.cast(oo, dd, model=model, sigma=sigma)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = r["t"].cpu().numpy().astype(np.float64)
        lab = r["labels"].cpu().numpy().astype(np.int64) & 0xFFFF
        hit = np.isfinite(t)
        q = np.asarray(o.tx, np.float64)[None] + t[hit, None] * d[hit]
        err = np.array([abs(q[i, a] - off) for i, (a, off) in
                        enumerate(_face_plane(int(s_), boxes) for s_ in lab[hit])])
        out[name] = {"sigma": sigma if model == nrt.ISECT_SDF else None,
                     "ms": float(np.median(ms)), "casts_per_s": n / (float(np.median(ms)) / 1e3),
                     "hit_fraction": float(hit.mean()),
                     "plane_error_m": {"mean": float(err.mean()), "p50": float(np.median(err)),
                                       "p99": float(np.quantile(err, 0.99))}}
    out["sdf_over_disc_time"] = out["sdf"]["ms"] / out["disc"]["ms"]
    return out


def proposal_bench(scene, o):
    """Learned launch proposal (RX-sphere capture, 16 RX, 5 specular
    interactions): 5M labelled rays from 250 trajectory positions, training
    on the GPU, then at 6 held-out trajectory positions and the office TX the
    uniform 1M launch against 1e5 proposed rays (scoring + selection + trace)."""
    from paper_2507_04021_gb300 import inputs, nrt, proposal

    traj = inputs.trajectory(o.extra["boxes"])
    # training positions: the first 250 trajectory points, each at a seeded
    # height in [0.8, 2.2] m so that the network also sees TX heights like
    # the office TX's 2.0 m (the trajectory keeps 0.3 m from every box in x/y)
    train_tx = traj[:250].copy()
    train_tx[:, 2] = inputs.rng_for(inputs.SEED_MLP, 7).uniform(0.8, 2.2, 250).astype(np.float32)
    data = proposal.make_training_set(scene, train_tx, o.rx)
    net = nrt.Mlp(scene.ctx, inputs.mlp_init(), [0, 0, 0], [20, 10, 3], proposal.N_LAUNCH)
    loss, secs, wp = proposal.train(net, data)
    per_tx = []
    for tx in list(traj[250:256]) + [o.tx]:
        ev = proposal.evaluate(scene, net, tx, o.rx)
        ok = ev.p_uniform > 0
        within = np.abs(ev.db_err[ok]) <= 0.5
        per_tx.append({
            "tx": [round(float(x), 3) for x in tx], "rays": ev.n_proposed,
            "rx_within_0.5dB": int(within.sum()), "rx_with_paths": int(ok.sum()),
            "uniform_leaves_rx_empty": bool((~ok).any()),
            "max_abs_db": float(np.max(np.abs(ev.db_err[ok]))) if ok.any() else None,
            "power_recall": float(np.nanmean(ev.power_recall)),
            "fallback": ev.fallback, "ms_uniform": ev.ms_uniform,
            "ms_proposal": ev.ms_proposal, "ms_score": ev.ms_score})
    net.close()
    mu = sum(t["ms_uniform"] for t in per_tx)
    mp = sum(t["ms_proposal"] + (t["ms_uniform"] if t["fallback"] else 0.0) for t in per_tx)
    free = [t for t in per_tx if not t["uniform_leaves_rx_empty"]]
    mu_f = sum(t["ms_uniform"] for t in free)
    mp_f = sum(t["ms_proposal"] + (t["ms_uniform"] if t["fallback"] else 0.0) for t in free)
    return {
        "workload": ("office, RX sphere r 0.1 m, 16 RX, 5 specular interactions; training 250 "
                     "trajectory TX x 20,000 rays; evaluation 6 held-out trajectory TX + office TX, "
                     "1e5 proposed rays (90% Gumbel-top-k, 10% stratified) vs uniform 1M"),
        "training": {"rays": int(data.ray_id.shape[0]), "positive_rate": data.positive_rate,
                     "label_trace_s": data.trace_s, "steps": int(loss.size), "train_s": secs,
                     "loss_first": float(loss[:50].mean()), "loss_last": float(loss[-50:].mean())},
        "speedup": mu / mp,
        "speedup_note": "wall(uniform 1M trace) / wall(score + select + 1e5 trace), summed over the "
                        "evaluation TX; a fallback TX adds the uniform trace to its proposal time",
        "tx_all_rx_within_0.5dB": int(sum(t["rx_within_0.5dB"] == t["rx_with_paths"] for t in per_tx)),
        "fallback_forced": int(sum(t["uniform_leaves_rx_empty"] for t in per_tx)),
        "fallback_note": "the configured fallback runs the uniform launch when any RX has no path "
                         "under the proposal; a TX where the uniform 1M launch itself leaves an RX "
                         "without paths therefore always falls back (fallback_forced TX)",
        "speedup_without_forced": (mu_f / mp_f) if free else None,
        "rx_within_0.5dB": int(sum(t["rx_within_0.5dB"] for t in per_tx)),
        "rx_with_paths": int(sum(t["rx_with_paths"] for t in per_tx)),
        "mean_power_recall": float(np.mean([t["power_recall"] for t in per_tx])),
        "per_tx": per_tx,
    }


def score_only(args):
    """The proposal network's scoring of the whole 1M-direction launch, three
    times (a fixed workload for profiling the fused tensor-core kernel)."""
    import torch
    from paper_2507_04021_gb300 import inputs, nrt

    ctx = nrt.Context(0)
    net = nrt.Mlp(ctx, inputs.mlp_init(), [0, 0, 0], [20, 10, 3], N_RAYS)
    z = torch.empty(N_RAYS, dtype=torch.float32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for _ in range(3):
        ev[0].record()
        net.score(np.array([3.0, 5.0, 2.0], np.float32), None, N_RAYS, z)
        ev[1].record()
        torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    print(json.dumps({"score_ms": ms, "directions": N_RAYS,
                      "tflops": 2 * N_RAYS * (96 * 128 + 2 * 128 * 128 + 128) / (ms * 1e-3) / 1e12}))
    net.close()


def batch_only(args):
    """Only the robot-trajectory batch measurement (one GPU): one JSON line
    with the batch section (a fixed workload for profiling the batch)."""
    import torch
    from paper_2507_04021_gb300 import inputs, nrt

    stream = torch.cuda.Stream()
    ctx = nrt.Context(0, stream=stream.cuda_stream)
    o = inputs.office_scene()
    scene = nrt.Scene(ctx, o.pos, o.nrm, o.surf, o.mat, rho=0.0625, r_p=0.015, lambda_d=100.0)
    scene.set_materials(o.eps_r, o.sigma, o.scat)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    print(json.dumps({"batch": batch_bench(args, scene, o, 0, stream, flush)}), flush=True)
    scene.close()


def ours(args):
    import torch
    from paper_2507_04021_gb300 import inputs, nrt

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    ctx = nrt.Context(local, stream=stream.cuda_stream)

    o = inputs.office_scene()
    scene = nrt.Scene(ctx, o.pos, o.nrm, o.surf, o.mat, rho=0.0625, r_p=0.015, lambda_d=100.0)
    scene.set_materials(o.eps_r, o.sigma, o.scat)
    build_ms = scene.info()["build_ms"]
    # one office simulation; with N ranks, each traces its contiguous ray range
    # of the launch and the ranks' paths are merged on the device (strong
    # scaling: the total work is the same simulation at every N)
    tx = o.tx
    p = nrt.default_trace_params(max_depth=5, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=args.rays,
                                 rep_tries=0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    subset = None
    if world > 1:
        from paper_2507_04021_gb300 import shard as _shard
        lo, hi = _shard.shard_ranges(args.rays, world)[rank]
        subset = torch.arange(lo, hi, dtype=torch.int32, device=dev)
    merged_power = [None]

    def exchange(r):
        """All-gather every rank's exported paths and merge them on the device."""
        e = r.export_paths()
        n = torch.tensor([e["key_hi"].shape[0]], dtype=torch.int64, device=dev)
        sizes = [torch.zeros_like(n) for _ in range(world)]
        dist.all_gather(sizes, n)
        m = int(max(int(x) for x in sizes))
        pad = lambda t, v: torch.cat([t, t.new_full((m - t.shape[0],), v)])  # noqa: E731
        fields = {"key_hi": (e["key_hi"], -1), "key_lo": (e["key_lo"], -1),
                  "rep": (e["rep"], -1), "power": (e["power"], 0.0)}
        out = {}
        for f, (t, v) in fields.items():
            parts = [torch.empty(m, dtype=t.dtype, device=dev) for _ in range(world)]
            dist.all_gather(parts, pad(t, v))
            out[f] = torch.cat([q[:int(sizes[i])] for i, q in enumerate(parts)])
        sid = torch.cat([torch.full((int(sizes[i]),), i, dtype=torch.int32, device=dev)
                         for i in range(world)])
        _, pw = nrt.shard_merge(ctx, out["key_hi"], out["key_lo"], sid, out["rep"],
                                power=out["power"], n_rx=int(o.rx.shape[0]))
        return pw

    def step():
        with torch.cuda.stream(stream):
            flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        r = scene.trace(tx, o.rx, p, ray_subset=subset)
        if world > 1:
            with torch.cuda.stream(stream):
                merged_power[0] = exchange(r)
        ev1.record(stream)
        return r, ev0, ev1

    for _ in range(args.warmup):
        r, _, _ = step()
        r.close()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    evs, casts, trace_ms, launches, phases = [], 0, [], 0, []
    traced = 0
    last = None
    for _ in range(args.steps):
        r, e0, e1 = step()
        _, c = r.counts()
        casts += c["segments"] + c["vis_casts"] + c["los_casts"] + c["validation_casts"]
        traced += c["segments"]
        t = r.times()
        trace_ms.append(t["trace"])
        phases.append(t)
        launches += c["kernel_launches"] + 1  # + the L2 flush fill
        evs.append((e0, e1))
        if last is not None:
            last.close()
        last = r
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = float(sum(a.elapsed_time(b) for a, b in evs))
    counts = last.counts()[1]
    if dist:
        t = torch.tensor([total_ms, float(casts), float(traced)], device=dev, dtype=torch.float64)
        tm = t.clone()
        dist.all_reduce(tm[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:], op=dist.ReduceOp.SUM)
        total_ms, casts, traced = float(tm[0]), float(t[1]), float(t[2])
    value = casts / (total_ms / 1000.0)

    # end to end through the C ABI with host buffers: TX/RX from host memory in,
    # the step's result (per-RX received power and path counts) back to host
    e2e_ms, e2e_casts = [], 0
    hb = db = 0
    for _ in range(0 if args.no_e2e else max(1, min(args.steps, 5))):
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        r = scene.trace(np.asarray(tx, np.float32), o.rx, p, ray_subset=subset)
        per_rx, c = r.counts()
        if world > 1:  # the merged per-RX power of all ranks' paths
            with torch.cuda.stream(stream):
                pw = exchange(r).cpu().numpy()
        else:
            pw = r.power()
        e2e_ms.append((time.perf_counter() - t0) * 1000.0)
        e2e_casts += c["segments"] + c["vis_casts"] + c["los_casts"] + c["validation_casts"]
        hb = 12 + o.rx.nbytes
        db = pw.nbytes + per_rx.nbytes
        r.close()
    if dist and e2e_ms:
        t = torch.tensor([sum(e2e_ms), float(e2e_casts)], device=dev, dtype=torch.float64)
        tm = t.clone()
        dist.all_reduce(tm[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:], op=dist.ReduceOp.SUM)
        e2e_ms, e2e_casts = [float(tm[0]) / len(e2e_ms)] * len(e2e_ms), float(t[1])
    e2e = None if args.no_e2e else {"value": e2e_casts / (sum(e2e_ms) / 1000.0), "unit": "ray-segments/s",
           "h2d_bytes_per_step": int(hb), "d2h_bytes_per_step": int(db),
           "ms_per_step": float(np.mean(e2e_ms)),
           "result": "per-RX received power and path counts"}

    ab = _alg_bytes()
    peak, peak_kind = _peaks()
    l2_peak = ctx.measure_l2(48 << 20, 50)  # this GPU's L2 read bandwidth, GB/s
    ph = {k: float(np.mean([x[k] for x in phases])) for k in phases[0]}

    def roof_entry(name, units, per_unit, ms, unit_name, traffic_key):
        achieved = units * per_unit / (ms / 1000.0) / 1e9
        l2_unit = _l2_bytes(traffic_key)
        l2_ach = None if l2_unit is None else units * l2_unit / (ms / 1000.0) / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": _traffic(traffic_key), "kernel": name,
                "peak_kind": peak_kind, "algorithmic_bytes_per_unit": per_unit,
                "units_per_launch": units, "unit_kind": unit_name, "kernel_ms": ms,
                "l2_peak": l2_peak, "l2_peak_kind": "measured (nrt_measure_l2, 48 MB x 50 reads)",
                "l2_achieved": l2_ach, "l2_frac": None if l2_ach is None else l2_ach / l2_peak,
                "l2_bytes_per_unit": l2_unit}

    # the dominant work: the validation phase (specular refinement + diffuse
    # shadow casts); diffuse shadow casts are oracle-counted, specular
    # validation legs use the trace-segment figure
    n_diff = counts["diffuse_casts"]
    n_spec = counts["validation_casts"] - n_diff
    per_val = ((n_diff * ab["bytes_per_shadow_cast"] + n_spec * ab["bytes_per_segment"])
               / max(counts["validation_casts"], 1))
    roof = roof_entry("validation phase: validate_specular_items_kernel + spec_finish_kernel + "
                      "validate_diffuse_kernel (one launch each)", counts["validation_casts"], per_val,
                      ph["validate"], "validation cast", "validation")
    tr_ms = float(np.mean(trace_ms))
    roof_more = [
        roof_entry("trace_kernel", counts["segments"], ab["bytes_per_segment"], tr_ms,
                   "trace segment", "trace_kernel"),
        roof_entry("vis_kernel", counts["vis_casts"], ab["bytes_per_vis_cast"], ph["vis"],
                   "visibility cast", "vis_kernel"),
    ]

    line = {
        "metric": METRIC, "value": value, "unit": "ray-segments/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "points": int(o.n_points), "rays": args.rays, "max_depth": 5,
                   "parallelism": f"ray-range shards x{world}, device merge" if world > 1 else "1 GPU",
                   "rep_tries": "all candidates (the paper's rule)",
                   "n_rx": int(o.rx.shape[0]), "l2_flush": "256 MB fill between steps",
                   "r_p": 0.015, "rho": 0.0625},
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks, "roofline": roof,
        "roofline_other": roof_more,
        "phases_ms": ph, "scene_build_ms": build_ms,
        "counts": {k: counts[k] for k in ("segments", "vis_casts", "validation_casts",
                                          "diffuse_casts", "candidates", "keys", "paths",
                                          "n_dps")},
        # `value` counts every cast (trace, visibility, LOS, validation), so
        # removing casts that cannot succeed lowers it; these count the
        # simulations and the traced segments of the launched rays alone
        "throughput": {"simulations_per_s": 1000.0 / (total_ms / args.steps),
                       "traced_segments_per_s": traced / (total_ms / 1000.0)},
    }
    # channel frequency response of the last simulation (129 frequencies over
    # 1.5 GHz, all receivers) and its Eq. 5 gradient, device-timed
    import torch as _t
    if args.no_extras:
        if rank == 0:
            print(json.dumps(line), flush=True)
        last.close()
        if dist:
            dist.destroy_process_group()
        return
    cf_ev = [_t.cuda.Event(enable_timing=True) for _ in range(3)]
    cf_ev[0].record(stream)
    H = last.cfr(1.5e9, 129)
    cf_ev[1].record(stream)
    last.cfr_backward(H * 0.9, None, 1.5e9)
    cf_ev[2].record(stream)
    _t.cuda.synchronize()
    line["cfr"] = {"n_freq": 129, "bandwidth_hz": 1.5e9, "paths": counts["paths"],
                   "ms": cf_ev[0].elapsed_time(cf_ev[1]),
                   "backward_ms": cf_ev[1].elapsed_time(cf_ev[2]),
                   "note": "FP64 sums; includes the host copy of H (and of the target)"}
    if rank == 0 and not args.no_extras:
        line["launch_comparison"] = launch_bench(scene, o, tx, stream)
        line["diffraction"] = diffraction_bench(ctx, o, tx, stream, args.rays)
        line["intersection_ablation"] = isect_bench(scene, o, stream)
        line["r_p_variant"] = rp_variant_bench(ctx, o, tx, stream, args.rays)
    if args.proposal and rank == 0:
        line["proposal"] = proposal_bench(scene, o)
    if args.batch_pairs > 0:
        line["batch"] = batch_bench(args, scene, o, rank, stream, flush)
        launches += line["batch"]["gpu_launches"]
        line["gpu_launches"] = int(launches)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        info = run_oracle_sample(_env_int("NRT_CPU_SAMPLE", 150000))
        one = run_oracle_sample(_env_int("NRT_CPU_SAMPLE_1T", 8000), threads=1)
        line["cpu_baseline"] = {
            "value": info["casts"] / info["seconds"], "unit": "ray-segments/s",
            "cores": info["cores"], "kind": "oracle",
            "sample": f"{info['rays']} rays of the 1M launch, full pipeline, "
                      f"{info['casts']} casts in {info['seconds']:.1f} s",
            "single_thread": {"value": one["casts"] / one["seconds"], "unit": "ray-segments/s",
                              "cores": 1,
                              "sample": f"{one['rays']} rays of the 1M launch, full pipeline, "
                                        f"{one['casts']} casts in {one['seconds']:.1f} s"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    last.close()
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--rays", type=int, default=N_RAYS)
    ap.add_argument("--batch-pairs", type=int, default=256,
                    help="robot-trajectory batch size (0 skips the batch measurement)")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--no-proposal", dest="proposal", action="store_false",
                    help="skip the learned-proposal measurement")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the timed simulation steps (for profiling): no CFR, launch, "
                         "diffraction, intersection or r_p measurements")
    ap.add_argument("--score-only", action="store_true",
                    help="only the proposal network's scoring of the 1M-direction launch")
    ap.add_argument("--batch-only", action="store_true",
                    help="only the robot-trajectory batch measurement (for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    elif args.score_only:
        score_only(args)
    elif args.batch_only:
        batch_only(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
