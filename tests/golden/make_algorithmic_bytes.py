"""Write office_algorithmic_bytes.json: the algorithmic disc reads per cast of
the office workload (2M points, 16 RX, 1M-ray Fibonacci launch, 5
interactions), counted by the FP64 oracle on a ray sample.

A cast's algorithmic bytes are 32 B of ray state + 24 B (position + normal)
per disc of every DPS whose r_p-inflated box the cast enters before its hit
+ 32 B of hit record: trace segments, visibility casts (RX -> reception point)
and diffuse validation shadow casts (scatter point -> RX).  Only oracle/ and the seeded inputs are used.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2507_04021_gb300 import inputs  # noqa: E402


def main():
    o = inputs.office_scene()
    sc = oracle.OracleScene(o.pos, o.nrm, o.surf, o.mat, r_p=0.015, grid_cell=0.1)
    ids = np.arange(0, 1_000_000, 1000, dtype=np.int64)
    p = oracle.SimParams(max_depth=5, capture=1, diffuse=1, n_rays=1_000_000, validate=0)
    sim = oracle.OracleSim(sc, o.tx, o.rx, p, ray_ids=ids)
    dc = sim.disc_counts()
    seg = dc[dc >= 0]
    rng = np.random.default_rng(11)
    nd = sc.n_dps
    j = rng.integers(0, o.rx.shape[0], 2000).astype(np.int32)
    d = rng.integers(0, nd, 2000).astype(np.int32)
    vc = sc.vis_disc_counts(o.rx, j, d)
    # diffuse validation shadow casts (scatter point -> RX) of a validated run
    pv = oracle.SimParams(max_depth=5, capture=1, diffuse=1, n_rays=1_000_000, rep_tries=8)
    simv = oracle.OracleSim(sc, o.tx, o.rx, pv, ray_ids=np.arange(0, 1_000_000, 2000, dtype=np.int64))
    dsum, dn = simv.shadow_disc_counts(stride=4)
    out = {
        "_source": "tests/golden/make_algorithmic_bytes.py (FP64 oracle, office scene, seed 2)",
        "rays_sampled": int(ids.size),
        "segments_sampled": int(seg.size),
        "discs_per_segment": float(seg.mean()),
        "bytes_per_segment": float(32 + 24 * seg.mean() + 32),
        "vis_casts_sampled": int(vc.size),
        "discs_per_vis_cast": float(vc.mean()),
        "bytes_per_vis_cast": float(32 + 24 * vc.mean() + 4.0 / 32.0),
        "shadow_casts_sampled": dn,
        "discs_per_shadow_cast": dsum / dn,
        "bytes_per_shadow_cast": float(32 + 24 * dsum / dn + 32),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "office_algorithmic_bytes.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
