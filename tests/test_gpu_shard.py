"""Ray-range shards on the GPU (run one after the other on one device) merged
by the host-side rule equal one simulation of the whole launch, bit for bit:
same keys, representatives, coefficients and delays (office scene, 4
receivers, visibility capture with diffuse paths, 3 interactions)."""
import numpy as np
import pytest

from paper_2507_04021_gb300 import nrt, shard

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rep_tries", [2, 8])
def test_shards_merge_to_single_run(office, rep_tries):
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, office.pos, office.nrm, office.surf, office.mat, r_p=0.015)
    sc.set_materials(office.eps_r, office.sigma, office.scat)
    n_rays = 200_000
    rx = office.rx[:4]
    p = nrt.default_trace_params(max_depth=3, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=n_rays,
                                 rep_tries=rep_tries, keep_keys=1)
    sums = []
    for lo, hi in shard.shard_ranges(n_rays, 3):
        r = sc.trace(office.tx, rx, p, ray_subset=np.arange(lo, hi, dtype=np.uint32))
        sums.append(shard.summary(r.keys(), r.paths()))
        r.close()
    merged = shard.merge(sums, rep_tries)
    one = sc.trace(office.tx, rx, p)
    s = shard.summary(one.keys(), one.paths())
    want = {k: v for k, v in s.items() if v[2] is not None}
    print("keys", len(s), "paths", len(want), "merged", len(merged))
    assert merged.keys() == want.keys()
    for k, (rep, path) in merged.items():
        _, wrep, wpath = want[k]
        assert rep == wrep
        assert np.array_equal(path["a"], wpath["a"]) and path["tau"] == wpath["tau"]
    assert np.allclose(shard.merged_power(merged, rx.shape[0]),
                       one.power().astype(np.float64), rtol=1e-5)
