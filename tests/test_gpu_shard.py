"""Ray-range shards on the GPU (run one after the other on one device) merged
by the host-side rule equal one simulation of the whole launch, bit for bit:
same keys, representatives, coefficients and delays (office scene, 4
receivers, visibility capture with diffuse paths, 3 interactions)."""
import numpy as np
import pytest

from paper_2507_04021_gb300 import nrt, shard

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rep_tries", [2, 0])
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


def _np_u64(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("rep_tries", [0, 2])
def test_device_merge_equals_single_run(office, rep_tries):
    """The device-side merge (nrt_shard_merge, the multi-GPU path's exchange
    step after an all-gather) of three ray-range shards equals one
    simulation of the whole launch: the same (key, representative) set and
    the same per-RX power.  Without a cap the shards' exported paths are
    merged directly; with a cap, their per-key summaries (tries carried
    from shard to shard)."""
    import torch

    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, office.pos, office.nrm, office.surf, office.mat, r_p=0.015)
    sc.set_materials(office.eps_r, office.sigma, office.scat)
    n_rays, rx = 200_000, office.rx[:6]
    p = nrt.default_trace_params(max_depth=3, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=n_rays,
                                 rep_tries=rep_tries, keep_keys=1)
    parts, sums = [], []
    for s, (lo, hi) in enumerate(shard.shard_ranges(n_rays, 3)):
        r = sc.trace(office.tx, rx, p, ray_subset=np.arange(lo, hi, dtype=np.uint32))
        e = r.export_paths()
        e["shard"] = torch.full_like(e["rep"], s)
        parts.append(e)
        k = r.keys()
        sums.append({"key_hi": k["key_hi"], "key_lo": k["key_lo"], "tried": k["tried"],
                     "rep": k["rep"], "shard": np.full(len(k["rep"]), s, np.uint32)})
        r.close()
    one = sc.trace(office.tx, rx, p)
    P1 = one.paths()
    want = set(zip(P1["key_hi"].tolist(), P1["key_lo"].tolist()))
    cat = {f: torch.cat([e[f] for e in parts]) for f in parts[0]}
    win, pw = nrt.shard_merge(ctx, cat["key_hi"], cat["key_lo"], cat["shard"], cat["rep"],
                              power=cat["power"], n_rx=rx.shape[0])
    torch.cuda.synchronize()
    w = win.cpu().numpy().astype(bool)
    got_keys = set(zip(_np_u64(cat["key_hi"])[w].tolist(), _np_u64(cat["key_lo"])[w].tolist()))
    if rep_tries == 0:  # every exported path is valid: the merge keeps the lowest shard's
        assert got_keys == want
        got_rep = dict(zip(zip(_np_u64(cat["key_hi"])[w].tolist(),
                               _np_u64(cat["key_lo"])[w].tolist()),
                           cat["rep"].cpu().numpy().view(np.uint32)[w].tolist()))
        rep1 = np.where(P1["k"] == 0, 0, P1["rep"])
        for h, l, r_, t in zip(P1["key_hi"].tolist(), P1["key_lo"].tolist(), rep1.tolist(),
                               P1["type"].tolist()):
            if t != 2:
                assert got_rep[(h, l)] == r_
        e1 = one.export_paths()
        j1 = (_np_u64(e1["key_hi"]) >> np.uint64(56)).astype(np.int64)
        p1 = np.bincount(j1, e1["power"].cpu().numpy(), minlength=rx.shape[0])
        assert np.allclose(pw.cpu().numpy(), p1, rtol=1e-12, atol=0)
    # per-key summaries with the try budget (any cap), against the host rule
    S = {f: np.concatenate([s_[f] for s_ in sums]) for f in sums[0]}
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()  # noqa: E731
    win2, _ = nrt.shard_merge(ctx, dev(S["key_hi"], np.int64), dev(S["key_lo"], np.int64),
                              dev(S["shard"], np.int32), dev(S["rep"], np.int32),
                              tried=dev(S["tried"], np.int32), rep_tries=rep_tries)
    torch.cuda.synchronize()
    w2 = win2.cpu().numpy().astype(bool)
    got2 = dict(zip(zip(S["key_hi"][w2].tolist(), S["key_lo"][w2].tolist()),
                    S["rep"][w2].tolist()))
    host_in = [{(int(h), int(l)): (int(t), int(r_), {} if r_ != shard.NO_REP else None)
                for h, l, t, r_ in zip(s_["key_hi"], s_["key_lo"], s_["tried"], s_["rep"])}
               for s_ in sums]
    host = {k: r_ for k, (r_, _) in shard.merge(host_in, rep_tries).items()}
    assert got2 == host
    # and the single run's per-key representatives are the merged ones
    K1 = one.keys()
    v1 = K1["rep"] != shard.NO_REP
    assert dict(zip(zip(K1["key_hi"][v1].tolist(), K1["key_lo"][v1].tolist()),
                    K1["rep"][v1].tolist())) == got2
