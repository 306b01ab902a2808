"""Ray-range sharding with the host-side merge (paper_2507_04021_gb300.shard),
on CPU: two gloo ranks each run the FP64 oracle on half of the launch, all-
gather their per-key summaries and merge; the merged paths, representatives
and per-RX power equal one oracle run over the whole launch.  A small
rep_tries makes keys carry their try budget from one shard to the next."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2507_04021_gb300 import inputs, shard

RX = np.array([[4.0, 3.0, 1.2], [1.5, 3.2, 1.0], [2.5, 2.0, 0.5]], np.float32)
MATS = (np.array([5.3, 3.0]), np.array([0.03, 0.01]), np.array([0.0, 0.0]))


def _params(n_rays, rep_tries):
    return oracle.SimParams(max_depth=2, capture=0, diffuse=0, n_rays=n_rays, rep_tries=rep_tries,
                            r_rx=0.3, n_threads=2)


def _scene():
    room = inputs.room_scene()
    osc = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05,
                             grid_cell=0.25)
    return room, osc


def _summary(sim):
    K = sim.keys()
    P = sim.paths()
    a, _ = sim.field(*MATS)
    keys = {"key_hi": K["hi"], "key_lo": K["lo"], "tried": K["n_tried"],
            "rep": np.where(K["valid"] != 0, K["rep"], shard.NO_REP)}
    paths = {"key_hi": P["hi"], "key_lo": P["lo"], "rep": P["rep"], "rx": P["j"],
             "a": np.stack([a.real, a.imag], 1), "tau": P["tau"]}
    return shard.summary(keys, paths)


def _rank(rank, world, port, n_rays, rep_tries, out_q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    room, osc = _scene()
    lo, hi = shard.shard_ranges(n_rays, world)[rank]
    sim = oracle.OracleSim(osc, room.tx, RX, _params(n_rays, rep_tries),
                           ray_ids=np.arange(lo, hi, dtype=np.int64))
    merged = shard.merge_distributed(_summary(sim), rep_tries)
    if rank == 0:
        out_q.put({k: (int(r), [float(x) for x in p["a"]], float(p["tau"]), int(p["rx"]))
                   for k, (r, p) in merged.items()})
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("rep_tries", [2, 0])
def test_two_rank_merge_equals_single_run(rep_tries):
    n_rays = 30000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, n_rays, rep_tries, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    room, osc = _scene()
    single = oracle.OracleSim(osc, room.tx, RX, _params(n_rays, rep_tries))
    s = _summary(single)
    want = {k: (r, [float(x) for x in p["a"]], float(p["tau"]), int(p["rx"]))
            for k, (t, r, p) in s.items() if p is not None}
    assert len(want) > 10
    assert merged == want
    pw = np.zeros(RX.shape[0])
    for r, a, tau, j in merged.values():
        pw[j] += a[0] ** 2 + a[1] ** 2
    _, P_single = single.field(*MATS)
    assert np.allclose(pw, P_single, rtol=1e-12)


def test_merge_budget_rules():
    """Hand-made summaries: the try budget carries across shards in order."""
    path = {"a": np.array([1.0, 0.0]), "rx": 0}
    A = {(1, 0): (3, shard.NO_REP, None), (2, 0): (2, 7, path), (3, 0): (8, shard.NO_REP, None)}
    B = {(1, 0): (2, 105, path), (2, 0): (1, 101, path), (3, 0): (1, 130, path),
         (4, 0): (5, 140, path)}
    m = shard.merge([A, B], rep_tries=5)
    assert m[(1, 0)][0] == 105        # 3 + 2 <= 5 tries
    assert m[(2, 0)][0] == 7          # the lower shard's valid candidate wins
    assert (3, 0) not in m            # budget spent in shard A
    assert m[(4, 0)][0] == 140        # exactly the budget
    m4 = shard.merge([A, B], rep_tries=4)
    assert (1, 0) not in m4           # 3 + 2 > 4
