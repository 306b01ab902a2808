"""Batched TX-RX pairs (robot trajectory, one fixed RX, uneven ray budgets):
one persistent trace launch, CUDA-graph replays and the autotuner, against
single-pair simulations of the same rays and against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2507_04021_gb300 import inputs, nrt

from parity import compare_paths

pytestmark = pytest.mark.gpu

RXF = np.array([17.5, 8.0, 1.2], np.float32)
KEY_RX_MASK = np.uint64(0x00FFFFFFFFFFFFFF)


@pytest.fixture(scope="module")
def setup(office):
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, office.pos, office.nrm, office.surf, office.mat, r_p=0.015)
    sc.set_materials(office.eps_r, office.sigma, office.scat)
    traj = inputs.trajectory(office.extra["boxes"])
    return ctx, sc, traj


def _params(**kw):
    d = dict(max_depth=5, capture=nrt.CAPTURE_VIS, diffuse=1, rep_tries=8)
    d.update(kw)
    return nrt.default_trace_params(**d)


def _by_key(P, mask_rx):
    hi = P["key_hi"] & KEY_RX_MASK if mask_rx else P["key_hi"]
    return {(int(h), int(l)): i for i, (h, l) in enumerate(zip(hi, P["key_lo"]))}


@pytest.mark.parametrize("pol", [nrt.POL_TE, nrt.POL_VECTOR])
def test_batch_equals_single_pair_runs(setup, pol):
    ctx, sc, traj = setup
    budgets = np.array([3000, 12000, 700, 5000], np.int64)
    tx = traj[[0, 40, 80, 120]]
    p = _params(n_rays=1, pol=pol)
    b = sc.trace_batch(tx, RXF, budgets, p, packet=64, schedule=1)
    B = b.paths()
    Pb = b.power()
    for j in range(len(budgets)):
        r = sc.trace(tx[j], RXF[None], _params(n_rays=int(budgets[j]), pol=pol))
        S = r.paths()
        mine = B["rx"] == j
        sub = {k: v[mine] for k, v in B.items()}
        kb, ks = _by_key(sub, True), _by_key(S, True)
        assert kb.keys() == ks.keys()
        for key, i in ks.items():
            i2 = kb[key]
            assert sub["rep"][i2] == S["rep"][i]
            assert np.array_equal(sub["a"][i2], S["a"][i])
            assert sub["tau"][i2] == S["tau"][i]
        assert Pb[j] == pytest.approx(float(r.power()[0]), rel=1e-12)


def test_batch_pair_against_oracle(setup, office):
    ctx, sc, traj = setup
    budgets = np.array([4000, 2500], np.int64)
    tx = traj[[10, 200]]
    b = sc.trace_batch(tx, RXF, budgets, _params(n_rays=1))
    B = b.paths()
    osc = oracle.OracleScene(office.pos, office.nrm, office.surf, office.mat, r_p=0.015,
                             grid_cell=0.1)
    for j in range(2):
        kp = dict(max_depth=5, capture=1, diffuse=1, rep_tries=8, n_rays=int(budgets[j]))
        osim = oracle.OracleSim(osc, tx[j], RXF[None], oracle.SimParams(delta=1e-5 * office.diag, **kp))
        mine = B["rx"] == j
        sub = {k: v[mine] for k, v in B.items()}
        sub["key_hi"] = sub["key_hi"] & KEY_RX_MASK  # the oracle's RX field is 0
        s = compare_paths(sub, osim, office.eps_r, office.sigma, office.scat, strict=("los", "specular"))
        assert s["matched"] > 0.8 * s["keys"], s


def test_schedules_and_graph_replay_agree(setup):
    ctx, sc, traj = setup
    rng = np.random.default_rng(5)
    budgets = rng.integers(2000, 20000, 16).astype(np.int64)
    tx0 = traj[:16]
    tx1 = traj[100:116]
    p = _params(n_rays=1)
    ref0 = sc.trace_batch(tx0, RXF, budgets, p, schedule=0).paths()
    for packet in (32, 128):
        alt = sc.trace_batch(tx0, RXF, budgets, p, packet=packet, schedule=1).paths()
        for k in ("key_hi", "key_lo", "rep", "a", "tau"):
            assert np.array_equal(ref0[k], alt[k]), k
    g = sc.trace_batch(tx0, RXF, budgets, p, use_graph=True)
    G0 = g.paths()
    for k in ("key_hi", "key_lo", "rep", "a", "tau"):
        assert np.array_equal(ref0[k], G0[k]), k
    g.replay(tx1)
    G1 = g.paths()
    ref1 = sc.trace_batch(tx1, RXF, budgets, p).paths()
    for k in ("key_hi", "key_lo", "rep", "a", "tau"):
        assert np.array_equal(ref1[k], G1[k]), k
    pm, tot = g.batch_times()
    assert np.all(pm > 0) and tot > 0 and np.all(pm <= tot * 1.0 + 1e-6)


@pytest.mark.parametrize("schedule", [0, 1])
def test_pair_latency_stamps_under_graph_replay(setup, schedule):
    """Per-pair latency from device timestamps, for both trace schedules and
    under graph replay: every pair has a trace-done and a paths-validated
    time, inside the simulation's device time; validation starts once every
    pair is traced, so each pair's path set is known after the last trace."""
    ctx, sc, traj = setup
    rng = np.random.default_rng(11)
    budgets = rng.integers(2000, 20000, 12).astype(np.int64)
    g = sc.trace_batch(traj[:12], RXF, budgets, _params(n_rays=1), schedule=schedule,
                       use_graph=True)
    for tx in (None, traj[40:52]):
        if tx is not None:
            g.replay(tx)
        pm, tot, pv = g.batch_times(paths=True)
        slack = 5e-3  # ms: globaltimer against event clocks
        assert np.all(pm > 0) and np.all(pm <= tot + slack), (pm, tot)
        assert np.all(pv > 0) and np.all(pv <= tot + slack), (pv, tot)
        assert np.all(pv >= pm.max() - slack), (pv, pm)


def test_autotune_picks_a_configuration(setup):
    ctx, sc, traj = setup
    budgets = np.full(8, 20000, np.int64)
    b = sc.trace_batch(traj[:8], RXF, budgets, _params(n_rays=1))
    cfgs = [(32, 1), (64, 1), (128, 1), (64, 0)]
    ms, best = b.autotune(cfgs, repeats=2)
    assert np.all(ms > 0) and 0 <= best < len(cfgs)
    assert ms[best] == ms.min()


def test_graph_replay_over_capacity_reports_overflow(setup):
    """A recorded graph keeps the buffer capacities of its first run.  Recorded
    with the TX pairs far above the office (almost every ray escapes, so the
    capacities stay near their floors), a replay inside the office finds far
    more candidates and keys than that: every write stays bounded, the replay
    reports an overflow, and the context keeps working."""
    ctx, sc, traj = setup
    budgets = np.full(4, 4000, np.int64)
    far = np.tile(np.array([10.0, 5.0, 200.0], np.float32), (4, 1))
    g = sc.trace_batch(far, RXF, budgets, _params(n_rays=1), use_graph=True)
    assert g.counts()[1]["keys"] < 1024
    with pytest.raises(nrt.NrtError) as ei:
        g.replay(traj[[0, 40, 80, 120]])
    # reported as an overflow of the recorded buffers, not as a CUDA error:
    # every candidate position below the count is written even when the hash
    # table is full, so nothing reads an unwritten slot
    assert ei.value.status == 4, str(ei.value)
    assert "device buffer overflow (flags" in str(ei.value), str(ei.value)
    g.close()
    r = sc.trace(traj[0], RXF[None], _params(n_rays=4000))
    assert r.counts()[1]["paths"] >= 1
    r.close()
