"""The learned launch proposal on a GPU, through the C ABI: the tcgen05
tensor-core contraction against FP64 products of the same BF16 values,
features, logits and one training step's gradients against the oracle's
BF16-emulated network, the Gumbel-top-k selection against the oracle's
selection (exact), and the tracer's per-ray labels against the oracle's."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp as M
from paper_2507_04021_gb300 import inputs, nrt

pytestmark = pytest.mark.gpu

BOX_MIN = np.array([0.0, 0.0, 0.0], np.float32)
BOX_MAX = np.array([20.0, 10.0, 3.0], np.float32)
N_RAYS = 1_000_000


@pytest.fixture(scope="module")
def ctx():
    return nrt.Context(0)


def _bf16_bits(x: np.ndarray) -> torch.Tensor:
    """float64 values already representable in BF16 -> CUDA bfloat16 tensor."""
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("M_,N_,K_,split", [(128, 128, 128, 0), (300, 96, 96, 0),
                                            (257, 128, 200, 0), (128, 96, 4096, 1024),
                                            (1000, 16, 8, 0)])
def test_gemm_matches_fp64(ctx, M_, N_, K_, split):
    rng = np.random.default_rng(M_ + N_ + K_)
    A = M.bf16(rng.standard_normal((M_, K_)))
    B = M.bf16(rng.standard_normal((N_, K_)))
    want = A @ B.T
    C = torch.zeros((M_, N_), dtype=torch.float32, device="cuda")
    nrt.gemm_bf16(ctx, _bf16_bits(A), _bf16_bits(B), C, accumulate=False, k_split=split)
    got = C.cpu().numpy().astype(np.float64)
    bound = 1e-5 * (np.abs(A) @ np.abs(B).T) + 1e-30
    assert np.all(np.abs(got - want) <= bound), float(np.max(np.abs(got - want) / bound))
    # accumulate into an existing C
    nrt.gemm_bf16(ctx, _bf16_bits(A), _bf16_bits(B), C, accumulate=True)
    got2 = C.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got2 - 2 * want) <= 2 * bound)


def _net(ctx, theta=None):
    theta = inputs.mlp_init() if theta is None else theta
    return nrt.Mlp(ctx, theta, BOX_MIN, BOX_MAX, N_RAYS), theta


def _oracle_features(ids, tx):
    d = oracle.fib_dirs(N_RAYS, ids.astype(np.int64)).astype(np.float32)
    u = M.normalise_tx(tx, 0.5 * (BOX_MIN + BOX_MAX), 0.5 * (BOX_MAX - BOX_MIN))
    return M.features(d, u)


def test_features_match_oracle(ctx):
    net, _ = _net(ctx)
    ids = np.arange(0, N_RAYS, 97, dtype=np.uint32)
    tx = np.array([3.0, 5.0, 2.0], np.float32)
    out = torch.zeros((ids.size, 96), dtype=torch.bfloat16, device="cuda")
    net.features(tx, torch.from_numpy(ids).cuda(), ids.size, out)
    got = out.float().cpu().numpy().astype(np.float64)
    want = _oracle_features(ids, tx)
    diff = got != want
    # a value near a BF16 rounding boundary may round the other way (FP32 vs
    # FP64 sin/cos and direction); one BF16 step at most
    step = np.abs(want) * 2.0 ** -7 + 1e-38
    assert np.all(np.abs(got - want) <= step + 1e-6)
    assert diff.mean() < 2e-3, diff.mean()


@pytest.mark.parametrize("n_ids", [1, 100, 7634, 142857])
def test_logits_match_oracle_forward(ctx, n_ids):
    """The fused scoring kernel (four 128-row tiles in flight per SM) against
    the oracle's forward pass: one row, one partial tile, fewer tiles than
    the grid's groups, and more tiles than groups with a ragged last tile."""
    net, theta = _net(ctx)
    ids = np.linspace(3, N_RAYS - 1, n_ids).astype(np.uint32)
    tx = np.array([12.5, 4.0, 1.0], np.float32)
    z = torch.zeros(ids.size, dtype=torch.float32, device="cuda")
    net.score(tx, torch.from_numpy(ids).cuda(), ids.size, z)
    got = z.cpu().numpy().astype(np.float64)
    want = M.forward(M.unpack(theta), _oracle_features(ids, tx))["z"]
    err = np.abs(got - want)
    print("logit max abs err", err.max(), "scale", np.abs(want).max())
    assert np.all(err <= 1e-2 * (1.0 + np.abs(want)))


def _train_inputs(n, seed_tx=(0, 40, 80, 120, 160, 200, 240)):
    office_boxes = inputs.office_scene(n_points=20000).extra["boxes"]
    traj = inputs.trajectory(office_boxes)
    tx_table = traj[list(seed_tx)].astype(np.float32)
    ti, rid, lab = inputs.mlp_samples(n, tx_table.shape[0], N_RAYS)
    return tx_table, ti, rid, lab


def test_train_step_gradients_match_oracle(ctx):
    net, theta = _net(ctx)
    B = 2048
    tx_table, ti, rid, lab = _train_inputs(B)
    wp = 5.0
    loss = net.train(torch.from_numpy(tx_table).cuda(), torch.from_numpy(ti).cuda(),
                     torch.from_numpy(rid).cuda(), torch.from_numpy(lab).cuda(),
                     steps=1, lr=0.0, batch=B, pos_weight=wp)
    g = net.grads()
    # oracle: same samples, features from the oracle's own directions
    u = M.normalise_tx(tx_table[ti], 0.5 * (BOX_MIN + BOX_MAX), 0.5 * (BOX_MAX - BOX_MIN))
    d = oracle.fib_dirs(N_RAYS, rid.astype(np.int64)).astype(np.float32)
    X = M.features(d, u)
    lo, G = M.grads(M.unpack(theta), X, lab.astype(np.float64), wp)
    assert loss[0] == pytest.approx(lo, rel=1e-3)
    Gp = M.unpack(M.pack(G).astype(np.float64))
    Gg = M.unpack(g.astype(np.float64))
    for k in Gp:
        rel = np.linalg.norm(Gg[k] - Gp[k]) / max(np.linalg.norm(Gp[k]), 1e-30)
        print(k, "relative gradient error", rel)
        assert rel < 3e-3, k
    assert np.array_equal(net.params(), theta)  # lr = 0 leaves the parameters


def test_first_adam_step_moves_each_parameter_by_lr(ctx):
    """First Adam step from zero moments: theta -= lr g / (|g| + eps)."""
    net, theta = _net(ctx)
    B = 1024
    tx_table, ti, rid, lab = _train_inputs(B)
    lr = 1e-3
    net.train(torch.from_numpy(tx_table).cuda(), torch.from_numpy(ti).cuda(),
              torch.from_numpy(rid).cuda(), torch.from_numpy(lab).cuda(),
              steps=1, lr=lr, batch=B, pos_weight=2.0)
    g = net.grads().astype(np.float64)
    step = net.params().astype(np.float64) - theta.astype(np.float64)
    big = np.abs(g) > 1e-5
    want = -lr * g / (np.abs(g) + 1e-8)
    assert np.allclose(step[big], want[big], rtol=1e-3, atol=1e-9)


def test_training_learns_a_direction_rule(ctx):
    """Labels from a rule on the launch direction (z > 0.4): a few hundred
    steps on the GPU separate the classes."""
    net, _ = _net(ctx)
    n = 65536
    tx_table, ti, rid, _ = _train_inputs(n)
    d = oracle.fib_dirs(N_RAYS, rid.astype(np.int64))
    lab = (d[:, 2] > 0.4).astype(np.float32)
    dev = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    loss = net.train(dev(tx_table), dev(ti), dev(rid), dev(lab), steps=300, lr=2e-3, batch=4096)
    print("loss", loss[0], "->", loss[-1])
    assert loss[-1] < 0.25 * loss[0]
    ids = np.arange(0, N_RAYS, 50, dtype=np.uint32)
    z = torch.zeros(ids.size, dtype=torch.float32, device="cuda")
    net.score(tx_table[0], dev(ids), ids.size, z)
    zt = oracle.fib_dirs(N_RAYS, ids.astype(np.int64))[:, 2] > 0.4
    acc = np.mean((z.cpu().numpy() > 0) == zt)
    print("accuracy", acc)
    assert acc > 0.97


@pytest.mark.parametrize("n,k_top,k_u,seed", [(1_000_000, 90_000, 10_000, 5), (100_003, 9_000, 1_000, 7),
                                              (1000, 1000, 0, 1), (5000, 0, 37, 2)])
def test_propose_matches_oracle(ctx, n, k_top, k_u, seed):
    z = inputs.mlp_logits(n)
    ids = torch.zeros(k_top + k_u, dtype=torch.int32, device="cuda")
    m = nrt.propose(ctx, torch.from_numpy(z).cuda(), k_top, k_u, seed, ids)
    got = ids[:m].cpu().numpy().astype(np.int64)
    want = M.select(z, k_top, k_u, seed)
    assert np.array_equal(got, want)


def test_ray_labels_match_oracle(ctx, room):
    RX = np.array([[4.0, 3.0, 1.2], [1.5, 3.2, 1.0]], np.float32)
    n_rays = 60000
    sc = nrt.Scene(ctx, room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    p = nrt.default_trace_params(max_depth=2, capture=nrt.CAPTURE_SPHERE, diffuse=0,
                                 n_rays=n_rays, rep_tries=8, r_rx=0.3, ray_labels=1)
    r = sc.trace(room.tx, RX, p)
    lab = r.ray_labels()
    osc = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05,
                             grid_cell=0.25)
    osim = oracle.OracleSim(osc, room.tx, RX, oracle.SimParams(
        max_depth=2, capture=0, diffuse=0, n_rays=n_rays, rep_tries=8, r_rx=0.3,
        delta=1e-5 * float(np.linalg.norm([5, 4, 3]))))
    olab, amb = osim.ray_labels()
    ok = ~amb
    print("labels gpu", int(lab.sum()), "oracle", int(olab.sum()), "ambiguous", int(amb.sum()))
    assert olab.sum() > 50
    assert np.array_equal(lab[ok], olab[ok])


def test_bounded_wait_runs_out_and_context_recovers():
    """Failure detection without a GPU fault: with the watchdog lowered to one
    non-blocking poll, the tensor-core kernel's wait for its MMAs runs out;
    the kernel records the timeout, drains its own MMAs, frees its tensor
    memory and returns, the call reports NRT_ERR_TIMEOUT, and the same
    context then computes the product correctly with the default limit."""
    c = nrt.Context(0)
    rng = np.random.default_rng(99)
    A = M.bf16(rng.standard_normal((512, 4096)))
    B = M.bf16(rng.standard_normal((256, 4096)))
    C = torch.zeros((512, 256), dtype=torch.float32, device="cuda")
    c.set_wait_limit(1)
    with pytest.raises(nrt.NrtError) as e:
        nrt.gemm_bf16(c, _bf16_bits(A), _bf16_bits(B), C)
    assert e.value.status == 5  # NRT_ERR_TIMEOUT
    c.set_wait_limit(0)
    nrt.gemm_bf16(c, _bf16_bits(A), _bf16_bits(B), C)
    want = A @ B.T
    bound = 1e-5 * (np.abs(A) @ np.abs(B).T) + 1e-30
    assert np.all(np.abs(C.cpu().numpy().astype(np.float64) - want) <= bound)
    with pytest.raises(nrt.NrtError):
        c.set_wait_limit(-1)


def test_checkpoint_resume_continues_training(ctx, tmp_path):
    """Checkpoint/resume of the network's training state: 3 Adam steps, a
    checkpoint to disk, 4 more steps; a fresh network restored from the
    checkpoint and given the same 4 steps ends where the uninterrupted run
    did (up to the order of the split-K atomic sums of the weight
    gradients), while a restore of the parameters alone (fresh moments and
    step count) lands measurably elsewhere."""
    n, B = 8 * 2048, 2048
    tx_table, ti, rid, lab = _train_inputs(n)
    dev = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    data = (dev(tx_table), dev(ti), dev(rid), dev(lab))
    kw = dict(lr=2e-3, batch=B, pos_weight=3.0)
    net, _ = _net(ctx)
    net.train(*data, start=0, steps=3, **kw)
    ck = tmp_path / "mlp.npz"
    net.save(ck)
    st = net.state()
    assert st["step"] == 3 and np.abs(st["adam_v"]).max() > 0
    net.train(*data, start=3 * B, steps=4, **kw)
    want = net.params().astype(np.float64)
    moved = np.abs(want - st["params"]).max()

    net2, _ = _net(ctx, theta=inputs.mlp_init() * 0.5)  # different start, overwritten
    net2.restore(ck)
    assert np.array_equal(net2.params(), st["params"])
    net2.train(*data, start=3 * B, steps=4, **kw)
    got = net2.params().astype(np.float64)
    assert net2.state()["step"] == 7
    err = np.abs(got - want).max()

    net3, _ = _net(ctx, theta=st["params"])  # parameters only: Adam restarts
    net3.train(*data, start=3 * B, steps=4, **kw)
    err_fresh = np.abs(net3.params().astype(np.float64) - want).max()
    print("moved", moved, "resumed err", err, "fresh-Adam err", err_fresh)
    assert err <= 1e-2 * kw["lr"]
    assert err_fresh > 10 * max(err, 1e-9)
