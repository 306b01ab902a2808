"""Pins of the learned-proposal oracle (oracle/mlp.py) to things other than
itself: published SplitMix64 outputs, closed-form distribution moments,
PyTorch's bfloat16 cast, torch.nn / autograd / torch.optim.Adam in FP64 (the
library routines for the network, its gradients and the optimiser), closed
forms of the Fourier features and the Gumbel-max sampling law."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp as M
from paper_2507_04021_gb300 import inputs


def test_splitmix64_published_outputs():
    # Reference outputs of SplitMix64 seeded with 1234567 (S. Vigna's
    # splitmix64.c, as tabulated by the Rosetta Code SplitMix64 task).
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    got = [int(x) for x in M.splitmix64_stream(1234567, 5)]
    assert got == want


def test_counter_uniform_and_gumbel_moments():
    i = np.arange(1_000_000)
    u = M.counter_uniform(99, i)
    assert 0.0 < u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 2e-3 and abs(u.var() - 1.0 / 12.0) < 2e-3
    g = M.gumbel(99, i)
    # standard Gumbel: mean = Euler-Mascheroni constant, variance = pi^2 / 6
    assert abs(g.mean() - 0.5772156649015329) < 5e-3
    assert abs(g.var() - math.pi ** 2 / 6.0) < 2e-2
    # counter-based: element i does not depend on how many are drawn
    assert np.array_equal(M.counter_uniform(99, [5, 7]), u[[5, 7]])
    # counter i is output i + 1 of the SplitMix64 stream of the same seed
    # (pinned above to the published outputs), top 53 bits, half-ulp offset
    z = M.splitmix64_stream(1234567, 5)
    want = ((z >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    assert np.array_equal(M.counter_uniform(1234567, np.arange(5)), want)


def test_bf16_matches_torch_cast():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(100000).astype(np.float32) * 10.0 ** rng.integers(-6, 6, 100000),
                        np.array([1.0, -2.5, 0.0, 3.4e38, 1e-30], np.float32)])
    # exact ties between two bfloat16 values (the low 16 bits are 0x8000)
    ties = (rng.integers(0, 2 ** 31, 2000, dtype=np.uint64) & np.uint64(0x7F7F0000)) | np.uint64(0x8000)
    x = np.concatenate([x, ties.astype(np.uint32).view(np.float32)]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(x), want)


def test_features_closed_forms():
    d = np.array([[1.0, 0.0, 0.0], [0.0, 0.5, -0.25]], np.float32)
    u = np.zeros(3, np.float32)
    F = M.features(d, u, emulate=False)
    assert F.shape == (2, 96)
    for k in range(8):
        # x = 1: sin(pi 2^k) = 0, cos(pi 2^k) = -1 for k = 0 else 1
        assert abs(F[0, (0 * 8 + k) * 2]) < 1e-12
        assert F[0, (0 * 8 + k) * 2 + 1] == pytest.approx(-1.0 if k == 0 else 1.0, abs=1e-12)
        # normalised TX at the centre: sin 0 = 0, cos 0 = 1
        for c in (3, 4, 5):
            assert F[0, (c * 8 + k) * 2] == 0.0 and F[0, (c * 8 + k) * 2 + 1] == 1.0
    # y = 0.5: sin(pi/2) = 1 at k = 0, cos(pi) = -1 at k = 1
    assert F[1, (1 * 8 + 0) * 2] == pytest.approx(1.0, abs=1e-12)
    assert F[1, (1 * 8 + 1) * 2 + 1] == pytest.approx(-1.0, abs=1e-12)
    # z = -0.25: sin(-pi/4) = -sqrt(2)/2
    assert F[1, (2 * 8 + 0) * 2] == pytest.approx(-math.sqrt(0.5), abs=1e-12)
    un = M.normalise_tx([10.0, 5.0, 1.5], [10.0, 5.0, 1.5], [10.0, 5.0, 1.5])
    assert np.array_equal(un, np.zeros(3, np.float32))


def _torch_net(P):
    net = torch.nn.Sequential(torch.nn.Linear(96, 128), torch.nn.ReLU(),
                              torch.nn.Linear(128, 128), torch.nn.ReLU(),
                              torch.nn.Linear(128, 128), torch.nn.ReLU(),
                              torch.nn.Linear(128, 1)).double()
    with torch.no_grad():
        for i, (w, b) in enumerate((("W1", "b1"), ("W2", "b2"), ("W3", "b3"), ("w4", "b4"))):
            lin = net[2 * i]
            lin.weight.copy_(torch.from_numpy(P[w].reshape(lin.weight.shape)))
            lin.bias.copy_(torch.from_numpy(P[b].reshape(lin.bias.shape)))
    return net


def _batch(n=256, seed=3):
    rng = np.random.default_rng(seed)
    X = M.bf16(rng.uniform(-1, 1, (n, 96)))
    y = (rng.random(n) < 0.2).astype(np.float64)
    return X, y


def test_forward_and_gradients_match_torch_autograd():
    P = M.unpack(inputs.mlp_init())
    P["b1"] = np.linspace(-0.1, 0.1, 128)  # non-zero biases exercise the bias terms
    P["b4"] = np.array([-0.3])
    X, y = _batch()
    net = _torch_net(P)
    Xt = torch.from_numpy(X)
    z = net(Xt)[:, 0]
    A = M.forward(P, X, emulate=False)
    assert np.allclose(A["z"], z.detach().numpy(), rtol=1e-12, atol=1e-12)
    wp = 4.0
    lt = torch.nn.functional.binary_cross_entropy_with_logits(
        z, torch.from_numpy(y), pos_weight=torch.tensor(wp, dtype=torch.float64))
    lt.backward()
    loss, G = M.grads(P, X, y, wp, emulate=False)
    assert loss == pytest.approx(float(lt.detach()), rel=1e-12)
    pairs = (("W1", net[0].weight), ("b1", net[0].bias), ("W2", net[2].weight), ("b2", net[2].bias),
             ("W3", net[4].weight), ("b3", net[4].bias), ("w4", net[6].weight), ("b4", net[6].bias))
    for name, prm in pairs:
        want = prm.grad.numpy().reshape(G[name].shape)
        assert np.allclose(G[name], want, rtol=1e-10, atol=1e-14), name


def test_emulated_rounding_points_match_torch_bf16_casts():
    """The BF16 points of the emulated forward, placed with torch's own cast."""
    P = M.unpack(inputs.mlp_init())
    X, _ = _batch(64, 5)
    c = lambda a: a.to(torch.bfloat16).to(torch.float64)  # noqa: E731
    t = {k: torch.from_numpy(v) for k, v in P.items()}
    h = torch.from_numpy(X)
    for w, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
        h = c(torch.relu(h @ c(t[w]).T + t[b]))
    z = h @ c(t["w4"]) + t["b4"][0]
    assert np.allclose(M.forward(P, X)["z"], z.numpy(), rtol=1e-12, atol=1e-12)


def test_emulated_backward_rounding_points_match_torch():
    """Gradients with BF16 rounding of the pre-activation gradients dZ
    (hooks on Z) and of the stored activations (straight-through casts), all
    other arithmetic by torch autograd in FP64."""
    P = M.unpack(inputs.mlp_init())
    P["b2"] = np.linspace(-0.05, 0.05, 128)
    X, y = _batch(128, 9)
    c = lambda a: a.to(torch.bfloat16).to(torch.float64)  # noqa: E731
    st = lambda a: a + (c(a) - a).detach()  # noqa: E731  forward rounded, gradient unchanged
    t = {k: torch.from_numpy(v).requires_grad_(True) for k, v in P.items()}
    h = torch.from_numpy(X)
    for w, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
        Z = h @ st(t[w]).T + t[b]
        Z.register_hook(c)
        h = st(torch.relu(Z))
    z = h @ st(t["w4"]) + t["b4"][0]
    wp = 3.0
    torch.nn.functional.binary_cross_entropy_with_logits(
        z, torch.from_numpy(y), pos_weight=torch.tensor(wp, dtype=torch.float64)).backward()
    _, G = M.grads(P, X, y, wp)
    for k in G:
        assert np.allclose(G[k], t[k].grad.numpy().reshape(G[k].shape), rtol=1e-10, atol=1e-15), k


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(7)
    theta = rng.standard_normal(50)
    p = torch.nn.Parameter(torch.from_numpy(theta.copy()))
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(50)
    v = np.zeros(50)
    th = theta.copy()
    for t in range(1, 4):
        g = rng.standard_normal(50)
        p.grad = torch.from_numpy(g.copy())
        opt.step()
        th, m, v = M.adam(th, g, m, v, t, 3e-3)
    assert np.allclose(th, p.detach().numpy(), rtol=1e-12, atol=1e-15)


def test_select_structure():
    n = 10000
    z = inputs.mlp_logits(n)
    ids = M.select(z, 900, 100, seed=11)
    assert np.all(np.diff(ids) > 0) and ids[0] >= 0 and ids[-1] < n
    assert 900 <= ids.size <= 1000
    # every stratum holds at least one selected index
    s = np.arange(100)
    lo, hi = s * n // 100, (s + 1) * n // 100
    assert all(np.any((ids >= a) & (ids < b)) for a, b in zip(lo, hi))
    # everything selected when k_top = n
    assert M.select(z, n, 0, seed=1).size == n
    # logit gaps far beyond the Gumbel spread: top-k is the plain top-k
    big = (np.arange(n) % 977).astype(np.float32) * 1000.0
    want = np.sort(np.argsort(-big.astype(np.float64), kind="stable")[:50])
    assert np.array_equal(M.select(big, 50, 0, seed=2), want)
    # every key tied (logit = -its float32 Gumbel noise, so logit + noise is
    # exactly 0): ties go to the smaller index, so top-k is 0 .. k-1
    g32 = M.gumbel(3, np.arange(n)).astype(np.float32)
    assert np.array_equal(M.select(-g32, 40, 0, seed=3), np.arange(40))


def test_strata_draws_are_independent_of_the_gumbel_noise():
    """The uniform stratum picks use their own counters: across seeds, the
    position of the pick inside stratum 0 is uncorrelated with the Gumbel
    noise of index 0 (had they shared a counter, the two would be the same
    monotone function of one uniform, rank correlation 1)."""
    n, k_u, seeds = 1000, 10, 400
    pos, g0 = np.zeros(seeds), np.zeros(seeds)
    z = np.full(n, -1e4, np.float32)  # no top-k pick lands in stratum 0 by accident
    z[-1] = 0.0
    for s in range(seeds):
        ids = M.select(z, 1, k_u, seed=500 + s)
        in0 = ids[ids < n // k_u]
        assert in0.size == 1
        pos[s] = in0[0]
        g0[s] = M.gumbel(500 + s, [0])[0]
    rp = np.argsort(np.argsort(pos)).astype(np.float64)
    rg = np.argsort(np.argsort(g0)).astype(np.float64)
    rho = np.corrcoef(rp, rg)[0, 1]
    assert abs(rho) < 4.0 / np.sqrt(seeds)


def test_gumbel_max_samples_the_softmax():
    """k = 1 (Gumbel-max): index i is drawn with probability softmax(z)_i."""
    z = np.array([0.0, 1.0, -0.5, 2.0], np.float32)
    p = np.exp(z.astype(np.float64))
    p /= p.sum()
    trials = 20000
    cnt = np.zeros(4)
    for s in range(trials):
        cnt[M.select(z, 1, 0, seed=1000 + s)[0]] += 1
    assert np.all(np.abs(cnt / trials - p) < 4.5 * np.sqrt(p * (1 - p) / trials))
