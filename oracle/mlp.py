"""FP64 reference of the learned launch proposal (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this module; the product path never does.  It shares
no code with the CUDA library.

The paper traces a fixed Fibonacci launch (Sec. II-B); the proposal is an
addition on top of it: a small network maps a launch direction and the
transmitter position to the probability that the ray is a member of a
valid specular path key, and a Gumbel-top-k draw over its logits picks the
rays to trace.  Everything here is written from those definitions:

* features: 6 coordinates (the float32 direction and the transmitter
  position normalised to the scene box), 8 octaves, sin and cos of
  pi * 2^k * v: 96 inputs;
* network: 96 -> 128 -> 128 -> 128 (ReLU) -> 1 logit;
* BF16 storage of weights and activations, wider accumulation; with
  ``emulate=True`` every value the kernels store in BF16 is rounded here at
  the same point (round to nearest even), all arithmetic otherwise FP64;
* loss: binary cross-entropy on the logit with a positive-class weight,
  mean over the batch; gradients by the chain rule, layer by layer;
* Adam (Kingma and Ba, 2015) with bias correction;
* random numbers: SplitMix64 (Steele, Lea and Flood, 2014) used as a
  counter-based generator, u = (mix(seed + (i + 1) * gamma) >> 11 + 0.5) / 2^53;
  Gumbel noise -log(-log(u));
* selection: the k_top largest (logit + Gumbel) keys (ties: smaller index)
  plus one uniformly drawn index per stratum of k_uniform equal strata,
  merged, unique and ascending.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
N_COORD = 6
N_OCT = 8
N_IN = N_COORD * N_OCT * 2
H = 128

_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


# ---------------------------------------------------------------- random numbers
def splitmix64_mix(z):
    """The SplitMix64 output function (finaliser) on uint64 values."""
    z = np.asarray(z, np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_stream(seed: int, n: int) -> np.ndarray:
    """First n outputs of a SplitMix64 generator whose state starts at seed."""
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return splitmix64_mix(np.uint64(seed) + i * GAMMA)


def counter_uniform(seed: int, idx) -> np.ndarray:
    """u_i in (0, 1): the idx-th SplitMix64 output of stream `seed`, top 53 bits."""
    idx = np.asarray(idx, np.uint64)
    with np.errstate(over="ignore"):
        z = splitmix64_mix(np.uint64(seed) + (idx + np.uint64(1)) * GAMMA)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def gumbel(seed: int, idx) -> np.ndarray:
    return -np.log(-np.log(counter_uniform(seed, idx)))


# ---------------------------------------------------------------- bf16
def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# ---------------------------------------------------------------- features
def normalise_tx(tx, center, half) -> np.ndarray:
    """(tx - center) / half in float32 arithmetic."""
    tx = np.asarray(tx, np.float32)
    return ((tx - np.asarray(center, np.float32)) / np.asarray(half, np.float32)).astype(np.float32)


def features(dirs32, u32, emulate: bool = True) -> np.ndarray:
    """[n, 96] inputs from float32 directions [n,3] and the normalised TX
    (float32 [3] or [n,3]).  Column (c * 8 + k) * 2 + {0: sin, 1: cos}."""
    d = np.asarray(dirs32, np.float32).astype(np.float64)
    u = np.broadcast_to(np.asarray(u32, np.float32).astype(np.float64), d.shape)
    v = np.concatenate([d, u], axis=1)  # [n, 6]
    n = v.shape[0]
    out = np.zeros((n, N_IN))
    for c in range(N_COORD):
        for k in range(N_OCT):
            a = np.pi * (2.0 ** k) * v[:, c]
            out[:, (c * N_OCT + k) * 2] = np.sin(a)
            out[:, (c * N_OCT + k) * 2 + 1] = np.cos(a)
    return bf16(out) if emulate else out


# ---------------------------------------------------------------- network
def unpack(theta, n_in: int = N_IN, h: int = H) -> dict:
    """Packed float32 parameters -> dict (W1 [h,n_in], b1, W2, b2, W3, b3, w4 [h], b4)."""
    t = np.asarray(theta, np.float64)
    o = 0
    P = {}
    for name, shape in (("W1", (h, n_in)), ("b1", (h,)), ("W2", (h, h)), ("b2", (h,)),
                        ("W3", (h, h)), ("b3", (h,)), ("w4", (h,)), ("b4", (1,))):
        size = int(np.prod(shape))
        P[name] = t[o:o + size].reshape(shape).copy()
        o += size
    assert o == t.size
    return P


def pack(P: dict) -> np.ndarray:
    return np.concatenate([P[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3",
                                                       "w4", "b4")])


def forward(P: dict, X, emulate: bool = True) -> dict:
    """Activations of the network on inputs X [n, n_in] (already rounded if
    emulating).  Weights are used in BF16, biases in full precision."""
    r = bf16 if emulate else (lambda a: np.asarray(a, np.float64))
    W1, W2, W3, w4 = r(P["W1"]), r(P["W2"]), r(P["W3"]), r(P["w4"])
    A = {"X": np.asarray(X, np.float64)}
    Z1 = A["X"] @ W1.T + P["b1"]
    A["H1"] = r(np.maximum(Z1, 0.0))
    Z2 = A["H1"] @ W2.T + P["b2"]
    A["H2"] = r(np.maximum(Z2, 0.0))
    Z3 = A["H2"] @ W3.T + P["b3"]
    A["H3"] = r(np.maximum(Z3, 0.0))
    A["z"] = A["H3"] @ w4 + P["b4"][0]
    return A


def bce_loss(z, y, pos_weight: float) -> float:
    """mean over the batch of -[w_p y log s(z) + (1 - y) log(1 - s(z))]."""
    z = np.asarray(z, np.float64)
    y = np.asarray(y, np.float64)
    log_s = -np.logaddexp(0.0, -z)      # log sigmoid(z)
    log_1ms = -np.logaddexp(0.0, z)     # log (1 - sigmoid(z))
    return float(np.mean(-(pos_weight * y * log_s + (1.0 - y) * log_1ms)))


def grads(P: dict, X, y, pos_weight: float, emulate: bool = True):
    """(loss, gradient dict) of the batch loss w.r.t. the float32 master
    parameters.  Backward values the kernels store in BF16 (the
    pre-activation gradients dZ) are rounded when emulating."""
    r = bf16 if emulate else (lambda a: np.asarray(a, np.float64))
    A = forward(P, X, emulate)
    y = np.asarray(y, np.float64)
    B = y.shape[0]
    W2, W3, w4 = r(P["W2"]), r(P["W3"]), r(P["w4"])
    s = 1.0 / (1.0 + np.exp(-A["z"]))
    dz = (s * (pos_weight * y + 1.0 - y) - pos_weight * y) / B
    G = {"w4": A["H3"].T @ dz, "b4": np.array([dz.sum()])}
    dZ3 = r(np.outer(dz, w4) * (A["H3"] > 0))
    G["W3"] = dZ3.T @ A["H2"]
    G["b3"] = dZ3.sum(axis=0)
    dZ2 = r((dZ3 @ W3) * (A["H2"] > 0))
    G["W2"] = dZ2.T @ A["H1"]
    G["b2"] = dZ2.sum(axis=0)
    dZ1 = r((dZ2 @ W2) * (A["H1"] > 0))
    G["W1"] = dZ1.T @ A["X"]
    G["b1"] = dZ1.sum(axis=0)
    return bce_loss(A["z"], y, pos_weight), G


def adam(theta, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999,
         eps: float = 1e-8):
    """One Adam step on packed arrays; returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------- selection
def select(logits, k_top: int, k_uniform: int, seed: int) -> np.ndarray:
    """Gumbel-top-k over float32 keys fl32(logit + fl32(gumbel)), ties to the
    smaller index, plus one index per stratum [s n / k_u, (s + 1) n / k_u)
    drawn with the same stream at counters n + s; unique, ascending."""
    z = np.asarray(logits, np.float32)
    n = z.shape[0]
    g = gumbel(seed, np.arange(n)).astype(np.float32)
    key = (z + g).astype(np.float32)
    k_top = min(k_top, n)
    order = np.lexsort((np.arange(n), -key.astype(np.float64)))
    chosen = set(order[:k_top].tolist())
    if k_uniform > 0:
        s = np.arange(k_uniform, dtype=np.int64)
        lo = (s * n) // k_uniform
        hi = ((s + 1) * n) // k_uniform
        u = counter_uniform(seed, n + s)
        pick = lo + np.floor(u * (hi - lo)).astype(np.int64)
        chosen.update(pick[hi > lo].tolist())
    return np.array(sorted(chosen), np.int64)
