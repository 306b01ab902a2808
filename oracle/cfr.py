"""FP64 reference of the channel frequency response, the impulse response and
the loss of Eq. 5 (test infrastructure; only tests, smoke() and bench's
CPU-baseline leg use it).

Sec. III-B builds its training targets from channel responses: the CFR at
N equally spaced frequencies over a bandwidth B around the centre frequency,
with every path coefficient taken at the centre frequency, and the CIR
obtained from it.  Here:

* f_n = f_c + (n - (N - 1)/2) B / (N - 1), n = 0..N-1;
* H_j(f_n) = sum over the paths p of receiver j of a_p exp(-j 2 pi f_n tau_p)
  (a_p: phase-split coefficient at f_c, tau_p: delay);
* h_j = inverse DFT of H_j (numpy's ifft);
* Eq. 5: L_j = |h_j - h^_j|^2 / |h^_j|^2; by Parseval the same ratio on the
  CFR, so the loss and its gradient are evaluated on H;
* dL_j/dtheta = (2 / |H^_j|^2) sum_p Re( conj(g_p) da_p/dtheta ),
  g_p = sum_n (H_j(f_n) - H^_j(f_n)) exp(+j 2 pi f_n tau_p).
"""
from __future__ import annotations

import numpy as np


def freqs(fc: float, bandwidth: float, n: int) -> np.ndarray:
    k = np.arange(n, dtype=np.float64) - (n - 1) / 2.0
    return fc + k * (bandwidth / (n - 1))


def cfr(a, tau, rx, n_rx: int, f) -> np.ndarray:
    """[n_rx, N] complex: sum of a_p exp(-j 2 pi f tau_p) per receiver."""
    a = np.asarray(a, np.complex128)
    tau = np.asarray(tau, np.float64)
    rx = np.asarray(rx, np.int64)
    f = np.asarray(f, np.float64)
    H = np.zeros((n_rx, f.size), np.complex128)
    for j in range(n_rx):
        m = rx == j
        if m.any():
            H[j] = (a[m, None] * np.exp(-2j * np.pi * tau[m, None] * f[None, :])).sum(axis=0)
    return H


def cir(H) -> np.ndarray:
    return np.fft.ifft(np.asarray(H), axis=-1)


def eq5_loss(H, H_target) -> np.ndarray:
    """Per receiver: |H - H^|^2 / |H^|^2 (equal to Eq. 5 on the CIR)."""
    H = np.asarray(H)
    T = np.asarray(H_target)
    return np.sum(np.abs(H - T) ** 2, axis=-1) / np.sum(np.abs(T) ** 2, axis=-1)


def eq5_grad(path_grads, tau, rx, f, H, H_target, rx_weight) -> np.ndarray:
    """[3, n_labels] gradient of sum_j w_j L_j from the per-path complex
    derivatives path_grads [n_paths, 3, n_labels]."""
    H = np.asarray(H)
    T = np.asarray(H_target)
    D = np.sum(np.abs(T) ** 2, axis=-1)
    dH = H - T
    tau = np.asarray(tau, np.float64)
    rx = np.asarray(rx, np.int64)
    g = np.sum(dH[rx] * np.exp(2j * np.pi * tau[:, None] * np.asarray(f)[None, :]), axis=1)
    w = 2.0 * np.asarray(rx_weight, np.float64)[rx] / D[rx]
    return np.real(np.einsum("p,ptl->tl", w * np.conj(g), path_grads))
