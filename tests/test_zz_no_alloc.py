"""nrt_backward_noalloc against nrt_backward, through the C ABI, on a GPU.

The no-alloc variant serves callers that cannot allocate device memory (work
captured into CUDA graphs, real-time loops, hosts whose framework owns the
device memory): they hand in device buffers for dL/dP and the gradient, and
the reduction's partial sums live in a fixed array inside the library.  This
file is collected last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_backward_noalloc_matches_backward_twice():
    import torch

    from paper_2507_04021_gb300 import inputs, nrt

    room = inputs.room_scene()
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    # non-zero scattering so that every derivative (eps_r, sigma, S) is exercised
    eps = np.array([5.3, 3.0], np.float32)
    sig = np.array([0.03, 0.01], np.float32)
    sca = np.array([0.3, 0.2], np.float32)
    sc.set_materials(eps, sig, sca)
    rx = np.array([[4.0, 3.0, 1.2], [1.5, 3.2, 1.0], [4.2, 0.8, 2.1], [2.5, 2.0, 0.5]],
                  np.float32)
    p = nrt.default_trace_params(max_depth=2, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=4000)
    res = sc.trace(room.tx, rx, p)
    _, c = res.counts()
    assert c["paths"] > 100
    P = res.power()
    dLdP = (1.0 / P).astype(np.float32) * np.array([1.0, -0.5, 0.25, 2.0], np.float32)
    ge, gs, gc = res.backward(dLdP)
    want = np.concatenate([ge, gs, gc]).astype(np.float64)
    assert np.all(np.isfinite(want)) and np.abs(want).max() > 0
    dev = torch.device("cuda", 0)
    dl = torch.tensor(dLdP, device=dev)
    for _ in range(2):
        grad = torch.full((3 * 2,), float("nan"), dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        res.backward_noalloc(dl, grad)
        ctx.sync()
        got = grad.cpu().numpy().astype(np.float64)
        scale = np.abs(want).max()
        assert np.allclose(got, want, rtol=1e-5, atol=1e-6 * scale), (got, want)
