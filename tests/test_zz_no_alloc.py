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


def _room_batch(nrt, inputs, ctx):
    room = inputs.room_scene()
    sc = nrt.Scene(ctx, room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    sc.set_materials(np.array([5.3, 3.0], np.float32), np.array([0.03, 0.01], np.float32),
                     np.array([0.3, 0.2], np.float32))
    tx = np.array([[1.0, 1.0, 1.5], [1.4, 1.2, 1.5], [1.8, 1.0, 1.2], [2.2, 1.5, 1.0]],
                  np.float32)
    rx = np.array([4.0, 3.0, 1.2], np.float32)
    budgets = np.array([3000, 5000, 2000, 4000], np.int64)
    p = nrt.default_trace_params(max_depth=2, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=1)
    return sc, tx, rx, budgets, p


def test_backward_noalloc_batch_graph_follows_replay():
    """A call recorded into a CUDA graph on a batch result (per-pair dL/dP),
    replayed after the batch is re-traced with other TX positions, gives the
    gradient of the new paths: the path count is read on the device."""
    import torch

    from paper_2507_04021_gb300 import inputs, nrt

    dev = torch.device("cuda", 0)
    s = torch.cuda.Stream(device=dev)
    ctx = nrt.Context(0, stream=s.cuda_stream)
    sc, tx, rx, budgets, p = _room_batch(nrt, inputs, ctx)
    b = sc.trace_batch(tx, rx, budgets, p, use_graph=True)
    P = b.power()
    assert (P > 0).all()
    dLdP = ((1.0 / P) * np.array([1.0, -0.5, 0.25, 2.0])).astype(np.float32)
    dl = torch.tensor(dLdP, device=dev)
    grad = torch.zeros(3 * 2, dtype=torch.float32, device=dev)
    # the first call on the device resolves the scratch address: before any capture
    b.backward_noalloc(dl, grad)
    ctx.sync()
    want = np.concatenate(b.backward(dLdP)).astype(np.float64)
    got = grad.cpu().numpy().astype(np.float64)
    assert np.allclose(got, want, rtol=1e-5, atol=1e-6 * np.abs(want).max()), (got, want)

    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        b.backward_noalloc(dl, grad)
    n_before = b.counts()[1]["paths"]
    tx2 = tx + np.array([0.3, 0.4, -0.2], np.float32)
    b.replay(tx2)
    n_after = b.counts()[1]["paths"]
    assert n_after != n_before  # the recorded call must not keep the old count
    want2 = np.concatenate(b.backward(dLdP)).astype(np.float64)
    for _ in range(2):
        grad.fill_(float("nan"))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        got2 = grad.cpu().numpy().astype(np.float64)
        assert np.allclose(got2, want2, rtol=1e-5, atol=1e-6 * np.abs(want2).max()), (got2, want2)


def test_backward_noalloc_checks_its_buffers():
    """The binding checks what the C call cannot: device, dtype, layout, size."""
    import torch

    from paper_2507_04021_gb300 import inputs, nrt

    ctx = nrt.Context(0)
    sc, tx, rx, budgets, p = _room_batch(nrt, inputs, ctx)
    res = sc.trace(tx[0], rx[None], nrt.default_trace_params(max_depth=2, capture=nrt.CAPTURE_VIS,
                                                             diffuse=1, n_rays=2000))
    dev = torch.device("cuda", 0)
    ok_dl = torch.ones(1, dtype=torch.float32, device=dev)
    ok_g = torch.zeros(6, dtype=torch.float32, device=dev)
    bad = [
        (torch.ones(1, dtype=torch.float32), ok_g),                      # host tensor
        (torch.ones(1, dtype=torch.float64, device=dev), ok_g),          # wrong dtype
        (ok_dl, torch.zeros(5, dtype=torch.float32, device=dev)),        # too short
        (ok_dl, torch.zeros((6, 2), dtype=torch.float32, device=dev)[:, 0]),  # strided
    ]
    for dl, g in bad:
        with pytest.raises(ValueError):
            res.backward_noalloc(dl, g)
    res.backward_noalloc(ok_dl, ok_g)
    ctx.sync()
    assert torch.isfinite(ok_g).all()
