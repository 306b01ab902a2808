"""Thin Python binding of libnrt (include/nrt.h): argument marshalling only.

Every step of the simulation runs in the library's CUDA kernels.  The
library must have been built (``paper_2507_04021_gb300.build.build()``); if it
cannot be loaded the import of this module's functions fails loudly -- there
is no CPU fallback.  Host inputs are numpy arrays; device inputs are torch
CUDA tensors (their data pointers are passed with ``inputs_on_device``).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_lib = None

NRT_OK = 0
CAPTURE_SPHERE = 0
CAPTURE_VIS = 1
LAUNCH_FIB = 0
LAUNCH_DPS = 1
POL_TE = 0
POL_TM = 1
POL_VECTOR = 2
ISECT_DISC = 0
ISECT_SDF = 1


class NrtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"nrt status {status}: {msg}")
        self.status = status


class SceneParams(C.Structure):
    _fields_ = [("rho", C.c_float), ("r_p", C.c_float), ("lambda_d", C.c_float)]


class TraceParams(C.Structure):
    _fields_ = [
        ("max_depth", C.c_int32), ("capture", C.c_int32), ("diffuse", C.c_int32),
        ("pol", C.c_int32), ("kappa", C.c_int32), ("rep_tries", C.c_int32),
        ("record_hits", C.c_int32), ("ray_labels", C.c_int32), ("n_rays", C.c_int64),
        ("r_rx", C.c_float), ("t_min", C.c_float), ("t_a_deg", C.c_float), ("t_d", C.c_float),
        ("freq", C.c_float), ("keep_keys", C.c_int32), ("key_capacity", C.c_int64),
        ("cand_capacity", C.c_int64), ("launch", C.c_int32), ("diffraction", C.c_int32),
        ("spec_waves", C.c_int32),
    ]


class CastParams(C.Structure):
    _fields_ = [("model", C.c_int32), ("sigma", C.c_float), ("t_min", C.c_float),
                ("t_max", C.c_float)]


class Counters(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "rays", "segments", "vis_casts", "los_casts", "validation_casts", "candidates", "keys",
        "paths", "n_dps", "hash_probes_max", "error_flags", "kernel_launches", "diffuse_casts",
        "diffraction_casts", "pruned_legs", "spec_items", "spec_ended_without_cast",
        "spec_ended_at_first_leg")] + [("reserved", C.c_int64 * 1)]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_ if n != "reserved"}


class BatchOpts(C.Structure):
    _fields_ = [("packet", C.c_int32), ("schedule", C.c_int32), ("use_graph", C.c_int32),
                ("reserved", C.c_int32)]


class MlpTrainOpts(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("pos_weight", C.c_float), ("batch", C.c_int32)]


class PathView(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in (
        "key_hi", "key_lo", "rep", "rx", "type", "k", "pts", "mats", "cos_theta", "geo", "tau", "a",
        "normal")]


_P = C.c_void_p


def lib():
    """Load libnrt.so (building it in-tree first if it is missing or stale), or
    the prebuilt library the environment names in NRT_LIBRARY (a build of the
    same sources with other compile-time settings, for A/B measurements)."""
    global _lib
    if _lib is None:
        path = os.environ.get("NRT_LIBRARY") or _build.build()
        _lib = C.CDLL(path)
        L = _lib
        L.nrt_status_string.restype = C.c_char_p
        L.nrt_status_string.argtypes = [C.c_int]
        L.nrt_last_error.restype = C.c_char_p
        L.nrt_last_error.argtypes = [_P]
        L.nrt_create.argtypes = [C.POINTER(_P), C.c_int, _P]
        L.nrt_destroy.argtypes = [_P]
        L.nrt_sync.argtypes = [_P]
        L.nrt_trace_params_default.argtypes = [C.POINTER(TraceParams)]
        L.nrt_trace_params_default.restype = None
        L.nrt_scene_upload.argtypes = [_P, _P, _P, _P, _P, C.c_int64, C.POINTER(SceneParams),
                                       C.c_int, C.POINTER(_P)]
        L.nrt_scene_free.argtypes = [_P]
        L.nrt_scene_free.restype = None
        L.nrt_scene_info.argtypes = [_P, _P, _P, _P]
        L.nrt_scene_dps_read.argtypes = [_P, _P, _P, _P]
        L.nrt_set_materials.argtypes = [_P, _P, _P, _P, C.c_int]
        L.nrt_set_materials_device.argtypes = [_P, _P, C.c_int]
        L.nrt_scene_set_edges.argtypes = [_P, C.c_int64, _P, _P, _P, _P, _P, _P]
        L.nrt_cast.argtypes = [_P, _P, _P, C.c_int64, C.POINTER(CastParams), _P, _P, _P, _P]
        L.nrt_trace.argtypes = [_P, _P, _P, C.c_int, C.POINTER(TraceParams), _P, C.c_int64,
                                C.c_int, C.POINTER(_P)]
        L.nrt_result_free.argtypes = [_P]
        L.nrt_result_free.restype = None
        L.nrt_result_counts.argtypes = [_P, _P, C.POINTER(Counters)]
        L.nrt_result_times.argtypes = [_P, _P]
        L.nrt_paths_read.argtypes = [_P, C.POINTER(PathView)]
        L.nrt_hits_read.argtypes = [_P, _P, _P, _P, _P, _P]
        L.nrt_vis_read.argtypes = [_P, _P]
        L.nrt_field.argtypes = [_P]
        L.nrt_field_read.argtypes = [_P, _P]
        L.nrt_field_read_device.argtypes = [_P, _P]
        L.nrt_backward.argtypes = [_P, _P, _P, _P, _P]
        L.nrt_backward_noalloc.argtypes = [_P, _P, _P]
        L.nrt_trace_batch.argtypes = [_P, _P, _P, _P, C.c_int, C.POINTER(TraceParams),
                                      C.POINTER(BatchOpts), C.POINTER(_P)]
        L.nrt_batch_replay.argtypes = [_P, _P]
        L.nrt_batch_times.argtypes = [_P, _P, _P, _P]
        L.nrt_autotune_batch.argtypes = [_P, _P, _P, C.c_int, C.c_int, _P, _P]
        L.nrt_ray_labels_read.argtypes = [_P, _P]
        L.nrt_cfr.argtypes = [_P, C.c_double, C.c_int32, _P]
        L.nrt_cfr_backward.argtypes = [_P, C.c_double, C.c_int32, _P, _P, _P, _P, _P, _P]
        L.nrt_keys_read.argtypes = [_P, _P, _P, _P, _P]
        L.nrt_get_stream.argtypes = [_P, C.POINTER(_P)]
        L.nrt_set_wait_limit.argtypes = [_P, C.c_int64]
        L.nrt_measure_l2.argtypes = [_P, C.c_int64, C.c_int32, C.POINTER(C.c_float)]
        L.nrt_paths_export.argtypes = [_P, _P, _P, _P, _P]
        L.nrt_shard_merge.argtypes = [_P, C.c_int64, _P, _P, _P, _P, _P, C.c_int32, _P,
                                      C.c_int32, _P, _P]
        L.nrt_mlp_create.argtypes = [_P, _P, C.c_int64, _P, _P, C.c_int64, C.POINTER(_P)]
        L.nrt_mlp_free.argtypes = [_P]
        L.nrt_mlp_free.restype = None
        L.nrt_mlp_params_read.argtypes = [_P, _P]
        L.nrt_mlp_grads_read.argtypes = [_P, _P]
        L.nrt_mlp_state_read.argtypes = [_P, _P, _P, _P, C.POINTER(C.c_int64)]
        L.nrt_mlp_state_write.argtypes = [_P, _P, _P, _P, C.c_int64]
        L.nrt_mlp_features.argtypes = [_P, _P, _P, C.c_int64, _P]
        L.nrt_mlp_score.argtypes = [_P, _P, _P, C.c_int64, _P]
        L.nrt_mlp_train.argtypes = [_P, _P, C.c_int32, _P, _P, _P, C.c_int64, _P, C.c_int64,
                                    C.c_int32, C.POINTER(MlpTrainOpts), _P]
        L.nrt_propose.argtypes = [_P, _P, C.c_int64, C.c_int64, C.c_int64, C.c_uint64, _P,
                                  C.POINTER(C.c_int64)]
        L.nrt_gemm_bf16.argtypes = [_P, _P, C.c_int64, _P, C.c_int64, _P, C.c_int64, C.c_int64,
                                    C.c_int32, C.c_int64, C.c_int32, C.c_int64]
        L.nrt_destroy.restype = None
    return _lib


def exported_symbols():
    return [l.split("(")[0].split()[-1].lstrip("*") for l in _header_decls()]


def _header_decls():
    here = os.path.dirname(os.path.abspath(__file__))
    txt = open(os.path.join(os.path.dirname(here), "include", "nrt.h")).read()
    import re
    return re.findall(r"^(?:nrt_status|void|const char\*)\s+\**nrt_\w+\s*\(", txt, re.M)


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _ptr(a):
    """(pointer, on_device) of a numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr()), bool(a.is_cuda)
    return _np_ptr(a), False


class Context:
    def __init__(self, device: int = 0, stream: int | None = None):
        self._h = _P()
        self._check(lib().nrt_create(C.byref(self._h), device, _P(stream) if stream else None))
        self.device = device

    def _check(self, st):
        if st != NRT_OK:
            msg = lib().nrt_last_error(self._h if getattr(self, "_h", None) else None)
            raise NrtError(st, f"{lib().nrt_status_string(st).decode()}: {(msg or b'').decode()}")

    def sync(self):
        self._check(lib().nrt_sync(self._h))

    def set_wait_limit(self, polls: int):
        """Polls of a bounded tensor-core wait before it gives up (0 = default)."""
        self._check(lib().nrt_set_wait_limit(self._h, int(polls)))

    def measure_l2(self, nbytes: int = 48 << 20, reps: int = 50) -> float:
        """L2 read bandwidth in GB/s (nrt_measure_l2)."""
        g = C.c_float()
        self._check(lib().nrt_measure_l2(self._h, int(nbytes), int(reps), C.byref(g)))
        return float(g.value)

    def stream_handle(self) -> int:
        """The cudaStream_t the library enqueues on (for torch.cuda.ExternalStream)."""
        s = _P()
        self._check(lib().nrt_get_stream(self._h, C.byref(s)))
        return int(s.value or 0)

    def close(self):
        if self._h:
            lib().nrt_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_trace_params(**kw) -> TraceParams:
    p = TraceParams()
    lib().nrt_trace_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


class Scene:
    def __init__(self, ctx: Context, pos, nrm, surf, mat, rho=0.0625, r_p=0.015, lambda_d=100.0):
        self.ctx = ctx
        dev = hasattr(pos, "data_ptr") and pos.is_cuda
        if not dev:
            pos = np.ascontiguousarray(pos, np.float32)
            nrm = np.ascontiguousarray(nrm, np.float32)
            surf = np.ascontiguousarray(surf, np.uint16)
            mat = np.ascontiguousarray(mat, np.uint8)
        self._keep = (pos, nrm, surf, mat)
        n = int(pos.shape[0])
        sp = SceneParams(rho, r_p, lambda_d)
        self._h = _P()
        ctx._check(lib().nrt_scene_upload(ctx._h, _ptr(pos)[0], _ptr(nrm)[0], _ptr(surf)[0],
                                          _ptr(mat)[0], n, C.byref(sp), int(dev), C.byref(self._h)))
        self._keep = None
        self.n_points = n
        self.params = (rho, r_p, lambda_d)

    def info(self):
        nd = C.c_int64()
        bmin = np.zeros(3, np.float32)
        ms = C.c_float()
        self.ctx._check(lib().nrt_scene_info(self._h, C.byref(nd), _np_ptr(bmin), C.byref(ms)))
        return {"n_dps": nd.value, "bmin": bmin, "build_ms": ms.value}

    def dps(self):
        n = self.info()["n_dps"]
        vox = np.zeros((n, 3), np.int32)
        cnt = np.zeros(n, np.int32)
        recv = np.zeros((n, 3), np.float32)
        self.ctx._check(lib().nrt_scene_dps_read(self._h, _np_ptr(vox), _np_ptr(cnt), _np_ptr(recv)))
        return vox, cnt, recv

    def set_materials(self, eps_r, sigma, scat):
        e = np.ascontiguousarray(eps_r, np.float32)
        s = np.ascontiguousarray(sigma, np.float32)
        c = np.ascontiguousarray(scat, np.float32)
        self.ctx._check(lib().nrt_set_materials(self._h, _np_ptr(e), _np_ptr(s), _np_ptr(c),
                                                int(e.shape[0])))
        self.n_labels = int(e.shape[0])

    def set_materials_device(self, mat_dev):
        """nrt_set_materials_device: mat_dev a contiguous float32 CUDA tensor
        [3, n_labels] (eps_r, sigma, S rows) on the context's device, read on
        the context stream; values are clamped into range there."""
        import torch

        if not (isinstance(mat_dev, torch.Tensor) and mat_dev.is_cuda):
            raise ValueError("mat_dev must be a CUDA tensor")
        if mat_dev.device.index != self.ctx.device:
            raise ValueError(f"mat_dev is on cuda:{mat_dev.device.index}, the context on "
                             f"cuda:{self.ctx.device}")
        if mat_dev.dtype != torch.float32 or not mat_dev.is_contiguous() or mat_dev.dim() != 2 \
                or mat_dev.shape[0] != 3:
            raise ValueError("mat_dev must be a contiguous float32 [3, n_labels] tensor")
        self.ctx._check(lib().nrt_set_materials_device(self._h, _P(mat_dev.data_ptr()),
                                                       int(mat_dev.shape[1])))
        self.n_labels = int(mat_dev.shape[1])

    def set_edges(self, edges):
        """Edges for the diffraction of Sec. II-B-3 (an object with arrays a, b,
        n0, n1 [n, 3] and m0, m1 [n], e.g. inputs.Edges); None clears them."""
        if edges is None:
            self.ctx._check(lib().nrt_scene_set_edges(self._h, 0, None, None, None, None, None,
                                                      None))
            return
        f = lambda x: np.ascontiguousarray(x, np.float32).reshape(-1, 3)  # noqa: E731
        u = lambda x: np.ascontiguousarray(x, np.uint8).reshape(-1)  # noqa: E731
        arrs = (f(edges.a), f(edges.b), f(edges.n0), f(edges.n1), u(edges.m0), u(edges.m1))
        self.ctx._check(lib().nrt_scene_set_edges(self._h, int(arrs[4].shape[0]),
                                                  *[_np_ptr(x) for x in arrs]))

    def cast(self, o, d, model=ISECT_DISC, sigma=0.0, t_min=1e-3, t_max=float("inf")):
        """Closest hits of rays o + t d (CUDA float32 tensors [n, 3]) under the
        disc model or the SDF model (nrt_cast); returns CUDA tensors t [n],
        normal [n, 3], dps [n], labels [n]."""
        import torch

        o = o.contiguous()
        d = d.contiguous()
        n = int(o.shape[0])
        dev = o.device
        out = {"t": torch.empty(n, dtype=torch.float32, device=dev),
               "normal": torch.empty((n, 3), dtype=torch.float32, device=dev),
               "dps": torch.empty(n, dtype=torch.int32, device=dev),
               "labels": torch.empty(n, dtype=torch.int32, device=dev)}
        prm = CastParams(int(model), float(sigma), float(t_min), float(t_max))
        self.ctx._check(lib().nrt_cast(self._h, _P(o.data_ptr()), _P(d.data_ptr()), n,
                                       C.byref(prm), *[_P(out[k].data_ptr()) for k in
                                                       ("t", "normal", "dps", "labels")]))
        return out

    def trace(self, tx, rx, params: TraceParams, ray_subset=None) -> "Result":
        return Result(self, tx, rx, params, ray_subset)

    def trace_batch(self, tx, rx, budgets, params: TraceParams, packet=64, schedule=1,
                    use_graph=False) -> "BatchResult":
        return BatchResult(self, tx, rx, budgets, params, packet, schedule, use_graph)

    def close(self):
        if getattr(self, "_h", None):
            lib().nrt_scene_free(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Result:
    def __init__(self, scene: Scene, tx, rx, params: TraceParams, ray_subset=None):
        self.scene = scene
        self.ctx = scene.ctx
        tx = np.ascontiguousarray(tx, np.float32).reshape(3)
        rx = np.ascontiguousarray(rx, np.float32).reshape(-1, 3)
        self.n_rx = int(rx.shape[0])
        self.params = params
        sub_ptr, n_sub, on_dev = None, 0, False
        if ray_subset is not None:
            if not (hasattr(ray_subset, "data_ptr") and ray_subset.is_cuda):
                ray_subset = np.ascontiguousarray(ray_subset, np.uint32)
            sub_ptr, on_dev = _ptr(ray_subset)
            n_sub = int(ray_subset.shape[0])
        self._h = _P()
        self.ctx._check(lib().nrt_trace(scene._h, _np_ptr(tx), _np_ptr(rx), self.n_rx,
                                        C.byref(params), sub_ptr, n_sub, int(on_dev),
                                        C.byref(self._h)))
        self.n_seg = params.max_depth + (1 if params.capture == CAPTURE_SPHERE else 0)
        if ray_subset is not None:
            self.n_traced = n_sub
        elif params.launch == LAUNCH_DPS:
            self.n_traced = int(scene.info()["n_dps"])
        else:
            self.n_traced = int(params.n_rays)

    def counts(self):
        c = Counters()
        per = np.zeros(self.n_rx, np.int64)
        self.ctx._check(lib().nrt_result_counts(self._h, _np_ptr(per), C.byref(c)))
        return per, c.as_dict()

    def times(self):
        t = np.zeros(8, np.float32)
        self.ctx._check(lib().nrt_result_times(self._h, _np_ptr(t)))
        return {"vis": float(t[0]), "trace": float(t[2]), "dedup": float(t[3]),
                "validate": float(t[4]), "field": float(t[5]), "total": float(t[6]),
                "sizing_wait": float(t[7])}

    def paths(self):
        per, c = self.counts()
        n = c["paths"]
        out = {"key_hi": np.zeros(n, np.uint64), "key_lo": np.zeros(n, np.uint64),
               "rep": np.zeros(n, np.uint32), "rx": np.zeros(n, np.int32),
               "type": np.zeros(n, np.int32), "k": np.zeros(n, np.int32),
               "pts": np.zeros((n, 5, 3), np.float32), "mats": np.zeros((n, 5), np.uint8),
               "cos_theta": np.zeros((n, 5), np.float32), "geo": np.zeros(n, np.float32),
               "tau": np.zeros(n, np.float32), "a": np.zeros((n, 2), np.float32),
               "normal": np.zeros((n, 3), np.float32)}
        v = PathView(**{k: _np_ptr(a) for k, a in out.items()})
        self.ctx._check(lib().nrt_paths_read(self._h, C.byref(v)))
        return out

    def hits(self):
        S, n = self.n_seg, self.n_traced
        out = {"idx": np.zeros((n, S), np.int32), "dps": np.zeros((n, S), np.int32),
               "q": np.zeros((n, S, 3), np.float32), "n": np.zeros((n, S, 3), np.float32),
               "t": np.zeros((n, S), np.float32)}
        self.ctx._check(lib().nrt_hits_read(self._h, *[_np_ptr(out[k]) for k in
                                                        ("idx", "dps", "q", "n", "t")]))
        return out

    def vis(self):
        nd = self.scene.info()["n_dps"]
        words = (nd + 31) // 32
        bits = np.zeros((self.n_rx, words), np.uint32)
        self.ctx._check(lib().nrt_vis_read(self._h, _np_ptr(bits)))
        return np.unpackbits(bits.view(np.uint8), axis=1, bitorder="little")[:, :nd].astype(bool)

    def field(self):
        self.ctx._check(lib().nrt_field(self._h))

    def power(self):
        p = np.zeros(self.n_rx, np.float32)
        self.ctx._check(lib().nrt_field_read(self._h, _np_ptr(p)))
        return p

    def power_device(self, out_dev):
        """nrt_field_read_device: per-RX power (float64) into out_dev, a
        contiguous float64 CUDA tensor of at least n_rx elements on the
        context's device, copied on the context stream."""
        import torch

        if not (isinstance(out_dev, torch.Tensor) and out_dev.is_cuda):
            raise ValueError("out_dev must be a CUDA tensor")
        if out_dev.device.index != self.ctx.device:
            raise ValueError(f"out_dev is on cuda:{out_dev.device.index}, the context on "
                             f"cuda:{self.ctx.device}")
        if out_dev.dtype != torch.float64 or not out_dev.is_contiguous() \
                or out_dev.numel() < self.n_rx:
            raise ValueError(f"out_dev must be contiguous float64 with >= {self.n_rx} elements")
        self.ctx._check(lib().nrt_field_read_device(self._h, _P(out_dev.data_ptr())))

    def backward(self, dL_dP):
        g = np.ascontiguousarray(dL_dP, np.float32)
        L = self.scene.n_labels
        ge, gs, gc = (np.zeros(L, np.float32) for _ in range(3))
        self.ctx._check(lib().nrt_backward(self._h, _np_ptr(g), _np_ptr(ge), _np_ptr(gs),
                                           _np_ptr(gc)))
        return ge, gs, gc

    def keys(self):
        """Per-key validation summary (trace parameter keep_keys = 1):
        key_hi, key_lo, tried, rep (ray id, 0xFFFFFFFF = no valid candidate)."""
        n = self.counts()[1]["keys"]
        out = {"key_hi": np.zeros(n, np.uint64), "key_lo": np.zeros(n, np.uint64),
               "tried": np.zeros(n, np.uint32), "rep": np.zeros(n, np.uint32)}
        self.ctx._check(lib().nrt_keys_read(self._h, *[_np_ptr(out[k]) for k in
                                                        ("key_hi", "key_lo", "tried", "rep")]))
        return out

    def cfr(self, bandwidth=1.5e9, n_freq=129):
        """[n_rx, n_freq] complex channel frequency response around the
        simulation frequency (nrt_cfr)."""
        H = np.zeros((self.n_rx, n_freq, 2), np.float64)
        self.ctx._check(lib().nrt_cfr(self._h, float(bandwidth), int(n_freq), _np_ptr(H)))
        return H[..., 0] + 1j * H[..., 1]

    def cfr_backward(self, H_target, rx_weight=None, bandwidth=1.5e9):
        """Eq. 5 losses per RX and the gradient of sum_j w_j L_j (nrt_cfr_backward)."""
        T = np.asarray(H_target)
        n_freq = T.shape[1]
        Tr = np.ascontiguousarray(np.stack([T.real, T.imag], -1), np.float64)
        w = np.ascontiguousarray(np.ones(self.n_rx) if rx_weight is None else rx_weight, np.float32)
        L = self.scene.n_labels
        loss = np.zeros(self.n_rx, np.float64)
        ge, gs, gc = (np.zeros(L, np.float32) for _ in range(3))
        self.ctx._check(lib().nrt_cfr_backward(self._h, float(bandwidth), int(n_freq), _np_ptr(Tr),
                                               _np_ptr(w), _np_ptr(loss), _np_ptr(ge), _np_ptr(gs),
                                               _np_ptr(gc)))
        return loss, (ge, gs, gc)

    def ray_labels(self):
        """Per traced row (ascending ray id): 1 if the ray is a member of a valid
        specular key (needs trace parameter ray_labels = 1)."""
        out = np.zeros(self.n_traced, np.uint8)
        self.ctx._check(lib().nrt_ray_labels_read(self._h, _np_ptr(out)))
        return out

    def export_paths(self):
        """The paths as CUDA tensors (nrt_paths_export): key_hi, key_lo (int64
        bits of the uint64 words), rep (int32 bits of the uint32 ray id) and
        power |a|^2 (float64)."""
        import torch

        n = self.counts()[1]["paths"]
        dev = torch.device("cuda", self.ctx.device)
        out = {"key_hi": torch.empty(n, dtype=torch.int64, device=dev),
               "key_lo": torch.empty(n, dtype=torch.int64, device=dev),
               "rep": torch.empty(n, dtype=torch.int32, device=dev),
               "power": torch.empty(n, dtype=torch.float64, device=dev)}
        if n:
            self.ctx._check(lib().nrt_paths_export(self._h, *[_P(out[k].data_ptr()) for k in
                                                              ("key_hi", "key_lo", "rep", "power")]))
        return out

    def backward_noalloc(self, dL_dP_dev, grad_dev):
        """nrt_backward_noalloc on caller-owned device buffers (torch CUDA tensors):
        dL_dP_dev float32[n_rx] in, grad_dev float32[3 * n_labels] out.  Enqueued on
        the context stream; call ctx.sync() before reading grad_dev.  The C call
        cannot see the buffers' sizes, so they are checked here: both must be
        contiguous float32 CUDA tensors on the context's device, dL_dP_dev at
        least n_rx long and grad_dev at least 3 * n_labels long."""
        import torch

        for name, t, need in (("dL_dP_dev", dL_dP_dev, self.n_rx),
                              ("grad_dev", grad_dev, 3 * self.scene.n_labels)):
            if not (isinstance(t, torch.Tensor) and t.is_cuda):
                raise ValueError(f"{name} must be a CUDA tensor")
            if t.device.index != self.ctx.device:
                raise ValueError(f"{name} is on cuda:{t.device.index}, the context on "
                                 f"cuda:{self.ctx.device}")
            if t.dtype != torch.float32 or not t.is_contiguous():
                raise ValueError(f"{name} must be contiguous float32")
            if t.numel() < need:
                raise ValueError(f"{name} has {t.numel()} elements, needs {need}")
        self.ctx._check(lib().nrt_backward_noalloc(self._h, _P(dL_dP_dev.data_ptr()),
                                                   _P(grad_dev.data_ptr())))

    def close(self):
        if getattr(self, "_h", None):
            lib().nrt_result_free(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchResult(Result):
    """nrt_trace_batch: TX-RX pairs (one fixed RX) with per-pair ray budgets; the
    per-RX outputs of Result (counts, power, paths' rx field) are per pair."""

    def __init__(self, scene, tx, rx, budgets, params, packet=64, schedule=1, use_graph=False):
        self.scene = scene
        self.ctx = scene.ctx
        tx = np.ascontiguousarray(tx, np.float32).reshape(-1, 3)
        rx = np.ascontiguousarray(rx, np.float32).reshape(3)
        b = np.ascontiguousarray(budgets, np.int64).reshape(-1)
        self.n_rx = int(tx.shape[0])
        self.n_pairs = self.n_rx
        self.params = params
        self.budgets = b
        o = BatchOpts(int(packet), int(schedule), int(bool(use_graph)), 0)
        self._h = _P()
        self.ctx._check(lib().nrt_trace_batch(scene._h, _np_ptr(tx), _np_ptr(rx), _np_ptr(b),
                                              self.n_rx, C.byref(params), C.byref(o),
                                              C.byref(self._h)))
        self.n_seg = params.max_depth
        self.n_traced = int(b.sum())

    def replay(self, tx=None):
        p = None
        if tx is not None:
            tx = np.ascontiguousarray(tx, np.float32).reshape(self.n_pairs, 3)
            p = _np_ptr(tx)
        self.ctx._check(lib().nrt_batch_replay(self._h, p))

    def batch_times(self, paths=False):
        """(per-pair ms at which the pair's last ray was traced, total ms); with
        paths, also the per-pair ms at which its last path key was validated."""
        pm = np.zeros(self.n_pairs, np.float64)
        pv = np.zeros(self.n_pairs, np.float64)
        tot = C.c_float()
        self.ctx._check(lib().nrt_batch_times(self._h, _np_ptr(pm), C.byref(tot), _np_ptr(pv)))
        if paths:
            return pm, float(tot.value), pv
        return pm, float(tot.value)

    def autotune(self, configs, repeats=2):
        """configs: [(packet, schedule), ...]; returns (ms per config, best index)."""
        pk = np.ascontiguousarray([c[0] for c in configs], np.int32)
        sc = np.ascontiguousarray([c[1] for c in configs], np.int32)
        ms = np.zeros(len(configs), np.float32)
        best = C.c_int32()
        self.ctx._check(lib().nrt_autotune_batch(self._h, _np_ptr(pk), _np_ptr(sc), len(configs),
                                                 int(repeats), _np_ptr(ms), C.byref(best)))
        return ms, int(best.value)


# ---------------------------------------------------------------- learned proposal
N_MLP_PARAMS = 45569


def _dev(t):
    """Device pointer of a torch CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    if not (hasattr(t, "data_ptr") and t.is_cuda):
        raise TypeError("expected a torch CUDA tensor")
    return _P(t.data_ptr())


class Mlp:
    """The proposal network (nrt_mlp_*): FP32 master parameters and Adam state
    on the device, BF16 tensor-core contractions."""

    def __init__(self, ctx: Context, params, box_min, box_max, n_rays: int):
        self.ctx = ctx
        p = np.ascontiguousarray(params, np.float32)
        lo = np.ascontiguousarray(box_min, np.float32)
        hi = np.ascontiguousarray(box_max, np.float32)
        self._h = _P()
        ctx._check(lib().nrt_mlp_create(ctx._h, _np_ptr(p), int(p.size), _np_ptr(lo), _np_ptr(hi),
                                        int(n_rays), C.byref(self._h)))
        self.n_rays = int(n_rays)

    def params(self):
        out = np.zeros(N_MLP_PARAMS, np.float32)
        self.ctx._check(lib().nrt_mlp_params_read(self._h, _np_ptr(out)))
        return out

    def grads(self):
        out = np.zeros(N_MLP_PARAMS, np.float32)
        self.ctx._check(lib().nrt_mlp_grads_read(self._h, _np_ptr(out)))
        return out

    def state(self) -> dict:
        """Training state (nrt_mlp_state_read): params, adam_m, adam_v, step."""
        out = {k: np.zeros(N_MLP_PARAMS, np.float32) for k in ("params", "adam_m", "adam_v")}
        step = C.c_int64()
        self.ctx._check(lib().nrt_mlp_state_read(self._h, _np_ptr(out["params"]),
                                                 _np_ptr(out["adam_m"]), _np_ptr(out["adam_v"]),
                                                 C.byref(step)))
        out["step"] = int(step.value)
        return out

    def load_state(self, st: dict):
        """Restore a state from state() (nrt_mlp_state_write)."""
        arr = {k: np.ascontiguousarray(st[k], np.float32) for k in ("params", "adam_m", "adam_v")}
        for k, a in arr.items():
            if a.size != N_MLP_PARAMS:
                raise ValueError(f"{k}: {a.size} values, expected {N_MLP_PARAMS}")
        self.ctx._check(lib().nrt_mlp_state_write(self._h, _np_ptr(arr["params"]),
                                                  _np_ptr(arr["adam_m"]), _np_ptr(arr["adam_v"]),
                                                  int(st["step"])))

    def save(self, path):
        """Checkpoint the training state to an .npz file."""
        np.savez(path, **self.state())

    def restore(self, path):
        """Resume from a checkpoint written by save()."""
        with np.load(path) as z:
            self.load_state({k: z[k] for k in ("params", "adam_m", "adam_v", "step")})

    def features(self, tx, ray_ids_dev, n, out_dev, sync=True):
        t = np.ascontiguousarray(tx, np.float32).reshape(3)
        self.ctx._check(lib().nrt_mlp_features(self._h, _np_ptr(t), _dev(ray_ids_dev), int(n),
                                               _dev(out_dev)))
        if sync:
            self.ctx.sync()

    def score(self, tx, ray_ids_dev, n, logits_dev, sync=True):
        """Logits into logits_dev; the work is enqueued on the context stream
        and, with sync, waited for before returning."""
        t = np.ascontiguousarray(tx, np.float32).reshape(3)
        self.ctx._check(lib().nrt_mlp_score(self._h, _np_ptr(t), _dev(ray_ids_dev), int(n),
                                            _dev(logits_dev)))
        if sync:
            self.ctx.sync()

    def train(self, tx_table_dev, tx_index_dev, ray_id_dev, label_dev, order_dev=None, start=0,
              steps=1, lr=1e-3, batch=4096, pos_weight=1.0, beta1=0.9, beta2=0.999, eps=1e-8):
        """Adam steps on device samples (torch CUDA tensors); returns the per-step losses."""
        n = int(ray_id_dev.shape[0])
        o = MlpTrainOpts(lr, beta1, beta2, eps, pos_weight, int(batch))
        loss = np.zeros(int(steps), np.float32)
        self.ctx._check(lib().nrt_mlp_train(self._h, _dev(tx_table_dev), int(tx_table_dev.shape[0]),
                                            _dev(tx_index_dev), _dev(ray_id_dev), _dev(label_dev),
                                            n, _dev(order_dev), int(start), int(steps), C.byref(o),
                                            _np_ptr(loss)))
        return loss

    def close(self):
        if getattr(self, "_h", None):
            lib().nrt_mlp_free(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def shard_merge(ctx: Context, key_hi, key_lo, shard, rep, power=None, n_rx=0, tried=None,
                rep_tries=0):
    """nrt_shard_merge on CUDA tensors (int64 key words, int32 shard / rep /
    tried, float64 power): returns (win uint8 tensor, per-RX power float64
    tensor or None)."""
    import torch

    n = int(key_hi.shape[0])
    dev = key_hi.device
    for t in (key_hi, key_lo, shard, rep) + ((tried,) if tried is not None else ()):
        if not (t.is_cuda and t.is_contiguous() and t.shape[0] == n):
            raise ValueError("shard_merge: contiguous CUDA tensors of one length expected")
    win = torch.empty(n, dtype=torch.uint8, device=dev)
    pout = torch.empty(n_rx, dtype=torch.float64, device=dev) if power is not None else None
    ctx._check(lib().nrt_shard_merge(ctx._h, n, _dev(key_hi), _dev(key_lo), _dev(shard),
                                     _dev(tried), _dev(rep), int(rep_tries), _dev(power), int(n_rx),
                                     _dev(win), _dev(pout)))
    return win, pout


def propose(ctx: Context, logits_dev, k_top: int, k_uniform: int, seed: int, ids_dev) -> int:
    """nrt_propose: selected launch indices into ids_dev (uint32 capacity
    k_top + k_uniform); returns how many."""
    n_out = C.c_int64()
    ctx._check(lib().nrt_propose(ctx._h, _dev(logits_dev), int(logits_dev.shape[0]), int(k_top),
                                 int(k_uniform), C.c_uint64(seed), _dev(ids_dev), C.byref(n_out)))
    return int(n_out.value)


def gemm_bf16(ctx: Context, A, B, C_out, accumulate=False, k_split=0):
    """C_out[M][N] (+)= A[M][K] B[N][K]^T on the tensor cores; A, B torch bfloat16
    CUDA tensors (row-major), C_out float32."""
    M, K = A.shape
    N = B.shape[0]
    ctx._check(lib().nrt_gemm_bf16(ctx._h, _dev(A), int(A.stride(0)), _dev(B), int(B.stride(0)),
                                   _dev(C_out), int(C_out.stride(0)), int(M), int(N), int(K),
                                   int(bool(accumulate)), int(k_split)))
