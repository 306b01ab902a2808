"""FP64 CPU oracle for the point-cloud radio ray tracer (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does.  The
oracle shares no code with the CUDA library: it is a separate C++17 source
(``nrt_oracle.cpp``) compiled with g++ and loaded through ctypes.

Functions follow the paper (Vaara et al., arXiv 2507.04021):
Sec. II-A voxelisation, Sec. II-B path computation, Sec. II-C ray/disc
intersection with Eq. 3 / Eq. 4; EM formulas are readings (Fresnel with the
ITU-R P.2040 permittivity, effective roughness, Lambertian lobe).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nrt_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    """The oracle library: built from nrt_oracle.cpp, or, when the environment
    names one in NRT_ORACLE_LIB, that prebuilt file instead (the
    planted-mistake tests load deliberately broken copies this way)."""
    global _lib
    if _lib is None:
        _lib = C.CDLL(os.environ.get("NRT_ORACLE_LIB") or build())
        _declare(_lib)
    return _lib


class OrcParams(C.Structure):
    _fields_ = [
        ("max_depth", C.c_int32), ("capture", C.c_int32), ("diffuse", C.c_int32),
        ("pol", C.c_int32), ("kappa", C.c_int32), ("rep_tries", C.c_int32),
        ("validate", C.c_int32), ("n_threads", C.c_int32), ("n_rays", C.c_int64),
        ("r_rx", C.c_double), ("t_min", C.c_double), ("delta", C.c_double),
        ("t_a_deg", C.c_double), ("t_d", C.c_double), ("freq", C.c_double),
        ("launch", C.c_int32), ("diffraction", C.c_int32),
    ]


_P = C.c_void_p
_D = C.POINTER(C.c_double)


def _declare(L):
    L.orc_scene_create.restype = _P
    L.orc_scene_create.argtypes = [_P, _P, _P, _P, C.c_int64, C.c_double, C.c_double,
                                   C.c_double, C.c_double, C.c_double]
    L.orc_scene_destroy.argtypes = [_P]
    L.orc_scene_n_dps.restype = C.c_int64
    L.orc_scene_n_dps.argtypes = [_P]
    L.orc_scene_bmin.argtypes = [_P, _P]
    L.orc_scene_dps.argtypes = [_P, _P, _P, _P]
    L.orc_scene_point_dps.argtypes = [_P, _P]
    L.orc_cast.restype = C.c_int
    L.orc_cast.argtypes = [_P, _P, _P, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_int,
                           _P, _P, _P, _P]
    L.orc_fib_dirs.argtypes = [C.c_int64, _P, C.c_int64, _P]
    L.orc_sim_run.restype = _P
    L.orc_sim_run.argtypes = [_P, _P, _P, C.c_int, C.POINTER(OrcParams), _P, C.c_int64]
    L.orc_sim_destroy.argtypes = [_P]
    L.orc_sim_n_seg.restype = C.c_int
    L.orc_sim_n_seg.argtypes = [_P]
    L.orc_sim_hits.argtypes = [_P] + [_P] * 9
    L.orc_sim_los.argtypes = [_P, _P, _P]
    L.orc_sim_n_vis.restype = C.c_int64
    L.orc_sim_n_vis.argtypes = [_P]
    L.orc_sim_vis.argtypes = [_P, _P, _P, _P, _P]
    L.orc_vis_pairs.argtypes = [_P, _P, _P, _P, C.c_int64, C.c_double, C.c_double, _P, _P]
    L.orc_sim_n_keys.restype = C.c_int64
    L.orc_sim_n_keys.argtypes = [_P]
    L.orc_sim_keys.argtypes = [_P] + [_P] * 8
    L.orc_sim_n_paths.restype = C.c_int64
    L.orc_sim_n_paths.argtypes = [_P]
    L.orc_sim_paths.argtypes = [_P] + [_P] * 13
    L.orc_cast_sdf.restype = C.c_int
    L.orc_cast_sdf.argtypes = [_P, _P, _P, C.c_double, C.c_double, C.c_double, C.c_double, _P,
                               C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.orc_sim_diffraction.restype = None
    L.orc_sim_diffraction.argtypes = [_P, C.c_int64, _P, _P, _P, _P, _P, _P]
    L.orc_utd_F.restype = None
    L.orc_utd_F.argtypes = [C.c_double, _D, _D]
    L.orc_diffraction_amplitude.restype = C.c_int
    L.orc_diffraction_amplitude.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, C.c_double, C.c_int,
                                            _D, _D]
    L.orc_diffraction_geometry.restype = C.c_int
    L.orc_diffraction_geometry.argtypes = [_P, _P, _P, _P, _P, _P, _P]
    L.orc_sim_path_normals.restype = None
    L.orc_sim_path_normals.argtypes = [_P, _P]
    L.orc_jones_amplitude.restype = None
    L.orc_jones_amplitude.argtypes = [_P, _P, _P, C.c_int, C.c_int, _P, _P, C.POINTER(C.c_double),
                                      C.POINTER(C.c_double)]
    L.orc_sim_path_grads.restype = None
    L.orc_sim_path_grads.argtypes = [_P, _P, _P, _P, C.c_int, _P]
    L.orc_sim_shadow_disc_counts.restype = None
    L.orc_sim_shadow_disc_counts.argtypes = [_P, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.orc_sim_ray_labels.restype = None
    L.orc_sim_ray_labels.argtypes = [_P, _P, _P]
    L.orc_sim_cand_status.restype = C.c_int
    L.orc_sim_cand_status.argtypes = [_P, C.c_uint64, C.c_uint64, C.c_int64]
    L.orc_sim_n_tried.restype = C.c_int64
    L.orc_sim_n_tried.argtypes = [_P]
    L.orc_sim_tried.argtypes = [_P, _P, _P, _P]
    L.orc_sim_field.argtypes = [_P, _P, _P, _P, _P, _P, _P, C.c_int]
    L.orc_sim_backward.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, C.c_int]
    for name in ("orc_fresnel",):
        getattr(L, name).argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int,
                                     _D, _D]
    L.orc_dfresnel.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, _D, _D]
    L.orc_fresnel_eta.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, _D, _D]
    L.orc_max_threads.restype = C.c_int
    L.orc_sim_disc_counts.argtypes = [_P, _P]
    L.orc_sim_cast_counts.argtypes = [_P, _P]
    L.orc_sim_path_sens.argtypes = [_P, _P, _P, _P, _P, _P]
    L.orc_sim_hit_sens.argtypes = [_P, _P, _P]
    L.orc_vis_disc_counts.argtypes = [_P, _P, _P, _P, C.c_int64, C.c_double, _P]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------------------
class OracleScene:
    """Voxelised point cloud (Sec. II-A) with an optional uniform acceleration grid.

    grid_cell <= 0 selects brute force over all discs.  band_cap bounds the
    ambiguity band and sets how far around each disc the grid lists it.
    """

    def __init__(self, pos, nrm, surf, mat, rho=0.0625, r_p=0.015, lambda_d=100.0,
                 grid_cell=0.0, band_cap=5e-3):
        self.pos = np.ascontiguousarray(pos, np.float32)
        self.nrm = np.ascontiguousarray(nrm, np.float32)
        self.surf = np.ascontiguousarray(surf, np.uint16)
        self.mat = np.ascontiguousarray(mat, np.uint8)
        self.rho, self.r_p, self.lambda_d = float(rho), float(r_p), float(lambda_d)
        self._h = lib().orc_scene_create(_ptr(self.pos), _ptr(self.nrm), _ptr(self.surf),
                                         _ptr(self.mat), self.pos.shape[0], self.rho, self.r_p,
                                         self.lambda_d, float(grid_cell), float(band_cap))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_scene_destroy(h)
            self._h = None

    @property
    def n_dps(self) -> int:
        return int(lib().orc_scene_n_dps(self._h))

    def bmin(self) -> np.ndarray:
        out = np.zeros(3, np.float32)
        lib().orc_scene_bmin(self._h, _ptr(out))
        return out

    def dps(self):
        """(voxel [D,3] int32, count [D], reception point [D,3] float64), lexicographic voxel order."""
        n = self.n_dps
        vox = np.zeros((n, 3), np.int32)
        cnt = np.zeros(n, np.int32)
        recv = np.zeros((n, 3), np.float64)
        lib().orc_scene_dps(self._h, _ptr(vox), _ptr(cnt), _ptr(recv))
        return vox, cnt, recv

    def point_dps(self) -> np.ndarray:
        out = np.zeros(self.pos.shape[0], np.int32)
        lib().orc_scene_point_dps(self._h, _ptr(out))
        return out

    def cast(self, o, d, skip_dps=-1, t_min=1e-3, t_max=np.inf, delta=0.0, weighted=True):
        """One closest-hit cast; returns dict or None on a miss."""
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        out = np.zeros(8, np.float64)
        idx = np.zeros(1, np.int64)
        dps = np.zeros(1, np.int32)
        amb = np.zeros(1, np.int32)
        hit = lib().orc_cast(self._h, _ptr(o), _ptr(d), int(skip_dps), float(t_min), float(t_max),
                             float(delta), int(weighted), _ptr(out), _ptr(idx), _ptr(dps), _ptr(amb))
        res = {"hit": bool(hit), "t": out[0], "q": out[1:4].copy(), "n": out[4:7].copy(),
               "cos_in": out[7], "idx": int(idx[0]), "dps": int(dps[0]), "amb": bool(amb[0])}
        return res

    def cast_sdf(self, o, d, sigma, t_min=1e-3, t_max=np.inf, delta=0.0):
        """Closest hit under the SDF model of Eq. 2 (the ablation); dict or None."""
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        out = np.zeros(7, np.float64)
        dps, lab, amb = C.c_int32(), C.c_int32(), C.c_int32()
        hit = lib().orc_cast_sdf(self._h, _ptr(o), _ptr(d), float(t_min), float(t_max),
                                 float(sigma), float(delta), _ptr(out), C.byref(dps), C.byref(lab),
                                 C.byref(amb))
        return {"hit": bool(hit), "t": out[0], "q": out[1:4].copy(), "n": out[4:7].copy(),
                "dps": int(dps.value), "labels": int(lab.value), "amb": bool(amb.value)}

    def vis_disc_counts(self, rx, j, dps, t_min=1e-3):
        rx = np.ascontiguousarray(rx, np.float64)
        j = np.ascontiguousarray(j, np.int32)
        dps = np.ascontiguousarray(dps, np.int32)
        out = np.zeros(j.shape[0], np.int64)
        lib().orc_vis_disc_counts(self._h, _ptr(rx), _ptr(j), _ptr(dps), j.shape[0],
                                  float(t_min), _ptr(out))
        return out

    def vis_pairs(self, rx, j, dps, t_min=1e-3, delta=0.0):
        rx = np.ascontiguousarray(rx, np.float64)
        j = np.ascontiguousarray(j, np.int32)
        dps = np.ascontiguousarray(dps, np.int32)
        bit = np.zeros(j.shape[0], np.int32)
        amb = np.zeros(j.shape[0], np.int32)
        lib().orc_vis_pairs(self._h, _ptr(rx), _ptr(j), _ptr(dps), j.shape[0], float(t_min),
                            float(delta), _ptr(bit), _ptr(amb))
        return bit.astype(bool), amb.astype(bool)


def fib_dirs(n_rays: int, ids) -> np.ndarray:
    ids = np.ascontiguousarray(ids, np.int64)
    out = np.zeros((ids.shape[0], 3), np.float64)
    lib().orc_fib_dirs(int(n_rays), _ptr(ids), ids.shape[0], _ptr(out))
    return out


@dataclass
class SimParams:
    max_depth: int = 2
    capture: int = 0          # 0 RX sphere, 1 visibility matrix
    diffuse: int = 0
    pol: int = 0              # 0 TE, 1 TM, 2 vector (Jones chain)
    kappa: int = 10
    rep_tries: int = 0        # candidates tried per key in ray order; 0 = all (the paper's rule)
    validate: int = 1
    n_threads: int = 0
    n_rays: int = 20000
    r_rx: float = 0.1
    t_min: float = 1e-3
    delta: float = 0.0
    t_a_deg: float = 1.0
    t_d: float = 0.01
    freq: float = 28e9
    launch: int = 0           # 0 Fibonacci sphere, 1 one ray per DPS (Morton order)
    diffraction: int = 0      # 1: single-bounce edge diffraction over the given edges

    def to_c(self) -> OrcParams:
        return OrcParams(**{k: getattr(self, k) for k, _ in OrcParams._fields_})


class OracleSim:
    """One full simulation for one TX (Sec. II-B), run on construction."""

    def __init__(self, scene: OracleScene, tx, rx, params: SimParams, ray_ids=None, edges=None):
        self.scene = scene
        self.params = params
        self.tx = np.ascontiguousarray(tx, np.float64).reshape(3)
        self.rx = np.ascontiguousarray(rx, np.float64).reshape(-1, 3)
        if ray_ids is None:
            ray_ids = np.arange(scene.n_dps if params.launch == 1 else params.n_rays, dtype=np.int64)
        self.ray_ids = np.ascontiguousarray(ray_ids, np.int64)
        cp = params.to_c()
        if params.launch == 1:  # one ray per DPS: the launch has n_dps rays
            cp.n_rays = scene.n_dps
        self._h = lib().orc_sim_run(scene._h, _ptr(self.tx), _ptr(self.rx), self.rx.shape[0],
                                    C.byref(cp), _ptr(self.ray_ids), self.ray_ids.shape[0])
        if params.diffraction and edges is not None and len(edges.m0) > 0:
            f = lambda x: np.ascontiguousarray(x, np.float32)  # noqa: E731
            u = lambda x: np.ascontiguousarray(x, np.uint8)  # noqa: E731
            self._edges = (f(edges.a), f(edges.b), f(edges.n0), f(edges.n1), u(edges.m0), u(edges.m1))
            lib().orc_sim_diffraction(self._h, len(edges.m0), *[_ptr(x) for x in self._edges])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_sim_destroy(h)
            self._h = None

    def hits(self):
        n, S = self.ray_ids.shape[0], lib().orc_sim_n_seg(self._h)
        r = {
            "idx": np.zeros((n, S), np.int64), "dps": np.zeros((n, S), np.int32),
            "t": np.zeros((n, S)), "q": np.zeros((n, S, 3)), "n": np.zeros((n, S, 3)),
            "cos_in": np.zeros((n, S)), "amb": np.zeros((n, S), np.int32),
            "excl": np.zeros(n, np.int32), "n_hits": np.zeros(n, np.int32),
        }
        lib().orc_sim_hits(self._h, *[_ptr(r[k]) for k in
                                      ("idx", "dps", "t", "q", "n", "cos_in", "amb", "excl", "n_hits")])
        return r

    def los(self):
        M = self.rx.shape[0]
        clear = np.zeros(M, np.int32)
        amb = np.zeros(M, np.int32)
        lib().orc_sim_los(self._h, _ptr(clear), _ptr(amb))
        return clear.astype(bool), amb.astype(bool)

    def vis(self):
        n = lib().orc_sim_n_vis(self._h)
        j, d, b, a = (np.zeros(n, np.int32) for _ in range(4))
        lib().orc_sim_vis(self._h, _ptr(j), _ptr(d), _ptr(b), _ptr(a))
        return j, d, b.astype(bool), a.astype(bool)

    def keys(self):
        n = lib().orc_sim_n_keys(self._h)
        r = {"hi": np.zeros(n, np.uint64), "lo": np.zeros(n, np.uint64),
             "n_tried": np.zeros(n, np.int32), "n_cand": np.zeros(n, np.int64),
             "rep": np.zeros(n, np.int64), "valid": np.zeros(n, np.int32),
             "certain": np.zeros(n, np.int32), "path": np.zeros(n, np.int32)}
        lib().orc_sim_keys(self._h, *[_ptr(r[k]) for k in
                                      ("hi", "lo", "n_tried", "n_cand", "rep", "valid", "certain", "path")])
        return r

    def paths(self):
        n = lib().orc_sim_n_paths(self._h)
        r = {"hi": np.zeros(n, np.uint64), "lo": np.zeros(n, np.uint64),
             "j": np.zeros(n, np.int32), "type": np.zeros(n, np.int32), "k": np.zeros(n, np.int32),
             "rep": np.zeros(n, np.int64), "pts": np.zeros((n, 5, 3)),
             "mats": np.zeros((n, 5), np.int32), "cos": np.zeros((n, 5)),
             "geo": np.zeros(n), "tau": np.zeros(n), "length": np.zeros(n),
             "certain": np.zeros(n, np.int32)}
        lib().orc_sim_paths(self._h, *[_ptr(r[k]) for k in
                                       ("hi", "lo", "j", "type", "k", "rep", "pts", "mats", "cos",
                                        "geo", "tau", "length", "certain")])
        return r

    def path_normals(self) -> np.ndarray:
        """[n_paths, 3] scatter-point normal of each diffuse path (0 otherwise)."""
        out = np.zeros((lib().orc_sim_n_paths(self._h), 3))
        lib().orc_sim_path_normals(self._h, _ptr(out))
        return out

    def cast_counts(self) -> dict:
        out = np.zeros(4, np.int64)
        lib().orc_sim_cast_counts(self._h, _ptr(out))
        return {"segments": int(out[0]), "vis_casts": int(out[1]),
                "validation_casts": int(out[2]), "los_casts": int(out[3])}

    def disc_counts(self) -> np.ndarray:
        """[n_rays, n_seg] discs in DPS boxes each cast enters before its hit (-1: no cast)."""
        out = np.zeros((self.ray_ids.shape[0], lib().orc_sim_n_seg(self._h)), np.int64)
        lib().orc_sim_disc_counts(self._h, _ptr(out))
        return out

    def path_grads(self, eps_r, sigma, scat) -> np.ndarray:
        """[n_paths, 3, n_labels] complex d a_p / d(eps_r, sigma, S)_l."""
        eps = np.ascontiguousarray(eps_r, np.float64)
        sig = np.ascontiguousarray(sigma, np.float64)
        sca = np.ascontiguousarray(scat, np.float64)
        L = eps.shape[0]
        n = lib().orc_sim_n_paths(self._h)
        out = np.zeros((n, 3, L, 2))
        lib().orc_sim_path_grads(self._h, _ptr(eps), _ptr(sig), _ptr(sca), L, _ptr(out))
        return out[..., 0] + 1j * out[..., 1]

    def shadow_disc_counts(self, stride: int = 1):
        """(discs entered, casts) of the diffuse validation shadow casts of every
        `stride`-th tried diffuse candidate."""
        s = C.c_int64()
        n = C.c_int64()
        lib().orc_sim_shadow_disc_counts(self._h, int(stride), C.byref(s), C.byref(n))
        return int(s.value), int(n.value)

    def cand_status(self, hi, lo, ray) -> int:
        """0 certainly not a candidate, 1 certainly a candidate, 2 uncertain."""
        return int(lib().orc_sim_cand_status(self._h, int(hi), int(lo), int(ray)))

    def ray_labels(self):
        """Per row (ray_ids order): 1 if the ray is a member of a valid
        specular key; and whether that is ambiguous under rounding."""
        n = self.ray_ids.shape[0]
        lab = np.zeros(n, np.int32)
        amb = np.zeros(n, np.int32)
        lib().orc_sim_ray_labels(self._h, _ptr(lab), _ptr(amb))
        return lab.astype(np.uint8), amb.astype(bool)

    def tried(self):
        """Flattened tried lists (ray, valid, ambiguous) in key order; see keys()['n_tried']."""
        n = lib().orc_sim_n_tried(self._h)
        ray = np.zeros(n, np.int64)
        valid = np.zeros(n, np.int32)
        amb = np.zeros(n, np.int32)
        lib().orc_sim_tried(self._h, _ptr(ray), _ptr(valid), _ptr(amb))
        return ray, valid.astype(bool), amb.astype(bool)

    def field(self, eps_r, sigma, scat):
        eps = np.ascontiguousarray(eps_r, np.float64)
        sig = np.ascontiguousarray(sigma, np.float64)
        sca = np.ascontiguousarray(scat, np.float64)
        n = lib().orc_sim_n_paths(self._h)
        M = self.rx.shape[0]
        a_re, a_im, P = np.zeros(n), np.zeros(n), np.zeros(M)
        lib().orc_sim_field(self._h, _ptr(eps), _ptr(sig), _ptr(sca), _ptr(a_re), _ptr(a_im),
                            _ptr(P), M)
        return a_re + 1j * a_im, P

    def path_sens(self, eps_r, sigma, scat):
        """(a_sens, tau_sens) per path from the shadow trajectories; -1 = fragile."""
        eps = np.ascontiguousarray(eps_r, np.float64)
        sig = np.ascontiguousarray(sigma, np.float64)
        sca = np.ascontiguousarray(scat, np.float64)
        n = lib().orc_sim_n_paths(self._h)
        a, t = np.zeros(n), np.zeros(n)
        lib().orc_sim_path_sens(self._h, _ptr(eps), _ptr(sig), _ptr(sca), _ptr(a), _ptr(t))
        return a, t

    def hit_sens(self):
        n, S = self.ray_ids.shape[0], lib().orc_sim_n_seg(self._h)
        dq, dn = np.zeros((n, S)), np.zeros((n, S))
        lib().orc_sim_hit_sens(self._h, _ptr(dq), _ptr(dn))
        return dq, dn

    def backward(self, eps_r, sigma, scat, dL_dP):
        eps = np.ascontiguousarray(eps_r, np.float64)
        sig = np.ascontiguousarray(sigma, np.float64)
        sca = np.ascontiguousarray(scat, np.float64)
        g = np.ascontiguousarray(dL_dP, np.float64)
        L = eps.shape[0]
        ge, gs, gc = np.zeros(L), np.zeros(L), np.zeros(L)
        lib().orc_sim_backward(self._h, _ptr(eps), _ptr(sig), _ptr(sca), _ptr(g), _ptr(ge),
                               _ptr(gs), _ptr(gc), L)
        return ge, gs, gc


def fresnel(eps_r, sigma, freq, cos_t, pol=0) -> complex:
    re, im = C.c_double(), C.c_double()
    lib().orc_fresnel(eps_r, sigma, freq, cos_t, pol, C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def fresnel_eta(eta: complex, cos_t, pol=0) -> complex:
    re, im = C.c_double(), C.c_double()
    lib().orc_fresnel_eta(eta.real, eta.imag, cos_t, pol, C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def dfresnel_deta(eta: complex, cos_t, pol=0) -> complex:
    re, im = C.c_double(), C.c_double()
    lib().orc_dfresnel(eta.real, eta.imag, cos_t, pol, C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def jones_amplitude(tx, rx, pts, D, diffuse=False, nd=(0.0, 0.0, 1.0)) -> complex:
    """Vector-polarisation a / geo of an explicit path (pol = 2 reading):
    pts [k,3] interaction points, D [k,2] complex (c Gamma_TE, c Gamma_TM)."""
    tx = np.ascontiguousarray(tx, np.float64)
    rx = np.ascontiguousarray(rx, np.float64)
    pts = np.ascontiguousarray(np.asarray(pts, np.float64).reshape(-1, 3))
    D = np.asarray(D, np.complex128).reshape(-1, 2)
    Dr = np.ascontiguousarray(np.stack([D.real, D.imag], -1))
    nd = np.ascontiguousarray(nd, np.float64)
    re, im = C.c_double(), C.c_double()
    lib().orc_jones_amplitude(_ptr(tx), _ptr(rx), _ptr(pts), pts.shape[0], int(diffuse), _ptr(nd),
                              _ptr(Dr), C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def utd_F(x: float) -> complex:
    """UTD transition function F(x) = 2j sqrt(x) e^{jx} int_{sqrt x}^inf e^{-j t^2} dt."""
    re, im = C.c_double(), C.c_double()
    lib().orc_utd_F(float(x), C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def _d3(x):
    return np.ascontiguousarray(x, np.float64).reshape(3)


def diffraction_amplitude(tx, rx, a, b, n0, n1, eta0, eta1, freq=28e9, pol=0):
    """a of the single-bounce diffracted path TX -> edge (a, b; face normals
    n0, n1; face permittivities eta0, eta1) -> RX, or None without a path."""
    e0 = np.array([complex(eta0).real, complex(eta0).imag])
    e1 = np.array([complex(eta1).real, complex(eta1).imag])
    re, im = C.c_double(), C.c_double()
    args = [_d3(v) for v in (tx, rx, a, b, n0, n1)] + [e0, e1]
    ok = lib().orc_diffraction_amplitude(*[_ptr(v) for v in args], float(freq), int(pol),
                                         C.byref(re), C.byref(im))
    return complex(re.value, im.value) if ok else None


def diffraction_geometry(tx, rx, a, b, n0, n1):
    """(ok, D, s', s, phi', phi, n, sin b0) of the diffracted path."""
    out = np.zeros(9)
    args = [_d3(v) for v in (tx, rx, a, b, n0, n1)]
    ok = lib().orc_diffraction_geometry(*[_ptr(v) for v in args], _ptr(out))
    return bool(ok), out[:3].copy(), *[float(v) for v in out[3:]]


def max_threads() -> int:
    return int(lib().orc_max_threads())
