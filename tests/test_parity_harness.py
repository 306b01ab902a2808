"""The parity harness itself, on the CPU: the vectorised path comparison
(used for full-size launches) against its key-by-key form on inputs made
by the oracle alone -- the oracle's own paths rounded to float32 as a
stand-in for a GPU result, then with planted differences: a dropped
uncertain key must be explained, a coefficient moved beyond the fixed
tolerance must be caught, and both forms must agree on every count."""
import copy

import numpy as np
import pytest

import oracle
from parity import compare_paths, compare_paths_loop

NONE = 0xFFFFFFFF


@pytest.fixture(scope="module")
def room_sim(room):
    osc = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, rho=0.0625, r_p=0.05)
    rx = np.array([[4.0, 3.0, 1.2], [1.5, 3.2, 1.0], [4.2, 0.8, 2.1]], np.float32)
    p = oracle.SimParams(max_depth=2, capture=1, diffuse=1, n_rays=3000, rep_tries=8,
                         delta=1e-5 * room.diag)
    osim = oracle.OracleSim(osc, room.tx, rx, p)
    mats = (np.array([5.3, 3.0]), np.array([0.03, 0.01]), np.array([0.3, 0.2]))
    return osim, mats


def _as_gpu(osim, mats):
    O = osim.paths()
    a, _ = osim.field(*mats)
    rep = O["rep"].copy()
    rep[rep < 0] = NONE
    return {"key_hi": O["hi"].copy(), "key_lo": O["lo"].copy(), "rep": rep.astype(np.uint32),
            "rx": O["j"].copy(), "type": O["type"].copy(), "k": O["k"].copy(),
            "a": np.stack([a.real, a.imag], 1).astype(np.float32),
            "tau": O["tau"].astype(np.float32)}


def _same_summary(a, b):
    """Equal counts; floats equal up to summation order."""
    def flat(s, pre=""):
        out = {}
        for k, v in s.items():
            if isinstance(v, dict):
                out.update(flat(v, pre + k + "."))
            else:
                out[pre + k] = v
        return out
    fa, fb = flat(copy.deepcopy(a)), flat(copy.deepcopy(b))
    assert fa.keys() == fb.keys()
    for k in fa:
        if isinstance(fa[k], (int, np.integer)):
            assert fa[k] == fb[k], k
        else:
            assert fa[k] == pytest.approx(fb[k], rel=1e-9, abs=1e-12), k


def test_vectorised_harness_equals_loop(room_sim):
    osim, mats = room_sim
    gp = _as_gpu(osim, mats)
    a = compare_paths(gp, osim, *mats)
    b = compare_paths_loop(gp, osim, *mats)
    assert a["matched"] > 200 and a["explained"] == 0 and a["field_checked"] > 10
    _same_summary(a, b)
    # float32 rounding of a and tau alone stays far inside the fixed tolerances
    assert a["max_da"] < 1e-6 and a["max_dtau"] < 1e-6


def test_dropped_uncertain_key_is_explained(room_sim):
    osim, mats = room_sim
    gp = _as_gpu(osim, mats)
    O = osim.paths()
    unc = np.nonzero((O["certain"] == 0) & (O["k"] > 0))[0]
    if unc.size == 0:
        pytest.skip("no uncertain path in this sample")
    keep = np.ones(len(gp["rep"]), bool)
    keep[unc[0]] = False
    sub = {k: v[keep] for k, v in gp.items()}
    a = compare_paths(sub, osim, *mats)
    b = compare_paths_loop(sub, osim, *mats)
    assert a["explained"] == b["explained"] >= 1
    _same_summary(a, b)


def test_moved_coefficient_is_caught_when_strict(room_sim):
    osim, mats = room_sim
    gp = _as_gpu(osim, mats)
    O = osim.paths()
    a_sens, _ = osim.path_sens(*mats)
    cand = np.nonzero((O["certain"] != 0) & (a_sens >= 0) & (O["k"] > 0) & (O["type"] == 0))[0]
    assert cand.size
    i = int(cand[0])
    gp["a"][i] *= np.float32(1.0 + 3e-4)
    for f in (compare_paths, compare_paths_loop):
        with pytest.raises(AssertionError):
            f(gp, osim, *mats, strict=("specular", "los"))
    # a changed representative that the oracle cannot explain is caught too
    gp2 = _as_gpu(osim, mats)
    j = int(cand[-1])
    gp2["rep"][j] = np.uint32(999_999)
    for f in (compare_paths, compare_paths_loop):
        with pytest.raises(AssertionError):
            f(gp2, osim, *mats)
