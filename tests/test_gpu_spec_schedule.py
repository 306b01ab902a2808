"""The two schedules of the specular refinement (Sec. II-B-2) give the same
paths on these workloads (the waves are opt-in: two compiled copies of the
Eq. 4 normal round differently in rare cases, and on the office's
DPS-directed launch a representative they chose failed the re-refinement
check).  The persistent pass refines each (key, candidate) item in one lane
from start to end; the waves keep each candidate's planes and image-method
points in device memory and cast every leg in a lean kernel, deferring a
key's tail items until its first candidates are done.  Both take the same
decisions per candidate and keep the lowest valid rank per key, so paths,
counts and received power are bit-identical (the validation cast count, a
measure of work that the early stop makes timing-dependent, aside)."""
import numpy as np
import pytest

from paper_2507_04021_gb300 import nrt

pytestmark = pytest.mark.gpu

WAVES, PERSISTENT = 1, 2


def _run(sc, office, kp, ids, schedule):
    r = sc.trace(office.tx, office.rx, nrt.default_trace_params(spec_waves=schedule, **kp),
                 ray_subset=ids)
    out = (r.paths(), r.counts(), r.power())
    r.close()
    return out


def _same(a, b):
    (pa, (na, ca), wa), (pb, (nb, cb), wb) = a, b
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k
    assert np.array_equal(na, nb)
    for k in ("segments", "vis_casts", "candidates", "keys", "paths"):
        assert ca[k] == cb[k], k
    assert ca["error_flags"] == 0 and cb["error_flags"] == 0
    assert np.array_equal(wa, wb)


@pytest.mark.parametrize("rep_tries", [0, 8])
def test_waves_match_the_persistent_pass_on_the_office(office, rep_tries):
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, office.pos, office.nrm, office.surf, office.mat, r_p=0.015)
    sc.set_materials(office.eps_r, office.sigma, office.scat)
    kp = dict(max_depth=5, capture=nrt.CAPTURE_VIS, diffuse=1, n_rays=1_000_000,
              rep_tries=rep_tries)
    ids = np.arange(0, 1_000_000, 3, dtype=np.uint32)
    a = _run(sc, office, kp, ids, WAVES)
    b = _run(sc, office, kp, ids, PERSISTENT)
    assert len(a[0]["key_hi"]) > 100000
    _same(a, b)
    _same(b, _run(sc, office, kp, ids, 0))  # the default is the persistent pass


def test_waves_match_the_persistent_pass_with_sphere_capture(office):
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, office.pos, office.nrm, office.surf, office.mat, r_p=0.015)
    sc.set_materials(office.eps_r, office.sigma, office.scat)
    kp = dict(max_depth=5, capture=nrt.CAPTURE_SPHERE, diffuse=0, n_rays=1_000_000, r_rx=0.3)
    a = _run(sc, office, kp, None, WAVES)
    b = _run(sc, office, kp, None, PERSISTENT)
    assert len(a[0]["key_hi"]) > 16
    _same(a, b)


def test_unknown_schedule_is_rejected(office):
    ctx = nrt.Context(0)
    sc = nrt.Scene(ctx, office.pos, office.nrm, office.surf, office.mat, r_p=0.015)
    with pytest.raises(RuntimeError):
        sc.trace(office.tx, office.rx, nrt.default_trace_params(spec_waves=3, n_rays=1000))
