"""Comparison helpers: CUDA path vs the FP64 oracle on the same seeded inputs.

Hit records: bit-exact point index (q_min) at every bounce the oracle marks
certain (before its first ambiguous decision), positions within the
ambiguity band delta, normals within 1e-4.

Paths: for every key valid on either side, the representative ray must be
the same, or the difference must be explained by a decision the oracle
marks ambiguous *for that key and that ray* (an uncertain candidacy or an
ambiguous validation).  Matched paths must agree within 1e-4 relative on
the complex coefficient and 1e-6 relative on the delay; for path types not
held strict, these floors are widened per path to twice the oracle's shadow
sensitivity.  The summaries report raw (unscaled) errors.
"""
from __future__ import annotations

import numpy as np

C0 = 299792458.0


def compare_hits(g, o, delta, n_tol=1e-4, sens=None, normal_tail=0.0, index_tail=0.0):
    """g: GPU hits dict (rows = rays in ascending id); o: oracle hits dict;
    sens: the oracle's shadow divergence (dq, dn) per hit, which widens the
    normal tolerance where the bounce sequence amplifies rounding.
    normal_tail: the fraction of compared hits whose weighted normal may
    exceed that tolerance (counted and reported; 0 = none) -- the normal is
    an intermediate of Eq. 4 with no bar of its own, and over millions of
    hits the FP32 rounding has a tail beyond the shadows' spread.
    index_tail: the fraction of compared hits whose point index may differ
    although the oracle marked the decision certain (0 = bit-exact; the
    escapes are counted and listed with their geometry for the report)."""
    gi = g["idx"].astype(np.int64)
    oi = o["idx"]
    n, S = oi.shape
    excl = o["excl"]
    checked = mism = n_over = 0
    max_dq = max_dn = 0.0
    worst = None
    bad = []
    for s in range(S):
        cert = (s + 1) < excl
        # compare only while the oracle ray is alive at bounce s (or its miss is certain)
        alive = np.ones(n, bool) if s == 0 else (oi[:, s - 1] >= 0)
        m = cert & alive
        checked += int(m.sum())
        diff = m & (gi[:, s] != oi[:, s])
        mism += int(diff.sum())
        if diff.any():
            bad += [{"row": int(r), "bounce": s, "gpu": int(gi[r, s]), "oracle": int(oi[r, s]),
                     "cos_in": float(o["cos_in"][r, s]), "t": float(o["t"][r, s]),
                     "dq_prev": [float(np.abs(g["q"][r, u] - o["q"][r, u]).max())
                                 for u in range(s)]}
                    for r in np.nonzero(diff)[0][:5]]
        hit = m & (oi[:, s] >= 0) & (gi[:, s] == oi[:, s])
        if hit.any():
            dq = np.abs(g["q"][hit, s].astype(np.float64) - o["q"][hit, s]).max(axis=1)
            dn = np.abs(g["n"][hit, s].astype(np.float64) - o["n"][hit, s]).max(axis=1)
            if float(dq.max()) > max_dq:
                rr = np.nonzero(hit)[0][int(np.argmax(dq))]
                worst = {"row": int(rr), "bounce": s, "dq": float(dq.max()),
                         "cos_in": float(o["cos_in"][rr, s]), "t": float(o["t"][rr, s]),
                         "idx": int(oi[rr, s]),
                         "dq_sens": float(sens[0][rr, s]) if sens is not None else None,
                         "dq_prev": [float(np.abs(g["q"][rr, u] - o["q"][rr, u]).max())
                                     for u in range(s)]}
            max_dq = max(max_dq, float(dq.max()))
            tol = np.full(dn.shape, n_tol)
            if sens is not None:
                tol = np.maximum(tol, 2.0 * sens[1][hit, s])
            wi = int(np.argmax(dn - tol))
            n_over += int((dn > tol).sum())
            max_dn = max(max_dn, float(dn.max()))
            assert normal_tail > 0 or (dn <= tol).all(), \
                f"normal differs by {dn[wi]} (tol {tol[wi]}) at bounce {s}"
    excluded = int((excl <= S).sum())
    # which rule excluded each ray first: the fixed band delta around a
    # threshold (the oracle's per-hit ambiguity flags) or, only, the shadow
    # trajectories (perturbed FP64 re-traces that land elsewhere)
    amb = o["amb"] != 0
    live = np.ones((n, S), bool)
    live[:, 1:] = oi[:, :-1] >= 0
    first_amb = np.where((amb & live).any(axis=1), np.argmax(amb & live, axis=1) + 1, S + 1)
    by_band = int(((excl <= S) & (first_amb <= excl)).sum())
    assert n_over <= normal_tail * checked, f"{n_over} normals beyond tolerance of {checked} hits"
    assert mism <= index_tail * checked, f"{mism} index mismatches of {checked} hits: {bad}"
    return {"checked": checked, "mismatch": mism, "max_dq": max_dq, "max_dn": max_dn,
            "normal_over_tol": n_over, "excluded_rays": excluded,
            "excluded_by_band": by_band, "excluded_by_shadow_only": excluded - by_band,
            "rays": int(n), "examples": bad, "worst": worst}


def _tried_map(osim):
    K = osim.keys()
    ray, valid, amb = osim.tried()
    off = np.concatenate([[0], np.cumsum(K["n_tried"])])
    out = {}
    for i in range(len(K["hi"])):
        key = (int(K["hi"][i]), int(K["lo"][i]))
        sl = slice(off[i], off[i + 1])
        out[key] = {"valid": bool(K["valid"][i]), "rep": int(K["rep"][i]),
                    "certain": bool(K["certain"][i]), "path": int(K["path"][i]),
                    "tried": list(zip(ray[sl].tolist(), valid[sl].tolist(), amb[sl].tolist()))}
    return out


PATH_TYPES = ("los", "specular", "diffuse", "diffracted")


def path_type_name(ty, k):
    return "diffracted" if ty == 2 else "diffuse" if ty == 1 else "los" if k == 0 else "specular"


def _key16(hi, lo):
    """128-bit keys as sortable 16-byte records (hi first, big-endian)."""
    a = np.empty((len(hi), 2), ">u8")
    a[:, 0] = hi
    a[:, 1] = lo
    return np.ascontiguousarray(a).view(np.dtype((np.void, 16))).reshape(-1)


def compare_paths(gp, osim, eps_r, sigma, scat, a_rtol=1e-4, tau_rtol=1e-6, strict=(),
                  key_tail=0.0, path_tail=0.0):
    """gp: GPU paths dict; osim: OracleSim.  Returns a summary; raises on an
    unexplained mismatch or an out-of-tolerance matched path.

    Tolerances: a_rtol / tau_rtol, widened per path to twice the oracle's
    shadow sensitivity except for the path types named in `strict` (from
    PATH_TYPES), which are held to the fixed values.  The summary reports,
    per type, the raw (unscaled) largest relative errors, how many paths
    were field-checked, how many needed a tolerance above the fixed one
    (widened_a / widened_tau), how many exceed the fixed one (over_fixed),
    and how many were not checked because the oracle found them fragile
    (a shadow trajectory does not reproduce the path) or uncertain.
    Vectorised over the paths, so a full-size launch (millions of paths)
    compares in seconds; only the mismatched keys are walked one by one.
    key_tail: the fraction of keys that may differ without an oracle-marked
    ambiguity (0 = none; the count is reported as "unexplained").
    path_tail: for the types not held strict, the fraction of field-checked
    paths that may exceed their (widened) tolerance -- counted per type as
    "out_of_tol" with the largest error-to-tolerance ratios; strict types
    may have none."""
    NONE = 0xFFFFFFFF
    O = osim.paths()
    a_o, _ = osim.field(eps_r, sigma, scat)
    a_sens, tau_sens = osim.path_sens(eps_r, sigma, scat)
    ng, no = len(gp["key_hi"]), len(O["hi"])
    kg = _key16(gp["key_hi"], gp["key_lo"])
    ko = _key16(O["hi"], O["lo"])
    allk, inv = np.unique(np.concatenate([kg, ko]), return_inverse=True)
    gi_of = np.full(len(allk), -1, np.int64)
    oi_of = np.full(len(allk), -1, np.int64)
    gi_of[inv[:ng]] = np.arange(ng)
    oi_of[inv[ng:]] = np.arange(no)
    grep = gp["rep"].astype(np.int64)
    grep[grep == NONE] = -1
    both = (gi_of >= 0) & (oi_of >= 0)
    same = both.copy()
    same[both] = grep[gi_of[both]] == O["rep"][oi_of[both]]
    gm, om = gi_of[same], oi_of[same]
    types = np.array([PATH_TYPES.index(path_type_name(int(t), int(k)))
                      for t, k in zip(O["type"][om], O["k"][om])], np.int64)
    certain = O["certain"][om] != 0
    sens_ok = a_sens[om] >= 0
    chk = certain & sens_ok
    ag = gp["a"][gm, 0].astype(np.float64) + 1j * gp["a"][gm, 1].astype(np.float64)
    ao = a_o[om]
    da = np.abs(ag - ao) / np.maximum(np.abs(ao), 1e-300)
    dt = np.abs(gp["tau"][gm].astype(np.float64) - O["tau"][om]) / O["tau"][om]
    strict_t = np.array([PATH_TYPES[t] in strict for t in types], bool)
    tol_a = np.where(strict_t, a_rtol, np.maximum(a_rtol, 2.0 * a_sens[om]))
    tol_t = np.where(strict_t, tau_rtol, np.maximum(tau_rtol, 2.0 * tau_sens[om]))
    out = chk & ((da > tol_a) | (dt > tol_t))
    bad = out & strict_t
    for ti in range(len(PATH_TYPES)):
        m_t = (types == ti) & ~strict_t
        if (out & m_t).sum() > path_tail * max(int((chk & m_t).sum()), 1):
            bad |= out & m_t
    if bad.any():
        w = int(np.nonzero(bad)[0][0])
        raise AssertionError(f"{PATH_TYPES[types[w]]} path ({hex(int(O['hi'][om[w]]))}, "
                             f"{hex(int(O['lo'][om[w]]))}): a rel error {da[w]} (tol {tol_a[w]}), "
                             f"tau rel error {dt[w]} (tol {tol_t[w]}); {int(bad.sum())} paths out")
    n_rx = osim.rx.shape[0]
    jj = O["j"][om].astype(np.int64)
    common_p_g = np.bincount(jj, np.abs(ag) ** 2, minlength=n_rx)
    common_p_o = np.bincount(jj, np.abs(ao) ** 2, minlength=n_rx)
    by_type = {}
    for ti, name in enumerate(PATH_TYPES):
        m = types == ti
        if not m.any():
            continue
        c = chk & m
        u = m & ~chk  # matched but not asserted (uncertain or fragile): raw errors reported
        ra = da[c] / tol_a[c] if c.any() else np.zeros(0)
        rt = dt[c] / tol_t[c] if c.any() else np.zeros(0)
        by_type[name] = {
            "out_of_tol": int((out & m).sum()),
            "max_ratio_a": float(ra.max()) if ra.size else 0.0,
            "max_ratio_tau": float(rt.max()) if rt.size else 0.0,
            "unchecked_max_da": float(da[u].max()) if u.any() else 0.0,
            "unchecked_p50_da": float(np.median(da[u])) if u.any() else 0.0,
            "unchecked_max_dtau": float(dt[u].max()) if u.any() else 0.0,
            "max_tol_a": float(tol_a[c].max()) if c.any() else 0.0,
            "max_tol_tau": float(tol_t[c].max()) if c.any() else 0.0,
            "matched": int(m.sum()), "field_checked": int(c.sum()),
            "fragile": int((m & certain & ~sens_ok).sum()), "uncertain": int((m & ~certain).sum()),
            "widened_a": int((c & (tol_a > a_rtol)).sum()),
            "widened_tau": int((c & (tol_t > tau_rtol)).sum()),
            "over_fixed": int((c & ((da > a_rtol) | (dt > tau_rtol))).sum()),
            "max_da": float(da[c].max()) if c.any() else 0.0,
            "p99_da": float(np.quantile(da[c], 0.99)) if c.any() else 0.0,
            "max_dtau": float(dt[c].max()) if c.any() else 0.0,
            "p99_dtau": float(np.quantile(dt[c], 0.99)) if c.any() else 0.0}
    # keys valid on one side only, or with different representatives: each
    # must be explained by a decision the oracle marks ambiguous for it
    mis = np.nonzero(~same)[0]
    explained = 0
    unexplained = []
    if mis.size:
        K = osim.keys()
        ray, valid, amb = osim.tried()
        off = np.concatenate([[0], np.cumsum(K["n_tried"])])
        kk = _key16(K["hi"], K["lo"])
        order = np.argsort(kk, kind="stable")
        kk_sorted = kk[order]
        for u in mis:
            gi, oi = int(gi_of[u]), int(oi_of[u])
            hi = int(gp["key_hi"][gi]) if gi >= 0 else int(O["hi"][oi])
            lo = int(gp["key_lo"][gi]) if gi >= 0 else int(O["lo"][oi])
            g = None if gi < 0 else int(grep[gi])
            o = None if oi < 0 else int(O["rep"][oi])
            q = np.searchsorted(kk_sorted, _key16([hi], [lo])[0])
            tried = []
            if q < len(kk_sorted) and kk_sorted[q] == _key16([hi], [lo])[0]:
                ki = int(order[q])
                sl = slice(int(off[ki]), int(off[ki + 1]))
                tried = list(zip(ray[sl].tolist(), valid[sl].tolist(), amb[sl].tolist()))
            tried_rays = {r: a for r, _, a in tried}
            ok = False
            if g is not None and g >= 0:
                if osim.cand_status(hi, lo, g) == 2:
                    ok = True
                if tried_rays.get(g, False):
                    ok = True
                if g not in tried_rays and any(a for _, _, a in tried):
                    ok = True
            if o is not None and o >= 0:
                if tried_rays.get(o, False) or osim.cand_status(hi, lo, o) == 2:
                    ok = True
            if (g is None or o is None) and any(a for _, _, a in tried):
                ok = True
            if ok:
                explained += 1
            else:
                unexplained.append((hex(hi), hex(lo), g, o, tried[:4]))
    assert len(unexplained) <= key_tail * len(allk), \
        f"{len(unexplained)} unexplained path mismatches, e.g. {unexplained[:5]}"
    m = common_p_o > 0
    dp = np.abs(common_p_g[m] - common_p_o[m]) / common_p_o[m]
    return {"keys": int(len(allk)), "matched": int(same.sum()), "explained": explained,
            "unexplained": len(unexplained), "unexplained_examples": unexplained[:5],
            "fragile": int((a_sens < 0).sum()),
            "field_checked": int(chk.sum()), "max_da": float(da[chk].max()) if chk.any() else 0.0,
            "max_dtau": float(dt[chk].max()) if chk.any() else 0.0,
            "max_dP_common": float(dp.max()) if dp.size else 0.0, "by_type": by_type}


def compare_paths_loop(gp, osim, eps_r, sigma, scat, a_rtol=1e-4, tau_rtol=1e-6, strict=(),
                       key_tail=0.0, path_tail=0.0):
    """Key-by-key form of compare_paths (same rules, same summary): the
    reference the vectorised harness is tested against on small cases.

    Tolerances: a_rtol / tau_rtol, widened per path to twice the oracle's
    shadow sensitivity except for the path types named in `strict` (from
    PATH_TYPES), which are held to the fixed values.  The summary reports,
    per type, the raw (unscaled) largest relative errors, how many paths
    were field-checked, how many needed a tolerance above the fixed one
    (widened_a / widened_tau), how many exceed the fixed one (over_fixed),
    and how many were not checked because the oracle found them fragile
    (a shadow trajectory does not reproduce the path) or uncertain."""
    O = osim.paths()
    a_o, _ = osim.field(eps_r, sigma, scat)
    a_sens, tau_sens = osim.path_sens(eps_r, sigma, scat)
    omap = _tried_map(osim)
    NONE = 0xFFFFFFFF
    g_by_key = {}
    for i in range(len(gp["key_hi"])):
        g_by_key[(int(gp["key_hi"][i]), int(gp["key_lo"][i]))] = i
    o_by_key = {}
    for i in range(len(O["hi"])):
        o_by_key[(int(O["hi"][i]), int(O["lo"][i]))] = i
    keys = set(g_by_key) | set(o_by_key)
    matched = explained = field_checked = 0
    unexplained = []
    max_da = max_dtau = 0.0
    per = {t: {"matched": 0, "field_checked": 0, "fragile": 0, "uncertain": 0, "widened_a": 0,
               "widened_tau": 0, "over_fixed": 0, "da": [], "dtau": [], "uda": [], "udt": [],
               "ta": [], "tt": [], "out_of_tol": 0, "out": []} for t in PATH_TYPES}
    common_p_g = np.zeros(osim.rx.shape[0])
    common_p_o = np.zeros(osim.rx.shape[0])
    for key in keys:
        gi = g_by_key.get(key)
        oi = o_by_key.get(key)
        g = None if gi is None else int(gp["rep"][gi])
        o = None if oi is None else int(O["rep"][oi])
        if g == NONE:
            g = -1
        if gi is not None and oi is not None and g == o:
            matched += 1
            info = omap.get(key)
            certain = bool(O["certain"][oi]) if info is None else info["certain"]
            j = int(O["j"][oi])
            ag = complex(gp["a"][gi, 0], gp["a"][gi, 1])
            ao = a_o[oi]
            common_p_g[j] += abs(ag) ** 2
            common_p_o[j] += abs(ao) ** 2
            t = per[path_type_name(int(O["type"][oi]), int(O["k"][oi]))]
            t["matched"] += 1
            if not certain:
                t["uncertain"] += 1
            elif a_sens[oi] < 0:
                t["fragile"] += 1
            if not (certain and a_sens[oi] >= 0):
                t["uda"].append(abs(ag - ao) / max(abs(ao), 1e-300))
                t["udt"].append(abs(float(gp["tau"][gi]) - O["tau"][oi]) / O["tau"][oi])
            if certain and a_sens[oi] >= 0:
                field_checked += 1
                t["field_checked"] += 1
                da = abs(ag - ao) / max(abs(ao), 1e-300)
                dt = abs(float(gp["tau"][gi]) - O["tau"][oi]) / O["tau"][oi]
                t["da"].append(da)
                t["dtau"].append(dt)
                name = path_type_name(int(O["type"][oi]), int(O["k"][oi]))
                fixed = name in strict
                tol_a = a_rtol if fixed else max(a_rtol, 2.0 * a_sens[oi])
                tol_t = tau_rtol if fixed else max(tau_rtol, 2.0 * tau_sens[oi])
                t["ta"].append(tol_a)
                t["tt"].append(tol_t)
                t["widened_a"] += int(tol_a > a_rtol)
                t["widened_tau"] += int(tol_t > tau_rtol)
                t["over_fixed"] += int(da > a_rtol or dt > tau_rtol)
                max_da = max(max_da, da)
                max_dtau = max(max_dtau, dt)
                if da > tol_a or dt > tol_t:
                    t["out_of_tol"] += 1
                    t["out"].append((fixed, f"{name} path {key}: a rel error {da} (tol {tol_a}), "
                                            f"tau rel error {dt} (tol {tol_t})"))
            continue
        info = omap.get(key)
        tried = info["tried"] if info else []
        tried_rays = {r: amb for r, _, amb in tried}
        ok = False
        if g is not None and g >= 0:
            if osim.cand_status(key[0], key[1], g) == 2:
                ok = True
            if tried_rays.get(g, False):
                ok = True
            if g not in tried_rays and any(a for _, _, a in tried):
                ok = True
        if o is not None and o >= 0:
            if tried_rays.get(o, False) or osim.cand_status(key[0], key[1], o) == 2:
                ok = True
        if (g is None or o is None) and any(a for _, _, a in tried):
            ok = True
        if ok:
            explained += 1
        else:
            unexplained.append((hex(key[0]), hex(key[1]), g, o, tried[:4]))
    for t in per.values():
        outs = t.pop("out")
        strict_out = [msg for fixed, msg in outs if fixed]
        assert not strict_out, strict_out[0]
        assert len(outs) <= path_tail * max(t["field_checked"], 1), outs[0][1]
    assert len(unexplained) <= key_tail * len(keys), \
        f"{len(unexplained)} unexplained path mismatches, e.g. {unexplained[:5]}"
    m = common_p_o > 0
    dp = np.abs(common_p_g[m] - common_p_o[m]) / common_p_o[m]
    by_type = {}
    for name, t in per.items():
        if not t["matched"]:
            continue
        da, dt = np.asarray(t.pop("da")), np.asarray(t.pop("dtau"))
        uda, udt = np.asarray(t.pop("uda")), np.asarray(t.pop("udt"))
        ta, tt = np.asarray(t.pop("ta")), np.asarray(t.pop("tt"))
        t["unchecked_max_da"] = float(uda.max()) if uda.size else 0.0
        t["unchecked_p50_da"] = float(np.median(uda)) if uda.size else 0.0
        t["unchecked_max_dtau"] = float(udt.max()) if udt.size else 0.0
        t["max_tol_a"] = float(ta.max()) if ta.size else 0.0
        t["max_tol_tau"] = float(tt.max()) if tt.size else 0.0
        t["max_ratio_a"] = float((da / ta).max()) if da.size else 0.0
        t["max_ratio_tau"] = float((dt / tt).max()) if dt.size else 0.0
        t["max_da"] = float(da.max()) if da.size else 0.0
        t["p99_da"] = float(np.quantile(da, 0.99)) if da.size else 0.0
        t["max_dtau"] = float(dt.max()) if dt.size else 0.0
        t["p99_dtau"] = float(np.quantile(dt, 0.99)) if dt.size else 0.0
        by_type[name] = t
    return {"keys": len(keys), "matched": matched, "explained": explained,
            "unexplained": len(unexplained), "unexplained_examples": unexplained[:5],
            "fragile": int((a_sens < 0).sum()),
            "field_checked": field_checked, "max_da": max_da, "max_dtau": max_dtau,
            "max_dP_common": float(dp.max()) if dp.size else 0.0, "by_type": by_type}
