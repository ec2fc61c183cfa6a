"""Per-ray grading of GPU results against the FP64 oracle.

Rules (the stated tolerances made precise):
  - both miss: correct;
  - both hit, same id: distance within 1e-5 relative;
  - both hit, different id: accepted if the GPU's triangle is in the oracle's
    near-tie set (t within 1e-6 relative of the best), or the ray passes within
    `edge_eps` rad of the GPU triangle and that triangle's plane distance is
    within 1e-6 relative of the best (a shared edge of the tie set);
  - hit/miss disagreement: accepted only within `silhouette_eps` rad of the
    boundary of the triangle involved.
"""
from __future__ import annotations

import numpy as np

import oracle

TIE_REL = 1e-6
DIST_REL = 1e-5


def grade(orc: "oracle.Oracle", tris: np.ndarray, ref: dict, gpu_t: np.ndarray, gpu_id: np.ndarray,
          edge_eps: float = 1e-7, silhouette_eps: float = 1e-12, dist_rel: float = DIST_REL) -> dict:
    tris = np.ascontiguousarray(tris, np.float32).reshape(-1, 9)
    ray_ids = ref["ray_ids"]
    ot, oid = ref["t"], ref["id"]
    gt = np.asarray(gpu_t, np.float64)
    gid = np.asarray(gpu_id).astype(np.int64) & 0xFFFFFFFF
    oid64 = oid.astype(np.int64)
    o_hit = oid64 != oracle.NO_HIT
    g_hit = gid != oracle.NO_HIT
    res = {"n": int(ray_ids.shape[0]), "hits": int(o_hit.sum()), "id_mismatch": 0, "hit_miss": 0, "dist_bad": 0,
           "tie_accepted": 0, "edge_accepted": 0, "silhouette_accepted": 0, "max_rel_err": 0.0, "bad_rays": []}
    both = o_hit & g_hit
    rel = np.zeros_like(gt)
    rel[both] = np.abs(gt[both] - ot[both]) / ot[both]
    if both.any():
        res["max_rel_err"] = float(rel[both].max())
    for k in np.nonzero(both & (rel > dist_rel))[0]:
        res["dist_bad"] += 1
        res["bad_rays"].append(("dist", int(ray_ids[k]), float(ot[k]), float(gt[k]), int(oid[k]), int(gid[k])))
    for k in np.nonzero(both & (gid != oid64))[0]:
        g = int(gid[k])
        nt = int(ref["n_ties"][k]) if "n_ties" in ref else 1
        if nt > 1 and g in set(int(x) for x in ref["tie_ids"][k][:min(nt, oracle.MAX_TIES)]):
            res["tie_accepted"] += 1
            continue
        tp, m = oracle.ray_tri_margin(orc, int(ray_ids[k]), tris[g])
        if m >= -edge_eps and abs(tp - ot[k]) <= TIE_REL * ot[k]:
            res["edge_accepted"] += 1
            continue
        res["id_mismatch"] += 1
        res["bad_rays"].append(("id", int(ray_ids[k]), float(ot[k]), float(gt[k]), int(oid[k]), g, float(m)))
    for k in np.nonzero(o_hit != g_hit)[0]:
        tri = int(oid[k]) if o_hit[k] else int(gid[k])
        tp, m = oracle.ray_tri_margin(orc, int(ray_ids[k]), tris[tri])
        if abs(m) <= silhouette_eps:
            res["silhouette_accepted"] += 1
            continue
        res["hit_miss"] += 1
        res["bad_rays"].append(("hitmiss", int(ray_ids[k]), float(ot[k]), float(gt[k]), int(oid[k]), int(gid[k]),
                                float(m)))
    res["bad_ids"] = [b[1] for b in res["bad_rays"]]
    res["bad_rays"] = res["bad_rays"][:20]
    res["errors"] = res["id_mismatch"] + res["hit_miss"] + res["dist_bad"]
    return res


def stratified_rays(sensors, n_per_sensor: int, seed: int = 0) -> np.ndarray:
    """About n_per_sensor rays per sensor: evenly strided channels (all of them
    when the budget allows), evenly strided rays with a seeded phase."""
    rng = np.random.default_rng(seed)
    out = []
    off = 0
    for s in sensors:
        if n_per_sensor >= s.n_channels:
            chans = np.arange(s.n_channels)
        else:
            step_c = s.n_channels / max(1, n_per_sensor)
            chans = np.unique((np.arange(n_per_sensor) * step_c + rng.uniform(0, step_c)).astype(np.int64))
            chans = chans[chans < s.n_channels]
        per_ch = max(1, n_per_sensor // len(chans))
        step = max(1, s.n_rays // per_ch)
        for j in chans:
            ph = int(rng.integers(step))
            i = np.arange(ph, s.n_rays, step)[:per_ch]
            out.append(off + int(j) * s.n_rays + i)
        off += s.n_channels * s.n_rays
    return np.unique(np.concatenate(out).astype(np.int64))
