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


def oracle_two_pass(orc: "oracle.Oracle", tris: np.ndarray, rays: np.ndarray, gpu_results, n_threads=None,
                    plain_ref: dict = None) -> dict:
    """Oracle reference for grading several GPU results on the same rays at the
    cost of one plain oracle pass: the closest hit of every ray first, then
    the near-tie data (runner-up, tie set) only for the rays where some GPU
    result differs from it in id or in hit/miss (the only rays where grade()
    reads that data).  gpu_results: list of (t, id) arrays over `rays`;
    plain_ref: the first pass, if it was already run."""
    ref = dict(plain_ref) if plain_ref is not None else oracle.cast(orc, tris, rays, n_threads=n_threads)
    oid = ref["id"].astype(np.int64)
    need = np.zeros(rays.shape[0], bool)
    for _, gid in gpu_results:
        need |= (np.asarray(gid).astype(np.int64) & 0xFFFFFFFF) != oid
    ref["second"] = np.full(rays.shape[0], np.nan)
    ref["n_ties"] = np.ones(rays.shape[0], np.uint32)
    ref["tie_ids"] = np.full((rays.shape[0], oracle.MAX_TIES), oracle.NO_HIT, np.uint32)
    ref["tie_ids"][:, 0] = ref["id"]
    if need.any():
        sub = oracle.cast(orc, tris, rays[need], ties=True, n_threads=n_threads)
        assert np.array_equal(sub["id"], ref["id"][need]) and np.array_equal(sub["t"], ref["t"][need])
        ref["second"][need] = sub["second"]
        ref["n_ties"][need] = sub["n_ties"]
        ref["tie_ids"][need] = sub["tie_ids"]
    ref["tie_pass_rays"] = int(need.sum())
    return ref


def summary(g: dict, ref: dict, gpu_t: np.ndarray, gpu_id: np.ndarray) -> dict:
    """Per-ray error statement of one graded result: counts by rule, and the
    relative distance error over the rays where both hit the same triangle."""
    gt = np.asarray(gpu_t, np.float64)
    gid = np.asarray(gpu_id).astype(np.int64) & 0xFFFFFFFF
    same = (gid == ref["id"].astype(np.int64)) & (gid != oracle.NO_HIT)
    rel = np.abs(gt[same] - ref["t"][same]) / ref["t"][same] if same.any() else np.zeros(0)
    n = max(1, g["n"])
    return {"rays": g["n"], "oracle_hits": g["hits"], "id_mismatch": g["id_mismatch"], "hit_miss": g["hit_miss"],
            "dist_bad": g["dist_bad"], "errors": g["errors"], "error_rate": g["errors"] / n,
            "tie_accepted": g["tie_accepted"], "edge_accepted": g["edge_accepted"],
            "silhouette_accepted": g["silhouette_accepted"],
            "max_rel_dist_err": float(rel.max()) if rel.size else 0.0,
            "median_rel_dist_err": float(np.median(rel)) if rel.size else 0.0}
