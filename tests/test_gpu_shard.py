"""GPU test of the triangle-sharded cast (grca_cast_shard / grca_flag_shard /
grca_resolve_shard / grca_decode_keys) through the C ABI.  The shards are contexts of one
process on one GPU, cast one after the other, with an element-wise minimum in
place of the collectives; the result must equal one cast of the whole
triangle set bit for bit (FP32 only and FP32 + FP64 re-test), and grade with
zero errors against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from grading import grade, stratified_rays
from scenes import make_config, scene_c1

pytestmark = pytest.mark.gpu


def _sharded(scene, tris, ranges, flags):
    import torch
    from paper_2605_10457_gb300 import grca
    from paper_2605_10457_gb300.shard import reduce_local
    cs = []
    for lo, hi in ranges:
        c = grca.Caster(0)
        ids = [c.add_sensor(s) for s in scene.sensors]
        c.upload(np.ascontiguousarray(tris[lo:hi]))
        cs.append((c, ids, lo))
    n = cs[0][0].n_rays(cs[0][1])
    local = [c.cast_shard(ids, lo, torch.empty(n, dtype=torch.int64, device="cuda"), flags) for c, ids, lo in cs]
    final = reduce_local(local)
    if flags & grca.CAST_FP64_RECHECK:
        fl = reduce_local([c.flag_shard(final, torch.empty(n, dtype=torch.uint8, device="cuda")) for c, _, _ in cs])
        final = reduce_local([c.resolve_shard(fl, torch.empty_like(final)) for c, _, _ in cs])
        st = [c.stats() for c, _, _ in cs]
        assert all(s["device_error"] == 0 for s in st)
    d, t = cs[0][0].decode_keys(final, cs[0][0].outputs(cs[0][1]))
    torch.cuda.synchronize()
    out = d.cpu().numpy(), t.cpu().numpy().view(np.uint32)
    for c, _, _ in cs:
        c.close()
    return out


def _whole(scene, tris, flags):
    import torch
    from paper_2605_10457_gb300 import grca
    c = grca.Caster(0)
    ids = [c.add_sensor(s) for s in scene.sensors]
    c.upload(tris)
    d, t = c.cast(ids, flags)
    torch.cuda.synchronize()
    out = d.cpu().numpy(), t.cpu().numpy().view(np.uint32)
    c.close()
    return out


@pytest.mark.parametrize("cfg,n_shards", [("c1", 2), ("c4m", 3), ("c5m", 2)])
def test_sharded_cast_equals_the_whole_cast(cfg, n_shards):
    from paper_2605_10457_gb300 import grca
    from paper_2605_10457_gb300.shard import split_ranges
    sc = scene_c1() if cfg == "c1" else make_config(cfg)
    tris = sc.tris(3 if cfg != "c1" else 0)
    # uneven cuts that split meshes
    ranges = split_ranges(tris.shape[0], n_shards)
    ranges = [(lo, hi) for lo, hi in ranges]
    for flags in (0, grca.CAST_FP64_RECHECK):
        d0, t0 = _whole(sc, tris, flags)
        d1, t1 = _sharded(sc, tris, ranges, flags)
        assert np.array_equal(t0, t1), (flags, np.nonzero(t0 != t1)[0][:8])
        assert np.array_equal(d0.view(np.uint32), d1.view(np.uint32))
    rays = stratified_rays(sc.sensors, 512 if cfg != "c1" else 8192, seed=9)
    if getattr(sc, "stress_rays", None) is not None:
        rays = np.unique(np.concatenate([rays, sc.stress_rays]))
    orc = oracle.Oracle(sc.sensors)
    ref = oracle.cast(orc, tris, rays, ties=True)
    g = grade(orc, tris, ref, d1[rays], t1[rays])
    assert g["errors"] == 0, g


def test_shard_calls_check_their_arguments():
    import torch
    from paper_2605_10457_gb300 import grca
    c = grca.Caster(0)
    sc = scene_c1()
    ids = [c.add_sensor(s) for s in sc.sensors]
    c.upload(sc.tris())
    keys = torch.empty(c.n_rays(ids), dtype=torch.int64, device="cuda")
    fl = torch.zeros(c.n_rays(ids), dtype=torch.uint8, device="cuda")
    with pytest.raises(grca.GrcaError):
        c.flag_shard(keys, fl)                        # no grca_cast_shard yet
    with pytest.raises(grca.GrcaError):
        c.resolve_shard(fl, keys)
    with pytest.raises(grca.GrcaError):
        c.cast_shard(ids, 0, keys, grca.CAST_GRAPH)   # graph replay is not offered
    c.close()
