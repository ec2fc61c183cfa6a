"""Triangle-sharded casts over several GPUs (host-side orchestration).

Each GPU (rank) holds a contiguous slice of the triangles and casts every
sensor against it; the per-ray u64 keys (FP32 bits of t << 32 | global
triangle id) are combined by a MIN across the ranks.  The closest hit over
the union of the slices is the minimum over the slices' closest hits, since
the problem's result is a minimum over triangles (Sec. 1.1, Eq. brute).  With
the FP64 re-test, each shard settles its flagged rays against the winner over
all shards, and a second MIN combines the settled keys (protocol in
include/grca.h, grca_cast_shard).

The collectives are caller-supplied in-place reductions: a MIN over int64
key tensors (keys are below 2^63, so the signed minimum is the unsigned one)
and a MAX over uint8 flag tensors; torch.distributed's all_reduce across
processes, or element-wise reductions when the shards are contexts of one
process.
"""
from __future__ import annotations

from typing import Callable, List, Sequence, Tuple

KEY_MISS = 0x7F800000FFFFFFFF
CAST_FP64_RECHECK = 1


def split_ranges(n_tris: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous slices [lo, hi) of n_tris triangles over `world` ranks, as
    even as possible."""
    q, r = divmod(n_tris, world)
    out, lo = [], 0
    for k in range(world):
        hi = lo + q + (1 if k < r else 0)
        out.append((lo, hi))
        lo = hi
    return out


def all_reduce_min(group=None) -> Callable:
    """In-place MIN over the ranks of a torch.distributed process group."""
    import torch.distributed as dist

    def f(t):
        dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
        return t
    return f


def all_reduce_max(group=None) -> Callable:
    """In-place MAX over the ranks of a torch.distributed process group."""
    import torch.distributed as dist

    def f(t):
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        return t
    return f


def sharded_cast(caster, ids: Sequence[int], tri_base: int, flags: int, reduce_min: Callable, reduce_max: Callable,
                 out=None, stream=None, launches: list = None):
    """One frame over this rank's slice of the triangles (uploaded to `caster`
    with global ids starting at tri_base); every rank calls it with the same
    sensors and flags.  Returns (distance, triangle id) of every ray, the same
    on every rank: the result over the union of the slices.  Exchanges: the
    keys (MIN), and with the FP64 re-test the per-ray flags (MAX) and the
    settled keys (MIN).  `launches`, if given, receives the number of
    kernels this rank launched."""
    import torch
    n = caster.n_rays(ids)
    dev = torch.device("cuda", caster.device)
    local = torch.empty(n, dtype=torch.int64, device=dev)
    caster.cast_shard(ids, tri_base, local, flags, stream)
    nl = caster.last_launch_count()
    final = reduce_min(local)
    if flags & CAST_FP64_RECHECK:
        fl = torch.empty(n, dtype=torch.uint8, device=dev)
        caster.flag_shard(final, fl, stream)
        nl += caster.last_launch_count()
        fl = reduce_max(fl)
        settled = torch.empty_like(local)
        caster.resolve_shard(fl, settled, stream)
        nl += caster.last_launch_count()
        final = reduce_min(settled)
    if out is None:
        out = caster.outputs(ids)
    res = caster.decode_keys(final, out, stream)
    if launches is not None:
        launches.append(nl + 1)
    return res


def reduce_local(tensors: Sequence):
    """Element-wise MIN (or MAX for uint8 flags) over a list of equal-length
    tensors: the exchange of sharded_cast for shards held by one process."""
    import torch
    out = tensors[0].clone()
    for t in tensors[1:]:
        out = torch.maximum(out, t) if t.dtype == torch.uint8 else torch.minimum(out, t)
    return out
