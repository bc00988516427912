"""Multi-GPU sharding of the sampler (one process per GPU).

Proposals are independent (Sec. IV.B: steps 2-5 need no communication), so
ranks split the work with no exchange on the data path: either each rank
takes a disjoint index range of every point (`shard_range`), or each rank
samples its own point streams (`rank_point_id`).  The one collective is the
final merge of statistics, a sum of integer counters and histograms plus a
max (`merge_stats`), done once after the runs.
"""
from __future__ import annotations

import numpy as np

from . import KMAX

INT_KEYS = ("n_proposals", "n_accepted", "n_near_threshold", "n_refined", "n_envelope_violations",
            "n_dropped", "n_fallback")


def shard_range(total: int, rank: int, world: int):
    """[start, start + count) of a range of `total` proposals for this rank
    (contiguous, sizes differ by at most one)."""
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def rank_point_id(rank: int, point: int, n_points: int) -> int:
    """Philox point id of `point` on `rank`: disjoint streams across ranks."""
    return rank * n_points + point


def merge_stats(stats, group=None):
    """Sum per-point statistics over ranks (torch.distributed all-reduce).
    stats: list of dicts as returned by Sampler.stats(); returns merged dicts
    with integer counters, histogram, exceedance counts, power sums and the
    spectrum sums added and max_delta maximised."""
    import torch
    import torch.distributed as dist
    P = len(stats)
    ints = np.array([[s[k] for k in INT_KEYS] + list(s["hist"]) + list(s["exceed"]) for s in stats],
                    dtype=np.int64)
    sums = np.array([list(s["sum_u0"]) + list(s.get("spectrum", np.zeros(KMAX))) for s in stats],
                    dtype=np.float64)
    mx = np.array([s["max_delta"] for s in stats], dtype=np.float64)
    ti, ts, tm = torch.from_numpy(ints), torch.from_numpy(sums), torch.from_numpy(mx)
    dist.all_reduce(ti, group=group)
    dist.all_reduce(ts, group=group)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX, group=group)
    ints, sums, mx = ti.numpy(), ts.numpy(), tm.numpy()
    nh = len(stats[0]["hist"])
    out = []
    for p in range(P):
        d = {k: int(ints[p, i]) for i, k in enumerate(INT_KEYS)}
        d["hist"] = ints[p, len(INT_KEYS):len(INT_KEYS) + nh].astype(np.uint64)
        d["exceed"] = ints[p, len(INT_KEYS) + nh:].astype(np.uint64)
        d["sum_u0"] = sums[p, :4]
        d["spectrum"] = sums[p, 4:]
        d["max_delta"] = float(mx[p])
        out.append(d)
    return out


def gather_records(raw, rec_bytes, group=None):
    """Concatenate the accepted records of all ranks (torch.distributed
    all-gather), in rank order, on every rank.  raw: this rank's records as
    a flat uint8 array of whole records (e.g. a buffer filled by
    Sampler.samples(host_dst=...), cut to n * rec_bytes); rec_bytes:
    tkdv_record_bytes(K).  Host tensors under gloo, device tensors under
    NCCL; one exchange after the runs, none on the sampling path."""
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")
    raw = np.ascontiguousarray(np.asarray(raw, dtype=np.uint8))
    if len(raw) % rec_bytes:
        raise ValueError("raw holds %d bytes, not whole %d-byte records" % (len(raw), rec_bytes))
    n = len(raw) // rec_bytes
    world = dist.get_world_size(group)
    cnt = torch.tensor([n], dtype=torch.int64, device=dev)
    cnts = [torch.zeros_like(cnt) for _ in range(world)]
    dist.all_gather(cnts, cnt, group=group)
    counts = [int(c.item()) for c in cnts]
    buf = torch.zeros(max(1, max(counts)) * rec_bytes, dtype=torch.uint8, device=dev)
    if n:
        buf[: n * rec_bytes] = torch.from_numpy(raw).to(dev)
    bufs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(bufs, buf, group=group)
    return np.concatenate([b[: c * rec_bytes].cpu().numpy() for b, c in zip(bufs, counts)])
