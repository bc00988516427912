"""Multi-GPU sharding of the sampler (one process per GPU).

Proposals are independent (Sec. IV.B: steps 2-5 need no communication), so
ranks split the work with no exchange on the data path: either each rank
takes a disjoint index range of every point (`shard_range`), or each rank
samples its own point streams (`rank_point_id`).  The one collective is the
final merge of statistics, a sum of integer counters, histograms and
fixed-point sums plus a max (`merge_stats`), done once after the runs; the
moments are then recomputed from the merged sums.
"""
from __future__ import annotations

import numpy as np

from . import KMAX

INT_KEYS = ("n_proposals", "n_accepted", "n_near_threshold", "n_refined", "n_envelope_violations",
            "n_dropped", "n_fallback", "n_kept")
# per-point constants that every rank holds alike (taken from the first rank's dict)
SAME_KEYS = ("logM", "alpha_star", "hist_lo", "hist_hi")


def shard_range(total: int, rank: int, world: int):
    """[start, start + count) of a range of `total` proposals for this rank
    (contiguous, sizes differ by at most one)."""
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def rank_point_id(rank: int, point: int, n_points: int) -> int:
    """Philox point id of `point` on `rank`: disjoint streams across ranks."""
    return rank * n_points + point


def _pack(stats):
    """(integer counters, float sums, max) arrays of a list of per-point dicts.
    The float sums are the u0 power sums, the spectrum and the SIR sums; the
    first two are integer multiples of 2^-28 .. 2^-16 (fixed point on the
    device), so adding them in FP64 is exact."""
    ints = np.array([[int(s.get(k, 0)) for k in INT_KEYS] + [int(v) for v in s["hist"]] +
                     [int(v) for v in s["exceed"]] for s in stats], dtype=np.int64)
    sums = np.array([list(s["sum_u0"]) + list(s.get("spectrum", np.zeros(KMAX))) +
                     [s.get("sir_sum_w", 0.0), s.get("sir_sum_w2", 0.0), s.get("sir_sum_wS", 0.0)] +
                     list(s.get("sir_sum_w_u0", np.zeros(4))) for s in stats], dtype=np.float64)
    mx = np.array([s["max_delta"] for s in stats], dtype=np.float64)
    return ints, sums, mx


def moments(n, sum_u0):
    """mean, variance, skewness and kurtosis of u0 from the accepted count and
    the raw power sums (the same reduction as sampler_stats)."""
    if n <= 0:
        return {"mean": float("nan"), "var": float("nan"), "skew": float("nan"), "kurt": float("nan")}
    m1, m2, m3, m4 = (float(v) / n for v in sum_u0)
    var = m2 - m1 * m1
    c3 = m3 - 3 * m1 * m2 + 2 * m1 * m1 * m1
    c4 = m4 - 4 * m1 * m3 + 6 * m1 * m1 * m2 - 3 * m1 * m1 * m1 * m1
    return {"mean": m1, "var": var, "skew": c3 / var ** 1.5, "kurt": c4 / (var * var)}


def _unpack(ints, sums, mx, template):
    nh = len(template[0]["hist"])
    ne = len(template[0]["exceed"])
    out = []
    for p in range(ints.shape[0]):
        d = {k: int(ints[p, i]) for i, k in enumerate(INT_KEYS)}
        o = len(INT_KEYS)
        d["hist"] = ints[p, o:o + nh].astype(np.uint64)
        d["exceed"] = ints[p, o + nh:o + nh + ne].astype(np.uint64)
        d["sum_u0"] = sums[p, :4].copy()
        d["spectrum"] = sums[p, 4:4 + KMAX].copy()
        d["sir_sum_w"], d["sir_sum_w2"], d["sir_sum_wS"] = (float(v) for v in sums[p, 4 + KMAX:7 + KMAX])
        d["sir_sum_w_u0"] = sums[p, 7 + KMAX:11 + KMAX].copy()
        d["max_delta"] = float(mx[p])
        for k in SAME_KEYS:
            if k in template[p]:
                d[k] = template[p][k]
        d.update(moments(d["n_accepted"], d["sum_u0"]))
        out.append(d)
    return out


def combine(per_rank):
    """Merge, in one process, the statistics of several shards of the same
    points (a list over shards of lists over points, as Sampler.stats()
    returns them): what merge_stats computes across ranks."""
    packed = [_pack(st) for st in per_rank]
    ints = sum(p[0] for p in packed)
    sums = sum(p[1] for p in packed)
    mx = np.max(np.stack([p[2] for p in packed]), axis=0)
    return _unpack(ints, sums, mx, per_rank[0])


def merge_stats(stats, group=None):
    """Merge per-point statistics over ranks (torch.distributed all-reduce).
    stats: list of dicts as returned by Sampler.stats(); returns merged dicts:
    integer counters (n_kept included), histogram, exceedance counts, power
    sums, spectrum and SIR sums added, max_delta maximised, and the moments
    recomputed from the merged sums."""
    import torch
    import torch.distributed as dist
    ints, sums, mx = _pack(stats)
    ti, ts, tm = torch.from_numpy(ints), torch.from_numpy(sums), torch.from_numpy(mx)
    dist.all_reduce(ti, group=group)
    dist.all_reduce(ts, group=group)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX, group=group)
    return _unpack(ti.numpy(), ts.numpy(), tm.numpy(), stats)


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
