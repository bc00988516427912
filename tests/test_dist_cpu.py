"""The multi-rank path on CPU: two gloo ranks split a run, merge their
statistics, and get exactly the statistics of one rank doing the whole run
(the per-rank sampling stands in by the oracle, which computes the same
statistics from the same stream)."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2411_16952_gb300 import dist as D


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _as_lib_stats(st):
    return {"n_proposals": st["n_prop"], "n_accepted": st["n_acc"], "n_near_threshold": st["n_near"],
            "n_refined": 0, "n_envelope_violations": st["n_viol"], "n_dropped": 0, "n_fallback": 0,
            "hist": st["hist"], "exceed": st["exceed"], "sum_u0": st["sum_u0"], "max_delta": st["max_delta"],
            "spectrum": np.concatenate([st["spectrum"], np.zeros(D.KMAX - len(st["spectrum"]))])}


def _encode(rec, K, point):
    """The library's record layout (include/tkdv.h: idx, point, flags, H2, H3,
    u0, log f/(Mg), xhat) of oracle records, as raw bytes."""
    import paper_2411_16952_gb300 as T
    rb = T.tkdv_record_bytes(K)
    n = len(rec["idx"])
    out = np.zeros((n, rb), dtype=np.uint8)
    out[:, 0:8] = rec["idx"].astype(np.uint64).reshape(n, 1).view(np.uint8)
    out[:, 8:12] = np.full((n, 1), point, dtype=np.uint32).view(np.uint8)
    for j, key in enumerate(("H2", "H3", "u0", "delta")):
        out[:, 16 + 4 * j:20 + 4 * j] = rec[key].astype(np.float32).reshape(n, 1).view(np.uint8)
    out[:, 32:32 + 8 * K] = rec["xhat"][:, :2 * K].astype(np.float32).view(np.uint8)
    return out.reshape(-1)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    K, E0, bp, r, n = 8, 1.0, 30.0, 50.0, 200_000
    pt = O.make_point(K, E0, bp, r, O.PAPER)
    pt.logM = O.log_M(pt, 0)
    start, count = D.shard_range(n, rank, world)
    st = O.run_stats(pt, 7, 3, start, count, 1)
    # a second point sampled on rank-specific streams
    pid = D.rank_point_id(rank, 1, 2)
    st2 = O.run_stats(pt, 7, pid, 0, 50_000, 1)
    merged = D.merge_stats([_as_lib_stats(st), _as_lib_stats(st2)])
    # accepted records of the shards, gathered in rank order
    import paper_2411_16952_gb300 as T
    _, rec = O.run_accepted(pt, 7, 3, start, count, cap=1 << 16)
    allrec = D.gather_records(_encode(rec, K, 0), T.tkdv_record_bytes(K))
    # a rank with no records contributes nothing
    mine = _encode(rec, K, 0) if rank == 0 else np.zeros(0, dtype=np.uint8)
    only0 = D.gather_records(mine, T.tkdv_record_bytes(K))
    if rank == 0:
        q.put((merged, allrec, only0, _encode(rec, K, 0)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_merge_to_one_run():
    pytest.importorskip("torch.distributed")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged, allrec, only0, rank0 = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    K, E0, bp, r, n = 8, 1.0, 30.0, 50.0, 200_000
    pt = O.make_point(K, E0, bp, r, O.PAPER)
    pt.logM = O.log_M(pt, 0)
    one = _as_lib_stats(O.run_stats(pt, 7, 3, 0, n, 1))
    for k in ("n_proposals", "n_accepted", "n_near_threshold", "n_envelope_violations"):
        assert merged[0][k] == one[k]
    assert np.array_equal(merged[0]["hist"], one["hist"])
    assert np.array_equal(merged[0]["exceed"], one["exceed"])
    assert np.allclose(merged[0]["sum_u0"], one["sum_u0"], rtol=1e-12)
    assert np.allclose(merged[0]["spectrum"], one["spectrum"], rtol=1e-12, atol=1e-9)
    assert merged[0]["max_delta"] == one["max_delta"]
    # moments recomputed from the merged sums; counters absent from the input stay zero
    m = D.moments(one["n_accepted"], one["sum_u0"])
    for k in ("mean", "var", "skew", "kurt"):
        assert abs(merged[0][k] - m[k]) <= 1e-9 * (1 + abs(m[k])), k
    assert merged[0]["n_kept"] == 0 and merged[0]["sir_sum_w"] == 0.0
    # rank-specific streams: point ids 1 and 3 are different draws
    assert merged[1]["n_proposals"] == 100_000
    # the gathered records are the one run's accepted draws, rank 0's first
    import paper_2411_16952_gb300 as T
    g = T.decode_records(allrec, K)
    total, rec = O.run_accepted(pt, 7, 3, 0, n, cap=1 << 16)
    assert len(g["idx"]) == total == merged[0]["n_accepted"]
    assert np.array_equal(np.sort(g["idx"]), np.sort(rec["idx"]))
    assert np.all(np.diff(g["idx"][g["idx"] < D.shard_range(n, 1, 2)[0]].astype(np.int64)) > 0)
    o = np.argsort(rec["idx"])
    assert np.array_equal(g["xhat"][np.argsort(g["idx"])], rec["xhat"][o][:, :2 * K].astype(np.float32))
    assert np.array_equal(only0, rank0)


def test_shard_range_covers_exactly():
    for total in (0, 1, 7, 1000, 2**33 + 5):
        for world in (1, 2, 3, 8):
            parts = [D.shard_range(total, r, world) for r in range(world)]
            assert sum(c for _, c in parts) == total
            pos = 0
            for s, c in parts:
                assert s == pos
                pos += c
