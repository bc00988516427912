"""Pins of the oracle's lowest-bucket scan (orc_tail_scan).

The scan lists the proposals whose stream holds a word below 512 (the lowest
bucket of the uniform map, refined from further Philox blocks) at a radius
position (word 0 of block j for mode 2j+1, word 2 of block j for mode 2j+2 <= K)
or at the accept position (word 0 of block ceil(K/2)).  It decides which draws
the refined-tail GPU tests expect, so it is checked here against the stream
itself (each reported index recomputed word by word from the oracle's Philox
block, which is pinned against Triton's implementation) and against the law
of the stream: every word is uniform on 2^32 values, so a proposal has a
lowest-bucket word at one of its K + 1 positions with probability
1 - (1 - 2^-23)^(K+1), and each position is hit equally often.
"""
import math

import numpy as np

import oracle as O

P_WORD = 2.0 ** -23


def positions(K):
    """(block, word, kind) of every position the scan checks."""
    out = []
    for j in range((K + 1) // 2):
        out.append((j, 0, "radius"))
        if 2 * j + 2 <= K:
            out.append((j, 2, "radius"))
    out.append(((K + 1) // 2, 0, "accept"))
    return out


def low_positions(K, seed, pid, idx):
    """Positions of proposal idx whose word is in the lowest bucket, and the
    lowest-bucket words at positions the scan must not look at."""
    key = (seed & 0xFFFFFFFF, seed >> 32)
    hit, stray = [], []
    checked = {(b, w) for b, w, _ in positions(K)}
    for b in range((K + 1) // 2 + 1):
        words = O.philox((b, idx & 0xFFFFFFFF, idx >> 32, pid), key)
        for w in range(4):
            if words[w] < 512:
                (hit if (b, w) in checked else stray).append((b, w))
    return hit, stray


def test_tail_scan_reports_exactly_lowest_bucket_positions_k2():
    """K = 2 over 2^27 indices crossing the 2^32 boundary of idx (both counter
    words): every reported index has a lowest-bucket word at a checked
    position; every position occurs; the count matches the stream's law; the
    accept-only scan returns exactly the hits at the accept position."""
    K, seed, pid = 2, (5 << 32) | 11, 9
    n = 1 << 27
    idx0 = (1 << 32) - (n // 2)
    idx, tot = O.tail_scan(K, seed, pid, idx0, n, which=3, cap=1 << 12)
    assert tot == len(idx)
    assert np.all(np.diff(idx.astype(np.int64)) > 0) and idx.min() >= idx0 and idx.max() < idx0 + n
    seen = {}
    accept_hits = []
    for i in idx.tolist():
        hit, _ = low_positions(K, seed, pid, i)
        assert hit, "index %d has no lowest-bucket word at a checked position" % i
        for h in hit:
            seen[h] = seen.get(h, 0) + 1
        if ((K + 1) // 2, 0) in hit:
            accept_hits.append(i)
    # all three positions (mode 1 radius, mode 2 radius, accept) occur
    assert set(seen) == {(b, w) for b, w, _ in positions(K)}, seen
    p = 1.0 - (1.0 - P_WORD) ** (K + 1)
    mean = n * p
    assert abs(tot - mean) <= 4 * math.sqrt(mean), (tot, mean)
    # which = 2: the accept position only
    acc, tot2 = O.tail_scan(K, seed, pid, idx0, n, which=2, cap=1 << 12)
    assert acc.tolist() == accept_hits and tot2 == len(accept_hits)


def test_tail_scan_radius_positions_stop_at_mode_k():
    """K = 3 (odd): block 1 carries mode 3 in word 0 and no mode in word 2, so
    a lowest-bucket word 2 of block 1 must not make a hit.  Every reported
    index of the radius-only scan is explained by a radius word of modes 1..3;
    the count matches 1 - (1 - 2^-23)^3."""
    K, seed, pid = 3, 123456789, 0
    n = 1 << 26
    idx, tot = O.tail_scan(K, seed, pid, 0, n, which=1, cap=1 << 12)
    assert tot == len(idx)
    radius = {(b, w) for b, w, kind in positions(K) if kind == "radius"}
    assert (1, 2) not in radius
    for i in idx.tolist():
        hit, _ = low_positions(K, seed, pid, i)
        assert any(h in radius for h in hit), "index %d: no lowest-bucket radius word of modes 1..3" % i
    mean = n * (1.0 - (1.0 - P_WORD) ** K)
    assert abs(tot - mean) <= 4 * math.sqrt(mean), (tot, mean)


def test_tail_scan_counts_beyond_cap_and_empty_range():
    K, seed, pid = 2, 3, 1
    idx, tot = O.tail_scan(K, seed, pid, 0, 1 << 25, which=3, cap=2)
    full, tot_full = O.tail_scan(K, seed, pid, 0, 1 << 25, which=3, cap=1 << 10)
    assert tot == tot_full and idx.tolist() == full[:2].tolist()
    e, te = O.tail_scan(K, seed, pid, 17, 0, which=3)
    assert te == 0 and len(e) == 0
