"""CPU emulation of sort mode 2's per-tile depth sort (Sec. 3.2 "Global
Sorting and Tiling": entries of a tile ordered front to back, ties by record).

Each tile's run arrives in record order and is sorted stably by the records'
depth bits, so the result is (depth, record) order.  The kernels (k_tile_sort,
k_tile_sort_long) do it as an LSD radix sort with 8-bit digits and skip a digit
whose value is the same for every entry of the run.  A warp takes the run in
rounds of 32 entries: the lanes holding the same digit are found with one
ballot per digit bit, a lane's rank among them is the number of such lanes
before it, and a running count per digit places each round after the earlier
ones.  A block holding a run of up to 2048 entries in shared memory gives
warp w the w-th contiguous share of it, ranks each share round by round, and
places an entry at its digit's start plus the earlier warps' counts of that
digit plus its rank within its warp.  A block sorting a longer run through
global memory takes it in chunks of 256 entries, ranks each chunk per warp,
adds the counts of the chunk's earlier warps for the same digit, and then the
running per-digit offsets.

This restates those steps in Python and checks them against numpy's stable
argsort on the (depth bits, record) pairs: runs of every length up to several
chunks, many equal depths, depths whose top bytes agree (skipped digits), and
extreme values.  It does not run the kernels; the GPU tests compare their
tile lists with the oracle bit for bit.  It needs no GPU."""
import numpy as np
import pytest


def digit_peers(digits, lane):
    """Lanes of the round whose digit equals this lane's, as the ballots find
    them: one ballot per bit of the digit field (9 bits; 256 marks no item)."""
    m = (1 << len(digits)) - 1
    d = digits[lane]
    for b in range(9):
        bit = (d >> b) & 1
        ballot = sum(1 << l for l, x in enumerate(digits) if (x >> b) & 1)
        m &= ballot if bit else ~ballot
    return m


def varying_digits(keys):
    o, a = 0, 0xFFFFFFFF
    for k in keys:
        o |= int(k)
        a &= int(k)
    diff = o & ~a
    return [s for s in range(0, 32, 8) if (diff >> s) & 255]


def warp_sort(keys, vals):
    """One warp's sort of a run (k_tile_sort): histogram, exclusive scan, then
    rounds of 32 entries in order."""
    keys, vals = list(keys), list(vals)
    n = len(keys)
    for shift in varying_digits(keys):
        cnt = [0] * 256
        for k in keys:
            cnt[(k >> shift) & 255] += 1
        off, run = [0] * 256, 0
        for d in range(256):
            off[d], run = run, run + cnt[d]
        nk, nv = [None] * n, [None] * n
        for base in range(0, n, 32):
            idx = list(range(base, min(base + 32, n)))
            digits = [(keys[i] >> shift) & 255 for i in idx] + [256] * (32 - len(idx))
            ranks, firsts = {}, {}
            for lane, i in enumerate(idx):
                peers = digit_peers(digits, lane)
                ranks[lane] = bin(peers & ((1 << lane) - 1)).count("1")
                if ranks[lane] == 0:
                    firsts[digits[lane]] = bin(peers).count("1")
            starts = {d: off[d] for d in firsts}          # read before the leaders add
            for d, c in firsts.items():
                off[d] += c
            for lane, i in enumerate(idx):
                pos = starts[digits[lane]] + ranks[lane]
                nk[pos], nv[pos] = keys[i], vals[i]
        keys, vals = nk, nv
    return keys, vals


def block_sort(keys, vals, threads=256):
    """A block's sort of a long run (k_tile_sort_long): per pass, digit counts
    and their scan, then chunks of `threads` entries in order, each ranked by
    warp, then by the counts of the chunk's earlier warps."""
    keys, vals = list(keys), list(vals)
    n, nw = len(keys), threads // 32
    for shift in varying_digits(keys):
        cnt = [0] * 256
        for k in keys:
            cnt[(k >> shift) & 255] += 1
        base, run = [0] * 256, 0
        for d in range(256):
            base[d], run = run, run + cnt[d]
        nk, nv = [None] * n, [None] * n
        for c0 in range(0, n, threads):
            chunk = list(range(c0, min(c0 + threads, n)))
            digit = {i: (keys[i] >> shift) & 255 for i in chunk}
            wcnt = [[0] * 256 for _ in range(nw)]
            rank = {}
            for w in range(nw):
                idx = [i for i in chunk if (i - c0) // 32 == w]
                if not idx:
                    continue
                digits = [digit[i] for i in idx] + [256] * (32 - len(idx))
                for lane, i in enumerate(idx):
                    peers = digit_peers(digits, lane)
                    rank[i] = bin(peers & ((1 << lane) - 1)).count("1")
                    if rank[i] == 0:
                        wcnt[w][digit[i]] = bin(peers).count("1")
            for i in chunk:
                w, d = (i - c0) // 32, digit[i]
                pos = base[d] + rank[i] + sum(wcnt[ww][d] for ww in range(w))
                nk[pos], nv[pos] = keys[i], vals[i]
            for d in range(256):
                base[d] += sum(wcnt[w][d] for w in range(nw))
        keys, vals = nk, nv
    return keys, vals


def block_sort_smem(keys, vals, threads=256, drop_earlier_warps=False):
    """A block's sort of a run held in shared memory (k_tile_sort_long, runs
    of up to 2048 entries): per pass, warp w takes the w-th contiguous share of
    the run (whole rounds of 32), ranks it round by round with a running count
    per (warp, digit), and an entry goes to its digit's start plus the counts
    of the earlier warps for that digit plus its rank within its warp."""
    keys, vals = list(keys), list(vals)
    n, nw = len(keys), threads // 32
    per_warp = ((n + nw - 1) // nw + 31) & ~31
    for shift in varying_digits(keys):
        wcnt = [[0] * 256 for _ in range(nw)]
        packed = {}                                   # entry -> (digit, rank within its warp)
        for w in range(nw):
            for r in range(per_warp // 32):
                idx = [i for i in range(w * per_warp + r * 32, w * per_warp + r * 32 + 32) if i < n]
                if not idx:
                    continue
                digits = [(keys[i] >> shift) & 255 for i in idx] + [256] * (32 - len(idx))
                base = {d: wcnt[w][d] for d in set(digits[:len(idx)])}   # read before the leaders add
                for lane, i in enumerate(idx):
                    peers = digit_peers(digits, lane)
                    rank = bin(peers & ((1 << lane) - 1)).count("1")
                    packed[i] = (digits[lane], base[digits[lane]] + rank)
                    if rank == 0:
                        wcnt[w][digits[lane]] = base[digits[lane]] + bin(peers).count("1")
        before = [[0 if drop_earlier_warps else sum(wcnt[ww][d] for ww in range(w)) for d in range(256)]
                  for w in range(nw)]
        totals = [sum(wcnt[w][d] for w in range(nw)) for d in range(256)]
        start, run = [0] * 256, 0
        for d in range(256):
            start[d], run = run, run + totals[d]
        nk, nv = [None] * n, [None] * n
        for i, (d, rank) in packed.items():
            w = i // per_warp
            pos = start[d] + before[w][d] + rank
            assert drop_earlier_warps or nk[pos] is None
            nk[pos], nv[pos] = keys[i], vals[i]
        keys, vals = nk, nv
    return keys, vals


def reference(keys, vals):
    order = np.lexsort((np.asarray(vals, np.uint64), np.asarray(keys, np.uint64)))
    return [int(keys[i]) for i in order], [int(vals[i]) for i in order]


def depth_bits(z):
    return np.asarray(z, np.float32).view(np.uint32)


def runs(seed):
    rng = np.random.default_rng(seed)
    yield depth_bits(rng.uniform(0.2, 30.0, 37))                       # ragged, all digits vary
    yield depth_bits(np.repeat(rng.uniform(1.0, 1.5, 13), 11)[:140])   # long runs of equal depths
    yield depth_bits(rng.uniform(2.0, 2.001, 300))                     # top bytes equal: digits skipped
    yield depth_bits(np.full(65, 7.0))                                 # one depth: nothing to sort
    z = rng.uniform(0.2, 1e30, 90)
    z[::7] = np.float32(np.finfo(np.float32).max)
    z[3::11] = np.float32(0.2)
    yield depth_bits(z)                                                # extremes
    yield depth_bits(rng.uniform(0.5, 40.0, 1))                        # a single entry
    yield depth_bits(rng.choice(rng.uniform(0.2, 5.0, 40), 700))       # several chunks, many ties
    yield depth_bits(rng.uniform(0.3, 12.0, 2048))                     # the largest run held in shared memory
    yield depth_bits(rng.choice(rng.uniform(1.0, 3.0, 9), 1531))       # ragged shares, few distinct depths


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_per_tile_sort_steps_are_stable_and_exact(seed):
    for keys in runs(seed):
        n = len(keys)
        vals = np.sort(np.random.default_rng(seed + n).choice(1 << 20, n, replace=False))  # record order
        want = reference(keys, vals)
        if n <= 512:
            assert warp_sort(keys, vals) == want, n
        assert block_sort(keys, vals) == want, n
        assert block_sort(keys, vals, threads=64) == want, n
        if n <= 2048:
            assert block_sort_smem(keys, vals) == want, n
            assert block_sort_smem(keys, vals, threads=64) == want, n


def test_skipped_digits_are_the_constant_ones():
    keys = depth_bits([2.0, 2.0000002, 2.0000005, 2.0000010])
    assert varying_digits(keys) == [0]                    # only the low byte differs
    keys = depth_bits([0.25, 16.0])
    assert 24 in varying_digits(keys)                     # exponents differ in the top byte
    assert varying_digits(depth_bits([3.0] * 5)) == []    # one value: no pass at all


def test_planted_instability_is_caught():
    """A rank that counts the lanes after a lane instead of before it (a
    plausible slip) reverses equal digits within a round, and the check sees
    it."""
    keys = depth_bits(np.repeat([1.0, 2.0], 20))
    vals = list(range(40))

    def unstable(keys, vals):
        keys, vals = list(keys), list(vals)
        n = len(keys)
        for shift in varying_digits(keys):
            digits = [(k >> shift) & 255 for k in keys]
            order = sorted(range(n), key=lambda i: (digits[i], -(i % 32), i // 32))
            keys, vals = [keys[i] for i in order], [vals[i] for i in order]
        return keys, vals

    assert unstable(keys, vals) != reference(keys, vals)
    assert warp_sort(keys, vals) == reference(keys, vals)


def test_planted_missing_warp_offsets_are_caught():
    """Leaving out the earlier warps' counts of a digit (a plausible slip in
    the shared-memory block form) puts two warps' entries in the same places,
    and the check sees it."""
    keys = depth_bits(np.random.default_rng(5).uniform(0.5, 9.0, 600))
    vals = list(range(600))
    try:
        got = block_sort_smem(keys, vals, drop_earlier_warps=True)
    except TypeError:     # holes left by the collisions reach the next pass
        got = None
    assert got != reference(keys, vals)
    assert block_sort_smem(keys, vals) == reference(keys, vals)
