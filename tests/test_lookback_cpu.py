"""CPU emulation of the onesweep sort's decoupled look-back (Sec. 3.2 "Global
Sorting and Tiling" asks for a stable sort; this is the protocol one pass of
the single-sweep form uses to find, for every digit, how many items of that
digit all earlier blocks hold).  It restates the protocol of
k_radix_scatter's look-back in Python; it does not run the kernel, whose
timeout path a GPU test drives with lp_debug_sort_stall.

Blocks take dynamic ids in start order.  Each block publishes its own count of
a digit as a status word (flag AGG, or INC for block 0), walks back over
earlier blocks' words -- a window of them read together, then taken in order,
re-reading a word that is not yet published -- summing counts until it meets
an INC word, and then publishes its inclusive count (INC).  Every wait is
bounded: a block that gives up latches a timeout status and its result is
invalid, but it still writes nothing outside the output.

The emulation interleaves blocks at random (each memory access is a
scheduling point) and checks: exact exclusive prefixes for every block and
digit without a stall, whatever the interleaving and window, with every output
slot written exactly once; with one block that never publishes, a latched
timeout and correct prefixes up to that block.  It needs no GPU."""
import random

import numpy as np

AGG, INC = 1 << 30, 2 << 30
FLAGS = AGG | INC
VAL = (1 << 30) - 1


def run(counts, window, seed, stall=-1, wait_limit=200, concurrency=6):
    """counts[b][d]: items of digit d in block b.  Returns (prefix[b][d] or
    None where the block timed out, timeout flag, writes per output slot).
    Block b's i-th item of digit d goes to slot base[d] + prefix + i, base[d]
    being all items of smaller digits; as in the kernel, a slot at or past n
    is never written."""
    nb, R = counts.shape
    status = np.zeros((nb, R), np.int64)
    rng = random.Random(seed)
    prefix = [[None] * R for _ in range(nb)]
    state = {"timeout": False}
    n_total = int(counts.sum())
    base = np.concatenate([[0], np.cumsum(counts.sum(0))[:-1]])
    written = np.zeros(n_total + 1, np.int64)

    def block(b):
        # publish own counts
        for d in range(R):
            if b != stall:
                status[b, d] = (INC if b == 0 else AGG) | int(counts[b, d])
            yield
        for d in range(R):
            pre, found, timed_out = 0, b == 0, False
            j0 = b - 1
            while j0 >= 0 and not found:
                win = []
                for u in range(window):
                    win.append(int(status[j0 - u, d]) if j0 - u >= 0 else INC)
                    yield
                for u in range(window):
                    if found:
                        break
                    v = win[u]
                    if not v & FLAGS:
                        spins = 0
                        while True:
                            v = int(status[j0 - u, d])
                            yield
                            if v & FLAGS:
                                break
                            spins += 1
                            if spins > wait_limit:
                                state["timeout"] = True
                                timed_out = True
                                v = INC
                                break
                    pre += v & VAL
                    found = bool(v & INC)
                j0 -= window
            if b != stall:
                status[b, d] = INC | ((pre + int(counts[b, d])) & VAL)
            prefix[b][d] = None if timed_out else pre
            for i in range(int(counts[b, d])):
                g = int(base[d]) + pre + i
                if g < n_total:
                    written[g] += 1
            yield

    pending = list(range(nb))       # dynamic ids: blocks start in id order
    running = []
    while pending or running:
        while pending and len(running) < concurrency:
            b = pending.pop(0)
            running.append((b, block(b)))
        i = rng.randrange(len(running))
        b, co = running[i]
        try:
            next(co)
        except StopIteration:
            running.pop(i)
    return prefix, state["timeout"], written[:n_total]


def _exclusive(counts):
    return np.vstack([np.zeros((1, counts.shape[1]), np.int64), np.cumsum(counts, 0)[:-1]])


def test_lookback_gives_exact_prefixes_under_any_interleaving():
    rng = np.random.default_rng(0)
    for trial in range(12):
        nb, R = int(rng.integers(1, 40)), int(rng.integers(1, 5))
        counts = rng.integers(0, 50, size=(nb, R))
        for window in (1, 3, 8):
            prefix, timeout, written = run(counts, window, seed=trial * 10 + window)
            assert not timeout
            np.testing.assert_array_equal(np.array(prefix, np.int64), _exclusive(counts))
            assert (written == 1).all()     # every output slot exactly once: a permutation


def test_a_block_that_never_publishes_times_out_the_blocks_after_it():
    rng = np.random.default_rng(1)
    counts = rng.integers(0, 50, size=(24, 3))
    for stall in (0, 5, 23):
        for window in (1, 8):
            prefix, timeout, written = run(counts, window, seed=stall + window, stall=stall)
            ex = _exclusive(counts)
            for b in range(stall + 1):      # up to the stalled block itself: exact
                assert prefix[b] == [int(x) for x in ex[b]], (b, stall)
            if stall < 23:
                assert timeout              # someone after it waited in vain
                assert any(prefix[b][d] is None for b in range(stall + 1, 24) for d in range(3))


def test_wait_bound_ends_the_emulation():
    """With the first block stalled and a tiny wait limit, the run still ends
    (every wait is bounded) with the timeout latched."""
    counts = np.ones((6, 2), np.int64)
    prefix, timeout, written = run(counts, 8, seed=3, stall=0, wait_limit=5, concurrency=6)
    assert timeout
