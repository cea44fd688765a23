"""The producer/consumer protocol of the packed-operator kernel (k_iface_sym.cu), on the CPU.

One producer thread bulk-copies 32 x 32 tiles of K into shared-memory slots; consumer warp
w takes the tiles J = w, w + CW, ... of every output row tile, and the consumer warps
meet at a barrier after each row tile (their partial sums are combined).  Each slot has a
"full" mbarrier (the copy landed) and an "empty" one (its warp is done with it).  The
waits use the parity form: ``mbarrier.try_wait.parity P`` succeeds when the barrier's
current phase has the other parity, i.e. after c completed phases it passes iff
``c % 2 != P`` (so before the first completion a wait for parity 1 passes at once).  A
parity wait is therefore only right when the waiter is at most one phase behind; the
model below checks that the kernel's slot assignment keeps it so.

Kernel protocol (CW consumer warps, D slots per warp, fills counted per warp):
* producer, tile J of a row tile: warp cw = J mod CW, its fill n; slot cw*D + n mod D;
  for n >= D wait on empty[slot] with parity (n/D - 1) & 1; then post the copy.
* consumer warp w, its n-th tile: slot w*D + n mod D; wait on full[slot] with parity
  (n/D) & 1; read; arrive on empty[slot].

The model runs the producer, the copies (landing in any order) and the consumers under
random interleavings and checks that every consumer read finds the tile it expects and
that the run never deadlocks.  A single ring shared by all warps in fill order (the
kernel's first form) is the negative control: consumers that drift more than one lap
apart alias parities there, and the model finds the stale reads that form produced.
"""
import os
import random
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2209_10886_gb300", "csrc", "k_iface_sym.cu")


def kernel_constants():
    text = open(SRC).read()
    cw = int(re.search(r"constexpr int CW = (\d+);", text).group(1))
    d = int(re.search(r"constexpr int D = (\d+);", text).group(1))
    return cw, d


def passes(completed, parity):
    """mbarrier.try_wait.parity after `completed` phases (one arrival per phase)."""
    return completed % 2 != parity


def simulate(row_tiles, CW, D, seed, shared_ring=0):
    """row_tiles: tile count nt of each output row tile a CTA streams in order.
    shared_ring > 0: one ring of that many slots filled in order (the negative control).
    Returns "ok", "stale read" or "deadlock"."""
    rnd = random.Random(seed)
    nslots = shared_ring if shared_ring else CW * D
    full = [0] * nslots                    # completed phases of each barrier
    empty = [0] * nslots
    content = [None] * nslots
    order = [(t, J) for t, nt in enumerate(row_tiles) for J in range(nt)]
    fills = [0] * CW
    p = 0                                  # next tile the producer posts
    in_flight = []                         # (slot, tile) copies not landed yet
    # consumer programs: ("tile", t, J, q) with q the tile's index in the producer's
    # order, then ("sync", t) after each row tile
    progs = []
    for w in range(CW):
        ops, base = [], 0
        for t, nt in enumerate(row_tiles):
            ops += [("tile", t, J, base + J) for J in range(w, nt, CW)]
            ops.append(("sync", t))
            base += nt
        progs.append(ops)
    pc = [0] * CW
    taken = [0] * CW                       # tiles warp w has taken from its slots
    arrived = {}
    at_sync = [None] * CW

    def consumer_slot(w, op):
        if shared_ring:
            q = op[3]
            return q % shared_ring, (q // shared_ring) & 1
        n = taken[w]
        return w * D + n % D, (n // D) & 1

    while True:
        moves = []
        if p < len(order):
            t, J = order[p]
            if shared_ring:
                slot, k = p % shared_ring, p // shared_ring
                ok = k == 0 or passes(empty[slot], (k - 1) & 1)
            else:
                cw = J % CW
                n = fills[cw]
                slot = cw * D + n % D
                ok = n < D or passes(empty[slot], (n // D - 1) & 1)
            if ok:
                moves.append(("post", slot))
        if in_flight:
            moves.append(("land",))
        for w in range(CW):
            if pc[w] >= len(progs[w]):
                continue
            op = progs[w][pc[w]]
            if op[0] == "tile":
                slot, parity = consumer_slot(w, op)
                if passes(full[slot], parity):
                    moves.append(("read", w, slot))
            else:
                moves.append(("sync", w))
        if not moves:
            done = p == len(order) and not in_flight and all(pc[w] >= len(progs[w]) for w in range(CW))
            return "ok" if done else "deadlock"
        m = rnd.choice(moves)
        if m[0] == "post":
            if not shared_ring:
                fills[order[p][1] % CW] += 1
            in_flight.append((m[1], order[p]))
            p += 1
        elif m[0] == "land":
            slot, tile = in_flight.pop(rnd.randrange(len(in_flight)))
            content[slot] = tile
            full[slot] += 1
        elif m[0] == "read":
            w, slot = m[1], m[2]
            op = progs[w][pc[w]]
            if content[slot] != (op[1], op[2]):
                return "stale read"
            empty[slot] += 1
            taken[w] += 1
            pc[w] += 1
        else:
            w = m[1]
            t = progs[w][pc[w]][1]
            if at_sync[w] != t:
                arrived[t] = arrived.get(t, 0) + 1
                at_sync[w] = t
            if arrived[t] == CW:
                pc[w] += 1


# tile counts per row tile: the bench workload's subdomains (512 boundary points: 16
# tiles), ragged ones, 256-node subdomains (32 tiles), fewer tiles than warps, and mixes
# of subdomains within one CTA's range
MIXES = [[16] * 4, [16] * 3, [4] * 10, [32], [16, 24, 32], [12, 16, 8], [2] * 30, [24, 16, 16, 32], [9, 17, 5]]


def test_model_reads_the_kernel_constants():
    cw, d = kernel_constants()
    assert cw >= 1 and d >= 1


@pytest.mark.parametrize("D", sorted({kernel_constants()[1], 1, 2}))
def test_per_warp_slots_never_read_stale_data_or_deadlock(D):
    CW = kernel_constants()[0]
    for nts in MIXES:
        results = {simulate(nts, CW, D, seed) for seed in range(60)}
        assert results == {"ok"}, (nts, D, results)


def test_a_shared_ring_aliases_parities():
    """The negative control: one ring of 12 slots shared by the warps in fill order
    reads stale tiles under some interleavings (consumers more than a lap apart)."""
    CW = kernel_constants()[0]
    results = set()
    for nts in MIXES:
        results |= {simulate(nts, CW, 1, seed, shared_ring=12) for seed in range(60)}
    assert "stale read" in results


def test_parity_rule_matches_the_ptx_semantics():
    """Before any completion a wait for parity 0 blocks and one for parity 1 passes;
    after one completion the reverse; after two, parity 0 blocks again (the alias)."""
    assert not passes(0, 0) and passes(0, 1)
    assert passes(1, 0) and not passes(1, 1)
    assert not passes(2, 0) and passes(2, 1)
