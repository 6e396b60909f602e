"""Model check of the barrier protocol of the persistent tensor-core expansion
(k_tc_expand): a CTA's contiguous range of output tiles (tile row mt = t // tiles_n), its
TMA thread, MMA thread and four epilogue warps as coroutines over phase-counted mbarriers,
run under random interleavings with delayed copy and commit completions.

As the kernel has them:
  TMA thread   at the first tile of each tile row, the row's A operand into the single A
               buffer once a_empty shows the previous row's products done (a_full, one
               arrival with its bytes); then per tile its KB B slabs into a ring of S slots,
               each once b_empty shows the slot released;
  MMA thread   at a new tile row, a_full; per tile, the TMEM buffer ti & 1 once t_empty shows
               its previous tile drained (from the third tile on); per slab b_full, the
               products, a commit to b_empty; a commit to t_full per tile and to a_empty after
               the row's last tile in the range;
  epilogue     per tile t_full of buffer ti & 1, the accumulator into registers, then
               t_empty (one arrival per warp) before the stores.
The checks: every run terminates, a product reads the A rows of its own tile row and a slot
holding its own (tile, slab), and each warp drains every tile's accumulator, in order, after
that tile's products."""
import random

import pytest


class Bar:
    def __init__(self, count):
        self.count, self.pending, self.phase = count, count, 0

    def arrive(self):
        self.pending -= 1
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count

    def done(self, parity):
        return (self.phase & 1) != parity


def run(t0, t1, tiles_n, KB, S, seed):
    rnd = random.Random(seed)
    a_full, a_empty = Bar(1), Bar(1)
    b_full = [Bar(1) for _ in range(S)]
    b_empty = [Bar(1) for _ in range(S)]
    t_full = [Bar(1), Bar(1)]
    t_empty = [Bar(4), Bar(4)]
    a_row, slot, acc = [None], [None] * S, [None, None]
    pending, drained = [], [[] for _ in range(4)]

    def tma():
        aload, slab, prev_m = 0, 0, -1
        for t in range(t0, t1):
            mt = t // tiles_n
            if mt != prev_m:
                if aload > 0:
                    while not a_empty.done((aload - 1) & 1):
                        yield False
                pending.append(lambda mt=mt: (a_row.__setitem__(0, mt), a_full.arrive()))
                aload += 1
                prev_m = mt
            for kb in range(KB):
                sl = slab % S
                if slab >= S:
                    while not b_empty[sl].done(((slab // S) - 1) & 1):
                        yield False
                pending.append(lambda sl=sl, t=t, kb=kb: (slot.__setitem__(sl, (t, kb)), b_full[sl].arrive()))
                slab += 1
                yield True

    def mma():
        slab, aload, prev_m = 0, 0, -1
        for ti, t in enumerate(range(t0, t1)):
            mt = t // tiles_n
            if mt != prev_m:
                while not a_full.done(aload & 1):
                    yield False
                aload += 1
                prev_m = mt
            buf = ti & 1
            while ti >= 2 and not t_empty[buf].done(((ti >> 1) - 1) & 1):
                yield False
            for kb in range(KB):
                sl = slab % S
                while not b_full[sl].done((slab // S) & 1):
                    yield False
                assert a_row[0] == mt, ("stale A rows", t, a_row[0])
                assert slot[sl] == (t, kb), ("stale B slab", t, kb, slot[sl])
                pending.append(lambda sl=sl: b_empty[sl].arrive())
                slab += 1
                yield True
            acc[buf] = t
            pending.append(lambda buf=buf: t_full[buf].arrive())
            if t + 1 >= t1 or (t + 1) // tiles_n != mt:
                pending.append(a_empty.arrive)

    def epilogue(w):
        for ti, t in enumerate(range(t0, t1)):
            buf = ti & 1
            while not t_full[buf].done((ti >> 1) & 1):
                yield False
            assert acc[buf] == t, ("stale accumulator", t, acc[buf])
            drained[w].append(t)
            t_empty[buf].arrive()  # released once in registers; the stores follow
            yield True

    roles = [tma(), mma()] + [epilogue(w) for w in range(4)]
    stalled = 0
    while roles or pending:
        if pending and (not roles or rnd.random() < 0.3):
            pending.pop(rnd.randrange(len(pending)))()
            stalled = 0
            continue
        role = rnd.choice(roles)
        try:
            stalled = 0 if next(role) else stalled + 1
        except StopIteration:
            roles.remove(role)
            stalled = 0
        assert stalled < 50000 or pending, ("deadlock", t0, t1, tiles_n, KB, S)
    assert all(d == list(range(t0, t1)) for d in drained), drained


@pytest.mark.parametrize("tiles_n,KB,S", [(1, 2, 4), (3, 2, 4), (4, 3, 2), (5, 1, 3), (2, 4, 8)])
def test_protocol_has_no_deadlock_and_no_stale_reads(tiles_n, KB, S):
    for t0, t1 in [(0, 1), (0, 7), (2, 9), (5, 6), (3, 20)]:
        for seed in range(4):
            run(t0, t1, tiles_n, KB, S, seed)
