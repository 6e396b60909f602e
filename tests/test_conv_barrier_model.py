"""Model check of the barrier protocol of the persistent tensor-core convolution
(k_conv3_tc): its five roles as coroutines over mbarriers with phase counts, run under
random interleavings, with the asynchronous completions (TMA copies landing, MMA commits
arriving) delayed at random.

Roles and barriers, as the kernel has them:
  TMA thread   raw row k (halo row k % HR of unit k // HR) into slot k % RS once
               st_empty[k % RS] shows the slot's previous row consumed; weight granules
               into ring slots once w_empty shows them released (or all at once when the
               layer's granules fit: resident);
  transposers  halo row hr of unit u from raw row k once st_full shows it landed and
               h_empty[hr] shows unit u - 1's products done with it; arrive h_full[hr],
               st_empty[k % RS] (four warps: count 4);
  MMA thread   per tile the accumulator (t_empty), per unit the halo rows and weights in
               the order of its form, commits to h_empty / w_empty / t_full;
  epilogue     per tile t_full, then t_empty (four warps); in the stacked form it first
               zeroes both accumulators and arrives on t_empty once each.
Forms: tap rows (Cout 64 / 128: a granule is the three boxes of one (channel block, dy),
halo rows released after the last tap row reading them), per-tap granules (Cout 256,
operands swapped), stacked (Cout 32: three (channel block, dx) granules per unit, each
halo row released after its own products, every tile waits for its zeroed accumulator).

The checks: every run terminates (no deadlock for any interleaving tried), a product reads
halo rows written for its own unit and weight slots holding its own boxes, and the
epilogue drains every tile's accumulator after that tile's products, in order. Parity
waits are modelled as the hardware does them (a phase of the given parity has completed),
so a wait that could pass on a stale phase shows up as a stale read."""
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

    def done(self, parity):  # the phase with this parity has completed
        return (self.phase & 1) != parity


def run(form, T, ncb, R, RS, seed):
    TR = 4 if form == "stacked" else 2
    HR = TR + 2
    if form == "taprows":
        GT, GPU, BPC = 3, 3, 9
    elif form == "pertap":
        GT, GPU, BPC = 1, 9, 9
    else:
        GT, GPU, BPC = 1, 3, 3
    rnd = random.Random(seed)
    U = T * ncb
    resident = GPU * ncb <= R
    st_full = [Bar(1) for _ in range(RS)]
    st_empty = [Bar(4) for _ in range(RS)]
    h_full = [Bar(4) for _ in range(HR)]
    h_empty = [Bar(1) for _ in range(HR)]
    t_full = [Bar(1), Bar(1)]
    t_empty = [Bar(4), Bar(4)]
    w_full = [Bar(1) for _ in range(R)]
    w_empty = [Bar(1) for _ in range(R)]
    raw, halo, wslot, acc = [None] * RS, [None] * HR, [None] * R, ["garbage", "garbage"]
    pending, drained, ndrained = [], [[] for _ in range(4)], [0] * T

    def tma():
        k = g = 0
        gtot = GPU * ncb if resident else GPU * U
        while k < U * HR or g < gtot:
            progress = False
            if k < U * HR and (k < RS or st_empty[k % RS].done(((k // RS) - 1) & 1)):
                def land(k=k):
                    raw[k % RS] = k
                    st_full[k % RS].arrive()
                pending.append(land)
                k += 1
                progress = True
            if g < gtot and (resident or g < R or w_empty[g % R].done(((g // R) - 1) & 1)):
                sl = g if resident else g % R
                box = GT * g if resident else ((g // GPU) % ncb) * BPC + (g % GPU) * GT

                def landw(sl=sl, box=box):
                    wslot[sl] = box
                    w_full[sl].arrive()
                pending.append(landw)
                g += 1
                progress = True
            yield progress

    def transposer():
        for k in range(U * HR):
            u, hr = divmod(k, HR)
            while not st_full[k % RS].done((k // RS) & 1):
                yield False
            while u > 0 and not h_empty[hr].done((u - 1) & 1):
                yield False
            assert raw[k % RS] == k, ("stale raw row", k)
            halo[hr] = u
            h_full[hr].arrive()
            st_empty[k % RS].arrive()
            yield True

    def wait_weights(u, cb, gi):
        """Wait for granule gi of unit u; returns its slot after checking its boxes."""
        g = u * GPU + gi
        sl = cb * GPU + gi if resident else g % R
        parity = 0 if resident else (g // R) & 1
        while not w_full[sl].done(parity):
            yield None
        assert wslot[sl] == cb * BPC + gi * GT, ("stale weights", u, gi)
        return sl

    def mma():
        for i in range(T):
            buf = i & 1
            if form == "stacked":
                while not t_empty[buf].done((i >> 1) & 1):
                    yield False
                # every product accumulates: the epilogue must have zeroed this accumulator
                assert acc[buf] == "zero", ("accumulator not zeroed", i)
            else:
                while i >= 2 and not t_empty[buf].done(((i >> 1) - 1) & 1):
                    yield False
            for cb in range(ncb):
                u = i * ncb + cb
                if form == "stacked":
                    slots = []
                    for dx in range(3):
                        sl = yield from wait_weights(u, cb, dx)
                        slots.append(sl)
                    for hr in range(HR):
                        while not h_full[hr].done(u & 1):
                            yield False
                        assert halo[hr] == u, ("stale halo", u, hr)
                        yield True
                        pending.append(lambda hr=hr: h_empty[hr].arrive())
                    if not resident:
                        for sl in slots:
                            pending.append(lambda sl=sl: w_empty[sl].arrive())
                    continue
                ready = 0
                for dy in range(3):
                    while ready < dy + TR:
                        while not h_full[ready].done(u & 1):
                            yield False
                        ready += 1
                    for r in range(TR):
                        assert halo[r + dy] == u, ("stale halo", u, r + dy)
                    for j in range(3 // GT):
                        sl = yield from wait_weights(u, cb, dy * (3 // GT) + j)
                        if not resident:
                            pending.append(lambda sl=sl: w_empty[sl].arrive())
                        yield True
                    if dy < 2:
                        pending.append(lambda dy=dy: h_empty[dy].arrive())
                    else:
                        for hr in range(2, HR):
                            pending.append(lambda hr=hr: h_empty[hr].arrive())
            acc[buf] = i
            pending.append(lambda buf=buf: t_full[buf].arrive())

    def epilogue(w):
        if form == "stacked":  # both accumulators zeroed before the first tile
            if w == 3:  # the four warps zero their lanes; modelled as one state change
                acc[0] = acc[1] = "zero"
            t_empty[0].arrive()
            t_empty[1].arrive()
            yield True
        for i in range(T):
            buf = i & 1
            while not t_full[buf].done((i >> 1) & 1):
                yield False
            assert acc[buf] == i, ("stale accumulator", i)
            drained[w].append(i)
            ndrained[i] += 1
            if form == "stacked" and ndrained[i] == 4:
                acc[buf] = "zero"  # drained by all four warps, then zeroed
            t_empty[buf].arrive()
            yield True

    roles = [tma()] + [transposer() for _ in range(4)] + [mma()] + [epilogue(w) for w in range(4)]
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
        assert stalled < 50000 or pending, ("deadlock", form, T, ncb, R, RS)
    assert all(d == list(range(T)) for d in drained), drained  # each warp drains every tile, in order


CASES = [("taprows", 3, 4), ("taprows", 2, 3), ("taprows", 6, 4),   # Cout 64 / 128 (and resident)
         ("pertap", 3, 2), ("pertap", 9, 2),                        # Cout 256, operands swapped
         ("stacked", 5, 3), ("stacked", 3, 3), ("stacked", 9, 3)]   # Cout 32, taps stacked


@pytest.mark.parametrize("form,R,RS", CASES)
def test_protocol_has_no_deadlock_and_no_stale_reads(form, R, RS):
    for ncb in (1, 2, 3):
        for T in (1, 2, 3, 7):
            for seed in range(4):
                run(form, T, ncb, R, RS, seed)
