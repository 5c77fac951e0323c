"""Host model of the contact substep loop's exchange protocol, with bounded waits.

The loop (k_iface_loop* with shared-memory replicas) runs one thread-block cluster of cs
CTAs. At each substep p a CTA sends its chunk to every peer with a bulk copy that
completes bytes on the receiver's mbarrier p & 1, arms its own barrier for the cs - 1
incoming chunks, and waits. A wait is bounded: if it gives up, the CTA stops exchanging
(sends and arms nothing more) and, after a cluster barrier at which every CTA has
published how many chunks it sent, drains the copies still addressed to it before a
closing cluster barrier (iface_drain). This model restates that protocol step by step
(mbarrier phases with pending arrivals and transaction counts; copies in flight that land
in any order; waits that give up at random) and checks, over many random schedules, that
  * without give-ups every CTA completes every substep;
  * every drain wait completes (it waits only for copies that were issued), and
  * at the closing barrier no copy is in flight, so no CTA exits while a copy from or into
    its shared memory can still land.
The device code's accounting (which phases a drain completes or arms, and with how many
bytes) is the function `drain` below, written as the kernel writes it.
"""

import random

import pytest

B = 1  # bytes of one chunk (any positive value)


class Barrier:
    def __init__(self):
        self.pending, self.tx, self.completed = 1, 0, 0

    def _check(self):
        if self.pending == 0 and self.tx == 0:
            self.completed += 1
            self.pending = 1

    def arrive_expect(self, nbytes):
        self.tx += nbytes
        self.pending -= 1
        assert self.pending >= 0, "arrive on a phase with no pending arrival"
        self._check()

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        self._check()

    def done(self, parity):  # mbarrier.try_wait.parity
        return (self.completed & 1) != parity


class Cta:
    def __init__(self, rank):
        self.rank = rank
        self.bar = [Barrier(), Barrier()]
        self.phase = [0, 0]
        self.p = 1
        self.n_sent = 0
        self.cta_to = False
        self.stage = "send"  # send -> wait -> (next p) ... -> end


def drain(x, sent, cs, P, bars):
    """iface_drain: the phases to wait for, after completing or arming them as the kernel does."""
    n = x.n_sent
    peers_sent = lambda p: sum(1 for q in range(cs) if q != x.rank and sent[q] >= p)
    done_phases = lambda b: n // 2 if b == 1 else (n - 1) // 2
    waits = []
    b = n & 1
    missing = (cs - 1 - peers_sent(n)) * B
    if missing:
        bars[b].complete_tx(missing)
    waits.append((b, done_phases(b) & 1))
    if n + 1 <= P:
        b = (n + 1) & 1
        arriving = peers_sent(n + 1) * B
        if arriving:
            bars[b].arrive_expect(arriving)
            waits.append((b, done_phases(b) & 1))
    return waits


def simulate(cs, P, p_give_up, rng):
    ctas = [Cta(r) for r in range(cs)]
    flight = []  # (dst, barrier index, substep)

    def land(k):
        dst, b, p = flight.pop(k)
        ctas[dst].bar[b].complete_tx(B)

    # the loop, until every CTA reached the first closing barrier
    steps = 0
    while any(c.stage != "end" for c in ctas):
        steps += 1
        assert steps < 100000, "loop did not end"
        live = [c for c in ctas if c.stage != "end"]
        if flight and rng.random() < 0.5:
            land(rng.randrange(len(flight)))
            continue
        x = rng.choice(live)
        if x.stage == "send":
            if x.cta_to or x.p > P:
                x.stage = "end"
                continue
            for q in range(cs):
                if q != x.rank:
                    flight.append((q, x.p & 1, x.p))
            x.bar[x.p & 1].arrive_expect((cs - 1) * B)
            x.n_sent = x.p
            x.stage = "wait"
        elif x.stage == "wait":
            b = x.p & 1
            if x.bar[b].done(x.phase[b]):
                x.phase[b] ^= 1
                x.p += 1
                x.stage = "send"
            elif rng.random() < p_give_up:  # the wait's poll budget ran out
                x.phase[b] ^= 1
                x.cta_to = True
                x.p += 1
                x.stage = "send"
    # every copy a CTA sends is issued before this barrier; the counts are published
    sent = [c.n_sent for c in ctas]
    for c in ctas:
        assert c.n_sent <= P
        if not c.cta_to:
            assert c.n_sent == P
    # a CTA whose waits all completed has nothing in flight towards it
    for dst, _, _ in flight:
        assert ctas[dst].cta_to
    waits = {c.rank: drain(c, sent, cs, P, c.bar) for c in ctas if c.cta_to}
    # the drains wait while the issued copies land, in any order
    guard = 0
    while True:
        pending = [(r, w) for r, ws in waits.items() for w in ws if not ctas[r].bar[w[0]].done(w[1])]
        if not pending:
            break
        assert flight, f"a drain waits for bytes no copy will bring: {pending}"
        land(rng.randrange(len(flight)))
        guard += 1
        assert guard < 100000
    # the closing barrier: nothing in flight
    assert not flight, flight
    return sum(c.cta_to for c in ctas)


@pytest.mark.parametrize("cs", [2, 3, 4, 16])
@pytest.mark.parametrize("P", [1, 2, 3, 20])
def test_no_give_up_completes_every_substep(cs, P):
    rng = random.Random(cs * 100 + P)
    for _ in range(20):
        assert simulate(cs, P, 0.0, rng) == 0


@pytest.mark.parametrize("cs", [2, 3, 4, 16])
@pytest.mark.parametrize("P", [1, 2, 3, 20])
@pytest.mark.parametrize("p_give_up", [0.02, 0.3, 1.0])
def test_drain_leaves_no_copy_in_flight(cs, P, p_give_up):
    rng = random.Random(cs * 1000 + P * 10 + int(100 * p_give_up))
    gave_up = 0
    for _ in range(60):
        gave_up += simulate(cs, P, p_give_up, rng)
    assert gave_up > 0  # the give-up path was exercised
