"""CPU models of the three shared-memory rings through which the adjoint kernels and the FMA
contraction stream their rows, checked over many step counts, ring depths and sequences of work
items.

* Per-lane cp.async ring (the checkpointing adjoint's strip tape, K = 4; the FD adjoint, D = 4, 6
  or 8). Each lane copies its own vectors. An item's steps t = n - 1 .. 0 live in slot t mod D.
  The prologue commits one group per step n - 1 .. n - D, empty past step 0. Then, per step,
  the lane waits until at most D - 1 of its groups are pending (cp.async.wait_group), reads the
  slot, and commits the group that refills it with step t - D.
* Bulk-copy ring with one mbarrier per slot (the tape adjoint, 4 slots). Lane 0 issues the
  copies. The warp waits on a slot's barrier for the phase parity it tracks in a register that
  persists across items, flips the bit, reads the slot, and then has lane 0 refill it with step
  t - 4.
* The FMA contraction's ring of three 32-row halves. Per strip and column window of ntiles
  tiles, half h goes to slot h mod 3: halves 0..min(2, ntiles) first. Tile b waits for half b
  (tile 0 only; later tiles got it as the upper half of the tile before) and for half b + 1,
  reads both, then refills slot b mod 3 with half b + 3 while b + 3 <= ntiles. The parity bits
  persist across strips and windows.

A copy's data may land at any moment until the wait that covers it returns. The model lets
every copy land as late as possible: at that wait. It then checks three things. A read sees the
step it expects. No copy into a slot is still in flight while that slot is read. And every
mbarrier wait finds its expected phase completed, so no wait can hang.
"""
import random

import pytest


def run_cp_async_ring(items, D, rng):
    """items: step counts of consecutive work items of one lane."""
    slots = {}              # slot -> step whose data has landed there
    groups = []             # committed groups, oldest first: (slot, step) or None for an empty group
    done = 0                # groups known complete (a prefix: wait_group completes all older ones)

    def commit(t):
        groups.append((t % D, t) if t >= 0 else None)

    def wait(pending_max):
        nonlocal done
        target = len(groups) - pending_max
        # groups older than the target must be complete now; newer ones may complete any time,
        # the adversary completes them as late as possible
        for g in groups[done:target]:
            if g is not None:
                slots[g[0]] = g[1]
        done = max(done, target)

    for n in items:
        for k in range(D):
            commit(n - 1 - k)
        for t in range(n - 1, -1, -1):
            wait(D - 1)
            sl = t % D
            assert slots.get(sl) == t, (n, D, t, slots.get(sl))
            # no copy into this slot may still be in flight while it is read
            assert all(g is None or g[0] != sl for g in groups[done:]), (n, D, t)
            if rng.random() < 0.3:      # the hardware may also complete newer groups early
                wait(rng.randint(0, D - 1))
            commit(t - D)
    # an item's real copies have all been waited for before the next item starts
    return True


def run_mbarrier_ring(items, R=4):
    """The tape adjoint: one barrier per slot; completions counted per slot."""
    completed = [0] * R     # completed phases (loads landed) per slot
    issued = [0] * R        # loads issued per slot
    data = {}               # slot -> step of the last load issued there (lands at its completion)
    parity = 0              # bit k: parity of slot k's next awaited phase (kept across items)
    waits = [0] * R

    def load(t):
        sl = t % R
        # a slot holds at most one load in flight: the previous one was awaited and read
        assert issued[sl] == completed[sl], (t, sl)
        issued[sl] += 1
        data[sl] = t

    for n in items:
        for k in range(R):
            if n - 1 - k >= 0:
                load(n - 1 - k)
        for t in range(n - 1, -1, -1):
            sl = t % R
            want = (parity >> sl) & 1
            # the adversary completes the load only now; the wait for phase `want` must be the
            # phase this load completes (phases alternate parity per slot)
            assert issued[sl] == completed[sl] + 1, (n, t)
            completed[sl] += 1
            assert (completed[sl] - 1) % 2 == want
            parity ^= 1 << sl
            waits[sl] += 1
            assert data[sl] == t
            if t - R >= 0:
                load(t - R)
    assert issued == completed == waits
    return True


@pytest.mark.parametrize("D", [4, 6, 8])
def test_cp_async_ring_reads_each_step_from_a_settled_slot(D):
    rng = random.Random(D)
    for n in list(range(1, 3 * D + 3)) + [31, 32, 33, 257, 543]:
        assert run_cp_async_ring([n], D, rng)
    for _ in range(200):
        items = [rng.randint(1, 60) for _ in range(rng.randint(2, 6))]
        assert run_cp_async_ring(items, D, rng)


def test_mbarrier_ring_waits_always_find_their_phase():
    rng = random.Random(7)
    for n in list(range(1, 14)) + [31, 32, 33, 543]:
        assert run_mbarrier_ring([n])
    for _ in range(500):
        items = [rng.randint(1, 40) for _ in range(rng.randint(2, 8))]
        assert run_mbarrier_ring(items)


def run_contraction_ring(ntiles_seq):
    """The FMA contraction: one warp's sequence of strip-window visits, each with its tile count."""
    completed = [0] * 3
    issued = [0] * 3
    holds = {}              # slot -> half whose load was issued last
    parity = 0

    def load(h):
        sl = h % 3
        assert issued[sl] == completed[sl], ("slot reloaded before its load was awaited", h)
        issued[sl] += 1
        holds[sl] = h

    def wait(sl):
        nonlocal parity
        want = (parity >> sl) & 1
        assert issued[sl] == completed[sl] + 1, ("wait with no load in flight: it would hang", sl)
        completed[sl] += 1
        assert (completed[sl] - 1) % 2 == want
        parity ^= 1 << sl

    for ntiles in ntiles_seq:
        for h in range(min(3, ntiles + 1)):
            load(h)
        for b in range(ntiles):
            if b == 0:
                wait(0)
            wait((b + 1) % 3)
            assert holds[b % 3] == b and holds[(b + 1) % 3] == b + 1
            if b + 3 <= ntiles:
                load(b + 3)
    assert issued == completed   # nothing left in flight or unawaited
    return True


def test_contraction_ring_waits_each_half_once():
    rng = random.Random(11)
    for n in range(1, 40):
        assert run_contraction_ring([n])
    for _ in range(500):
        assert run_contraction_ring([rng.randint(1, 40) for _ in range(rng.randint(2, 10))])
