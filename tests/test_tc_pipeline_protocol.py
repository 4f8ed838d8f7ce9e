"""CPU model of the warp-specialised pipelines of the two tensor-core kernels (csrc/sk_m_tc.cu and
csrc/sk_contract_tc.cu): a producer warp, an MMA-issuing thread and several epilogue warps hand
work to one another through mbarriers, and every interleaving of them must neither deadlock nor
let one role overrun another.

The barriers, as the kernels use them:
* full[s]: a stage's operands have landed.
* empty[s]: the MMAs that read stage s are done.
* tfull[a]: accumulator a holds finished sums.
* tempty[a]: every epilogue warp has read accumulator a. It needs one arrival per epilogue warp.

Roles:
* The producer waits empty[s] and loads stage s.
* The MMA role waits tempty[a] and full[s], issues its MMAs, and commits empty[s] and tfull[a].
* Each epilogue warp waits tfull[a], reads the accumulator and arrives on tempty[a].
* The M kernel uses one accumulator per tile. The contraction uses one per item, accumulated
  over the item's tiles.

mbarrier rule: a barrier starts in phase 0, and a wait on parity P returns once the barrier's
completed-phase count c has c mod 2 != P. So the first wait on parity 1 returns at once.

The model runs the roles in random order, and asynchronous completions (copies landing, MMAs
finishing) fire at random later times. It checks four things:
* each wait returns with exactly the phase it means, not an older one through parity aliasing
  and not one phase later;
* the MMA reads the tile its stage was loaded with;
* each epilogue warp reads its own tile's or item's finished sums;
* every run finishes.
"""
import random

import pytest


class Barrier:
    def __init__(self, count):
        self.count, self.arrived, self.completed = count, 0, 0

    def arrive(self):
        self.arrived += 1
        if self.arrived == self.count:
            self.arrived = 0
            self.completed += 1

    def ready(self, parity):
        return self.completed % 2 != parity


def simulate(kind, units, n_epi, seed):
    """kind 'm': one accumulator per tile; kind 'contract': one per processed item.  units: tiles
    per item (0 = an item every role skips, as the kernels skip items without cells)."""
    rng = random.Random(seed)
    full = [Barrier(1) for _ in range(2)]
    empty = [Barrier(1) for _ in range(2)]
    tfull = [Barrier(1) for _ in range(2)]
    tempty = [Barrier(n_epi) for _ in range(2)]
    stage = [None, None]            # tile whose operands sit in stage s
    acc = [None, None]              # (owner, tiles summed) in accumulator a
    events = []                     # pending asynchronous completions: callables
    tiles = [(i, t) for i, n in enumerate(units) for t in range(n)]

    def wait(bar, parity, phase):
        # block until ready; then the barrier must have completed exactly phase + 1 phases
        while not bar.ready(parity):
            yield
        assert bar.completed == phase + 1, (bar.completed, phase)

    def producer():
        for it, tile in enumerate(tiles):
            s, u = it % 2, it // 2
            yield from wait(empty[s], (u & 1) ^ 1, u - 1)

            def land(s=s, tile=tile):
                stage[s] = tile
                full[s].arrive()
            events.append(land)

    def mma():
        it = nitem = 0
        for i, n in enumerate(units):
            if not n:
                continue
            if kind == "contract":
                a, v = nitem % 2, nitem // 2
                yield from wait(tempty[a], (v & 1) ^ 1, v - 1)
                acc[a] = (i, 0)
            for t in range(n):
                s, u = it % 2, it // 2
                if kind == "m":
                    a = s
                    yield from wait(tempty[a], (u & 1) ^ 1, u - 1)
                    acc[a] = ((i, t), 0)
                yield from wait(full[s], u & 1, u)
                assert stage[s] == (i, t)           # the operands of this tile
                owner, k = acc[a]
                acc[a] = (owner, k + 1)             # the MMAs add this tile into accumulator a

                def mma_done(s=s, tile=(i, t)):
                    assert stage[s] == tile          # the stage held still until the MMAs finished
                    empty[s].arrive()
                events.append(mma_done)
                if kind == "m":
                    events.append(tfull[a].arrive)
                it += 1
            if kind == "contract":
                events.append(tfull[a].arrive)
                nitem += 1

    def epilogue(w):
        it = nitem = 0
        for i, n in enumerate(units):
            if not n:
                continue
            if kind == "contract":
                a, v = nitem % 2, nitem // 2
                yield from wait(tfull[a], v & 1, v)
                assert acc[a] == (i, n), (w, i, acc[a])   # the item's finished sums
                tempty[a].arrive()
                nitem += 1
            else:
                for t in range(n):
                    a, u = it % 2, it // 2
                    yield from wait(tfull[a], u & 1, u)
                    assert acc[a] == ((i, t), 1), (w, i, t, acc[a])
                    tempty[a].arrive()
                    it += 1

    live = [producer(), mma()] + [epilogue(w) for w in range(n_epi)]
    idle = 0                        # consecutive role steps without any state change
    while live or events:
        if events and (not live or rng.random() < 0.3):
            events.pop(rng.randrange(len(events)))()
            idle = 0
            continue
        r = rng.choice(live)
        snapshot = (tuple(b.completed for b in full + empty + tfull + tempty),
                    tuple(b.arrived for b in tempty), len(events), len(live))
        try:
            next(r)
        except StopIteration:
            live.remove(r)
        after = (tuple(b.completed for b in full + empty + tfull + tempty),
                 tuple(b.arrived for b in tempty), len(events), len(live))
        idle = idle + 1 if after == snapshot else 0
        # every live role blocked with nothing left to complete: a deadlock
        assert events or idle < 50 * (len(live) + 1), "deadlock"
    return True


@pytest.mark.parametrize("seed", range(40))
def test_m_kernel_pipeline(seed):
    rng = random.Random(seed)
    units = [rng.randint(0, 7) for _ in range(rng.randint(1, 6))]
    assert simulate("m", units, 8, seed)


@pytest.mark.parametrize("seed", range(40))
def test_contraction_pipeline(seed):
    rng = random.Random(1000 + seed)
    units = [rng.randint(0, 7) for _ in range(rng.randint(1, 6))]
    assert simulate("contract", units, 4, seed)
