"""CPU model of the cooperative strip pipeline's schedule (the forward kernels' CW > 1 sweeps).

W warps share one pair; warp w runs strips w, w + W, ...; its 32 lanes advance in lockstep, lane r
at local step tau working on local strip (tau - r) // P, column (tau - r) mod P.  Lane 0 of strip
g > 0 may run column j only after lane 31 of strip g - 1 has published column j; a warp whose lane 0
waits makes no step at all.  The model advances every warp that can advance until none can; the
schedule is sound when every warp finishes.

The kernels pick the period P = cols + 31 (a warp finishes a strip before starting the next) unless
cols > 31 W, where the overlapped P = cols is used.  These tests check that rule on many shapes and
show that plain overlap (P = max(cols, 32)) can deadlock when rows are short.
"""
import pytest


def schedule_completes(rows, cols, W, P, K=1):
    nstrips = (rows + 31) // 32
    last_lane = rows - 1 - 32 * (nstrips - 1)
    done = [0] * nstrips
    warps = []
    for w in range(min(W, nstrips)):
        nloc = (nstrips - 1 - w) // W + 1
        has_last = (nstrips - 1) % W == w
        warps.append([w, nloc, (nloc - 1) * P + (last_lane if has_last else 31) + cols, 0])

    def cell(w, nloc, tau, r):
        t = tau - r
        if t < 0:
            return None
        s, j = divmod(t, P)
        g = w + s * W
        if s >= nloc or j >= cols or g * 32 + r >= rows:
            return None
        return g, j

    moved = True
    while moved:
        moved = False
        for st in warps:
            w, nloc, nsteps, tau = st
            if tau >= nsteps:
                continue
            c0 = cell(w, nloc, tau, 0)
            if c0 and c0[0] > 0 and done[c0[0] - 1] < c0[1] + 1:
                continue
            c31 = cell(w, nloc, tau, 31)
            if c31 and c31[0] + 1 < nstrips and ((c31[1] + 1) % K == 0 or c31[1] + 1 == cols):
                done[c31[0]] = c31[1] + 1  # published every K columns and at the row's end
            st[3] += 1
            moved = True
    return all(st[3] >= st[2] for st in warps)


def kernel_period(cols, W):
    return max(cols if cols > 31 * W else cols + 31, 32)


@pytest.mark.parametrize("W", [2, 3, 4, 8])
def test_kernel_period_rule_never_deadlocks(W):
    for cols in list(range(1, 34)) + list(range(31 * W - 2, 31 * W + 6)) + [400, 1024]:
        for nst in (2, 3, 5, 8, 9, 17):
            for k in (0, 1, 31):
                assert schedule_completes(nst * 32 - k, cols, W, kernel_period(cols, W)), (W, cols, nst, k)


def test_plain_overlap_deadlocks_on_short_rows():
    # two warps, 2-column rows: warp 0's lane 0 waits on strip 1 in the step in which its lane 31
    # would publish the column of strip 0 that warp 1 needs
    assert not schedule_completes(3 * 32 - 5, 2, 2, 32)
    assert not schedule_completes(9 * 32 - 5, 200, 8, 200)   # cols <= 31 W
    assert schedule_completes(9 * 32 - 5, 260, 8, 260)       # cols > 31 W


@pytest.mark.parametrize("W", [16, 32, 64])
def test_kernel_period_rule_on_wide_rings(W):
    """Rings as the kernels build them: one block of 16 warps, and rings of 2 or 4 such blocks
    (the grid strip pipeline for few long pairs)."""
    for cols in (1, 31, 33, 31 * W - 1, 31 * W, 31 * W + 1, 1024):
        for nst in (W - 1, W + 1, 2 * W + 3):
            assert schedule_completes(nst * 32 - 5, cols, W, kernel_period(cols, W)), (W, cols, nst)


@pytest.mark.parametrize("W", [32, 64])
def test_batched_publishing_needs_the_longer_lag(W):
    """Rings that span blocks publish their progress every 8 columns.  The overlapped schedule is
    then safe only above cols > (31 + 8) W: just above 31 W it deadlocks."""
    K = 8

    def grid_period(cols):
        return max(cols if cols > (31 + K) * W else cols + 31, 32)

    for cols in (1, 8, 9, 33, 31 * W + 1, 31 * W + 32, (31 + K) * W, (31 + K) * W + 1, 4000):
        for nst in (W - 1, W + 1, 2 * W + 3):
            assert schedule_completes(nst * 32 - 5, cols, W, grid_period(cols), K), (cols, nst)
    assert not schedule_completes((W + 1) * 32 - 5, 31 * W + 32, W, 31 * W + 32, K)
