"""CPU model of the dk/dM buffer shared by the tape adjoint and the FMA-pipe contraction
(bwd_contract_kernel), with the index arithmetic of csrc/sk_bwd_poly.cuh restated in Python.

* The adjoint stores cell (32 s + r, j) of a pair at buffer row `step` (warp step s P + j + r,
  with P = max(cols, 32)), position (r + step) mod 32.
* The contraction takes strip s in windows of WIN columns and each window in tiles of 32
  columns. A tile spans buffer rows t0 + 32 b .. t0 + 32 b + 62, with t0 = s P + w0. It streams
  them as 32-row halves into a circular ring of three: half h goes to slot h mod 3, halves 0..2
  first, then half b + 3 once tile b is done.
* In tile b, lane r's x-walk and lane q's y-walk read cell (r, j0 + q) at ring row
  (32 (b mod 3) + r + q) mod 96, position (2 r + q + coff) mod 32, with coff = (s P + j0) mod 32.

The model checks three things. Both walks read every cell of the grid exactly once, at the
buffer row and position where the adjoint stored it. The ring slot holds the half the tile
needs. Every bulk copy stays inside the item's buffer: the longest pair's warp steps plus
kContractSlack = 64 rows.
"""
import pytest

K_SLACK = 64


def nsteps(rows, cols):
    return ((rows + 31) // 32 - 1) * max(cols, 32) + 31 + cols


def adjoint_stores(rows, cols):
    P = max(cols, 32)
    out = {}
    for i in range(rows):
        s, r = divmod(i, 32)
        for j in range(cols):
            step = s * P + j + r
            out[(i, j)] = (step, (r + step) & 31)
    return out


def contraction_reads(rows, cols, win):
    P = max(cols, 32)
    xr, yr, loaded = {}, {}, set()
    for s in range((rows + 31) // 32):
        nr = min(32, rows - 32 * s)
        for w0 in range(0, cols, win):
            wcols = min(win, cols - w0)
            ntiles = (wcols + 31) // 32
            t0 = s * P + w0
            halves = {}                       # slot -> half it holds
            for h in range(min(3, ntiles + 1)):
                halves[h % 3] = h
                loaded.update(range(t0 + 32 * h, t0 + 32 * h + 32))
            for b in range(ntiles):
                j0 = w0 + 32 * b
                nc = min(32, cols - j0)
                coff = (s * P + j0) & 31
                s0 = b % 3
                hb = 32 * s0
                assert halves[s0] == b and halves[(b + 1) % 3] == b + 1  # both halves of the tile are in

                def buffer_row(u):
                    ring_row = hb + u
                    if s0 < 2:
                        assert ring_row < 96       # these tiles are read without the wrap
                    ring_row %= 96
                    slot, off = divmod(ring_row, 32)
                    return t0 + 32 * halves[slot] + off

                for lane in range(32):
                    for q0 in range(32):          # x-walk of row `lane`
                        q = (q0 + (lane >> 4)) & 31
                        u = lane + q
                        if lane < nr and q < nc:
                            key = (32 * s + lane, j0 + q)
                            assert key not in xr
                            xr[key] = (buffer_row(u), (lane + u + coff) & 31)
                    for r in range(32):           # y-walk of column `lane`
                        u = r + lane
                        if r < nr and lane < nc:
                            key = (32 * s + r, j0 + lane)
                            assert key not in yr
                            yr[key] = (buffer_row(u), (r + u + coff) & 31)
                if b + 3 <= ntiles:               # refill the slot just read
                    halves[s0] = b + 3
                    loaded.update(range(t0 + 32 * (b + 3), t0 + 32 * (b + 3) + 32))
    return xr, yr, loaded


@pytest.mark.parametrize("rows,cols,win", [
    (1, 1, 1024), (31, 5, 1024), (32, 32, 1024), (33, 33, 1024), (64, 256, 1024), (256, 256, 1024),
    (70, 95, 64), (100, 300, 256), (45, 1300, 1024), (129, 97, 32), (96, 200, 96),
])
def test_contraction_reads_what_the_adjoint_stored(rows, cols, win):
    stored = adjoint_stores(rows, cols)
    xr, yr, loaded = contraction_reads(rows, cols, win)
    assert xr == stored
    assert yr == stored
    assert min(loaded) >= 0
    assert max(loaded) < nsteps(rows, cols) + K_SLACK


@pytest.mark.parametrize("rows,cols", [(300, 40), (33, 1000), (64, 64)])
def test_a_shorter_pair_stays_inside_the_longest_pairs_stride(rows, cols):
    """Every item's buffer has the stride of the call's longest pair; a shorter pair's copies stay
    below it too."""
    _, _, loaded = contraction_reads(rows, cols, 1024)
    for longest in ((rows, cols), (rows + 7, cols), (rows, cols + 40)):
        assert max(loaded) < nsteps(*longest) + K_SLACK
