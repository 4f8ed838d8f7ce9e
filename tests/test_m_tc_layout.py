"""CPU model of where m_tc_kernel's epilogue writes each cell's M (the index arithmetic of
csrc/sk_m_tc.cu restated in Python), checked for bounds and coverage over every alignment, block
width and lane, and over pair shapes with ragged strips and column blocks.

The layout: one warp sweeps a pair, with cell (32 s + r, j) at warp step s P + j + r and
P = max(cols, 32). The steps go in groups of four, and group G holds lane r's M of steps
4G .. 4G + 3 as the float4 at index 32 G + r of the item's buffer. An item's buffer holds
ceil(nsteps / 4) groups, where nsteps counts the warp steps of the longest pair of the call.

The epilogue warp of strip sg and columns jb .. jb + ncol - 1 stages lane r's cell of block
column c at staging float c + r + a, with a = T0 mod 4 and T0 = sg P + jb. It then stores groups
g = 0 .. ng - 1 of the staging row at group (T0 >> 2) + g. Interior groups go out whole; the
others go element by element, for the cells inside the block only.
"""
import pytest

K_MT_ROW = 100  # staging floats per lane


def block_writes(a, ncol, rows_in_strip):
    """{(lane, group, k): block column c} that one epilogue block stores, following the kernel:
    whole float4s for interior groups of a full strip, single elements otherwise."""
    ng = (ncol + 30 + a) // 4 + 1
    gin0 = (31 + a + 3) // 4
    num = ncol - 4 + a
    gin1 = int(num / 4)  # C division truncates toward zero
    rows_full = rows_in_strip >= 32
    out = {}
    for lane in range(32):
        row_ok = lane < rows_in_strip
        for g in range(ng):
            # the float4 read from the staging row
            assert 4 * g + 3 < K_MT_ROW
            if rows_full and gin0 <= g <= gin1:
                for k in range(4):
                    c = 4 * g + k - lane - a
                    assert 0 <= c < ncol, (a, ncol, lane, g, k)  # a whole store holds only the block's cells
                    out[(lane, g, k)] = c
            elif row_ok:
                for k in range(4):
                    c = 4 * g + k - lane - a
                    if 0 <= c < ncol:
                        out[(lane, g, k)] = c
    return out


@pytest.mark.parametrize("a", range(4))
def test_every_cell_of_a_block_is_stored_once_and_only_its_cells(a):
    for ncol in range(1, 65):
        for rows_in_strip in (32, 31, 17, 1):
            # staging writes of the block's cells stay in the lane's row
            assert 63 + 31 + a < K_MT_ROW
            w = block_writes(a, ncol, rows_in_strip)
            want = {(lane, c) for lane in range(min(rows_in_strip, 32)) for c in range(ncol)}
            got = [(lane, c) for (lane, g, k), c in w.items()]
            assert len(got) == len(set(got)) == len(want)
            assert set(got) == want
            for (lane, g, k), c in w.items():
                assert 4 * g + k == c + lane + a  # the cell's step relative to 4 (T0 >> 2)


def nsteps(rows, cols):
    """Warp steps of one pair in the one-warp-per-pair schedule (plan_forward's count)."""
    return ((rows + 31) // 32 - 1) * max(cols, 32) + 31 + cols


@pytest.mark.parametrize("rows,cols,max_rows,max_cols", [
    (1, 1, 1, 1), (31, 5, 31, 5), (32, 32, 32, 32), (33, 129, 200, 300), (128, 128, 128, 128),
    (129, 127, 129, 127), (256, 256, 256, 256), (200, 31, 512, 512), (512, 512, 512, 512),
    (300, 65, 300, 65), (97, 191, 1000, 40),
])
def test_writes_stay_inside_the_item_buffer_and_cover_its_cells(rows, cols, max_rows, max_cols):
    """Every tile of a pair of rows x cols cells (in a call whose longest pair is max_rows x
    max_cols) writes groups below the item's ceil(nsteps / 4), each cell exactly once, at the
    step the sweep reads it."""
    groups = (nsteps(max(max_rows, rows), max(max_cols, cols)) + 3) // 4
    period = max(cols, 32)
    seen = {}
    nrb, ncb = (rows + 127) // 128, (cols + 127) // 128
    for rb in range(nrb):
        for cb in range(ncb):
            for q in range(4):
                for half in range(2):
                    sg = rb * 4 + q
                    jb = cb * 128 + 64 * half
                    ncol = min(64, cols - jb)
                    if 32 * sg >= rows or ncol <= 0:
                        continue
                    T0 = sg * period + jb
                    a = T0 & 3
                    for (lane, g, k), c in block_writes(a, ncol, rows - 32 * sg).items():
                        G = (T0 >> 2) + g
                        assert 0 <= G < groups
                        step = 4 * G + k
                        cell = (32 * sg + lane, jb + c)
                        assert step == sg * period + cell[1] + lane  # where the sweep reads it
                        assert (G, lane, k) not in seen
                        seen[(G, lane, k)] = cell
    assert sorted(seen.values()) == [(i, j) for i in range(rows) for j in range(cols)]
    # the sweep reads group 0 first, then group step / 4 + 1 on entering each group while
    # 4 (step / 4 + 1) < nsteps of this pair: all inside the item's buffer
    n = nsteps(rows, cols)
    reads = {0} | {s // 4 + 1 for s in range(0, n, 4) if 4 * (s // 4 + 1) < n}
    assert max(reads) < groups
    # and every group holding a cell is read before its steps are swept
    assert {G for (G, lane, k) in seen} <= reads
