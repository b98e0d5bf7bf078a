"""CPU checks of two device-side index schemes, with the kernels' formulas written out here:

* the TMA-staged x pass (`k_fft_wx_tma`): the 64-byte-swizzled tile addressing, the per-lane
  base plus compile-time row offsets, and the tile coordinates against the TMA rules (the
  innermost coordinate times the element size a multiple of 16 bytes, boxes inside the tensor);
* the work queue of the batched persistent launch (`k_batch_persist`): the (pass, group) item
  table, the decode of an item into (pass, solve, tiles), coverage of every tile exactly once,
  and the ordering that makes the launch deadlock-free (every item an item waits on comes
  earlier in the queue).
"""

import itertools
import math

import pytest

# ---------------------------------------------------------------------------
# TMA-staged x pass
# ---------------------------------------------------------------------------
N_X, LINES, BOX_ROWS, ELEM = 512, 8, 256, 8


def tma_x_offset(m, c):
    """Byte offset of element (row m, line c) in a tile: 64-byte rows, 16-byte chunk c/2 XOR bits 1..2 of m."""
    return m * 64 + (((c >> 1) ^ ((m >> 1) & 3)) << 4) + ((c & 1) << 3)


def swizzle64(linear):
    """The 64-byte swizzle of the tensor memory accelerator on a 1024-byte-aligned buffer: the
    16-byte chunk index (address bits 4..5) XOR address bits 7..8."""
    return linear ^ (((linear >> 7) & 3) << 4)


def test_tile_offsets_are_the_swizzled_dense_box():
    slots = set()
    for m in range(N_X):
        for c in range(LINES):
            dense = m * LINES * ELEM + c * ELEM          # the box as the tensor lays it out, row m, element c
            o = tma_x_offset(m, c)
            assert o == swizzle64(dense)
            assert 0 <= o < N_X * LINES * ELEM and o % ELEM == 0
            slots.add(o)
    assert len(slots) == N_X * LINES                     # a bijection onto the 32 KB tile


def test_lane_rows_are_base_plus_constant_offsets():
    for lane, warp, k in itertools.product(range(32), range(LINES), range(16)):
        assert tma_x_offset(lane, warp) + 2048 * k == tma_x_offset(lane + 32 * k, warp)
    # the second box (rows 256..511) starts 16 KB in, on a 1024-byte boundary, so the swizzle
    # pattern of its rows is the one of the first box
    assert (BOX_ROWS * LINES * ELEM) % 1024 == 0


def test_line_reads_use_eight_bank_slots():
    # a warp's read of its line (rows lane + 32 k) touches 8 distinct 8-byte bank slots: 4 wavefronts
    for w in range(LINES):
        assert len({(tma_x_offset(l, w) // 4) % 32 for l in range(32)}) == 8


@pytest.mark.parametrize("n2,n3,batch", [(512, 512, 1), (24, 16, 3), (16, 8, 1), (8, 30, 2)])
def test_tile_coordinates_follow_the_tma_rules(n2, n3, batch):
    n3h = n3 // 2 + 1
    assert n2 % LINES == 0
    seen = set()
    for s in range(batch):
        ntiles = n3h * n2 // LINES
        for t in range(ntiles):
            l = t * LINES
            kz, ky = divmod(l, n2)
            z = s * n3h + kz
            assert (ky * ELEM) % 16 == 0                  # innermost coordinate x element size
            assert 0 <= ky and ky + LINES <= n2            # the box stays in one plane
            for y0 in (0, BOX_ROWS):
                assert 0 <= y0 and y0 + BOX_ROWS <= N_X
            assert 0 <= z < n3h * batch
            for c in range(LINES):
                seen.add((s, kz, ky + c))
    assert len(seen) == batch * n3h * n2                   # every x line once


# ---------------------------------------------------------------------------
# Work queue of the batched persistent launch
# ---------------------------------------------------------------------------
PASSES = 6
P, L = 16, 32                # line pairs per z tile, lines per y / x tile (variant 0)
CHUNK = 256 * 16             # thread groups per update chunk


def group_tiles(n1, n2, n3, upd_w):
    n3h = n3 // 2 + 1
    pairs = math.ceil(n1 * n2 / 2)
    nchunks = math.ceil(n1 * n2 * n3 // upd_w / CHUNK)
    return [math.ceil(pairs / P), math.ceil(n3h * n1 / L), math.ceil(n3h * n2 / L),
            math.ceil(n3h * n1 / L), math.ceil(pairs / P), nchunks]


def build_queue(groups, grid):
    """groups: list of (shape, solves). Returns per-group tiles, tiles per item, items per solve,
    the (pass, group) base table and each group's first solve index."""
    tiles = [group_tiles(*sh, upd_w=2) for sh, _ in groups]
    tile_bytes = [lambda sh: 2 * P * sh[2] * 52, lambda sh: L * sh[1] * 16, lambda sh: L * sh[0] * 16,
                  lambda sh: L * sh[1] * 16, lambda sh: 2 * P * sh[2] * 8, lambda sh: 1]
    tpi = [[1 if q == PASSES - 1 else max(1, int(256 * 1024 / tile_bytes[q](sh))) for q in range(PASSES)]
           for sh, _ in groups]
    for q in range(PASSES):
        total = sum(tiles[b][q] * groups[b][1] for b in range(len(groups)))
        cap = max(1, total // (4 * grid))
        for b in range(len(groups)):
            tpi[b][q] = min(tpi[b][q], cap)
    items = [[math.ceil(tiles[b][q] / tpi[b][q]) for q in range(PASSES)] for b in range(len(groups))]
    base, acc = [], 0
    for q in range(PASSES):
        for b, (_, ns) in enumerate(groups):
            base.append(acc)
            acc += items[b][q] * ns
    base.append(acc)
    gstart = [sum(ns for _, ns in groups[:b]) for b in range(len(groups))]
    return tiles, tpi, items, base, gstart


def decode(item, base, items, gstart, ng):
    """The kernel's decode: pass by scan, group by scan, then solve and item inside the group."""
    p = 0
    while p + 1 < PASSES and item >= base[(p + 1) * ng]:
        p += 1
    g = 0
    while g + 1 < ng and item >= base[p * ng + g + 1]:
        g += 1
    off = item - base[p * ng + g]
    nt = items[g][p]
    q, tile = divmod(off, nt)
    return p, g, q, gstart[g] + q, tile


@pytest.mark.parametrize("groups,grid", [
    ([((96, 96, 96), 48), ((160, 160, 160), 48), ((64, 64, 64), 45), ((128, 128, 128), 51)], 456),
    ([((8, 8, 8), 2), ((12, 10, 6), 2), ((16, 12, 10), 2), ((6, 10, 15), 1), ((9, 5, 1), 1), ((1, 1, 20), 1)], 456),
    ([((128, 128, 128), 1)], 456),
])
def test_queue_covers_every_tile_once_in_dependency_order(groups, grid):
    tiles, tpi, items, base, gstart = build_queue(groups, grid)
    ng = len(groups)
    total = base[-1]
    first, last = {}, {}
    covered = {}
    for it in range(total):
        p, g, q, j, tile = decode(it, base, items, gstart, ng)
        assert 0 <= tile < items[g][p] and 0 <= q < groups[g][1]
        first.setdefault((j, p), it)
        last[(j, p)] = it
        t0 = tile * tpi[g][p]
        t1 = min(t0 + tpi[g][p], tiles[g][p])
        assert t0 < t1
        for t in range(t0, t1):
            key = (j, p, t)
            assert key not in covered
            covered[key] = it
    nsolve = sum(ns for _, ns in groups)
    for j in range(nsolve):
        g = max(b for b in range(ng) if gstart[b] <= j)
        for p in range(PASSES):
            assert all((j, p, t) in covered for t in range(tiles[g][p]))
            if p > 0:
                # every item of pass p - 1 of the solve precedes every item of pass p: the
                # earliest unfinished item never waits on a later one
                assert last[(j, p - 1)] < first[(j, p)]
    # the update pass keeps one item per chunk (one partial-sum slot each)
    assert all(tpi[b][PASSES - 1] == 1 for b in range(ng))


def test_shared_memory_tables_do_not_overlap():
    for ng in range(1, 40):
        off_sc = ((PASSES * ng + 1) * 8 + 15) // 16 * 16
        off_start = off_sc + ng * 8
        table = (off_start + ng * 4 * (1 + PASSES) + 15) // 16 * 16
        assert off_sc >= (PASSES * ng + 1) * 8         # item bases (8 bytes each)
        assert off_start - off_sc == 8 * ng             # scalar-slot pointers
        assert table >= off_start + 4 * ng + 4 * PASSES * ng and table % 16 == 0
