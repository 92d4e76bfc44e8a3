"""Host-side model of the column-march kernel's schedule (step_march.cuh), checked on CPU.

The model replays, for one block and each kind of warp (upwind row y-1 or y+1), the order
in which the kernel issues row copies into its ring of S slots and consumes them, with the
kernel's item numbering (chunk-major, first three items per block fixed, the rest from a
counter) and the host's choice of the chunk count, for rings of 2, 4 and 5 slots and for the
deferred-relaxation variant (item ids published through mbarrier phases, visible one row
later than at a block barrier).  It checks what a GPU run could only
show as a fault or a wrong answer: every copy starts 16-byte aligned inside one grid row,
a slot is refilled only after its last use, each row computed finds its own row and its
upwind row in the slots, an item id is read only after the barrier that published it,
and the interior x in [32, nx-32), y in [1, ny-2] is written exactly once.
"""
import pytest


def march_row0(k, rows, nchunks, first=1):
    return first + (k * rows) // nchunks


def choose_chunks(nx, ny, grid):
    strips, rows = (nx - 64) // 64, ny - 2
    lo_len = 16 if rows >= 64 else 8
    cmax = max(rows // lo_len, 1)
    cmin = min((4 * grid + strips - 1) // strips, cmax)
    chunks, best = cmax, 1e300
    for c in range(cmin, cmax + 1):
        items = strips * c
        rounds = (items + grid - 1) // grid
        cost = rounds * grid / items * (1.0 + c / rows)
        if cost < best - 1e-12:
            best, chunks = cost, c
    return strips, chunks


def simulate(nx, ny, S, grid, defer=False, order=1):
    """order 2: the second-order march (rows [2, ny - 3], an item's rows plus two upwind
    rows copied, own row and both upwind rows read; the host plans ny - 4 rows)."""
    strips, nchunks = choose_chunks(nx, ny - 2 * (order - 1), grid)
    rows, nitems, ncells = ny - 2 * order, strips * nchunks, nx * ny
    written = {}
    counter = [3 * grid]

    def decode(it):
        k = it // strips
        r0 = march_row0(k, rows, nchunks, order)
        return it - k * strips, r0, march_row0(k + 1, rows, nchunks, order) - r0

    for b in range(grid):
        fetched = []                       # dynamic ids of this block, in fetch order
        for ypos in (False, True):
            items = {0: b, 1: grid + b, 2: 2 * grid + b}
            visible = {0, 1, 2}
            pending = []
            pending_old = []
            dyn = iter(fetched) if ypos else None
            l_pos, l_i, nl = 0, 0, 0
            l_item = items[0]
            if l_item < nitems:
                l_strip, l_row0, l_len = decode(l_item)
            loads = []
            c_pos, c_u, gb = 0, 0, 0
            c_item = items[0]
            if c_item < nitems:
                c_strip, c_row0, c_len = decode(c_item)
            while c_item < nitems:
                while l_item < nitems and nl <= gb + c_u + S - 1:
                    if nl - S >= 0:
                        assert nl - S < gb + c_u            # slot's previous row no longer needed
                    row = l_row0 - (order if ypos else 0) + l_i
                    assert 0 <= row < ny
                    if order == 1:    # the planar copy of a row line (load paths 4-7)
                        start = row * nx + 28 + 64 * l_strip
                        assert start % 4 == 0 and start >= 0 and start + 72 <= ncells
                        assert start // nx == row and (start + 71) // nx == row
                    loads.append((row, l_strip))
                    nl += 1
                    l_i += 1
                    if l_i > l_len + order - 1:
                        l_i, l_pos = 0, l_pos + 1
                        assert l_pos in visible
                        l_item = items[l_pos]
                        if l_item < nitems:
                            l_strip, l_row0, l_len = decode(l_item)
                assert gb + c_u + order < nl
                jo = gb + c_u + (order if ypos else 0)
                jy = gb + c_u + (order - 1 if ypos else 1)
                y = c_row0 + c_u
                assert loads[jo] == (y, c_strip)
                assert loads[jy] == (y - 1 if ypos else y + 1, c_strip)
                if order == 2:
                    jq = gb + c_u + (0 if ypos else 2)
                    assert loads[jq] == (y - 2 if ypos else y + 2, c_strip)
                    assert nl - 1 < min(jo, jy, jq) + S         # all three still in the ring
                assert nl - 1 < min(jo, jy) + S                 # both still in the ring
                if defer:
                    # deferred relaxation: an id written after row t's moments were published
                    # is released with row t+1's and acquired at the wait for row t+1, which
                    # follows row t+2's copies: visible one row later than at a block barrier
                    visible |= set(pending_old)
                    pending_old, pending = pending, []
                else:
                    visible |= set(pending)                      # the row barrier
                    pending = []
                if not ypos:
                    for xx in range(64):
                        c = y * nx + 32 + 64 * c_strip + xx
                        written[c] = written.get(c, 0) + 1
                c_u += 1
                if c_u == c_len:
                    gb, c_u, c_pos = gb + c_len + order, 0, c_pos + 1
                    assert c_pos in visible
                    c_item = items[c_pos]
                    if c_item < nitems:
                        c_strip, c_row0, c_len = decode(c_item)
                    if ypos:
                        items[c_pos + 2] = next(dyn)
                    else:
                        items[c_pos + 2] = counter[0]
                        counter[0] += 1
                        fetched.append(items[c_pos + 2])
                    pending.append(c_pos + 2)
    interior = {y * nx + x for y in range(order, ny - order) for x in range(32, nx - 32)}
    assert set(written) == interior and all(v == 1 for v in written.values())
    return strips, nchunks


@pytest.mark.parametrize("nx,ny", [(128, 10), (192, 45), (256, 70), (384, 522), (640, 33), (1024, 1000),
                                   (2048, 2048)])
@pytest.mark.parametrize("slots,defer", [(4, False), (5, False), (2, False), (4, True)])
@pytest.mark.parametrize("grid", [7, 152, 304])
def test_march_schedule_covers_interior_once(nx, ny, slots, defer, grid):
    """Load paths 4, 5 (rings of 4 and 5 slots), 6 (a ring of 2: nothing read ahead) and 7
    (ring of 4, relaxation deferred by one row)."""
    simulate(nx, ny, slots, grid, defer)


@pytest.mark.parametrize("nx,ny", [(128, 12), (192, 45), (256, 70), (640, 33), (1024, 300), (2048, 130)])
@pytest.mark.parametrize("slots", [4, 5])
@pytest.mark.parametrize("grid", [7, 152, 304])
def test_second_order_march_schedule_covers_interior_once(nx, ny, slots, grid):
    """Second-order march (load paths 8 and 9 after lbm_set_transport(sim, 2)): rings of five
    and four slots, rows [2, ny - 3]."""
    simulate(nx, ny, slots, grid, order=2)


def _library():
    from paper_1308_0692_gb300 import build, lbm
    build.build()
    return lbm


@pytest.mark.parametrize("nx,ny", [(128, 10), (192, 45), (256, 70), (384, 522), (640, 33), (1024, 1000),
                                   (1024, 1024), (2048, 2048), (4096, 1030)])
@pytest.mark.parametrize("grid", [7, 152, 304])
def test_library_plan_equals_model(nx, ny, grid):
    assert _library().lbm_march_plan(nx, ny, grid) == choose_chunks(nx, ny, grid)


def test_library_plan_rejects_unfit_grids():
    lbm = _library()
    for nx, ny in [(160, 64), (64, 64), (128, 9)]:
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_march_plan(nx, ny, 152)
        assert e.value.status == lbm.LBM_EUNSUPPORTED


def test_chunk_choice_fills_rounds():
    # 2048^2 on 152 blocks: 31 strips x 44 chunks = 1364 items = 8.97 rounds of 152
    assert choose_chunks(2048, 2048, 152) == (31, 44)
    strips, c = choose_chunks(1024, 1024, 152)
    items = strips * c
    assert items % 152 == 0 or items % 152 > 0.9 * 152
    for nx, ny, g in [(2048, 2048, 152), (1024, 1024, 152), (384, 522, 152), (256, 70, 304)]:
        _, c = choose_chunks(nx, ny, g)
        assert (ny - 2) // c >= 8


# ---- strip-tiled state (load path 8): tile t holds x in [64 t - 32, 64 t + 32) as [y][a][64]

TILE_W, TILE_SHIFT = 64, 32


def tiles_for(nx):
    return (nx + TILE_SHIFT + TILE_W - 1) // TILE_W


def tile_off(x, y, n, tile_pitch):
    xs = x + TILE_SHIFT
    return (xs // TILE_W) * tile_pitch + y * n * TILE_W + xs % TILE_W


def tiled_cell(off, n, tile_pitch):
    """(x, y, a) stored at float offset `off` of the tiled state, or None for padding."""
    t, rem = divmod(off, tile_pitch)
    y, rem = divmod(rem, n * TILE_W)
    a, p = divmod(rem, TILE_W)
    return t * TILE_W - TILE_SHIFT + p, y, a


@pytest.mark.parametrize("nx,ny", [(128, 10), (192, 11), (256, 13), (640, 12)])
@pytest.mark.parametrize("n", [64, 144])
def test_tiled_offsets_are_a_bijection_onto_the_buffer(nx, ny, n):
    tp = ny * n * TILE_W
    size = tiles_for(nx) * tp
    seen = set()
    for y in range(ny):
        for x in range(nx):
            for a in (0, n // 2, n - 1):
                off = tile_off(x, y, n, tp) + a * TILE_W
                assert 0 <= off < size and off not in seen
                assert tiled_cell(off, n, tp) == (x, y, a)
                seen.add(off)
    # the buffer holds every (cell, velocity) once plus one tile column of padding
    assert size == (nx + TILE_W) * ny * n


@pytest.mark.parametrize("nx,ny", [(128, 10), (192, 45), (384, 30), (2048, 12)])
@pytest.mark.parametrize("m,g", [(12, 6), (8, 4)])
@pytest.mark.parametrize("order", [1, 2])
def test_tiled_march_copies(nx, ny, m, g, order):
    """Every row copy of the tiled march (one contiguous bulk copy of the warp's lines, one
    4-byte asynchronous copy of the x halo per velocity) lies inside the buffer, the bulk copy
    starts 16-byte aligned and covers exactly the warp's velocities of the strip's cells in
    that row, and each halo copy takes the upwind x neighbour of the strip's edge cell for that
    velocity into the position the kernel reads (index 3 of the velocity's 4-float halo slot
    for the left neighbour, index 0 for the right one)."""
    n, half = m * m, m // 2
    rpl = m // g
    nvw = rpl * m
    tp = ny * n * TILE_W
    size = tiles_for(nx) * tp
    strips = (nx - 64) // 64
    for s in range(strips):
        x0 = 32 + 64 * s
        for row in range(ny):
            left_row = s * tp + row * n * TILE_W
            for w in range(g):
                big = left_row + tp + w * nvw * TILE_W
                assert big % 4 == 0 and 0 <= big and big + nvw * TILE_W <= size
                for q in range(nvw * TILE_W):
                    x, y, a = tiled_cell(big + q, n, tp)
                    assert (y, a) == (row, w * nvw + q // TILE_W) and x == x0 + q % TILE_W
                dsts = set()
                for k in range(nvw):
                    ix = k % m
                    a = w * nvw + k
                    # order 1: the upwind cell next to the strip (4 bytes); order 2: the two
                    # upwind cells (8 bytes, 8-byte aligned on both sides)
                    if ix >= m - half:
                        halo = left_row + a * TILE_W + (TILE_W - order)
                        want, dst = x0 - order, nvw * TILE_W + 4 * k + 4 - order
                    else:
                        halo = left_row + 2 * tp + a * TILE_W
                        want, dst = x0 + 64, nvw * TILE_W + 4 * k
                    for j in range(order):
                        assert 0 <= halo + j < size
                        x, y, aa = tiled_cell(halo + j, n, tp)
                        assert (x, y, aa) == (want + j, row, a) and 0 <= x < nx
                        # inside the warp's slot (dense lines, then 4 floats per velocity), one each
                        assert nvw * TILE_W <= dst + j < nvw * (TILE_W + 4) and dst + j not in dsts
                        dsts.add(dst + j)
                    if order == 2:
                        assert halo % 2 == 0 and dst % 2 == 0


# ---- batched column march on strip-tiled cavity instances: 32-column tiles, velocity pairs
# side by side per cell: value (a, x, y) at (x/32) tp + 32 n y + 64 (a/2) + 2 (x mod 32) + a mod 2

def batch_tile_index(a, x, y, n, ny):
    return (x >> 5) * (32 * n * ny) + y * 32 * n + (a >> 1) * 64 + (x & 31) * 2 + (a & 1)


def batch_tiled_cell(off, n, ny):
    """(a, x, y) stored at offset `off` of a tiled instance (x may lie in the last tile's padding)."""
    t, rem = divmod(off, 32 * n * ny)
    y, rem = divmod(rem, 32 * n)
    pair, rem = divmod(rem, 64)
    xc, odd = divmod(rem, 2)
    return 2 * pair + odd, 32 * t + xc, y


@pytest.mark.parametrize("nx,ny", [(3, 2), (64, 5), (70, 9), (96, 4), (97, 6), (128, 3)])
@pytest.mark.parametrize("m,g", [(8, 4), (8, 8), (4, 2), (4, 4)])
def test_batch_tiled_march_copies(nx, ny, m, g):
    """The batched column march's row copies on a strip-tiled cavity instance (the kernel's own
    arithmetic): the bulk copy of a warp's velocity pairs of a row starts 16-byte aligned inside
    the instance and covers exactly those pairs of the strip's 32 columns (padding past nx in a
    ragged last tile); each 8-byte halo copy takes, for a pair moving right, the cell left of
    the strip, for a pair moving left the cell right of it, both inside the instance; at a side
    wall it takes a cell of the strip itself (the wall lane uses the ghost instead)."""
    n = m * m
    rpl, half_pairs, p_row = m // g, m // 4, m // 2
    pw = rpl * m // 2
    ntiles = (nx + 31) // 32
    vals = ntiles * ny * n * 32
    tp, trow = 32 * n * ny, 32 * n
    # every (a, x, y) of the grid has its own place; the rest is padding
    places = {batch_tile_index(a, x, y, n, ny) for a in range(n) for x in range(nx) for y in range(ny)}
    assert len(places) == n * nx * ny and max(places) < vals
    off = 16 * 37                                   # an instance offset as the batch lays them out
    assert off % 16 == 0
    for tile in range(ntiles):
        x0 = 32 * tile
        for w in range(g):
            iy0 = w * rpl
            wbase = off + tile * tp + (iy0 * m // 2) * 64
            for r in range(ny):
                src = wbase + r * trow
                assert src % 4 == 0 and off <= src and src + pw * 64 <= off + vals
                for k in range(pw * 64):
                    a, x, y = batch_tiled_cell(src - off + k, n, ny)
                    assert y == r and x0 <= x < x0 + 32 and a // 2 == iy0 * m // 2 + k // 64
                for hq in range(pw):
                    j = hq % p_row
                    if j >= half_pairs:
                        halo = -tp + 62 if tile > 0 else 0
                        want = x0 - 1 if tile > 0 else None
                    else:
                        halo = tp if tile + 1 < ntiles else 0
                        want = x0 + 32 if tile + 1 < ntiles else None
                    h = wbase + hq * 64 + halo + r * trow
                    assert h % 2 == 0 and off <= h and h + 2 <= off + vals
                    a, x, y = batch_tiled_cell(h - off, n, ny)
                    assert y == r and a == 2 * (iy0 * m // 2 + hq)
                    if want is not None:
                        assert x == want and 0 <= x < nx
                    else:
                        assert x0 <= x < x0 + 32
