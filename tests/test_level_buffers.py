"""Geometry checks (CPU) of the swept blocks' level buffers: the positions the
kernels copy each level's ring (downward pyramid, Algorithm 5) and strips
(bridges, Algorithms 2 and 3) into, restated from the kernels' index formulas,
against the squares and rectangles each level computes and reads.

* Two buffers, every level's copies issued before the first level: rings
  (strips) of one parity never overlap, no level's writes or reads touch a
  later level's ring (strip) in the same buffer, and a bridge's panel reads
  of a level never see a later level's strip.
* One buffer (in-place levels): the next level's ring (strip), copied during a
  level, never lands in the square (rectangle) that level computes, and a
  bridge's panel reads of a level see only that level's values (the rectangle
  the previous level computed and the level's own strip). The updates whose
  first pass reads the neighbours (heat, wave) copy the next ring only after
  that pass, so the overlap with the current ring's inner line is harmless.
* Packed aux values: a level's pair sums (heat, wave) and fluxes (Euler) are
  packed for its own rectangle; every level of a block fits the block's aux
  buffer, the second pass finds each neighbour's value where the first pass
  put it, and the flux pitch keeps a column-pair walk conflict-free.
* Panel lines start on even elements (pair stores), and the downward
  pyramid's two-part staging keeps every ring in one part with 16-byte copies.
"""
import pytest

SIZES = [4, 6, 8, 16, 32, 64, 128]


def down_ring(n, k):
    h, L, pos = n // 2, 2 * k + 2, set()
    for side in range(4):
        for d in range(2):
            if side == 0:
                bx, by, ax, ay = h - 1 - k - d, h - k - 2, 0, 1
            elif side == 1:
                bx, by, ax, ay = h + k + d, h - k, 0, 1
            elif side == 2:
                bx, by, ax, ay = h - k, h - 1 - k - d, 1, 0
            else:
                bx, by, ax, ay = h - k - 2, h + k + d, 1, 0
            pos |= {(bx + p * ax, by + p * ay) for p in range(L)}
    return pos


def down_square(n, k):
    h = n // 2
    return {(x, y) for x in range(h - k - 1, h + k + 1) for y in range(h - k - 1, h + k + 1)}


def nbhd(points):
    return {(x + a, y + b) for (x, y) in points for a in (-1, 0, 1) for b in (-1, 0, 1)}


def bridge_strip(n, k):     # (along, across)
    h, L = n // 2, n - 2 * k
    return {(k + p, (h + k + d) if which else (h - 1 - k - d))
            for which in (0, 1) for d in (0, 1) for p in range(L)}


def bridge_rect(n, k):      # (along, across) of the points level k computes
    h = n // 2
    return {(u, w) for u in range(k + 1, n - k - 1) for w in range(h - k - 1, h + k + 1)}


def bridge_panel_reads(n, k, xb):
    h, L = n // 2, 2 * k + 2
    lo, hi = (-2, 0) if xb else (0, -2)
    return {((n - 1 - k - d) if which else (k + d), h - k + (hi if which else lo) + p)
            for which in (0, 1) for d in (0, 1) for p in range(L)}


@pytest.mark.parametrize("n", SIZES)
def test_down_rings_preloaded_into_two_buffers(n):
    h = n // 2
    for i in range(h):
        writes, reads = down_square(n, i), nbhd(down_square(n, i))
        for j in range(i + 1, h):
            if j % 2 == (i + 1) % 2:
                assert not writes & down_ring(n, j), (n, i, j)
            if j % 2 == i % 2:
                assert not reads & down_ring(n, j), (n, i, j)
        # level i's inputs are its ring and the square level i-1 wrote
        have = down_ring(n, i) | (down_square(n, i - 1) if i else set())
        assert reads <= have, (n, i)
    for j in range(h):
        for jj in range(j + 2, h, 2):
            assert not down_ring(n, j) & down_ring(n, jj), (n, j, jj)


@pytest.mark.parametrize("n", SIZES)
def test_bridge_strips_preloaded_into_two_buffers(n):
    h = n // 2
    for k in range(h - 1):
        writes, reads = bridge_rect(n, k), nbhd(bridge_rect(n, k))
        for j in range(k + 1, h):
            if j % 2 == (k + 1) % 2:
                assert not writes & bridge_strip(n, j), (n, k, j)
            if j % 2 == k % 2:
                assert not reads & bridge_strip(n, j), (n, k, j)
    for k in range(h):
        for xb in (0, 1):
            for j in range(k + 2, h, 2):
                assert not bridge_panel_reads(n, k, xb) & bridge_strip(n, j), (n, k, xb, j)
    for j in range(h):
        for jj in range(j + 2, h, 2):
            assert not bridge_strip(n, j) & bridge_strip(n, jj), (n, j, jj)


@pytest.mark.parametrize("n", SIZES)
def test_in_place_levels_copy_the_next_ring_outside_the_computed_points(n):
    h = n // 2
    for k in range(h - 1):
        assert not down_square(n, k) & down_ring(n, k + 1), (n, k)
        assert not bridge_rect(n, k) & bridge_strip(n, k + 1), (n, k)


@pytest.mark.parametrize("n", SIZES)
def test_in_place_bridge_panel_reads_see_only_the_current_level(n):
    h = n // 2
    for k in range(h):
        have = bridge_strip(n, k) | (bridge_rect(n, k - 1) if k else set())
        for xb in (0, 1):
            assert bridge_panel_reads(n, k, xb) <= have, (n, k, xb)



# ---- packed aux values of a level (pair sums; Euler fluxes), restated from
# aux_elems, flux_pitch and the index formulas of the level computations

def kernel_levels(n, kind):
    """(W, H) of every level rectangle a block of the kind computes."""
    h = n // 2
    if kind == "up":
        return [(n - 2 * k - 2, n - 2 * k - 2) for k in range(h - 1)]
    if kind == "bridge":
        out = []
        for k in range(h - 1):
            out += [(n - 2 * k - 2, 2 * k + 2), (2 * k + 2, n - 2 * k - 2)]
        return out
    return [(2 * k + 2, 2 * k + 2) for k in range(h)]          # down (and octahedron's down)


def flux_pitch(W):
    return W + 4 if (W + 2) % 4 == 0 else W + 2


def aux_elems(n, bridge, pair_sums):
    h = n // 2
    if pair_sums:
        return (h + 1) ** 2 if bridge else (n + 1) ** 2
    return (h + 3) ** 2 if bridge else flux_pitch(n) * (n + 2)


EVEN_SIZES = [4, 6, 8, 10, 16, 18, 32, 34, 64, 128]


@pytest.mark.parametrize("n", EVEN_SIZES)
def test_packed_pair_sums_fit_and_index_the_right_neighbours(n):
    for kind in ("up", "bridge", "down"):
        cap = aux_elems(n, kind == "bridge", True)
        for W, H in kernel_levels(n, kind):
            W1, cnt1 = W + 1, (W + 1) * (H + 1)
            assert cnt1 <= cap, (n, kind, W, H)
            # pass 1: entry e holds Pr(x0 - 1 + e % W1, y0 - 1 + e // W1)
            where = {e: (e % W1 - 1, e // W1 - 1) for e in range(cnt1)}
            for e in range(W * H):
                yy, xx = divmod(e, W)
                a = e + yy
                assert where[a] == (xx - 1, yy - 1)        # Pr(x-1, y-1)
                assert where[a + W1 + 1] == (xx, yy)        # Pr(x, y)


@pytest.mark.parametrize("n", EVEN_SIZES)
def test_packed_flux_planes_fit_index_and_keep_column_pairs_on_distinct_banks(n):
    for kind in ("up", "bridge", "down"):
        cap = aux_elems(n, kind == "bridge", False)
        for W, H in kernel_levels(n, kind):
            A = flux_pitch(W)
            assert A >= W + 2 and A * (H + 2) <= cap, (n, kind, W, H)
            # pass 2 of point (xx, yy): its own slot and the four neighbours'
            for yy in range(H):
                for xx in range(W):
                    a = (yy + 1) * A + xx + 1
                    for d in (1, -1, A, -A):
                        q = a + d
                        assert 0 <= q < A * (H + 2) and q % A < W + 2
            # 32 consecutive points of a column pair (16 rows x 2 columns) in
            # 4-byte fluxes fall on 32 different banks
            if H + 2 >= 16:
                banks = {(r * A + c) % 32 for r in range(16) for c in range(2)}
                assert len(banks) == 32, (n, W, A)


@pytest.mark.parametrize("n", EVEN_SIZES)
def test_bridge_plan_is_not_larger_than_the_pyramids(n):
    for pair_sums in (True, False):
        assert aux_elems(n, True, pair_sums) <= aux_elems(n, False, pair_sums)


@pytest.mark.parametrize("n", EVEN_SIZES)
def test_panel_lines_of_8_byte_elements_start_on_16_bytes(n):
    """The pair stores of 8-byte panel elements (two per 16-byte store) need
    every line to start at an even element with an even length: up lines
    L = n - 2k at 2k(n-k+1) + dL, bridge lines L = 2k + 2 at 2k(k+1) + dL, and
    every panel at a multiple of panel_stride(n) (a multiple of 8 elements)."""
    h = n // 2
    ps = ((n * n // 2 + n) + 7) & ~7
    assert ps % 8 == 0 and ps >= n * n // 2 + n
    for k in range(h):
        for L, off in ((n - 2 * k, 2 * k * (n - k + 1)), (2 * k + 2, 2 * k * (k + 1))):
            assert L % 2 == 0
            for d in (0, 1):
                start = off + d * L
                assert start % 2 == 0 and start + L <= n * n // 2 + n


def stage_split(n, esize):
    """The downward pyramid's two-part staging, restated: the level k1 whose
    ring offset 2 k1 (k1 + 1) starts on 16 bytes and makes the larger part
    smallest (0: one part)."""
    h, ps = n // 2, ((n * n // 2 + n) + 7) & ~7
    best, best_span = 0, ps
    for k in range(1, h):
        off = 2 * k * (k + 1)
        if (off * esize) % 16:
            continue
        span = max(off, ps - off)
        if span < best_span:
            best, best_span = k, span
    return best, best_span, ps


@pytest.mark.parametrize("n", [8, 16, 32, 64, 128])
@pytest.mark.parametrize("esize", [2, 4, 8])
def test_two_part_staging_keeps_rings_whole_and_copies_aligned(n, esize):
    """Each ring lies wholly in one part; both parts start on 16 bytes and
    their byte counts are multiples of 16 (bulk copies); each fits the
    staging slot; and every part-1 ring is read at an offset within it."""
    h = n // 2
    k1, span, ps = stage_split(n, esize)
    assert (span * esize) % 16 == 0 and span <= ps
    if not k1:
        return
    cut = 2 * k1 * (k1 + 1)
    assert (cut * esize) % 16 == 0 and ((ps - cut) * esize) % 16 == 0
    assert cut <= span and ps - cut <= span
    for k in range(h):
        off, L = 2 * k * (k + 1), 2 * k + 2
        lo, hi = off, off + 2 * L                 # the ring's two lines
        if k < k1:
            assert hi <= cut
        else:
            assert lo >= cut and hi - cut <= span
    # the staging area is smaller than the whole panel set
    assert span < ps
