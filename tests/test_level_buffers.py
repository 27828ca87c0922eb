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

