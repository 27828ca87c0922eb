"""Pins for the component walk-through (oracle/swept_sim.py): the paper's
worked-example numbers (tests/golden/paper_worked_examples.json), the exact
partition / no-redundancy claim, and equality with plain time marching."""
import json
import os

import numpy as np
import pytest

from oracle import swept_sim

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                     "paper_worked_examples.json")))
PRIME = (1 << 61) - 1


class Mixer:
    """A position- and order-sensitive stencil on nv int64 components (any wrong,
    missing or stale neighbour changes its output); counts its calls."""

    def __init__(self, nv):
        self.nv = nv
        self.calls = 0

    def __call__(self, g, nb):
        self.calls += 1
        flat = [int(v) for v in nb.reshape(-1)]
        out = np.empty(self.nv, dtype=np.int64)
        for c in range(self.nv):
            h = (g * 1000003 + c * 7919 + 12345) % PRIME
            for v in flat:
                h = (h * 1099511628211 + v) % PRIME
            out[c] = h
        return out


def _state(nx, ny, nv, seed):
    return np.random.default_rng(seed).integers(0, PRIME, size=(nx, ny, nv), dtype=np.int64)


@pytest.mark.parametrize("nx,ny,n,cycles", [(16, 16, 8, 1), (24, 16, 8, 2), (12, 8, 4, 3)])
def test_swept_equals_plain_marching_without_redundancy(nx, ny, n, cycles):
    """Abstract / Section 4: the swept decomposition computes every (point, level)
    exactly once, from the same neighbourhood as plain time marching."""
    st = Mixer(nv=2)
    u0 = _state(nx, ny, 2, seed=nx * 100 + ny)
    swept = swept_sim.swept2d(st, u0, n, cycles)
    assert st.calls == nx * ny * n * cycles          # no redundant computation
    ref = swept_sim.plain_steps(Mixer(nv=2), u0, n * cycles)
    assert np.array_equal(swept, ref)


def test_literal_latitudinal_extents_misplace_the_corners():
    """Algorithm 3's printed output extents put the 2 x 2 corners of the north and
    south bridge panels on the opposite side from where Algorithm 5 places them;
    taken literally, the result differs from plain time marching."""
    u0 = _state(16, 16, 1, seed=1)
    ref = swept_sim.plain_steps(Mixer(1), u0, 8)
    assert np.array_equal(swept_sim.swept2d(Mixer(1), u0, 8, 1), ref)
    assert not np.array_equal(swept_sim.swept2d(Mixer(1), u0, 8, 1, literal_alg3=True), ref)


def test_paper_worked_example_numbers():
    """Section 3.1, 3.2, 3.3 and 4 on 8 x 8 tiles with the 'increment by 1' stencil
    starting from level 1 on a domain of 4 subdomains."""
    up = GOLDEN["upward_pyramid_8x8"]
    br = GOLDEN["bridge_panels_8x8"]
    dn = GOLDEN["downward_pyramid_8x8"]
    cy = GOLDEN["swept_cycle_8x8"]
    n = up["n"]
    inc = lambda g, nb: nb[1, 1] + 1
    u0 = np.full((2 * n, 2 * n, 1), float(cy["initial_level"]))
    tr = swept_sim.Trace()
    out = swept_sim.swept2d(inc, u0, n, 1, trace=tr)
    assert tr.up_panel_level_sizes == up["panel_values_added_per_level"]
    assert [int(round(np.sqrt(c))) for c in tr.up_compute_sizes[:-1]] == up["computed_square_sides"]
    assert tr.up_compute_sizes[-1] == 0                 # "no further computation is possible"
    assert tr.bridge_panel_level_sizes == br["panel_values_per_level"]
    assert tr.down_square_sides == dn["computed_square_sides"]
    assert [s + 2 for s in tr.down_square_sides[:2]] == dn["first_working_square_sides"]
    assert tr.exchanges == cy["communications_per_full_cycle"]
    assert np.all(out == cy["initial_level"] + cy["levels_per_full_cycle"])
    # tip of the upward pyramid: the last panel level holds values at level 4
    (N, S, W, E), _ = swept_sim.upward_pyramid(inc, u0[:n, :n], 0)
    assert np.all(N[-1] == cy["pyramid_tip_level"]) and N[-1].size == 4
    # level squares 8, 6, 4, 2: each panel level is the 2-wide ring of that square
    assert [p.shape[0] for p in N] == up["level_square_sides"]


def test_half_cycle_shifts_the_frame_by_half_a_tile():
    """Section 4: after a half cycle the tiles are shifted by (n/2, n/2); after a
    full cycle the original arrangement is restored. A cycle count that is not
    whole is not expressible by Algorithm 4; we check the full-cycle restore and
    that a half cycle leaves the Down tile at the south-east corner."""
    n = 8
    u0 = _state(16, 16, 1, seed=3)
    inc = lambda g, nb: nb[1, 1]                 # identity: positions only
    out = swept_sim.swept2d(inc, u0, n, 1)
    assert np.array_equal(out, u0)
    # one half cycle by hand: Down of tile (0,0) covers x, y in [n/2, 3n/2)
    up = {(I, J): swept_sim.upward_pyramid(inc, u0[I * n:(I + 1) * n, J * n:(J + 1) * n], 0)[0]
          for I in range(2) for J in range(2)}
    W_D, E_D = swept_sim.longitudinal_bridge(inc, up[(0, 0)][1], up[(0, 1)][0], n, 0)
    N_D, S_D = swept_sim.latitudinal_bridge(inc, up[(0, 0)][3], up[(1, 0)][2], n, 0)
    W_D1, _ = swept_sim.longitudinal_bridge(inc, up[(1, 0)][1], up[(1, 1)][0], n, 0)
    N_D1, _ = swept_sim.latitudinal_bridge(inc, up[(0, 1)][3], up[(1, 1)][2], n, 0)
    B, _ = swept_sim.downward_pyramid(inc, S_D, N_D1, E_D, W_D1, n, 0)
    assert np.array_equal(B, u0[n // 2:n // 2 + n, n // 2:n // 2 + n])


def test_two_substep_scheme_through_the_swept_components(oracle_lib):
    """Eqs. (substep1)-(substep2) run as a 2-stage, 5-component stencil through
    Algorithms 1-5 reproduce eq. (complex_step) computed directly by the C oracle."""
    M = (1 << 64) - 1

    def st(g, nb):
        c = nb[1, 1]
        if g % 2 == 0:   # eq. (substep1): push u and its 4 neighbours
            return np.array([c[0], nb[0, 1][0], nb[2, 1][0], nb[1, 0][0], nb[1, 2][0]],
                            dtype=object)
        v = (int(nb[0, 1][1]) + int(nb[2, 1][2]) + int(nb[1, 0][3]) + int(nb[1, 2][4])
             - 4 * int(c[0])) & M                 # eq. (substep2)
        return np.array([v, 0, 0, 0, 0], dtype=object)

    rng = np.random.default_rng(12)
    words = rng.integers(0, 2**64, size=(16, 8), dtype=np.uint64)   # (ny, nx)
    u0 = np.zeros((8, 16, 5), dtype=object)
    u0[:, :, 0] = np.array([[int(v) for v in row] for row in words.T], dtype=object)
    out = swept_sim.swept2d(st, u0, 4, 2)          # 8 sub-steps = 4 steps
    ref = oracle_lib.wide2(words, 4)
    got = np.array([[int(v) for v in row] for row in out[:, :, 0].T], dtype=np.uint64)
    assert np.array_equal(got, ref)
