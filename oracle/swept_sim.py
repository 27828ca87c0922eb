"""Slow CPU walk-through of the Swept 2D components (TEST INFRASTRUCTURE ONLY).

Only ``tests/`` use this module. It restates, in plain numpy and Python loops,
the four components of Section 3 and the glue of Algorithm 4, on tiny grids:

* ``upward_pyramid``      Algorithm 1 (Section 3.1)
* ``longitudinal_bridge`` Algorithm 2 (Section 3.2)
* ``latitudinal_bridge``  Algorithm 3 (Section 3.2)
* ``downward_pyramid``    Algorithm 5 (Section 3.3)
* ``swept2d``             Algorithm 4 (Section 4): each tile is one "process",
                          panels are messages between processes.

Notation follows the paper: every component works on two (n+2) x (n+2) arrays
``D`` and ``U`` indexed ``[i, j]`` with ``i`` along x (west -> east) and ``j``
along y (north -> south), interior indices 1..n. An inclusive paper range
``a:b`` becomes the Python slice ``a:b+1``. A point state is a vector of ``nv``
values, so arrays are (n+2, n+2, nv).

The stencil ``St(g, nb)`` receives the global sub-step index ``g`` and the
3 x 3 neighbourhood ``nb[di, dj, :]`` (di, dj in 0..2, centre at [1, 1]) and
returns the new point state.

Readings of the printed algorithms (where the text is garbled or inconsistent):

* Algorithms 2 and 3 print the bridge compute range as ``n/2-k .. n/2-k+1``;
  the bridge grows by one row on each side per level (its panels have
  ``2(2k+2)`` values), so the range is read as ``n/2-k .. n/2+k+1``.
* Algorithm 5 prints ``k = 0 .. n/2``; at ``k = n/2`` the ranges leave the
  (n+2) x (n+2) array, and the last level is ``n/2``, so the loop is read as
  ``k = 0 .. n/2-1`` (levels 1 .. n/2).
* Algorithm 3's two outputs carry the 2 x 2 corner on the side that
  Algorithm 5 places them on: Algorithm 5 puts the north input at columns
  ``n/2-k+1 .. n/2+k+2`` and the south input at ``n/2-k-1 .. n/2+k``, and
  Algorithm 4 feeds it the latitudinal bridge's *south* output as its north
  input. So S^k is taken over ``n/2-k+1 .. n/2+k+2`` and N^k over
  ``n/2-k-1 .. n/2+k`` (the printed extents are the other way round, which
  puts every corner two columns away from where it belongs; ``literal_alg3``
  keeps the printed extents so that a test can show this).
"""
from __future__ import annotations

import numpy as np


def _nb(D, i, j):
    return D[i - 1:i + 2, j - 1:j + 2]


def upward_pyramid(St, B, g0):
    """Algorithm 1. ``B`` is (n, n, nv) at level 0 of the half cycle whose first
    sub-step is ``g0``. Returns the panels (N, S, W, E), each a list over
    k = 0..n/2-1 of (2-wide) arrays, and a trace of computed square sizes."""
    n = B.shape[0]
    h = n // 2
    D = np.zeros((n + 2, n + 2) + B.shape[2:], dtype=B.dtype)
    U = np.zeros_like(D)
    D[1:n + 1, 1:n + 1] = B
    N, S, W, E = [], [], [], []
    sizes = []
    for k in range(h):
        N.append(D[k + 1:n - k + 1, k + 1:k + 3].copy())
        S.append(D[k + 1:n - k + 1, n - k - 1:n - k + 1].copy())
        W.append(D[k + 1:k + 3, k + 1:n - k + 1].copy())
        E.append(D[n - k - 1:n - k + 1, k + 1:n - k + 1].copy())
        count = 0
        for i in range(2 + k, n - k):          # i = 2+k .. n-k-1
            for j in range(2 + k, n - k):
                U[i, j] = St(g0 + k, _nb(D, i, j))
                count += 1
        sizes.append(count)
        D, U = U, D
    return (N, S, W, E), sizes


def longitudinal_bridge(St, Nin, Sin, n, g0):
    """Algorithm 2. ``Nin`` is placed on the north side (it is the south panel
    of the pyramid to the north), ``Sin`` on the south side. Returns (W, E)."""
    h = n // 2
    shape = (n + 2, n + 2) + Nin[0].shape[2:]
    D = np.zeros(shape, dtype=Nin[0].dtype)
    U = np.zeros_like(D)
    W, E = [], []
    for k in range(h):
        D[k + 1:n - k + 1, h - k - 1:h - k + 1] = Nin[k]
        D[k + 1:n - k + 1, h + k + 1:h + k + 3] = Sin[k]
        W.append(D[k + 1:k + 3, h - k + 1:h + k + 3].copy())
        E.append(D[n - k - 1:n - k + 1, h - k - 1:h + k + 1].copy())
        for i in range(2 + k, n - k):          # i = 2+k .. n-k-1
            for j in range(h - k, h + k + 2):  # j = n/2-k .. n/2+k+1 (read, see module doc)
                U[i, j] = St(g0 + k, _nb(D, i, j))
        D, U = U, D
    return W, E


def latitudinal_bridge(St, Win, Ein, n, g0, literal_alg3=False):
    """Algorithm 3. ``Win`` is placed on the west side (east panel of the
    pyramid to the west), ``Ein`` on the east side. Returns (N, S)."""
    h = n // 2
    shape = (n + 2, n + 2) + Win[0].shape[2:]
    D = np.zeros(shape, dtype=Win[0].dtype)
    U = np.zeros_like(D)
    N, S = [], []
    for k in range(h):
        D[h - k - 1:h - k + 1, k + 1:n - k + 1] = Win[k]
        D[h + k + 1:h + k + 3, k + 1:n - k + 1] = Ein[k]
        if literal_alg3:
            N.append(D[h - k + 1:h + k + 3, k + 1:k + 3].copy())
            S.append(D[h - k - 1:h + k + 1, n - k - 1:n - k + 1].copy())
        else:
            N.append(D[h - k - 1:h + k + 1, k + 1:k + 3].copy())
            S.append(D[h - k + 1:h + k + 3, n - k - 1:n - k + 1].copy())
        for i in range(h - k, h + k + 2):      # i = n/2-k .. n/2+k+1 (read)
            for j in range(2 + k, n - k):
                U[i, j] = St(g0 + k, _nb(D, i, j))
        D, U = U, D
    return N, S


def downward_pyramid(St, N, S, W, E, n, g0):
    """Algorithm 5 (loop read as k = 0..n/2-1). Returns the n x n tile at level
    n/2 and the trace of computed square sides per level."""
    h = n // 2
    shape = (n + 2, n + 2) + W[0].shape[2:]
    D = np.zeros(shape, dtype=W[0].dtype)
    U = np.zeros_like(D)
    sides = []
    for k in range(h):
        D[h - k - 1:h - k + 1, h - k - 1:h + k + 1] = W[k]
        D[h + k + 1:h + k + 3, h - k + 1:h + k + 3] = E[k]
        D[h - k + 1:h + k + 3, h - k - 1:h - k + 1] = N[k]
        D[h - k - 1:h + k + 1, h + k + 1:h + k + 3] = S[k]
        for i in range(h - k, h + k + 2):
            for j in range(h - k, h + k + 2):
                U[i, j] = St(g0 + k, _nb(D, i, j))
        sides.append(2 * k + 2)
        D, U = U, D
    return D[1:n + 1, 1:n + 1].copy(), sides


class Trace:
    """What the walk-through observed: messages and panel sizes."""

    def __init__(self):
        self.exchanges = 0          # exchange rounds (one per communication step)
        self.messages = 0           # panels sent, all processes
        self.up_panel_level_sizes = None
        self.bridge_panel_level_sizes = None
        self.up_compute_sizes = None
        self.down_square_sides = None


def swept2d(St, state, n, cycles, g0=0, literal_alg3=False, trace=None):
    """Algorithm 4 on a periodic grid ``state`` of shape (nx, ny, nv) (indexed
    [i, j, :]) split into (nx/n) x (ny/n) tiles, one process per tile.
    Runs ``cycles`` full cycles (n sub-steps each) and returns the new grid.

    First half cycle: send N_U north and W_U west, receive from south/east;
    y-bridge south and x-bridge east of the own pyramid; send N_D north and
    W_D west; the downward pyramid fills the south-east corner (frame shifted
    by +n/2 in x and y). Second half: the same with S/E sent south/east, the
    bridges north/west of the own pyramid and the downward pyramid at the
    north-west corner, which restores the original frame."""
    nx, ny = state.shape[:2]
    assert nx % n == 0 and ny % n == 0 and n % 2 == 0 and n >= 4
    P, Q = nx // n, ny // n
    h = n // 2
    tr = trace if trace is not None else Trace()
    B = {(I, J): state[I * n:(I + 1) * n, J * n:(J + 1) * n].copy()
         for I in range(P) for J in range(Q)}
    g = g0
    for _ in range(cycles):
        # ---- first half cycle
        up = {}
        for key, b in B.items():
            up[key], sizes = upward_pyramid(St, b, g)
            tr.up_compute_sizes = sizes
        tr.up_panel_level_sizes = [int(np.prod(p.shape[:2])) for p in up[(0, 0)][0]]
        tr.exchanges += 1
        tr.messages += 2 * len(B)
        recvN = {(I, J): up[(I, (J + 1) % Q)][0] for (I, J) in B}   # N_U from the south
        recvW = {(I, J): up[((I + 1) % P, J)][2] for (I, J) in B}   # W_U from the east
        yb, xb = {}, {}
        for (I, J) in B:
            N_U, S_U, W_U, E_U = up[(I, J)]
            yb[(I, J)] = longitudinal_bridge(St, S_U, recvN[(I, J)], n, g)          # (W_D, E_D)
            xb[(I, J)] = latitudinal_bridge(St, E_U, recvW[(I, J)], n, g, literal_alg3)  # (N_D, S_D)
        tr.bridge_panel_level_sizes = [int(np.prod(p.shape[:2])) for p in yb[(0, 0)][0]]
        tr.exchanges += 1
        tr.messages += 2 * len(B)
        newB = {}
        for (I, J) in B:
            W_D, E_D = yb[(I, J)]
            N_D, S_D = xb[(I, J)]
            rN_D = xb[(I, (J + 1) % Q)][0]      # N_D received from the south
            rW_D = yb[((I + 1) % P, J)][0]      # W_D received from the east
            newB[(I, J)], sides = downward_pyramid(St, S_D, rN_D, E_D, rW_D, n, g)
            tr.down_square_sides = sides
        B = newB
        g += h
        # ---- second half cycle (frame shifted by +n/2; own tile (I, J) now
        # covers x in [I n + n/2, I n + 3n/2), likewise y)
        up = {key: upward_pyramid(St, b, g)[0] for key, b in B.items()}
        tr.exchanges += 1
        tr.messages += 2 * len(B)
        recvS = {(I, J): up[(I, (J - 1) % Q)][1] for (I, J) in B}   # S_U from the north
        recvE = {(I, J): up[((I - 1) % P, J)][3] for (I, J) in B}   # E_U from the west
        yb, xb = {}, {}
        for (I, J) in B:
            N_U, S_U, W_U, E_U = up[(I, J)]
            yb[(I, J)] = longitudinal_bridge(St, recvS[(I, J)], N_U, n, g)
            xb[(I, J)] = latitudinal_bridge(St, recvE[(I, J)], W_U, n, g, literal_alg3)
        tr.exchanges += 1
        tr.messages += 2 * len(B)
        newB = {}
        for (I, J) in B:
            W_D, E_D = yb[(I, J)]
            N_D, S_D = xb[(I, J)]
            rS_D = xb[(I, (J - 1) % Q)][1]      # S_D received from the north
            rE_D = yb[((I - 1) % P, J)][1]      # E_D received from the west
            newB[(I, J)], _ = downward_pyramid(St, rS_D, N_D, rE_D, W_D, n, g)
        B = newB
        g += h
    out = np.empty_like(state)
    for (I, J), b in B.items():
        out[I * n:(I + 1) * n, J * n:(J + 1) * n] = b
    return out


def plain_steps(St, state, nsub, g0=0):
    """The plain definition on the same (nx, ny, nv) layout: ``nsub`` sweeps."""
    nx, ny = state.shape[:2]
    u = state.copy()
    for s in range(nsub):
        v = np.empty_like(u)
        for i in range(nx):
            for j in range(ny):
                nb = u[np.ix_([(i - 1) % nx, i, (i + 1) % nx], [(j - 1) % ny, j, (j + 1) % ny])]
                v[i, j] = St(g0 + s, nb)
        u = v
    return u
