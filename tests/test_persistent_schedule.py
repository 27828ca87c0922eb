"""Model check of the persistent form's dependency rule (no GPU). Every tile
counts its finished work items; an item of half cycle j on tile (I, J) starts
once every tile of its periodic 3 x 3 neighbourhood has finished all of its
items of the previous phase (count >= 1 + 3j for a bridge item, >= 3 + 3j for
an octahedron or final Down item). Random interleavings of concurrent items
(each a start event, reads at any time while it runs, and an end event that
writes and counts) must never let an item read a panel slot that is not the
version it needs, nor let a writer overwrite a slot that a running item still
reads. The one-launch batch form is modelled too: several classes, each with
its own items and counter, run by blocks of teams that take the classes in
order and wait at a block barrier between classes.

Items (the launch-per-phase schedule of Algorithm 4 on one GPU, as work items;
panel slots are per tile and side group):
  first Up(I, J), frame 0: reads the state, writes up slot (I, J)
  half cycle j, y-bridge(I, J): reads up (I, J) and (I, J+1), writes the
                     bridge slot (I, J) W/E sides
  half cycle j, x-bridge(I, J): reads up (I, J) and (I+1, J), writes the
                     bridge slot (I, J) N/S sides
  half cycle j, octahedron (j < H-1) or final Down (j = H-1): reads the W/E
                     sides of bridge slots (I, J), (I+1, J) and the N/S sides of
                     (I, J), (I, J+1); the octahedron writes up slot (I, J) for
                     even j and (I+1, J+1) for odd j (its Up is in the shifted
                     frame); the final Down writes the state of the four tiles
                     its shifted tile overlaps (the first Ups read the state of
                     their own tile).
"""
import random

import pytest


def items_of(T, Q, H):
    """(phase, I, J, reads, writes, need) in the kernel's item order; phase
    numbers the launch-per-phase schedule (1, then 2 + 2j bridges and 3 + 2j
    octahedra) and `need` is the neighbourhood count the item waits for."""
    out = []
    wrap = lambda i, j: ((i % T), (j % Q))
    for J in range(Q):
        for I in range(T):
            out.append((1, I, J, [("st",) + wrap(I, J)], [("up",) + wrap(I, J)], 0))
    for j in range(H):
        for J in range(Q):
            for I in range(T):
                for xb in (False, True):
                    if xb:
                        reads = [("up",) + wrap(I, J), ("up",) + wrap(I + 1, J)]
                        writes = [("brNS",) + wrap(I, J)]
                    else:
                        reads = [("up",) + wrap(I, J), ("up",) + wrap(I, J + 1)]
                        writes = [("brWE",) + wrap(I, J)]
                    out.append((2 + 2 * j, I, J, reads, writes, 1 + 3 * j))
        for J in range(Q):
            for I in range(T):
                reads = [("brWE",) + wrap(I, J), ("brWE",) + wrap(I + 1, J),
                         ("brNS",) + wrap(I, J), ("brNS",) + wrap(I, J + 1)]
                if j + 1 < H:
                    writes = [("up",) + (wrap(I, J) if j % 2 == 0 else wrap(I + 1, J + 1))]
                else:   # the final Down writes the state of the tile shifted by (h, h)
                    writes = [("st",) + wrap(I + a, J + b) for a in (0, 1) for b in (0, 1)]
                out.append((3 + 2 * j, I, J, reads, writes, 3 + 3 * j))
    return out


def needed_version(p, kind):
    """The phase whose write an item of phase p must read in a slot of `kind`
    (the first Up reads the state as set, which no item has written)."""
    return None if kind == "st" else p - 1


def run_model(T, Q, H, rng):
    items = items_of(T, Q, H)
    done = {(I, J): 0 for J in range(Q) for I in range(T)}   # finished items per tile
    version = {}                                               # slot -> phase of last write
    pending = list(range(len(items)))
    running = []
    while pending or running:
        ready = []
        for k in pending:
            p, I, J, _, _, need = items[k]
            if all(done[((I + di) % T, (J + dj) % Q)] >= need
                   for di in (-1, 0, 1) for dj in (-1, 0, 1)):
                ready.append(k)
        choices = [("start", k) for k in ready] + [("end", k) for k in running]
        assert choices, "deadlock"
        what, k = rng.choice(choices)
        p, I, J, reads, writes, _ = items[k]
        if what == "start":
            for slot in reads:
                assert version.get(slot) == needed_version(p, slot[0]), (p, I, J, slot, version.get(slot))
            pending.remove(k)
            running.append(k)
        else:
            for slot in writes:
                for r in running:
                    if r != k:
                        assert slot not in items[r][3], ("overwrite while read", items[k][:3], items[r][:3], slot)
                version[slot] = p
            running.remove(k)
            done[(I, J)] += 1


def test_item_counts_and_needs_follow_the_kernel_layout():
    """NT (1 + 3H) items; a tile's count after its first Up is 1, after the
    bridges of half cycle j it is 3 + 3j, after the octahedron 4 + 3j."""
    T, Q, H = 3, 2, 4
    items = items_of(T, Q, H)
    assert len(items) == T * Q * (1 + 3 * H)
    per_tile = {}
    for p, I, J, _, _, need in items:
        per_tile.setdefault((I, J), []).append(need)
    for needs in per_tile.values():
        # the count a tile has reached when it starts each of its items
        assert needs == [0] + sum(([1 + 3 * j, 1 + 3 * j, 3 + 3 * j] for j in range(H)), [])


@pytest.mark.parametrize("T,Q", [(1, 1), (2, 1), (2, 2), (3, 2), (4, 3), (5, 5)])
@pytest.mark.parametrize("H", [1, 2, 3, 4])
def test_neighbourhood_waits_order_every_panel_exchange(T, Q, H):
    rng = random.Random(1000 * T + 10 * Q + H)
    for _ in range(40):
        run_model(T, Q, H, rng)


def test_a_smaller_neighbourhood_is_not_enough():
    """Waiting only for the tile itself (not its neighbours) lets an item read a
    slot before its producer wrote it: the model detects it."""
    rng = random.Random(7)
    T, Q, H = 3, 3, 2
    items = items_of(T, Q, H)
    done = {(I, J): 0 for J in range(Q) for I in range(T)}
    version, pending, failures = {}, list(range(len(items))), 0
    while pending:
        ready = [k for k in pending if done[(items[k][1], items[k][2])] >= items[k][5]]
        k = rng.choice(ready)
        p, I, J, reads, writes, _ = items[k]
        if any(version.get(s) != needed_version(p, s[0]) for s in reads):
            failures += 1
        for s in writes:
            version[s] = p
        done[(I, J)] += 1
        pending.remove(k)
    assert failures > 0


# ---- the one-launch batch form: several classes, blocks of teams

def run_one_launch_model(classes, blocks, teams, rng):
    """classes: list of (T, Q, H). Every block takes the classes in order;
    each of its teams takes the current class's items one at a time from the
    class's counter, waits for the item's neighbourhood counts, runs it (start
    and end events, reads checked against the versions the item needs), and
    when the counter is past the class's last item waits at the block's
    barrier; once all of a block's teams wait there, the block moves on to the
    next class. Returns when every item of every class has ended; asserts that
    some action is always possible (no deadlock)."""
    cls = []
    for (T, Q, H) in classes:
        items = items_of(T, Q, H)
        cls.append(dict(T=T, Q=Q, items=items, next=0,
                        done={(I, J): 0 for J in range(Q) for I in range(T)}, version={}))
    # team state: (block, team) -> ("fetch" | ("hold", k, started) | "barrier", class index)
    state = {(b, t): ["fetch", 0] for b in range(blocks) for t in range(teams)}
    running = {c: [] for c in range(len(cls))}   # items started, not ended
    finished = 0
    total = sum(len(c["items"]) for c in cls)
    while finished < total:
        actions = []
        for key, (st, c) in state.items():
            if c >= len(cls):
                continue
            C = cls[c]
            if st == "fetch":
                actions.append(("fetch", key))
            elif st == "barrier":
                b = key[0]
                if all(state[(b, t)][0] == "barrier" and state[(b, t)][1] == c
                       for t in range(teams)):
                    actions.append(("release", key))
            else:
                _, k, started = st
                p, I, J, reads, writes, need = C["items"][k]
                if not started:
                    if all(C["done"][((I + di) % C["T"], (J + dj) % C["Q"])] >= need
                           for di in (-1, 0, 1) for dj in (-1, 0, 1)):
                        actions.append(("start", key))
                else:
                    actions.append(("end", key))
        assert actions, "deadlock"
        what, key = rng.choice(actions)
        st, c = state[key]
        C = cls[c] if c < len(cls) else None
        if what == "fetch":
            if C["next"] < len(C["items"]):
                state[key] = [("hold", C["next"], False), c]
                C["next"] += 1
            else:
                state[key] = ["barrier", c]
        elif what == "release":
            b = key[0]
            for t in range(teams):
                state[(b, t)] = ["fetch", c + 1]
        elif what == "start":
            _, k, _ = st
            p, I, J, reads, writes, need = C["items"][k]
            for slot in reads:
                assert C["version"].get(slot) == needed_version(p, slot[0]), (c, p, I, J, slot)
            running[c].append(k)
            state[key] = [("hold", k, True), c]
        else:
            _, k, _ = st
            p, I, J, reads, writes, need = C["items"][k]
            for slot in writes:
                for r in running[c]:
                    if r != k:
                        assert slot not in C["items"][r][3], ("overwrite while read", c, p, slot)
                C["version"][slot] = p
            running[c].remove(k)
            C["done"][(I, J)] += 1
            finished += 1
            state[key] = ["fetch", c]
    return True


@pytest.mark.parametrize("blocks,teams", [(1, 1), (1, 3), (2, 2), (3, 4)])
def test_one_launch_classes_and_teams_never_deadlock_or_race(blocks, teams):
    """Several tile classes (their own grids, half cycles and counters) run by
    blocks of teams that wait at a block barrier between classes: every item
    still sees the panel versions it needs, no writer overwrites a slot being
    read, and the launch always finishes, even with a single team in a single
    block."""
    rng = random.Random(97 * blocks + teams)
    for classes in ([(2, 2, 3), (3, 1, 2)], [(1, 1, 2), (2, 3, 1), (3, 3, 2)]):
        for _ in range(15):
            run_one_launch_model(classes, blocks, teams, rng)

