"""Model check of the engine's wait/publish protocol (host logic, no GPU).

The persistent engine's control warp (`engine_kernel` in csrc/hh_engine.cu)
walks its block's tiles phase by phase.  Before a system's slot it waits until
every tile of that system has published the previous phase; it posts the slot
to the compute warps and publishes the *previous* task only after preparing
the next one, unless

  * the next task is of the same system as the pending one, or
  * the next task is at a later phase (level) and the launch is not
    homogeneous (every block holds one tile of each system in the same order).

This test executes that schedule as a discrete simulation over random tile
layouts (blocks progress in random interleavings; a waiting block is blocked
until its condition holds) and checks that every run completes, i.e. the rule
admits no cycle of waits.  It also checks the rule is necessary: publishing
after the next preparation unconditionally deadlocks on layouts that are not
homogeneous, and so does a homogeneous layout with a single system.
"""
import random

import pytest


def simulate(block_tiles, nsys, levels, rule, rng, max_steps=200000, done_at=None):
    """block_tiles: per block, the list of systems of its tiles (in order).
    done_at: per system, the level from which it is done (its tasks are then
    skipped by every block, as all blocks take the same decision).
    Returns True if every block finishes all levels, False on deadlock."""
    tiles_of = {s: [] for s in range(nsys)}
    for b, lst in enumerate(block_tiles):
        for j, s in enumerate(lst):
            tiles_of[s].append((b, j))
    published = {}          # (b, j) -> highest published level
    homogeneous = all(lst == list(range(nsys)) for lst in block_tiles) and nsys >= 2

    # Per block: its task list (level, j, sys) and a cursor.
    done_at = done_at or [levels] * nsys
    tasks = [[(lv, j, s) for lv in range(levels) for j, s in enumerate(lst) if lv < done_at[s]]
             for lst in block_tiles]
    cur = [0] * len(block_tiles)
    pend = [None] * len(block_tiles)      # (level, j, sys) posted but not published
    stage = ["prep"] * len(block_tiles)   # prep -> (post) -> finish_pending

    def ready(lv, s):
        if lv == 0:
            return True
        return all(published.get(t, -1) >= lv - 1 for t in tiles_of[s])

    def must_finish_first(b, lv, s):
        p = pend[b]
        if p is None:
            return False
        if rule == "always_delay":
            return p[2] == s and False
        if rule == "never_delay":
            return True
        same_sys = p[2] == s
        return same_sys or (not homogeneous and p[0] != lv)

    for _ in range(max_steps):
        live = [b for b in range(len(block_tiles)) if cur[b] < len(tasks[b]) or pend[b] is not None]
        if not live:
            return True
        progressed = False
        for b in rng.sample(live, len(live)):
            if cur[b] >= len(tasks[b]):
                # all posted: publish the last pending task
                lv, j, s = pend[b]
                published[(b, j)] = lv
                pend[b] = None
                progressed = True
                continue
            lv, j, s = tasks[b][cur[b]]
            if stage[b] == "prep":
                if must_finish_first(b, lv, s):
                    plv, pj, ps = pend[b]
                    published[(b, pj)] = plv
                    pend[b] = None
                    progressed = True
                    continue
                if not ready(lv, s):
                    continue            # waiting on other blocks' signals
                # prepared and posted; the pending one is published after
                stage[b] = "posted"
                progressed = True
            if stage[b] == "posted":
                if pend[b] is not None:
                    plv, pj, ps = pend[b]
                    published[(b, pj)] = plv
                pend[b] = (lv, j, s)
                cur[b] += 1
                stage[b] = "prep"
                progressed = True
        if not progressed:
            return False
    raise AssertionError("simulation did not terminate")


def random_layout(rng, nblocks, nsys, max_tiles):
    """Tiles of each system in contiguous runs, dealt round-robin to blocks
    (tile t -> block t % nblocks), as the engine's tile lists are built."""
    tiles = []
    for s in range(nsys):
        tiles += [s] * rng.randint(1, max_tiles)
    blocks = [[] for _ in range(nblocks)]
    for t, s in enumerate(tiles):
        blocks[t % nblocks].append(s)
    return [b for b in blocks if b]


@pytest.mark.parametrize("seed", range(40))
def test_level_rule_never_deadlocks(seed):
    rng = random.Random(seed)
    layout = random_layout(rng, rng.randint(2, 7), rng.randint(1, 5), 6)
    nsys = 1 + max(max(b) for b in layout)
    for trial in range(5):
        assert simulate(layout, nsys, levels=6, rule="engine", rng=random.Random(seed * 10 + trial))


@pytest.mark.parametrize("nsys", [2, 3, 4])
def test_homogeneous_layout_never_deadlocks(nsys):
    """Including systems that finish at different iterations (down to one
    live system, whose next phase then publishes first)."""
    layout = [list(range(nsys)) for _ in range(5)]
    for trial in range(20):
        rng = random.Random(trial)
        done_at = [rng.randint(1, 8) for _ in range(nsys)]
        assert simulate(layout, nsys, levels=8, rule="engine", rng=random.Random(trial))
        assert simulate(layout, nsys, levels=8, rule="engine", rng=random.Random(trial), done_at=done_at)


@pytest.mark.parametrize("seed", range(20))
def test_level_rule_with_finished_systems(seed):
    rng = random.Random(1000 + seed)
    layout = random_layout(rng, rng.randint(2, 6), rng.randint(2, 5), 5)
    nsys = 1 + max(max(b) for b in layout)
    done_at = [rng.randint(1, 6) for _ in range(nsys)]
    assert simulate(layout, nsys, levels=6, rule="engine", rng=random.Random(seed), done_at=done_at)


def test_delaying_every_publication_deadlocks_somewhere():
    """Without the rule (always publish after the next preparation), some
    layout and interleaving deadlock: the rule is needed."""
    found = False
    for seed in range(200):
        rng = random.Random(seed)
        layout = random_layout(rng, rng.randint(2, 6), rng.randint(1, 4), 5)
        nsys = 1 + max(max(b) for b in layout)
        if not simulate(layout, nsys, levels=5, rule="always_delay", rng=random.Random(seed)):
            found = True
            break
    assert found


def test_single_system_needs_publish_first():
    """One system per block (noalloc, single right-hand side): its next phase
    waits for its own pending signal."""
    layout = [[0], [0], [0]]
    assert not simulate(layout, 1, levels=3, rule="always_delay", rng=random.Random(1))
    assert simulate(layout, 1, levels=3, rule="engine", rng=random.Random(1))
