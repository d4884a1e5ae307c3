"""Monotone Scene Generation tree search over the oracle (Sec. III, Fig. 2;
variant 2.0-B of Sec. VI-A).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the reference for
the library's tree search.  Level l of the tree places one more object; an
edge's cost is the oracle's score_tree of that object at one of its poses
against the parent state (refused edges are dropped).  A goal is a state with
every object placed; the task is the goal with the lowest path cost.

beam_search keeps, at every level, the `beam` cheapest children of the
current states, ordered by (path cost, parent rank, object, pose index);
exhaustive enumerates every order and pose choice (tiny cases only).  With a
beam at least as wide as a level, the two agree.
"""
from __future__ import annotations

import itertools

from . import oracle as O


def beam_search(scene, objects, beam):
    """objects: list of (OracleMesh, label, roi, poses (n,12)).  Returns
    (order, pose_index, level_cost) of the best goal, or None when every path
    is refused."""
    K = len(objects)
    states = [(0, (), (), (), O.empty_state(scene))]    # (g, order, poses, level costs, images)
    for _ in range(K):
        cands = []
        for b, (g, order, pidx, lc, img) in enumerate(states):
            for j in range(K):
                if j in order:
                    continue
                mesh, label, roi, poses = objects[j]
                costs, _ = O.score_tree(scene, mesh, poses, img, label=label, roi=roi)
                for h in range(len(poses)):
                    if costs[h, 0] >= 0:
                        cands.append((g + int(costs[h, 0]) + int(costs[h, 1]), b, j, h))
        if not cands:
            return None
        cands.sort()
        nxt = []
        for (c, b, j, h) in cands[:beam]:
            g, order, pidx, lc, img = states[b]
            mesh, label, roi, poses = objects[j]
            _, _, child = O.score_tree(scene, mesh, poses[h:h + 1], img, label=label, roi=roi, child=True)
            nxt.append((c, order + (j,), pidx + (h,), lc + (c,), child))
        states = nxt
    g, order, pidx, lc, _ = states[0]
    return list(order), list(pidx), list(lc)


def exhaustive(scene, objects):
    """Lowest path cost over every order and pose choice: (cost, order, pose_index)."""
    K = len(objects)
    best = None
    for order in itertools.permutations(range(K)):
        def rec(level, img, g, pidx):
            nonlocal best
            if level == K:
                cand = (g, list(order), list(pidx))
                if best is None or cand[0] < best[0]:
                    best = cand
                return
            mesh, label, roi, poses = objects[order[level]]
            costs, _ = O.score_tree(scene, mesh, poses, img, label=label, roi=roi)
            for h in range(len(poses)):
                if costs[h, 0] < 0:
                    continue
                _, _, child = O.score_tree(scene, mesh, poses[h:h + 1], img, label=label, roi=roi,
                                           child=True)
                rec(level + 1, child, g + int(costs[h, 0]) + int(costs[h, 1]), pidx + [h])
        rec(0, O.empty_state(scene), 0, [])
    return best
