"""Level-restricted adaptive octree, near/far lists and colouring (oracle).

Test infrastructure: used only by tests, the smoke check and the benchmark's
CPU baseline.

Follows Sec. 4 (preamble) and Sec. 4.3:
  * the root cube C is level 0; a box at level l is split into its eight
    children (empty children dropped) while it holds more than s points;
  * level restriction: two leaves that share a boundary point (faces, edges and
    corners) differ by at most one level; a coarser leaf that violates it is
    split, repeated until nothing changes (the minimal balanced refinement);
  * near field N(B): other current boxes that touch B (same level, and coarser
    leaves -- Fig. adaptive); far field F: the rest;
  * Q(B): current far boxes that lie within one box side h_l of B (see the
    reading below); P = F minus Q.

Readings where the paper is silent or does not carry over to 3-D:
  * Cube: centre of the bounding box, side = max extent * (1 + 1e-12).
    Integer coordinates q = floor((x - corner)/side * 2^21) clipped to
    [0, 2^21 - 1]; child intervals are half-open, a point on a midpoint goes to
    the upper child. Depth cap 21.
  * "Current" boxes while level l is processed: all boxes of level l plus all
    leaves of coarser levels; they partition the points.
  * Q(B) = current boxes C with 0 < gap(B, C) <= h_l, gap being the
    max-norm distance between the closed boxes. The paper's sphere of radius
    5R/2 around B misses the eight corner boxes at offset (2,2,2), whose
    nearest point lies 1.5*sqrt(3) R ~ 2.6 R away, although a box touching both
    (offset (1,1,1)) updates their block with B by a Schur complement. The ring
    rule contains the 5R/2 ball and every pair the Schur updates of this level
    can create, so A_PB stays pure kernel as Sec. 4.3 requires.
  * Order inside a level: colour-major, then Morton. Two boxes of a level
    conflict when gap(B1,B2) <= h_l or their closed neighbourhoods {B}+N(B)
    share a box; colours are greedy in Morton order (smallest colour unused by
    earlier conflicting boxes). Boxes of one colour touch disjoint sets of
    blocks and see none of each other's actives in N or Q, so the colour-major
    order gives the same arithmetic as any order within a colour.

Pins (tests/test_oracle_tree.py): every point in exactly one leaf, leaf counts,
children partition parents, the split rule, the 2:1 balance checked over all
leaf pairs with float box bounds, N/Q lists against float geometry, colour
validity over all pairs.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BITS = 21
ONE = 1 << BITS


def bounding_cube(points: np.ndarray):
    lo = points.min(axis=0)
    hi = points.max(axis=0)
    center = (lo + hi) / 2.0
    extent = float((hi - lo).max())
    side = extent * (1.0 + 1e-12)
    if not side > 0.0:
        side = 1.0
    corner = center - side / 2.0
    return corner, side


def int_coords(points: np.ndarray, corner: np.ndarray, side: float) -> np.ndarray:
    q = np.floor((points - corner[None, :]) / side * float(ONE))
    return np.clip(q, 0, ONE - 1).astype(np.int64)


def morton(q: np.ndarray) -> np.ndarray:
    """Interleave 21-bit x, y, z: bit 3b <- x_b, 3b+1 <- y_b, 3b+2 <- z_b."""
    key = np.zeros(q.shape[0], dtype=np.int64)
    for b in range(BITS):
        for c in range(3):
            key |= ((q[:, c] >> b) & 1) << (3 * b + c)
    return key


def morton3(cx: int, cy: int, cz: int) -> int:
    key = 0
    for b in range(BITS):
        key |= ((cx >> b) & 1) << (3 * b)
        key |= ((cy >> b) & 1) << (3 * b + 1)
        key |= ((cz >> b) & 1) << (3 * b + 2)
    return key


@dataclass
class Box:
    level: int
    cell: tuple
    start: int
    end: int
    parent: int = -1
    children: list = field(default_factory=list)

    @property
    def count(self):
        return self.end - self.start

    @property
    def leaf(self):
        return not self.children

    def bounds(self):
        """Closed integer bounds [lo, hi] per axis at the finest resolution."""
        sh = BITS - self.level
        lo = np.array(self.cell, dtype=np.int64) << sh
        return lo, lo + (1 << sh)


def gap(b1: Box, b2: Box) -> int:
    """Max-norm distance between two closed boxes (0 when they touch)."""
    lo1, hi1 = b1.bounds()
    lo2, hi2 = b2.bounds()
    g = np.maximum(0, np.maximum(lo2 - hi1, lo1 - hi2))
    return int(g.max())


@dataclass
class Tree:
    perm: np.ndarray            # sorted position -> original index
    corner: np.ndarray
    side: float
    keys: np.ndarray            # sorted Morton keys
    boxes: list                 # Box, ids ordered by (level, Morton)
    nlevels: int                # deepest level + 1
    leaf_size: int
    levels: dict                # level -> LevelLists (levels >= 2)

    def h(self, level: int) -> int:
        return 1 << (BITS - level)


@dataclass
class LevelLists:
    level: int
    boxes: list                 # level-l box ids, Morton order
    current: list               # current box ids ordered by point start
    near: dict                  # B -> list of current box ids (touching, != B)
    farq: dict                  # B -> list of current box ids (0 < gap <= h)
    colour: dict                # B -> colour
    order: list                 # elimination order: (colour, Morton)


def _split(box: Box, keys: np.ndarray) -> list:
    l = box.level
    sh = 3 * (BITS - l - 1)
    codes = (keys[box.start:box.end] >> sh) & 7
    cuts = np.flatnonzero(np.diff(codes)) + 1
    starts = np.concatenate([[0], cuts])
    ends = np.concatenate([cuts, [codes.size]])
    kids = []
    for s0, e0 in zip(starts, ends):
        c = int(codes[s0])
        cell = (2 * box.cell[0] + (c & 1), 2 * box.cell[1] + ((c >> 1) & 1),
                2 * box.cell[2] + ((c >> 2) & 1))
        kids.append(Box(l + 1, cell, box.start + int(s0), box.start + int(e0)))
    return kids


def build_tree(points: np.ndarray, leaf_size: int = 64) -> Tree:
    points = np.asarray(points, dtype=np.float64)
    corner, side = bounding_cube(points)
    q = int_coords(points, corner, side)
    keys_all = morton(q)
    perm = np.argsort(keys_all, kind="stable")
    keys = keys_all[perm]
    n = points.shape[0]

    # ---- subdivision while count > s (Sec. 4 preamble) --------------------
    nodes = [Box(0, (0, 0, 0), 0, n)]
    work = [0]
    while work:
        i = work.pop()
        b = nodes[i]
        if b.count > leaf_size and b.level < BITS:
            for kid in _split(b, keys):
                kid.parent = i
                nodes.append(kid)
                b.children.append(len(nodes) - 1)
                work.append(len(nodes) - 1)

    # ---- level restriction: split coarse leaves touching leaves 2+ finer --
    while True:
        leaves = [i for i, b in enumerate(nodes) if b.leaf]
        lo = np.array([nodes[i].bounds()[0] for i in leaves])
        hi = np.array([nodes[i].bounds()[1] for i in leaves])
        lev = np.array([nodes[i].level for i in leaves])
        touch = np.all((lo[:, None, :] <= hi[None, :, :])
                       & (lo[None, :, :] <= hi[:, None, :]), axis=2)
        finer = lev[None, :] >= lev[:, None] + 2
        need = np.any(touch & finer, axis=1)
        todo = [leaves[j] for j in np.flatnonzero(need) if nodes[leaves[j]].level < BITS]
        if not todo:
            break
        for i in todo:
            b = nodes[i]
            for kid in _split(b, keys):
                kid.parent = i
                nodes.append(kid)
                b.children.append(len(nodes) - 1)

    # ---- canonical ids: (level, Morton) ------------------------------------
    sort_key = [(b.level, morton3(*b.cell)) for b in nodes]
    order = sorted(range(len(nodes)), key=lambda i: sort_key[i])
    remap = {old: new for new, old in enumerate(order)}
    boxes = []
    for old in order:
        b = nodes[old]
        nb = Box(b.level, b.cell, b.start, b.end,
                 remap[b.parent] if b.parent >= 0 else -1,
                 sorted(remap[c] for c in b.children))
        boxes.append(nb)
    nlevels = max(b.level for b in boxes) + 1
    tree = Tree(perm=perm, corner=corner, side=side, keys=keys, boxes=boxes,
                nlevels=nlevels, leaf_size=leaf_size, levels={})
    for lev_ in range(2, nlevels):
        tree.levels[lev_] = level_lists(tree, lev_)
    return tree


def current_boxes(tree: Tree, level: int) -> list:
    cur = [i for i, b in enumerate(tree.boxes)
           if b.level == level or (b.leaf and b.level < level)]
    return sorted(cur, key=lambda i: tree.boxes[i].start)


def _bounds_arrays(bx, ids):
    lo = np.array([bx[i].bounds()[0] for i in ids], dtype=np.int64).reshape(-1, 3)
    hi = np.array([bx[i].bounds()[1] for i in ids], dtype=np.int64).reshape(-1, 3)
    return lo, hi


def gap_matrix(bx, rows, cols) -> np.ndarray:
    """gap(rows[i], cols[j]) for all pairs (max-norm distance, 0 = touching)."""
    lo1, hi1 = _bounds_arrays(bx, rows)
    lo2, hi2 = _bounds_arrays(bx, cols)
    g = np.maximum(0, np.maximum(lo2[None, :, :] - hi1[:, None, :],
                                 lo1[:, None, :] - hi2[None, :, :]))
    return g.max(axis=2)


def level_lists(tree: Tree, level: int) -> LevelLists:
    bx = tree.boxes
    h = tree.h(level)
    mine = [i for i, b in enumerate(bx) if b.level == level]
    cur = current_boxes(tree, level)
    g = gap_matrix(bx, mine, cur)
    cur_arr = np.array(cur)
    near, farq = {}, {}
    for r, B in enumerate(mine):
        self_mask = cur_arr == B
        near[B] = [int(c) for c in cur_arr[(g[r] == 0) & ~self_mask]]
        farq[B] = [int(c) for c in cur_arr[(g[r] > 0) & (g[r] <= h)]]
    # closed neighbourhoods as a boolean (mine x cur) matrix; B touches itself
    closed = (g == 0).astype(np.int64)
    share = (closed @ closed.T) > 0
    gm = gap_matrix(bx, mine, mine)
    conflict = share | (gm <= h)
    colour = {}
    cols = np.full(len(mine), -1, dtype=np.int64)
    for idx, B in enumerate(mine):
        used = set(cols[:idx][conflict[idx, :idx]].tolist())
        c = 0
        while c in used:
            c += 1
        cols[idx] = c
        colour[B] = c
    pos = {B: i for i, B in enumerate(mine)}
    order = sorted(mine, key=lambda B: (colour[B], pos[B]))
    return LevelLists(level, mine, cur, near, farq, colour, order)
