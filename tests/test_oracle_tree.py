"""Pins for the oracle octree (CPU only).

The oracle builds the tree with integer Morton coordinates; these checks use
float geometry of the original points and brute force over all pairs:
  * leaves partition the points, children partition parents, every point lies
    inside the float bounds of its box;
  * the split rule of Sec. 4: leaves hold <= s points; a non-leaf holding
    <= s points was split by the level restriction, so a leaf two or more
    levels finer touches it;
  * the level restriction: touching leaves differ by at most one level;
  * N(B), Q(B) agree with float box distances; the current boxes of a level
    partition the points;
  * colouring: no two boxes of one colour conflict.
"""
import numpy as np
import pytest

import synth
from oracle import tree as otree


def _float_bounds(T, b):
    h = T.side / (1 << b.level)
    lo = T.corner + np.array(b.cell, dtype=np.float64) * h
    return lo, lo + h


def _dist_inf(T, b1, b2):
    lo1, hi1 = _float_bounds(T, b1)
    lo2, hi2 = _float_bounds(T, b2)
    return float(np.max(np.maximum(0.0, np.maximum(lo2 - hi1, lo1 - hi2))))


SURFACES = [
    ("sphere", lambda: synth.sphere_fibonacci(3000), 32),
    ("torus", lambda: synth.torus_graded(4000, seed=5), 24),
    ("ellipsoid", lambda: synth.ellipsoid_graded_tip(3000, seed=6), 32),
]


@pytest.fixture(scope="module", params=SURFACES, ids=[s[0] for s in SURFACES])
def built(request):
    name, mk, ls = request.param
    s = mk()
    return s, otree.build_tree(s.points, ls), ls


def test_partition_and_bounds(built):
    s, T, ls = built
    n = s.n
    leaves = [b for b in T.boxes if b.leaf]
    cover = np.zeros(n, dtype=np.int64)
    for b in leaves:
        cover[b.start:b.end] += 1
    assert np.all(cover == 1)
    assert np.array_equal(np.sort(T.perm), np.arange(n))
    pts = s.points[T.perm]
    tol = 1e-9 * T.side
    for i, b in enumerate(T.boxes):
        lo, hi = _float_bounds(T, b)
        p = pts[b.start:b.end]
        assert np.all(p >= lo - tol) and np.all(p <= hi + tol)
        if b.children:
            ch = [T.boxes[c] for c in b.children]
            assert all(c.parent == i and c.level == b.level + 1 for c in ch)
            assert ch[0].start == b.start and ch[-1].end == b.end
            assert all(ch[j].end == ch[j + 1].start for j in range(len(ch) - 1))


def test_split_rule_and_balance(built):
    s, T, ls = built
    leaves = [b for b in T.boxes if b.leaf]
    tol = 1e-9 * T.side
    for b in leaves:
        assert b.count <= ls or b.level == otree.BITS
    for b in leaves:
        for c in leaves:
            if b is not c and _dist_inf(T, b, c) <= tol:
                assert abs(b.level - c.level) <= 1
    for b in T.boxes:
        if not b.leaf and b.count <= ls:
            assert any(c.level >= b.level + 2 and _dist_inf(T, b, c) <= tol
                       for c in leaves), "split not forced by the level restriction"


def test_lists_and_colouring(built):
    s, T, ls = built
    tol = 1e-9 * T.side
    for lev, L in T.levels.items():
        h = T.side / (1 << lev)
        cov = np.zeros(s.n, dtype=np.int64)
        for C in L.current:
            cov[T.boxes[C].start:T.boxes[C].end] += 1
        assert np.all(cov == 1)
        for B in L.boxes:
            near = [C for C in L.current if C != B and _dist_inf(T, T.boxes[B], T.boxes[C]) <= tol]
            farq = [C for C in L.current if C != B
                    and tol < _dist_inf(T, T.boxes[B], T.boxes[C]) <= h + tol]
            assert sorted(near) == sorted(L.near[B])
            assert sorted(farq) == sorted(L.farq[B])
        for B1 in L.boxes:
            for B2 in L.boxes:
                if B1 < B2 and L.colour[B1] == L.colour[B2]:
                    assert _dist_inf(T, T.boxes[B1], T.boxes[B2]) > h + tol
                    c1 = set(L.near[B1]) | {B1}
                    c2 = set(L.near[B2]) | {B2}
                    assert not (c1 & c2)
        cols = [L.colour[B] for B in L.order]
        assert cols == sorted(cols)


def test_single_box_tree():
    s = synth.sphere_fibonacci(40)
    T = otree.build_tree(s.points, 64)
    assert len(T.boxes) == 1 and T.nlevels == 1 and T.levels == {}
