"""Pins of the oracle's integer stage: Morton codes (Sec. 3.1), the
cardinality-based cluster tree ((C1)-(C4), Sec. 2.3) and the block cluster
tree of Algorithm 1 under Eq. 5."""
import math

import numpy as np
import pytest

import meshgen


def test_morton_interleave_known_values(orc):
    q = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [2, 0, 0], [3, 3, 3],
                  [2 ** 21 - 1] * 3, [2 ** 20, 0, 0]], dtype=np.uint64)
    want = [4, 2, 1, 32, 63, 2 ** 63 - 1, 2 ** 62]
    assert [int(c) for c in orc.morton_interleave(q)] == want


def test_morton_roundtrip_and_msb_order(orc):
    rng = np.random.default_rng(5)
    q = rng.integers(0, 2 ** 21, size=(2000, 3)).astype(np.uint64)
    code = orc.morton_interleave(q)
    # de-interleave recovers q
    back = np.zeros_like(q)
    for b in range(21):
        for ax, sh in ((0, 2), (1, 1), (2, 0)):
            back[:, ax] |= ((code >> np.uint64(3 * b + sh)) & np.uint64(1)) << np.uint64(b)
    assert np.array_equal(back, q)

    # Z-order: compare two points by the axis holding the most significant
    # differing bit (x before y before z at equal bit position)
    def zless(a, b):
        best, axis = -1, -1
        for ax in range(3):
            x = int(a[ax]) ^ int(b[ax])
            if x:
                msb = x.bit_length() - 1
                # priority x > y > z at the same bit: bit 3b+2 > 3b+1 > 3b
                key = 3 * msb + (2 - ax)
                if key > best:
                    best, axis = key, ax
        return axis >= 0 and int(a[axis]) < int(b[axis])

    for k in range(0, 1998, 2):
        assert zless(q[k], q[k + 1]) == (code[k] < code[k + 1])


def test_morton_quantisation(orc):
    cent = np.array([[0.0, 0.0, 0.0], [1.0, 0.5, 0.25], [0.5, 0.5, 0.5], [0.25, 0.0, 1.0]])
    q = orc.morton_quantise(cent)
    # lo = 0, ext = 1, s = 2^21: exact dyadic values, top clamped
    assert q.tolist() == [[0, 0, 0], [2 ** 21 - 1, 2 ** 20, 2 ** 19], [2 ** 20] * 3, [2 ** 19, 0, 2 ** 21 - 1]]
    # one point: ext = 0 gives code 0
    assert orc.morton_codes(np.array([[0.3, 0.2, 0.1]])).tolist() == [0]


def test_morton_order_stable_on_ties(orc):
    codes = np.array([5, 3, 5, 3, 0], dtype=np.uint64)
    assert orc.morton_order(codes).tolist() == [4, 1, 3, 0, 2]


@pytest.mark.parametrize("n,leaf", [(5120, 64), (1000, 7), (65, 64), (129, 32), (1, 4)])
def test_cluster_tree_conditions(orc, n, leaf):
    cl = orc.cluster_tree(n, leaf)
    by = {(b, e): d for b, e, d in cl}
    assert (0, n, 0) in cl  # (C2)
    for b, e, d in cl:
        assert e > b  # (C1)
        if e - b > leaf:  # (C4): two children, disjoint union, |tau1| = floor(|tau|/2)
            m = b + (e - b) // 2
            assert (b, m) in by and (m, e) in by
        else:  # (C3)
            assert e - b <= leaf
    leaves = sorted((b, e) for b, e, _ in cl if e - b <= leaf)
    assert leaves[0][0] == 0 and leaves[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(leaves, leaves[1:]))


def _box(c, b, e):
    return c[b:e].min(0), c[b:e].max(0)


def _adm_sqrt(c, blk, eta):
    """Eq. 5 with true Euclidean diam / dist (no squares)."""
    rb, re, cb, ce = blk
    (lt, ht), (ls, hs) = _box(c, rb, re), _box(c, cb, ce)
    diam = min(np.linalg.norm(ht - lt), np.linalg.norm(hs - ls))
    gap = np.maximum(0, np.maximum(ls - ht, lt - hs))
    return diam <= eta * np.linalg.norm(gap)


@pytest.mark.parametrize("level,leaf,eta", [(3, 64, 1.5), (3, 16, 1.0), (4, 64, 1.5), (2, 5, 2.0)])
def test_block_tree_is_algorithm1(orc, level, leaf, eta):
    V, T = meshgen.icosphere(level)
    tr = orc.Tree(V, T, leaf, eta)
    n = tr.n
    c = tr.cent_sorted
    cover = np.zeros((n, n), dtype=np.int8)
    for blk in np.concatenate([tr.dense, tr.adm]):
        rb, re, cb, ce = blk
        cover[rb:re, cb:ce] += 1
    assert (cover == 1).all()  # the leaves partition I x I
    clusters = {(b, e) for b, e, _ in orc.cluster_tree(n, leaf)}
    parent = {}
    for b, e, _ in orc.cluster_tree(n, leaf):
        if e - b > leaf:
            m = b + (e - b) // 2
            parent[(b, m)] = (b, e)
            parent[(m, e)] = (b, e)

    def boxes(blk):
        rb, re, cb, ce = blk
        return _box(c, rb, re), _box(c, cb, ce)

    for kind, lst in (("dense", tr.dense), ("adm", tr.adm)):
        for blk in lst:
            rb, re, cb, ce = (int(v) for v in blk)
            assert (rb, re) in clusters and (cb, ce) in clusters
            adm = orc.admissible(*boxes(blk), eta)
            if kind == "adm":
                assert adm and _adm_sqrt(c, blk, eta)
            else:
                assert not adm and (re - rb <= leaf or ce - cb <= leaf)
            # the parent block was subdivided: not admissible, both clusters > leaf
            if (rb, re) != (0, n):
                pr, pc = parent[(rb, re)], parent[(cb, ce)]
                assert pr[1] - pr[0] > leaf and pc[1] - pc[0] > leaf
                assert not orc.admissible(_box(c, *pr), _box(c, *pc), eta)


def test_admissibility_squared_form_matches_definition(orc):
    rng = np.random.default_rng(2)
    for _ in range(2000):
        a = np.sort(rng.uniform(-1, 1, (2, 3)), axis=0)
        b = np.sort(rng.uniform(-1, 1, (2, 3)), axis=0) + rng.uniform(-1.5, 1.5, 3)
        eta = rng.uniform(0.5, 2.0)
        diam = min(np.linalg.norm(a[1] - a[0]), np.linalg.norm(b[1] - b[0]))
        gap = np.maximum(0, np.maximum(b[0] - a[1], a[0] - b[1]))
        dist = np.linalg.norm(gap)
        want = diam <= eta * dist
        if abs(diam - eta * dist) > 1e-12:
            assert orc.admissible((a[0], a[1]), (b[0], b[1]), eta) == want
    # overlapping boxes are never admissible
    assert not orc.admissible((np.zeros(3), np.ones(3)), (np.full(3, 0.5), np.full(3, 2.0)), 10.0)
