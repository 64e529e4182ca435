"""Pins of the oracle's LBVH integer definitions (Morton codes, sorting,
binary radix tree), against published examples and independent methods."""
import json
import os

import numpy as np
import pytest

from oracle import bvh
from paper_2307_15412_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _spread10(v):
    """Independent bit spreading by the multiply-and-mask method: 10-bit v ->
    bits at positions 0, 3, 6, ..."""
    v = np.asarray(v, np.uint64) & np.uint64(0x3FF)
    v = (v * np.uint64(0x00010001)) & np.uint64(0xFF0000FF)
    v = (v * np.uint64(0x00000101)) & np.uint64(0x0F00F00F)
    v = (v * np.uint64(0x00000011)) & np.uint64(0xC30C30C3)
    v = (v * np.uint64(0x00000005)) & np.uint64(0x49249249)
    return v


def test_interleave_known_values():
    q = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1023, 1023, 1023], [0, 0, 0], [5, 3, 6]])
    c = bvh.interleave3(q)
    assert list(c[:5]) == [4, 2, 1, 2 ** 30 - 1, 0]
    # x=101, y=011, z=110 -> bit triples (x y z) from bit 2 down: 101, 011, 110
    assert int(c[5]) == 0b101_011_110


def test_interleave_matches_magic_number_spreading():
    rng = np.random.default_rng(0)
    q = rng.integers(0, 1024, size=(5000, 3))
    ref = (_spread10(q[:, 0]) << np.uint64(2)) | (_spread10(q[:, 1]) << np.uint64(1)) | _spread10(q[:, 2])
    np.testing.assert_array_equal(bvh.interleave3(q).astype(np.uint64), ref)


def test_quantise_extremes_and_degenerate_axis():
    c = np.array([[0.0, 1.0, 5.0], [1.0, 1.0, 5.0], [0.5, 1.0, 5.0]], np.float32)
    q = bvh.quantise(c)
    assert q[0, 0] == 0 and q[1, 0] == 1023 and q[2, 0] == 512
    assert (q[:, 1] == 0).all() and (q[:, 2] == 0).all()


def test_sorted_order_is_code_then_id():
    rng = np.random.default_rng(1)
    codes = rng.integers(0, 50, size=300).astype(np.uint32)
    order = bvh.sorted_order(codes)
    ref = sorted(range(300), key=lambda i: (int(codes[i]), i))
    assert list(order) == ref


def test_radix_tree_karras_fig3():
    g = json.load(open(os.path.join(GOLDEN, "karras2012_fig3.json")))
    left, right, rl, rr, root = bvh.radix_tree(np.array(g["keys"], np.uint32))
    assert root == g["root"]
    assert list(left) == g["left"] and list(right) == g["right"]
    assert list(rl) == g["range_l"] and list(rr) == g["range_r"]


def _check_tree(codes, left, right, rl, rr, root):
    n = len(codes)
    seen_leaf = np.zeros(n, int)
    seen_node = np.zeros(max(n - 1, 0), int)
    stack = [(root, 0, n - 1)]
    while stack:
        node, lo, hi = stack.pop()
        if node < 0:
            assert lo == hi == ~node
            seen_leaf[~node] += 1
            continue
        seen_node[node] += 1
        assert (rl[node], rr[node]) == (lo, hi)
        assert lo <= node < hi
        stack.append((left[node], lo, node))
        stack.append((right[node], node + 1, hi))
    assert (seen_leaf == 1).all() and (seen_node == 1).all()


@pytest.mark.parametrize("n,span", [(2, 4), (3, 1), (17, 8), (200, 1000), (500, 3)])
def test_radix_tree_invariants(n, span):
    rng = np.random.default_rng(n)
    codes = np.sort(rng.integers(0, span, size=n)).astype(np.uint32)
    _check_tree(codes, *bvh.radix_tree(codes))


def test_radix_tree_single_leaf():
    left, right, rl, rr, root = bvh.radix_tree(np.array([42], np.uint32))
    assert root == ~0 and len(left) == 0


def test_hand_codes_and_tree():
    s = I.hand_scene(0, 2000)
    codes = bvh.morton_codes(s.V, s.F)
    assert codes.dtype == np.uint32 and codes.max() < 2 ** 30
    order = bvh.sorted_order(codes)
    sc = codes[order]
    assert (np.diff(sc.astype(np.int64)) >= 0).all()
    _check_tree(sc, *bvh.radix_tree(sc))


def test_subtree_boxes_hand_worked_example():
    """Three triangles, two of them close together: the radix tree pairs the
    two near ones under internal node 0 and the root (node 1) takes that pair
    and the far triangle.  Every box below is worked out by hand from the
    vertex coordinates (the min / max of the triangles under each child)."""
    V = np.array([[0.0, 0.0, 0.0], [0.2, 0.1, 0.0], [0.1, 0.3, 0.2],      # T0
                  [0.3, 0.0, 0.1], [0.4, 0.2, 0.0], [0.2, 0.1, 0.3],      # T1
                  [10.0, 1.0, 2.0], [10.5, 1.5, 2.0], [10.2, 1.2, 2.5]],  # T2
                 np.float32)
    F = np.array([[0, 1, 2], [3, 4, 5], [6, 7, 8]], np.int32)
    codes = bvh.morton_codes(V, F)
    order = bvh.sorted_order(codes)
    assert list(order) == [1, 0, 2]  # T1's centre quantises below T0's
    L, R, rl, rr, root = bvh.radix_tree(codes[order])
    assert root == 1 and list(L) == [~0, 0] and list(R) == [~1, ~2]
    f = np.float32
    T0 = ([0.0, 0.0, 0.0], [0.2, 0.3, 0.2])
    T1 = ([0.2, 0.0, 0.0], [0.4, 0.2, 0.3])
    T2 = ([10.0, 1.0, 2.0], [10.5, 1.5, 2.5])
    T01 = ([0.0, 0.0, 0.0], [0.4, 0.3, 0.3])

    def row(lb, rb):
        (llo, lhi), (rlo, rhi) = lb, rb
        return [llo[0], lhi[0], llo[1], lhi[1], rlo[0], rhi[0], rlo[1], rhi[1], llo[2], lhi[2], rlo[2], rhi[2]]

    want = np.array([row(T1, T0), row(T01, T2)], f)
    got = bvh.subtree_boxes(V, F, order, L, R, rl, rr)
    assert got.dtype == np.float32 and np.array_equal(got, want)


def _union_boxes(V, F, order, L, R, root):
    """The same boxes by a different algorithm: a post-order walk that
    unites the two children's boxes (min / max are exact, so the order of
    the unions cannot change a bit)."""
    tri = np.asarray(V, np.float32)[np.asarray(F)[order]]
    tlo, thi = tri.min(axis=1), tri.max(axis=1)
    out = np.empty((len(L), 12), np.float32)
    memo = {}
    stack = [(root, False)]
    while stack:
        g, done = stack.pop()
        if g < 0:
            memo[g] = (tlo[~g], thi[~g])
            continue
        if not done:
            stack.append((g, True))
            stack.extend([(int(L[g]), False), (int(R[g]), False)])
            continue
        (llo, lhi), (rlo, rhi) = memo[int(L[g])], memo[int(R[g])]
        out[g] = [llo[0], lhi[0], llo[1], lhi[1], rlo[0], rhi[0], rlo[1], rhi[1], llo[2], lhi[2], rlo[2], rhi[2]]
        memo[g] = (np.minimum(llo, rlo), np.maximum(lhi, rhi))
    return out


def test_subtree_boxes_equal_bottom_up_unions_for_a_moved_pose():
    """The tree of one hand pose refit to another pose (same faces): the
    range definition and the bottom-up unions agree bit for bit, and every
    triangle of the new pose lies in all boxes on its root path."""
    a = I.hand_scene(11, 1500)
    b = I.hand_scene(12, 1500)
    assert np.array_equal(a.F, b.F)
    codes = bvh.morton_codes(a.V, a.F)
    order = bvh.sorted_order(codes)
    L, R, rl, rr, root = bvh.radix_tree(codes[order])
    got = bvh.subtree_boxes(b.V, b.F, order, L, R, rl, rr)
    assert np.array_equal(got, _union_boxes(b.V, b.F, order, L, R, root))
    tri = b.V[b.F[order]]
    for g in range(len(L)):
        for side, kid in ((0, L[g]), (1, R[g])):
            a_, z_ = (~kid, ~kid) if kid < 0 else (rl[kid], rr[kid])
            lo = got[g, [4 * side, 4 * side + 2, 8 + 2 * side]]
            hi = got[g, [4 * side + 1, 4 * side + 3, 9 + 2 * side]]
            pts = tri[a_:z_ + 1].reshape(-1, 3)
            assert (pts >= lo).all() and (pts <= hi).all()
