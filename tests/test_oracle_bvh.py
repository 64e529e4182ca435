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
