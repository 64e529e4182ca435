"""Oracle definitions of the LBVH's integer steps (numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper traces rays into a triangle mesh (Sec. III) and notes that its
cost grows with the number of faces; the CUDA path accelerates the nearest
hit query with a linear BVH.  The nearest hit itself is checked against the
brute-force trace; these definitions pin the builder's exact integer
outputs:

* ``morton_codes`` -- 30-bit Morton code (10 bits per axis, x highest) of
  each triangle's bounding-box centre quantised on the centre bounds.  The
  quantisation runs in float32, as in the CUDA builder, so that both sides
  take the same integer decision (the arithmetic is three correctly rounded
  float32 operations, which numpy reproduces exactly).
* ``sorted_order`` -- triangle ids sorted by (code, id).
* ``radix_tree`` -- the binary radix tree over the sorted keys (Karras, HPG
  2012), defined top-down: a range [l, r] splits at the last position whose
  key shares with k_l a longer prefix than k_r does.  Duplicate codes are
  made distinct by appending the sorted position (the 64-bit key
  code << 32 | position).  Internal nodes are numbered by their split
  position gamma, which is unique per internal node; leaves are encoded as
  ~position.
"""
from __future__ import annotations

import numpy as np


def centroids_f32(V: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Bounding-box centre of each triangle, float32: (min + max) * 0.5."""
    V = np.asarray(V, np.float32)
    T = V[np.asarray(F, np.int64)]  # [nt, 3 verts, 3 axes]
    lo = T.min(axis=1)
    hi = T.max(axis=1)
    return ((lo + hi) * np.float32(0.5)).astype(np.float32)


def quantise(c: np.ndarray) -> np.ndarray:
    """10-bit grid coordinate per axis: floor((c - lo) / (hi - lo) * 1024),
    clamped to [0, 1023]; an axis of zero extent maps to 0."""
    c = np.asarray(c, np.float32)
    lo = c.min(axis=0)
    hi = c.max(axis=0)
    ext = (hi - lo).astype(np.float32)
    q = np.zeros(c.shape, np.int64)
    for ax in range(3):
        if ext[ax] > 0:
            u = ((c[:, ax] - lo[ax]).astype(np.float32) / ext[ax]).astype(np.float32)
            u = (u * np.float32(1024.0)).astype(np.float32)
            q[:, ax] = np.clip(np.floor(u), 0, 1023).astype(np.int64)
    return q


def interleave3(q: np.ndarray) -> np.ndarray:
    """Morton interleave, bit-by-bit: bit 3i+2 = x_i, 3i+1 = y_i, 3i = z_i."""
    q = np.asarray(q, np.int64)
    code = np.zeros(q.shape[0], np.int64)
    for i in range(10):
        code |= ((q[:, 0] >> i) & 1) << (3 * i + 2)
        code |= ((q[:, 1] >> i) & 1) << (3 * i + 1)
        code |= ((q[:, 2] >> i) & 1) << (3 * i)
    return code.astype(np.uint32)


def morton_codes(V, F) -> np.ndarray:
    return interleave3(quantise(centroids_f32(V, F)))


def sorted_order(codes: np.ndarray) -> np.ndarray:
    """Triangle ids sorted by (code, id)."""
    return np.argsort(np.asarray(codes, np.uint32), kind="stable").astype(np.int32)


def _clz64(x: int) -> int:
    return 64 - int(x).bit_length()


def radix_tree(sorted_codes: np.ndarray):
    """Binary radix tree over n sorted codes.

    Returns (left, right, rng_l, rng_r, root) with internal node gamma in
    [0, n-2]; children are internal node ids (>= 0) or ~leaf position (< 0).
    For n == 1 the root is the leaf ~0 and the arrays are empty."""
    codes = [int(c) for c in np.asarray(sorted_codes, np.uint64)]
    n = len(codes)
    keys = [(c << 32) | i for i, c in enumerate(codes)]
    left = np.full(max(n - 1, 0), 0, np.int64)
    right = np.full(max(n - 1, 0), 0, np.int64)
    rl = np.full(max(n - 1, 0), -1, np.int64)
    rr = np.full(max(n - 1, 0), -1, np.int64)
    if n == 1:
        return left, right, rl, rr, ~0
    stack = [(0, n - 1)]
    root = None
    while stack:
        l, r = stack.pop()
        g = _node_of(l, r, keys)
        if root is None:
            root = g
        rl[g], rr[g] = l, r
        left[g] = ~g if g == l else _node_of(l, g, keys)
        right[g] = ~(g + 1) if g + 1 == r else _node_of(g + 1, r, keys)
        if g != l:
            stack.append((l, g))
        if g + 1 != r:
            stack.append((g + 1, r))
    return left, right, rl, rr, root


def _node_of(l: int, r: int, keys) -> int:
    """Split position (node id) of the internal node covering [l, r]: the
    last i in [l, r-1] whose key shares with k_l a longer prefix than k_r."""
    dlr = _clz64(keys[l] ^ keys[r])
    g = l
    for i in range(l, r):
        if _clz64(keys[l] ^ keys[i]) > dlr:
            g = i
    return g


def subtree_boxes(V: np.ndarray, F: np.ndarray, order: np.ndarray, left, right, rng_l, rng_r) -> np.ndarray:
    """Child boxes of every internal node of the radix tree, in the node
    layout of the CUDA builder: 12 float32 per node = left (lo.x, hi.x, lo.y,
    hi.y), right (lo.x, hi.x, lo.y, hi.y), left (lo.z, hi.z), right (lo.z,
    hi.z).  A child's box is the componentwise min / max over the vertices of
    the triangles in its range of sorted positions (a leaf: its triangle) --
    the definition of a bounding-volume hierarchy's boxes, whatever order
    they are computed in, and exact in float32.  The tree (left, right,
    rng_l, rng_r from ``radix_tree``) may have been built for other vertex
    positions: this is the box set a refit of that tree must produce."""
    tri = np.asarray(V, np.float32)[np.asarray(F)[np.asarray(order)]]  # [n, 3 vertices, 3]
    tlo, thi = tri.min(axis=1), tri.max(axis=1)
    m = len(left)
    out = np.empty((m, 12), np.float32)

    def box(kid):
        if kid < 0:
            return tlo[~kid], thi[~kid]
        a, b = int(rng_l[kid]), int(rng_r[kid])
        return tlo[a:b + 1].min(axis=0), thi[a:b + 1].max(axis=0)

    for g in range(m):
        (llo, lhi), (rlo, rhi) = box(int(left[g])), box(int(right[g]))
        out[g] = [llo[0], lhi[0], llo[1], lhi[1], rlo[0], rhi[0], rlo[1], rhi[1], llo[2], lhi[2], rlo[2], rhi[2]]
    return out
