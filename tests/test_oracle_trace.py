"""Pins of the oracle's ray generation and brute-force closest-hit trace.

Checked against closed forms that do not reuse the oracle's formulas:
plate and sphere hit sets, exact axis-permuting rotations, duplicated
triangles (lowest id wins), rays through shared edges and vertices
(watertightness) and hand-computed single-triangle cases."""
import math

import numpy as np
import pytest

import oracle
from paper_2307_15412_gb300 import inputs as I


def test_ray_dirs_grid_closed_form():
    g = I.RayGrid(4, 2, math.radians(40.0), math.radians(10.0))
    dirs, omega = oracle.ray_dirs(g)
    # unit vectors
    assert np.allclose(np.linalg.norm(dirs, axis=1), 1.0, atol=1e-15)
    # ray id = i_el * n_az + i_az; cell centres: az = -40 + 20*(i+0.5)
    az = np.radians(-40.0 + 20.0 * (np.arange(4) + 0.5))
    el = np.radians(-10.0 + 10.0 * (np.arange(2) + 0.5))
    for j in range(2):
        for i in range(4):
            u = dirs[j * 4 + i]
            assert math.isclose(math.atan2(u[0], u[2]), az[i], abs_tol=1e-14)
            assert math.isclose(math.asin(u[1]), el[j], abs_tol=1e-14)
    # solid angles add up to the integral of cos(el) over the field of view
    # only in the limit; for the 2x2 el cells check the per-cell formula's total
    exact = 2 * math.radians(40.0) * (math.sin(math.radians(10)) - math.sin(math.radians(-10)))
    assert abs(omega.sum() - exact) / exact < 2e-3
    # a fine grid converges to the exact solid angle of the field of view
    gf = I.RayGrid(256, 256, math.radians(30.0), math.radians(30.0))
    _, om = oracle.ray_dirs(gf)
    exact = 2 * math.radians(30.0) * 2 * math.sin(math.radians(30.0))
    assert abs(om.sum() - exact) / exact < 1e-5


def test_ray_dirs_frame_rotation():
    g = I.RayGrid(5, 3, 0.3, 0.2)
    R = np.array([[0, 0, 1], [0, 1, 0], [-1, 0, 0]], np.float64)  # boresight +z -> -x
    d0, _ = oracle.ray_dirs(g)
    d1, _ = oracle.ray_dirs(g, R.reshape(-1))
    assert np.allclose(d1, d0 @ R.T, atol=1e-15)


def _single(V, F, d, o=(0.0, 0.0, 0.0)):
    tri, t = oracle.trace(np.asarray(V, np.float32), np.asarray(F, np.int32), np.asarray(o, float),
                          np.asarray(d, float).reshape(-1, 3))
    return int(tri[0]), float(t[0])


def test_single_triangle_hand_computed():
    V = [(-1, -1, 2), (1, -1, 2), (0, 1, 2)]
    F = [(0, 1, 2)]
    assert _single(V, F, (0, 0, 1)) == (0, 2.0)
    # direction (0.6, 0, 0.8): plane z=2 at t=2.5, point x=1.5 -> outside (|x| <= 0.5 at y=0)
    assert _single(V, F, (0.6, 0, 0.8))[0] == -1
    # direction (0.2, 0, sqrt(0.96)): x = 2*0.2/0.9798 = 0.408 -> inside
    tri, t = _single(V, F, (0.2, 0, math.sqrt(0.96)))
    assert tri == 0 and math.isclose(t, 2.0 / math.sqrt(0.96), rel_tol=1e-14)
    # behind the origin: miss (t > 0 strictly)
    assert _single(V, F, (0, 0, -1))[0] == -1
    # origin on the plane: t = 0 is not a hit
    assert _single(V, F, (0, 0, 1), o=(0, 0, 2))[0] == -1
    # back face is hit too (two-sided)
    assert _single([(-1, -1, 2), (0, 1, 2), (1, -1, 2)], F, (0, 0, 1)) == (0, 2.0)


def test_lowest_id_wins_on_equal_t():
    V = [(-1, -1, 1), (1, -1, 1), (0, 1, 1)]
    F = [(0, 1, 2), (2, 0, 1), (1, 2, 0)]
    assert _single(V, F, (0, 0, 1)) == (0, 1.0)
    # a nearer triangle with a higher id still wins
    V2 = V + [(-1, -1, 0.5), (1, -1, 0.5), (0, 1, 0.5)]
    F2 = F + [(3, 4, 5)]
    assert _single(V2, F2, (0, 0, 1)) == (3, 0.5)


def test_watertight_shared_edge_and_vertex():
    # fan of 6 triangles around (0, 0, 1): a ray through the shared vertex and
    # rays through each shared edge must hit
    c = (0.0, 0.0, 1.0)
    ring = [(math.cos(2 * math.pi * k / 6), math.sin(2 * math.pi * k / 6), 1.0) for k in range(6)]
    V = [c] + ring
    F = [(0, 1 + k, 1 + (k + 1) % 6) for k in range(6)]
    tri, t = _single(V, F, (0, 0, 1))
    assert tri >= 0 and t == 1.0
    Vf = np.asarray(V, np.float32)
    for k in range(6):
        p = 0.5 * Vf[1 + k].astype(np.float64) + 0.5 * Vf[0].astype(np.float64)
        tri, t = _single(V, F, p / np.linalg.norm(p))
        assert tri >= 0, k
        assert math.isclose(t, np.linalg.norm(p), rel_tol=1e-12)


def test_plate_hit_set_closed_form():
    D, hx, hy = 0.3, 0.05, 0.03
    V, F = I.plate((0.0, 0.0, D), hx, hy, nx=8, ny=6)
    D = float(V[0, 2])  # the plane sits at float32(0.3)
    g = I.RayGrid(64, 64, math.radians(20.0), math.radians(20.0))
    dirs, _ = oracle.ray_dirs(g)
    tri, t = oracle.trace(V, F, np.zeros(3), dirs)
    x = D * dirs[:, 0] / dirs[:, 2]
    y = D * dirs[:, 1] / dirs[:, 2]
    inside = (np.abs(x) < hx) & (np.abs(y) < hy)
    edge = (np.abs(np.abs(x) - hx) < 1e-9) | (np.abs(np.abs(y) - hy) < 1e-9)
    assert not edge.any()
    assert np.array_equal(tri >= 0, inside)
    assert inside.sum() > 100
    np.testing.assert_allclose(t[inside], D / dirs[inside, 2], rtol=1e-13)


def test_sphere_hit_set_and_depth_bounds():
    D, r = 0.3, 0.05
    V, F = I.icosphere((0.0, 0.0, D), r, subdiv=3)
    Vd = V.astype(np.float64) - np.array([0, 0, D])
    tri_v = Vd[F]
    n = np.cross(tri_v[:, 1] - tri_v[:, 0], tri_v[:, 2] - tri_v[:, 0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    r_in = np.abs(np.einsum("ij,ij->i", n, tri_v[:, 0])).min()
    r_out = np.linalg.norm(Vd, axis=1).max()
    g = I.RayGrid(96, 96, math.radians(12.0), math.radians(12.0))
    dirs, _ = oracle.ray_dirs(g)
    tri, t = oracle.trace(V, F, np.zeros(3), dirs)
    ang = np.arccos(np.clip(dirs[:, 2], -1, 1))
    must_hit = ang < math.asin(r_in / D) - 1e-9
    must_miss = ang > math.asin(r_out / D) + 1e-9
    assert must_hit.sum() > 500 and must_miss.sum() > 500
    assert (tri[must_hit] >= 0).all()
    assert (tri[must_miss] < 0).all()
    # the polyhedron lies between the inscribed and circumscribed spheres
    b = D * np.cos(ang[must_hit])
    t_out = b - np.sqrt(r_out ** 2 - (D * np.sin(ang[must_hit])) ** 2)
    t_in = b - np.sqrt(r_in ** 2 - (D * np.sin(ang[must_hit])) ** 2)
    th = t[must_hit]
    assert (th >= t_out - 1e-12).all() and (th <= t_in + 1e-12).all()


def test_rigid_rotation_invariance_exact():
    """A 90-degree rotation permutes float32 coordinates exactly, so rotating
    scene and radar frame together must give identical ids and equal t."""
    s = I.hand_scene(3, 600)
    R = np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]], np.float64)  # axis cycle
    g = I.RayGrid(48, 48, math.radians(30.0), math.radians(30.0))
    d0, _ = oracle.ray_dirs(g)
    d1, _ = oracle.ray_dirs(g, R.reshape(-1))
    V1 = (s.V.astype(np.float64) @ R.T).astype(np.float32)
    tri0, t0 = oracle.trace(s.V, s.F, np.zeros(3), d0)
    tri1, t1 = oracle.trace(V1, s.F, np.zeros(3), d1)
    assert (tri0 >= 0).sum() > 50
    assert np.array_equal(tri0, tri1)
    np.testing.assert_allclose(t1, t0, rtol=1e-12)


def test_rigid_rotation_invariance_generic():
    """A generic rotation re-rounds the float32 vertices, so ids may differ
    only on rays within rounding distance of an edge."""
    s = I.hand_scene(4, 600)
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    g = I.RayGrid(48, 48, math.radians(30.0), math.radians(30.0))
    d0, _ = oracle.ray_dirs(g)
    d1, _ = oracle.ray_dirs(g, Q.reshape(-1))
    V1 = (s.V.astype(np.float64) @ Q.T).astype(np.float32)
    tri0, t0 = oracle.trace(s.V, s.F, np.zeros(3), d0)
    tri1, t1 = oracle.trace(V1, s.F, np.zeros(3), d1)
    same = tri0 == tri1
    assert same.mean() >= 0.999
    hit = same & (tri0 >= 0)
    np.testing.assert_allclose(t1[hit], t0[hit], rtol=1e-5)


def test_hand_is_hit_near_expected_range():
    radar, grid, nt = I.workload_tiny()
    s = I.hand_scene(0, nt)
    r = oracle.frame(s.V, s.F, s.vel, radar, grid)
    th = r["t"][r["tri"] >= 0]
    assert 100 < len(th) < 2000
    # the hand spans about 0.2 - 0.32 m in front of the radar
    assert th.min() > 0.19 and th.max() < 0.34
