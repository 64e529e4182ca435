"""Pins of the oracle's per-triangle casting (rays cast to each mesh
triangle, Sec. III) and of the alpha mixing (Eq. 3), against closed forms
that do not reuse the oracle's formulas:

* the sample layout: k^2 distinct points inside the triangle whose mean is
  its centroid (the sub-triangles' centroids average to the centroid);
* visibility on a convex sphere: a sample is received iff its face turns
  toward the TX;
* visibility behind a plate: a sample on a farther plate is hidden iff its
  central projection from the TX onto the near plate falls inside it;
* solid angle: the samples of a finely tessellated plate facing the radar
  add up to the rectangle's exact solid angle 4 asin(ab / sqrt((a^2 + D^2)
  (b^2 + D^2))) within the midpoint rule's O(h^2);
* alpha: the IF is the exact linear blend of the alpha = 0 and alpha = 1
  cubes (amplitudes mix linearly, paths do not depend on alpha).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2307_15412_gb300 import inputs as I


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_sample_layout(k):
    V = np.array([[0.0, 0.0, 0.5], [0.03, 0.0, 0.5], [0.01, 0.02, 0.5]], np.float32)
    F = np.array([[0, 1, 2]], np.int32)
    P, tid, samp = oracle.triangle_samples(V, F, k)
    assert P.shape == (k * k, 3) and (tid == 0).all() and list(samp) == list(range(k * k))
    assert len({tuple(np.round(p, 15)) for p in P}) == k * k
    c = V.astype(np.float64).mean(axis=0)
    assert np.allclose(P.mean(axis=0), c, atol=1e-15)
    # strictly inside: barycentric coordinates in (0, 1)
    A = np.stack([V[1] - V[0], V[2] - V[0]], 1).astype(np.float64)[:2]
    bc = np.linalg.solve(A, (P[:, :2] - V[0, :2]).T).T
    assert (bc > 0).all() and (bc.sum(axis=1) < 1).all()


def _radar():
    return I.Radar(n_samples=64, n_chirps=4, rx=I.rx_l_array())


def test_convex_sphere_visible_iff_front_facing():
    V, F = I.icosphere((0.01, -0.02, 0.4), 0.05, subdiv=2)
    r = _radar()
    k = 2
    out = oracle.triangle_frame(V, F, np.zeros(3), r, k)
    P, tid, _ = oracle.triangle_samples(V, F, k)
    V64 = V.astype(np.float64)
    n = np.cross(V64[F[:, 1]] - V64[F[:, 0]], V64[F[:, 2]] - V64[F[:, 0]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    to_tx = np.asarray(r.tx) - P
    cos = (n[tid] * to_tx).sum(axis=1) / np.linalg.norm(to_tx, axis=1)
    outward = (n[tid] * (P - np.array([0.01, -0.02, 0.4]))).sum(axis=1) > 0
    front = np.where(outward, cos, -cos) > 0
    clear = np.abs(cos) > 1e-3   # grazing faces excluded
    assert (out["visible"][clear] == front[clear]).all()
    assert front.sum() > 100 and (~front).sum() > 100


def test_plate_shadow_closed_form():
    Vn, Fn = I.plate((0.0, 0.0, 0.30), 0.012, 0.012, 3, 3)
    Vf, Ff = I.plate((0.0, 0.0, 0.50), 0.05, 0.05, 10, 10)
    V = np.concatenate([Vn, Vf]).astype(np.float32)
    F = np.concatenate([Fn, Ff + len(Vn)]).astype(np.int32)
    r = _radar()
    k = 3
    out = oracle.triangle_frame(V, F, np.zeros(3), r, k)
    P, tid, _ = oracle.triangle_samples(V, F, k)
    far = tid >= len(Fn)
    scale = 0.30 / 0.50
    proj = P[:, :2] * scale
    hidden = far & (np.abs(proj[:, 0]) < 0.012) & (np.abs(proj[:, 1]) < 0.012)
    margin = np.minimum(np.abs(np.abs(proj[:, 0]) - 0.012), np.abs(np.abs(proj[:, 1]) - 0.012))
    clear = margin > 1e-6
    assert (out["visible"][clear] == ~hidden[clear]).all()
    assert hidden.sum() > 20 and (far & ~hidden).sum() > 1000
    assert out["visible"][~far].all()


def test_plate_solid_angle_closed_form():
    a, b, D = 0.02, 0.015, 0.4
    V, F = I.plate((0.0, 0.0, D), a, b, 24, 18)
    out = oracle.triangle_frame(V, F, np.zeros(3), _radar(), 4)
    exact = 4.0 * math.asin(a * b / math.sqrt((a * a + D * D) * (b * b + D * D)))
    assert out["visible"].all()
    assert abs(out["omega"].sum() - exact) <= 1e-6 * exact


def test_alpha_mix_is_linear():
    s = I.hand_scene(3, 800)
    r = _radar()
    cubes = {}
    for al in (0.0, 0.3, 1.0):
        r.alpha = al
        cubes[al] = oracle.triangle_frame(s.V, s.F, s.vel, r, 2)["if_cube"]
    blend = cubes[0.0] + 0.3 * (cubes[1.0] - cubes[0.0])
    assert np.linalg.norm(cubes[0.3] - blend) <= 1e-12 * np.linalg.norm(cubes[0.3])
    assert np.linalg.norm(cubes[1.0] - cubes[0.0]) > 1e-3 * np.linalg.norm(cubes[0.0])
