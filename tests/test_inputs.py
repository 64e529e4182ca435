"""Checks of the seeded synthetic input generators (no method arithmetic)."""
import numpy as np
import pytest

from paper_2307_15412_gb300 import inputs as I


@pytest.mark.parametrize("target", [2000, 20000, 5000, 50000])
def test_hand_triangle_count_and_closed(target):
    s = I.hand_scene(1, target)
    nt = s.F.shape[0]
    assert 0.8 * target < nt < 1.3 * target
    e = np.sort(np.concatenate([s.F[:, [0, 1]], s.F[:, [1, 2]], s.F[:, [2, 0]]]), axis=1)
    _, cnt = np.unique(e, axis=0, return_counts=True)
    assert (cnt == 2).all()  # every edge shared by exactly two triangles
    assert s.V.dtype == np.float32 and s.F.dtype == np.int32
    assert s.F.min() >= 0 and s.F.max() < s.V.shape[0]


def test_hand_is_seeded_and_sized():
    a = I.hand_scene(5, 2000)
    b = I.hand_scene(5, 2000)
    c = I.hand_scene(6, 2000)
    assert np.array_equal(a.V, b.V) and not np.array_equal(a.V, c.V)
    ext = a.V.max(0) - a.V.min(0)
    assert 0.03 < ext[0] < 0.2 and 0.05 < ext[1] < 0.2


def test_full_frame_scene_ranges():
    for seed in range(5):
        s = I.hand_scene(seed, 2000, range_m=I.FULL_FRAME_RANGE, speed=I.FULL_FRAME_SPEED)
        assert 0.2 <= s.center[2] <= 0.6
        v = float(np.linalg.norm(s.vel))
        assert v <= 1.0 + 1e-6


def test_random_hits_layout():
    d, a, dd = I.random_hits(0, 100, 3)
    assert d.shape == a.shape == dd.shape == (3, 100)
    assert d.dtype == np.float32
    assert np.abs(d[1] - d[0]).max() <= 2.5e-3 + 1e-7


def test_batched_hand_meshes_equal_single_meshes():
    r = I.surrogate_inputs(3, 5)
    V, F, vel = I.surrogate_scenes(r)
    for i in range(5):
        s = I.surrogate_scene(r[i])
        V1, F1 = I.hand_mesh(I.SURROGATE_TRIANGLES, r[i, :27], r[i, 27:30])
        assert np.array_equal(V[i], V1) and np.array_equal(F, F1)
        assert np.array_equal(s.V, V1) and np.allclose(s.vel, vel[i])


def test_surrogate_features_map_the_box_to_unit_cube():
    lo, hi = I.SURROGATE_LO, I.SURROGATE_HI
    f = I.surrogate_features(np.stack([lo, hi, 0.5 * (lo + hi)]))
    assert np.allclose(f[0], -1) and np.allclose(f[1], 1) and np.allclose(f[2], 0, atol=1e-6)
