"""CPU: pins of the imaging oracle (Sec. II and IV: SFCW MIMO baseband,
brute-force back-projection, maximum projection) against closed forms and
against the pinned single-radar frame."""
import math

import numpy as np
import pytest

import oracle
from oracle import imaging as oim
from paper_2307_15412_gb300 import inputs as I

C = 299_792_458.0


def _point_target(tx, rx, q, f):
    R = np.linalg.norm(q - tx, axis=1)[:, None] + np.linalg.norm(q - rx, axis=1)[None, :]
    return np.exp(-2j * np.pi * R[:, :, None] * f[None, None, :] / C)


def test_backproject_point_target_closed_form():
    """An ideal point scatterer's baseband back-projects to exactly
    n_pairs * n_f at the scatterer (every term's phase cancels) and to a
    smaller magnitude everywhere else."""
    tx, rx = I.mimo_square_array(4, 6e-3)
    n_f = 32
    f = I.IMAGING_F0 + I.IMAGING_DF * np.arange(n_f)
    q = np.array([0.011, -0.017, 0.302])
    s = _point_target(tx, rx, q, f)
    full = tx.shape[0] * rx.shape[0] * n_f
    at_q = oim.backproject(s, tx, rx, I.IMAGING_F0, I.IMAGING_DF, q[None])[0]
    assert abs(at_q - full) <= 1e-9 * full
    rng = np.random.default_rng(4)
    elsewhere = q + rng.uniform(-0.03, 0.03, size=(64, 3))
    assert np.all(np.abs(oim.backproject(s, tx, rx, I.IMAGING_F0, I.IMAGING_DF, elsewhere)) < full * (1 - 1e-6))
    # on a 1 mm grid around the scatterer the peak is the scatterer's voxel
    off = np.stack(np.meshgrid(*([np.arange(-2, 3) * 1e-3] * 3), indexing="ij"), -1).reshape(-1, 3)
    img = np.abs(oim.backproject(s, tx, rx, I.IMAGING_F0, I.IMAGING_DF, q + off))
    assert np.argmax(img) == len(off) // 2


def test_backproject_integer_and_quarter_cycle_phase():
    """One co-located TX/RX, one carrier, a voxel at R0 = 0.3 m (path 0.6 m):
    at f0 = 1000 c / 0.6 the voxel sees s itself; at 1000.25 c / 0.6 the
    phase advances a quarter cycle, so the image is s * (+j)."""
    o = np.zeros((1, 3))
    v = np.array([[0.0, 0.18, 0.24]])  # |v| = 0.3
    s = np.array([[[2.0 + 3.0j]]])
    got = oim.backproject(s, o, o, 1000.0 * C / 0.6, 1.0, v)[0]
    assert abs(got - (2.0 + 3.0j)) < 1e-9
    got = oim.backproject(s, o, o, 1000.25 * C / 0.6, 1.0, v)[0]
    assert abs(got - (-3.0 + 2.0j)) < 1e-9


def test_mimo_rows_equal_single_radar_frames():
    """Each TX-RX row is the pinned single-radar frame of a one-chirp radar
    whose sample n sees f0 + n df (slope * dt = df)."""
    s = I.hand_scene(3, 600, center=(0.0, 0.0, I.IMAGING_RANGE))
    tx, rx = I.mimo_square_array(5, 6e-3)
    grid = I.RayGrid(24, 24, math.radians(20.0), math.radians(20.0))
    n_f = 16
    tx3, rx10 = tx[[0, 4, 7]], rx
    got = oim.mimo_sfcw(s.V, s.F, tx3, rx10, grid, I.IMAGING_F0, I.IMAGING_DF, n_f)
    assert got.shape == (3, 10, n_f)
    for t in range(3):
        for j0 in (0, 8):
            rows = rx10[j0:j0 + 8]
            radar = I.Radar(f0=I.IMAGING_F0, bandwidth=I.IMAGING_DF * n_f, t_chirp=1e-3, n_samples=n_f, n_chirps=1,
                            tx=tuple(tx3[t]), rx=tuple(map(tuple, rows)))
            ref = oracle.frame(s.V, s.F, np.zeros(3), radar, grid)["if_cube"][:, 0, :]
            assert np.linalg.norm(ref) > 0
            assert np.allclose(got[t, j0:j0 + len(rows)], ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_mimo_unit_amplitude_plate_closed_form():
    """A plate facing the array, unit amplitude per hit (Eq. 4 as printed):
    the baseband is the sum over the rays that land on the plate of
    exp(-j 2 pi (f0 + n df) d / c), d = t + |p - rx|, with the rays and
    their hit points computed here from the grid's definition."""
    D = float(np.float32(0.3))
    h = float(np.float32(0.0213))
    V, F = I.plate((0.0, 0.0, D), h, h)
    tx = np.array([[0.01, 0.0, 0.0], [-0.004, 0.012, 0.0]])
    rx = np.array([[-0.02, 0.01, 0.0], [0.0, -0.015, 0.0], [0.03, 0.03, 0.0]])
    grid = I.RayGrid(16, 12, math.radians(10.0), math.radians(8.0))
    n_f = 24
    got = oim.mimo_sfcw(V, F, tx, rx, grid, I.IMAGING_F0, I.IMAGING_DF, n_f, amp_mode=1)
    f = I.IMAGING_F0 + I.IMAGING_DF * np.arange(n_f)
    az = -grid.half_az + 2 * grid.half_az * (np.arange(grid.n_az) + 0.5) / grid.n_az
    el = -grid.half_el + 2 * grid.half_el * (np.arange(grid.n_el) + 0.5) / grid.n_el
    E, A = np.meshgrid(el, az, indexing="ij")
    u = np.stack([np.cos(E) * np.sin(A), np.sin(E), np.cos(E) * np.cos(A)], -1).reshape(-1, 3)
    for t in range(2):
        tt = (D - tx[t, 2]) / u[:, 2]
        p = tx[t] + tt[:, None] * u
        on = (np.abs(p[:, 0]) < h) & (np.abs(p[:, 1]) < h)
        margin = np.minimum(h - np.abs(p[:, 0]), h - np.abs(p[:, 1]))
        assert np.all(np.abs(margin) > 1e-5)  # no ray grazes an edge
        assert 10 < on.sum() < len(on)
        for j in range(3):
            d = tt[on] + np.linalg.norm(p[on] - rx[j], axis=1)
            ref = np.exp(-2j * np.pi * d[:, None] * f[None, :] / C).sum(0)
            assert np.allclose(got[t, j], ref, rtol=0, atol=1e-9 * on.sum())


def test_max_projection_hand_built_volume():
    img = np.zeros((4, 2, 3), np.complex128)
    img[2, 0, 0] = 3 + 4j          # |.| = 5, the image maximum
    img[1, 0, 0] = 4.0
    img[0, 1, 2] = 0.5j            # 0.5: -20 dB, floored at -15
    img[3, 1, 2] = 0.25
    img[3, 0, 1] = -2.5            # 2.5: 20 log10(0.5) = -6.02 dB
    img[:, 1, 0] = 0.0             # all zero: floored, index 0
    img[1, 1, 1] = 5 * 10 ** (-12 / 20.0)
    db, z = oim.max_projection(img, 15.0)
    assert z.tolist() == [[2, 3, 0], [0, 1, 0]]
    want = np.array([[0.0, 20 * math.log10(0.5), -15.0], [-15.0, -12.0, -15.0]])
    assert np.allclose(db, want, atol=1e-12)
