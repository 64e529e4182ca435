"""Pins of the oracle's echo model, IF synthesis and range-Doppler map.

Each check rests on geometry or signal theory rather than on the oracle's
own formulas: normal-incidence and tilted-plate lobes, reciprocity of the
two legs, the FMCW beat frequency f_b = S d / c landing in range bin
B d / c, the Doppler bin f0 d-dot T_rep M / c, the carrier phase of the
peak, range migration across chirps, linearity, numpy's FFT and Parseval."""
import math

import numpy as np
import pytest

import oracle
from paper_2307_15412_gb300 import inputs as I

C = I.C_LIGHT


def _echo_one(p, n_hint_tri, origin, rx, alpha=0.5, m_s=8.0, vel=(0, 0, 0), omega=1.0, amp_mode=0):
    """Echo of a hit at point p on the triangle n_hint_tri, ray from origin."""
    V = np.asarray(n_hint_tri, np.float32)
    F = np.array([[0, 1, 2]], np.int32)
    o = np.asarray(origin, np.float64)
    u = np.asarray(p, np.float64) - o
    t = np.linalg.norm(u)
    u = u / t
    radar = I.Radar(rx=tuple(tuple(map(float, r)) for r in rx), alpha=alpha, spec_exp=m_s, amp_mode=amp_mode)
    d, a, dd = oracle.echo(V, F, o, u[None], np.array([t]), np.array([0], np.int32), np.array([omega]),
                           radar, np.asarray(vel, np.float64))
    return d[:, 0], a[:, 0], dd[:, 0]


def _plate_tri(D, tilt_deg):
    """Large triangle through (0, 0, D) whose normal is tilted by tilt_deg about y."""
    th = math.radians(tilt_deg)
    e1 = np.array([math.cos(th), 0.0, math.sin(th)])
    e2 = np.array([0.0, 1.0, 0.0])
    c = np.array([0.0, 0.0, D])
    return [c - 2 * e1 - 2 * e2, c + 2 * e1 - 2 * e2, c + 2 * e2]


def test_echo_normal_incidence_monostatic():
    D = 0.5
    tri = _plate_tri(D, 0.0)
    for alpha in (0.0, 0.5, 1.0):
        d, a, dd = _echo_one((0, 0, D), tri, (0, 0, 0), [(0, 0, 0)], alpha=alpha, omega=2e-5,
                             vel=(0, 0, 0.7))
        # mirror direction points straight back and both cosines are 1: g = 1
        assert math.isclose(d[0], 2 * D, rel_tol=1e-15)
        assert math.isclose(a[0], 2e-5 / (D * D), rel_tol=1e-12)
        # receding along the ray on both legs
        assert math.isclose(dd[0], 2 * 0.7, rel_tol=1e-12)


@pytest.mark.parametrize("tilt", [10.0, 25.0, 40.0, 50.0])
def test_echo_tilted_plate_lobes(tilt):
    """Monostatic radar, plate tilted by theta: incidence and exit cosines are
    cos(theta); the mirror ray leaves at 2 theta from the way back."""
    D = 0.4
    tri = _plate_tri(D, tilt)
    th = math.radians(tilt)
    # the triangle's vertices are rounded to float32, which tilts the face by
    # ~1e-7 rad: compare to 1e-6
    _, a_d, _ = _echo_one((0, 0, D), tri, (0, 0, 0), [(0, 0, 0)], alpha=1.0)
    assert math.isclose(a_d[0] * D * D, math.cos(th) ** 2, rel_tol=1e-6)
    _, a_s, _ = _echo_one((0, 0, D), tri, (0, 0, 0), [(0, 0, 0)], alpha=0.0, m_s=8.0)
    expect = max(0.0, math.cos(2 * th)) ** 8
    assert math.isclose(a_s[0] * D * D, expect, rel_tol=1e-5, abs_tol=1e-12)
    _, a_m, _ = _echo_one((0, 0, D), tri, (0, 0, 0), [(0, 0, 0)], alpha=0.3, m_s=8.0)
    assert math.isclose(a_m[0], 0.7 * a_s[0] + 0.3 * a_d[0], rel_tol=1e-12)


def test_echo_reciprocity():
    """Swapping the transmit and receive antennas leaves path, amplitude and
    path rate unchanged."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        tri = [rng.uniform(-0.1, 0.1, 3) + np.array([0, 0, 0.3]) for _ in range(3)]
        w = rng.dirichlet([1, 1, 1])
        p = sum(wi * np.asarray(v, np.float32).astype(np.float64) for wi, v in zip(w, tri))
        tx = rng.uniform(-0.01, 0.01, 3)
        rx = rng.uniform(-0.01, 0.01, 3)
        vel = rng.uniform(-1, 1, 3)
        alpha = rng.uniform()
        d1, a1, v1 = _echo_one(p, tri, tx, [rx], alpha=alpha, m_s=4.0, vel=vel)
        d2, a2, v2 = _echo_one(p, tri, rx, [tx], alpha=alpha, m_s=4.0, vel=vel)
        assert math.isclose(d1[0], d2[0], rel_tol=1e-14)
        assert math.isclose(a1[0], a2[0], rel_tol=1e-9, abs_tol=1e-300)
        assert math.isclose(v1[0], v2[0], rel_tol=1e-9, abs_tol=1e-12)


def test_echo_antenna_behind_face_is_silent():
    tri = _plate_tri(0.3, 0.0)
    d, a, _ = _echo_one((0, 0, 0.3), tri, (0, 0, 0), [(0, 0, 0), (0, 0, 0.6)], alpha=0.5)
    assert a[0] > 0 and a[1] == 0.0
    assert math.isclose(d[1], 0.6, rel_tol=1e-15)


def test_echo_unit_amplitude_mode():
    tri = _plate_tri(0.3, 20.0)
    _, a, _ = _echo_one((0, 0, 0.3), tri, (0, 0, 0), [(0, 0, 0)], amp_mode=1)
    assert a[0] == 1.0


def _radar(N=64, M=1, n_rx=1):
    return I.Radar(n_samples=N, n_chirps=M, rx=tuple((0.0, 0.0, 0.0) for _ in range(n_rx)))


@pytest.mark.parametrize("k0", [3, 8, 21])
def test_point_target_range_bin_and_carrier_phase(k0):
    """A static point target at path d = k0 c / B has beat frequency S d / c,
    i.e. exactly k0 cycles per chirp: the range DFT puts N a in bin k0, zero
    elsewhere, with the carrier phase -2 pi f0 d / c."""
    r = _radar(N=64)
    d = k0 * C / r.bandwidth
    a = 0.37
    s = oracle.synth(np.array([[d]]), np.array([[a]]), np.array([[0.0]]), r)
    X = oracle.range_doppler(s)[0, 0]
    assert int(np.argmax(np.abs(X))) == k0
    assert math.isclose(abs(X[k0]), a * 64, rel_tol=1e-12)
    mask = np.ones(64, bool)
    mask[k0] = False
    assert np.abs(X[mask]).max() < 1e-9
    phase = -2 * math.pi * ((r.f0 * d / C) % 1.0)
    assert abs(np.angle(X[k0] * np.exp(-1j * phase))) < 1e-9


@pytest.mark.parametrize("q0", [1, 2, -3])
def test_point_target_doppler_bin(q0):
    """Radial path rate d-dot advances the carrier phase by f0 d-dot T_rep / c
    per chirp: Doppler bin q0 = f0 d-dot T_rep M / c (after the shift, index
    q0 + M/2)."""
    M, N = 32, 32
    r = _radar(N=N, M=M)
    k0 = 5
    d = k0 * C / r.bandwidth
    ddot = q0 * C / (r.f0 * r.t_rep * M)
    s = oracle.synth(np.array([[d]]), np.array([[1.0]]), np.array([[ddot]]), r)
    X = np.abs(oracle.range_doppler(s)[0])
    q, k = np.unravel_index(np.argmax(X), X.shape)
    assert (q, k) == ((q0 + M // 2) % M, k0)
    # small range migration keeps almost all of the coherent gain
    assert X[q, k] > 0.95 * M * N


def test_range_migration_across_chirps():
    """With a path rate of c / (B T_rep) the target moves one range bin per
    chirp: chirp m's range DFT peaks exactly at k0 + m."""
    M, N = 8, 32
    r = _radar(N=N, M=M)
    k0 = 4
    d = k0 * C / r.bandwidth
    ddot = C / (r.bandwidth * r.t_rep)
    s = oracle.synth(np.array([[d]]), np.array([[1.0]]), np.array([[ddot]]), r)
    for m in range(M):
        X = N * np.fft.ifft(s[0, m])
        assert int(np.argmax(np.abs(X))) == k0 + m
        assert math.isclose(abs(X[k0 + m]), N, rel_tol=1e-9)


def test_synth_linearity_and_channels():
    r = _radar(N=32, M=4, n_rx=2)
    d, a, dd = I.random_hits(0, 40, 2)
    s_all = oracle.synth(d, a, dd, r)
    s_1 = oracle.synth(d[:, :25], a[:, :25], dd[:, :25], r)
    s_2 = oracle.synth(d[:, 25:], a[:, 25:], dd[:, 25:], r)
    np.testing.assert_allclose(s_all, s_1 + s_2, rtol=1e-12, atol=1e-18)
    # channel j depends only on channel j's hits
    d2 = d.copy()
    d2[1] += 0.01
    s_b = oracle.synth(d2, a, dd, r)
    np.testing.assert_array_equal(s_b[0], s_all[0])
    assert np.abs(s_b[1] - s_all[1]).max() > 1e-6


def test_synth_empty_hit_list_is_zero():
    r = _radar(N=16, M=2)
    s = oracle.synth(np.zeros((1, 0)), np.zeros((1, 0)), np.zeros((1, 0)), r)
    assert s.shape == (1, 2, 16) and np.all(s == 0)


@pytest.mark.parametrize("shape", [(1, 1, 64), (3, 8, 16), (2, 5, 12), (1, 16, 1)])
def test_range_doppler_matches_numpy(shape):
    rng = np.random.default_rng(3)
    x = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    n_rx, M, N = shape
    ref = np.fft.fftshift(M * N * np.fft.ifft2(x, axes=(1, 2)), axes=1)
    np.testing.assert_allclose(oracle.range_doppler(x), ref, rtol=1e-9, atol=1e-9)
    # Parseval
    X = oracle.range_doppler(x)
    assert math.isclose((np.abs(X) ** 2).sum(), M * N * (np.abs(x) ** 2).sum(), rel_tol=1e-10)


def test_range_doppler_hann_window():
    rng = np.random.default_rng(4)
    M, N = 8, 16
    x = rng.normal(size=(1, M, N)) + 1j * rng.normal(size=(1, M, N))
    hm = np.hanning(M)
    hn = np.hanning(N)  # numpy's symmetric Hann
    ref = np.fft.fftshift(M * N * np.fft.ifft2(x * hm[None, :, None] * hn[None, None, :], axes=(1, 2)), axes=1)
    np.testing.assert_allclose(oracle.range_doppler(x, window=1), ref, rtol=1e-9, atol=1e-9)


def test_tiny_frame_peak_at_hand_range():
    """The hand at 0.30 m gives a round trip of about 0.6 m: range bin ~ B d / c = 8."""
    radar, grid, nt = I.workload_tiny()
    s = I.hand_scene(0, nt)
    r = oracle.frame(s.V, s.F, s.vel, radar, grid)
    X = np.abs(oracle.range_doppler(r["if_cube"]))[0, 0]
    k = int(np.argmax(X))
    dmin, dmax = r["d"].min(), r["d"].max()
    assert math.floor(radar.bandwidth * dmin / C) - 1 <= k <= math.ceil(radar.bandwidth * dmax / C) + 1
