"""Pins of the oracle's stochastic material model (Eq. 1-3 with random
diffuse directions, reception cones, bounces) and of its random stream.

* Philox4x32-10: the published known-answer vectors of the generator
  (Salmon et al., SC 2011; the test vectors distributed with its reference
  implementation) for three (counter, key) pairs;
* alpha = 0 (pure mirror), a plate facing a TX with a colocated receiver:
  a ray at incidence theta leaves at 2 theta from the way back, so it is
  received iff 2 theta <= theta_r, with path 2 t (closed form);
* alpha = 1 (pure Eq. 1): (n + r) / |n + r| with r uniform on the unit
  sphere is the cosine-weighted (Lambertian) direction, so the chance that
  it falls in a cone of half-angle theta_r around a direction at beta from
  n (cone clear of the horizon) is sin^2(theta_r) cos(beta) exactly; the
  received count over a plate matches the sum of these chances within 5
  standard deviations;
* the stream is keyed by (ray, bounce): the first bounce of a three-bounce
  run is the one-bounce run, entry for entry.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2307_15412_gb300 import inputs as I


@pytest.mark.parametrize("ctr,key,want", [
    ((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff,) * 4, (0xffffffff,) * 2, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
])
def test_philox_known_answers(ctr, key, want):
    assert tuple(int(x) for x in oracle.philox4x32(ctr, key)) == want


def _colocated(**kw):
    return I.Radar(n_samples=64, n_chirps=4, rx=((0.0, 0.0, 0.0),), **kw)


def test_mirror_plate_closed_form():
    D = 0.4
    V, F = I.plate((0.0, 0.0, D), 0.3, 0.3, 4, 4)
    radar = _colocated(alpha=0.0)
    grid = I.RayGrid(48, 48, math.radians(20.0), math.radians(20.0))
    th = math.radians(8.0)
    out = oracle.stochastic_frame(V, F, np.zeros(3), radar, grid, 0.0, th, 1, seed=7, frame=1)
    dirs, omega = oracle.ray_dirs(grid)
    inc = np.arccos(np.clip(dirs[:, 2], -1, 1))
    want = 2 * inc <= th
    clear = np.abs(2 * inc - th) > 1e-9
    got = np.zeros(len(dirs), bool)
    got[out["ray"]] = True
    assert (got[clear] == want[clear]).all() and want.sum() > 20
    t = float(np.float32(D)) / dirs[out["ray"], 2]   # the plate's float32 height
    assert np.allclose(out["d"][0], 2 * t, rtol=1e-12)
    assert np.allclose(out["a"][0], omega[out["ray"]] / (2 * math.pi * (1 - math.cos(th))), rtol=1e-12)


def test_lambertian_reception_probability():
    D = 0.4
    V, F = I.plate((0.0, 0.0, D), 0.5, 0.5, 2, 2)
    radar = _colocated(alpha=1.0)
    grid = I.RayGrid(96, 96, math.radians(30.0), math.radians(30.0))
    th = math.radians(10.0)
    out = oracle.stochastic_frame(V, F, np.zeros(3), radar, grid, 1.0, th, 1, seed=3, frame=5)
    dirs, _ = oracle.ray_dirs(grid)
    beta = np.arccos(dirs[:, 2])        # the way back makes the incidence angle with the normal
    P = math.sin(th) ** 2 * np.cos(beta)
    mean, sd = P.sum(), math.sqrt((P * (1 - P)).sum())
    assert abs(len(out["ray"]) - mean) <= 5 * sd
    assert mean > 200


def test_bounce_prefix_is_the_single_bounce_run():
    s = I.hand_scene(2, 1000)
    radar = I.Radar(n_samples=64, n_chirps=4, rx=I.rx_l_array(), alpha=0.5)
    grid = I.RayGrid(32, 32, math.radians(25.0), math.radians(25.0))
    one = oracle.stochastic_frame(s.V, s.F, s.vel, radar, grid, 0.5, math.radians(20.0), 1, seed=11, frame=2)
    three = oracle.stochastic_frame(s.V, s.F, s.vel, radar, grid, 0.5, math.radians(20.0), 3, seed=11, frame=2)
    first = three["bounce"] == 0
    assert np.array_equal(three["ray"][first], one["ray"])
    for k in ("d", "a", "ddot"):
        assert np.array_equal(three[k][:, first], one[k])
    assert (three["bounce"] > 0).any()
