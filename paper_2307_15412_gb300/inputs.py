"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds geometry and parameter generation only: the hand mesh, the
radar and ray-grid descriptions, and synthetic hit lists.  It contains none of
the method's arithmetic (no ray tracing, no echo model, no signal synthesis,
no range-Doppler processing), so both the CUDA path and the FP64 oracle can
consume its arrays without sharing any of the computation that is compared.

The paper's scene is a photogrammetric, rigged hand mesh posed in Maya
(Sec. III); that mesh is not available, so a procedural hand of the same scale
stands in: a tessellated palm box (6 x 4 x 1.5 cm) plus five fingers of three
capsules each, posed by 27 joint angles and placed about 0.3 m in front of the
radar (the measurement distance of Sec. IV-A is 31.5 cm).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

C_LIGHT = 299_792_458.0  # m/s

# --------------------------------------------------------------------------
# Radar and ray grid descriptions
# --------------------------------------------------------------------------


@dataclasses.dataclass
class Radar:
    """FMCW radar description, SI units.

    The IF sample n of chirp m sees the instantaneous frequency f0 + S*t_n
    with S = bandwidth / t_chirp and t_n = n * t_chirp / n_samples; this is
    the CW term of Eq. 4 with f0 + n*df replaced by the chirp's frequency.
    """

    f0: float = 60e9
    bandwidth: float = 4e9
    t_chirp: float = 64e-6
    t_rep: float = 64e-6
    n_samples: int = 64
    n_chirps: int = 1
    tx: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    rx: Tuple[Tuple[float, float, float], ...] = ((0.0, 0.0, 0.0),)
    frame: Tuple[float, ...] = (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0)
    alpha: float = 0.5      # Eq. 3 mixture weight (0 specular, 1 diffuse)
    spec_exp: float = 8.0   # exponent of the specular lobe
    amp_mode: int = 0       # 0: lobe amplitude, 1: unit amplitude per hit (Eq. 4)

    @property
    def n_rx(self) -> int:
        return len(self.rx)

    @property
    def slope(self) -> float:
        return self.bandwidth / self.t_chirp

    @property
    def dt(self) -> float:
        return self.t_chirp / self.n_samples


@dataclasses.dataclass
class RayGrid:
    """Uniform azimuth/elevation grid of n_az x n_el rays over +-half angles (rad)."""

    n_az: int = 64
    n_el: int = 64
    half_az: float = math.radians(30.0)
    half_el: float = math.radians(30.0)

    @property
    def n_rays(self) -> int:
        return self.n_az * self.n_el


def rx_l_array(f_center: float = 62e9) -> Tuple[Tuple[float, float, float], ...]:
    """1 TX / 3 RX in an L at lambda/2 spacing: RX0 colocated with the TX at
    the origin, RX1 at +x, RX2 at +y (boresight +z)."""
    half_lambda = 0.5 * C_LIGHT / f_center
    return ((0.0, 0.0, 0.0), (half_lambda, 0.0, 0.0), (0.0, half_lambda, 0.0))


# --------------------------------------------------------------------------
# Procedural hand mesh
# --------------------------------------------------------------------------

_CM = 0.01
PALM_HALF = (3.0 * _CM, 2.0 * _CM, 0.75 * _CM)
PHALANX_LEN = (4.5 * _CM, 2.5 * _CM, 2.0 * _CM)
# thumb, index, middle, ring, little
FINGER_SCALE = (0.8, 0.95, 1.0, 0.95, 0.75)
FINGER_RADIUS = (0.9 * _CM, 0.75 * _CM, 0.75 * _CM, 0.75 * _CM, 0.75 * _CM)
FINGER_BASE_X = (None, -2.25 * _CM, -0.75 * _CM, 0.75 * _CM, 2.25 * _CM)
THUMB_BASE = (-3.0 * _CM, -0.5 * _CM, 0.0)
THUMB_SPLAY_DEG = 50.0
N_ANGLES = 27


def _rx(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=np.float64)


def _ry(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], dtype=np.float64)


def _rz(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]], dtype=np.float64)


def _capsule(segments: int, length: float, radius: float):
    """Closed capsule along local +y from y=0 to y=length.

    segments around the axis, H = segments//2 latitude bands per hemisphere
    plus the cylinder band: 4*S*H triangles (2*S^2 for even S)."""
    S = segments
    H = max(1, S // 2)
    rings = []  # (y, ring radius)
    for i in range(1, H + 1):  # bottom hemisphere, pole side first
        phi = 0.5 * math.pi * i / H
        rings.append((-radius * math.cos(phi), radius * math.sin(phi)))
    for i in range(H, 0, -1):  # top hemisphere, equator first
        phi = 0.5 * math.pi * i / H
        rings.append((length + radius * math.cos(phi), radius * math.sin(phi)))
    verts = [(0.0, -radius, 0.0)]
    for (y, rr) in rings:
        for s in range(S):
            th = 2.0 * math.pi * s / S
            verts.append((rr * math.cos(th), y, rr * math.sin(th)))
    verts.append((0.0, length + radius, 0.0))
    V = np.array(verts, dtype=np.float64)
    top = len(verts) - 1
    F = []
    ring0 = 1
    for s in range(S):  # bottom fan
        F.append((0, ring0 + (s + 1) % S, ring0 + s))
    for b in range(len(rings) - 1):
        r0 = 1 + b * S
        r1 = r0 + S
        for s in range(S):
            a0, a1 = r0 + s, r0 + (s + 1) % S
            b0, b1 = r1 + s, r1 + (s + 1) % S
            F.append((a0, a1, b1))
            F.append((a0, b1, b0))
    rl = 1 + (len(rings) - 1) * S
    for s in range(S):  # top fan
        F.append((top, rl + s, rl + (s + 1) % S))
    return V, np.array(F, dtype=np.int64)


def _box(half: Sequence[float], quad: float):
    """Closed, tessellated axis-aligned box centred at the origin."""
    hx, hy, hz = half
    verts: List[Tuple[float, float, float]] = []
    faces: List[Tuple[int, int, int]] = []

    def face(origin, du, dv, nu, nv):
        base = len(verts)
        for j in range(nv + 1):
            for i in range(nu + 1):
                p = np.asarray(origin) + np.asarray(du) * (i / nu) + np.asarray(dv) * (j / nv)
                verts.append(tuple(p))
        for j in range(nv):
            for i in range(nu):
                a = base + j * (nu + 1) + i
                b = a + 1
                c = a + (nu + 1)
                d = c + 1
                faces.append((a, b, d))
                faces.append((a, d, c))

    def n_of(extent):
        return max(1, int(round(extent / quad)))

    X, Y, Z = 2 * hx, 2 * hy, 2 * hz
    # -z face (palm, facing the radar) and +z face (back of the hand)
    face((-hx, -hy, -hz), (0, Y, 0), (X, 0, 0), n_of(Y), n_of(X))
    face((-hx, -hy, hz), (X, 0, 0), (0, Y, 0), n_of(X), n_of(Y))
    # -y and +y faces
    face((-hx, -hy, -hz), (X, 0, 0), (0, 0, Z), n_of(X), n_of(Z))
    face((-hx, hy, -hz), (0, 0, Z), (X, 0, 0), n_of(Z), n_of(X))
    # -x and +x faces
    face((-hx, -hy, -hz), (0, 0, Z), (0, Y, 0), n_of(Z), n_of(Y))
    face((hx, -hy, -hz), (0, Y, 0), (0, 0, Z), n_of(Y), n_of(Z))
    # weld duplicated edge vertices so the box is one closed mesh
    V = np.array(verts, dtype=np.float64)
    key = np.round(V / 1e-9).astype(np.int64)
    inv = np.unique(key, axis=0, return_inverse=True)[1].reshape(-1)
    uniq, first = np.unique(inv, return_index=True)
    Vw = V[first]
    remap = np.empty(len(uniq), dtype=np.int64)
    remap[uniq] = np.arange(len(uniq))
    Fw = remap[inv.reshape(-1)[np.asarray(faces, dtype=np.int64)]]
    return Vw, Fw


def segments_for_triangles(n_tri_target: int) -> int:
    """Capsule segment count S for a total of about 33*S^2 triangles (even S)."""
    S = int(round(math.sqrt(max(n_tri_target, 1) / 33.0)))
    S = max(4, S + (S % 2))
    return S


def random_hand_angles(rng: np.random.Generator) -> np.ndarray:
    """27 joint/pose angles, each drawn U(0, 60 deg) (returned in degrees)."""
    return rng.uniform(0.0, 60.0, size=N_ANGLES)


def hand_mesh(n_tri_target: int, angles_deg: Sequence[float],
              center: Sequence[float] = (0.0, 0.0, 0.30)):
    """Procedural hand: V float32 [nv,3] (metres), F int32 [nt,3].

    angles_deg: 15 flexions (3 per finger, thumb first, used as drawn: bending
    toward the palm side, which faces -z, i.e. the radar), then 5 abductions,
    5 twists and 2 global tilts; the last 12 are drawn in [0, 60] deg and
    mapped to (a - 30)/3, i.e. +-10 deg.
    """
    ang = np.asarray(angles_deg, dtype=np.float64)
    if ang.shape != (N_ANGLES,):
        raise ValueError("expected 27 angles")
    flex = np.radians(ang[0:15]).reshape(5, 3)
    small = np.radians((ang[15:27] - 30.0) / 3.0)
    abd, twist, tilt = small[0:5], small[5:10], small[10:12]
    S = segments_for_triangles(n_tri_target)
    quad = 7.2 * _CM / S

    parts_v, parts_f = [], []
    nbase = 0
    Vb, Fb = _box(PALM_HALF, quad)
    parts_v.append(Vb)
    parts_f.append(Fb)
    nbase += len(Vb)
    for f in range(5):
        if f == 0:
            base = np.array(THUMB_BASE)
            Q = _rz(math.radians(THUMB_SPLAY_DEG))
        else:
            base = np.array([FINGER_BASE_X[f], PALM_HALF[1], 0.0])
            Q = np.eye(3)
        Q = Q @ _rz(abd[f]) @ _ry(twist[f])
        p = base.copy()
        for k in range(3):
            Q = Q @ _rx(-flex[f, k])
            L = PHALANX_LEN[k] * FINGER_SCALE[f]
            Vc, Fc = _capsule(S, L, FINGER_RADIUS[f])
            parts_v.append(p + Vc @ Q.T)
            parts_f.append(Fc + nbase)
            nbase += len(Vc)
            p = p + L * Q[:, 1]
    V = np.concatenate(parts_v, axis=0)
    F = np.concatenate(parts_f, axis=0)
    G = _rx(tilt[0]) @ _ry(tilt[1])
    V = V @ G.T + np.asarray(center, dtype=np.float64)
    return V.astype(np.float32), F.astype(np.int32)


def _rot_batch(axis: int, a: np.ndarray) -> np.ndarray:
    """[P][3][3] rotations by angles a[P] about x (0), y (1) or z (2)."""
    c, s = np.cos(a), np.sin(a)
    R = np.zeros((a.size, 3, 3))
    i, j = [(1, 2), (0, 2), (0, 1)][axis]
    R[:, axis, axis] = 1.0
    R[:, i, i] = c
    R[:, j, j] = c
    if axis == 1:
        R[:, 0, 2], R[:, 2, 0] = s, -s
    else:
        R[:, i, j], R[:, j, i] = -s, s
    return R


_TEMPLATES = {}


def _hand_templates(S: int):
    """Box and the 15 capsule templates of segment count S (shared by all poses)."""
    if S not in _TEMPLATES:
        quad = 7.2 * _CM / S
        box = _box(PALM_HALF, quad)
        caps = [[_capsule(S, PHALANX_LEN[k] * FINGER_SCALE[f], FINGER_RADIUS[f]) for k in range(3)] for f in range(5)]
        _TEMPLATES[S] = (box, caps)
    return _TEMPLATES[S]


def hand_meshes(n_tri_target: int, angles_deg: np.ndarray, centers: np.ndarray):
    """The procedural hand of hand_mesh for P poses at once: V float32
    [P][nv][3], F int32 [nt][3] (one topology).  Same construction, evaluated
    with batched rotations (values agree with hand_mesh to float32 rounding)."""
    ang = np.atleast_2d(np.asarray(angles_deg, dtype=np.float64))
    centers = np.atleast_2d(np.asarray(centers, dtype=np.float64))
    P = ang.shape[0]
    flex = np.radians(ang[:, 0:15]).reshape(P, 5, 3)
    small = np.radians((ang[:, 15:27] - 30.0) / 3.0)
    abd, twist, tilt = small[:, 0:5], small[:, 5:10], small[:, 10:12]
    S = segments_for_triangles(n_tri_target)
    (Vb, Fb), caps = _hand_templates(S)
    parts_v = [np.broadcast_to(Vb, (P,) + Vb.shape)]
    parts_f = [Fb]
    nbase = len(Vb)
    for f in range(5):
        if f == 0:
            base = np.broadcast_to(np.array(THUMB_BASE), (P, 3)).copy()
            Q = np.broadcast_to(_rz(math.radians(THUMB_SPLAY_DEG)), (P, 3, 3)).copy()
        else:
            base = np.broadcast_to(np.array([FINGER_BASE_X[f], PALM_HALF[1], 0.0]), (P, 3)).copy()
            Q = np.broadcast_to(np.eye(3), (P, 3, 3)).copy()
        Q = Q @ _rot_batch(2, abd[:, f]) @ _rot_batch(1, twist[:, f])
        pos = base
        for k in range(3):
            Q = Q @ _rot_batch(0, -flex[:, f, k])
            L = PHALANX_LEN[k] * FINGER_SCALE[f]
            Vc, Fc = caps[f][k]
            parts_v.append(pos[:, None, :] + np.einsum("vj,pij->pvi", Vc, Q))
            parts_f.append(Fc + nbase)
            nbase += len(Vc)
            pos = pos + L * Q[:, :, 1]
    V = np.concatenate(parts_v, axis=1)
    F = np.concatenate(parts_f, axis=0)
    G = _rot_batch(0, tilt[:, 0]) @ _rot_batch(1, tilt[:, 1])
    V = np.einsum("pvj,pij->pvi", V, G) + centers[:, None, :]
    return V.astype(np.float32), F.astype(np.int32)


@dataclasses.dataclass
class Scene:
    V: np.ndarray          # float32 [nv,3]
    F: np.ndarray          # int32 [nt,3]
    vel: np.ndarray        # float32 [3], rigid translation velocity (m/s)
    center: np.ndarray     # float64 [3]
    angles_deg: np.ndarray


def hand_scene(seed: int, n_tri_target: int, range_m: Optional[Tuple[float, float]] = None,
               speed: Optional[Tuple[float, float]] = None, angles_deg=None,
               center=None) -> Scene:
    """Seeded hand scene.  range_m=(lo, hi) draws the hand's distance along
    boresight; speed=(lo, hi) draws a radial velocity (rigid translation along
    the unit vector from the radar to the hand centre; positive = receding)."""
    rng = np.random.default_rng(seed)
    ang = random_hand_angles(rng) if angles_deg is None else np.asarray(angles_deg, dtype=np.float64)
    if center is None:
        R = 0.30 if range_m is None else float(rng.uniform(*range_m))
        center = np.array([0.0, 0.0, R])
    center = np.asarray(center, dtype=np.float64)
    v = 0.0 if speed is None else float(rng.uniform(*speed))
    chat = center / np.linalg.norm(center)
    V, F = hand_mesh(n_tri_target, ang, center)
    return Scene(V=V, F=F, vel=(v * chat).astype(np.float32), center=center, angles_deg=ang)


# --------------------------------------------------------------------------
# Simple test geometries (closed forms live in the tests, not here)
# --------------------------------------------------------------------------


def plate(center, half_x, half_y, nx=1, ny=1):
    """Rectangular plate in the plane z = center[2], facing the radar."""
    cx, cy, cz = center
    xs = np.linspace(cx - half_x, cx + half_x, nx + 1)
    ys = np.linspace(cy - half_y, cy + half_y, ny + 1)
    V = np.array([(x, y, cz) for y in ys for x in xs], dtype=np.float32)
    F = []
    for j in range(ny):
        for i in range(nx):
            a = j * (nx + 1) + i
            F.append((a, a + 1, a + nx + 2))
            F.append((a, a + nx + 2, a + nx + 1))
    return V, np.array(F, dtype=np.int32)


def icosphere(center, radius, subdiv=2):
    """Geodesic sphere (subdivided icosahedron) with vertices on the sphere."""
    t = (1.0 + 5 ** 0.5) / 2.0
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    V = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in V]
    for _ in range(subdiv):
        cache = {}
        newF = []

        def mid(a, b):
            k = (min(a, b), max(a, b))
            if k not in cache:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                cache[k] = len(V) - 1
            return cache[k]
        for (a, b, c) in F:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            newF += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = newF
    Vn = np.array(V) * radius + np.asarray(center, dtype=np.float64)
    return Vn.astype(np.float32), np.array(F, dtype=np.int32)


# --------------------------------------------------------------------------
# Synthetic hit lists (for the synthesis-only workloads)
# --------------------------------------------------------------------------


def random_hits(seed: int, K: int, n_rx: int, d_range=(0.4, 1.2), amp_range=(1e-6, 1e-4),
                ddot_range=(-2.0, 2.0)):
    """Seeded hit list in the [n_rx][K] float32 layout: total path d (m),
    amplitude a and path rate d-dot (m/s).  Paths of the RX channels of one
    hit differ by at most a few millimetres, as for antennas lambda/2 apart."""
    rng = np.random.default_rng(seed)
    d0 = rng.uniform(*d_range, size=K)
    off = rng.uniform(-2.5e-3, 2.5e-3, size=(n_rx, K))
    off[0] = 0.0
    d = (d0[None, :] + off).astype(np.float32)
    a = rng.uniform(*amp_range, size=(n_rx, K)).astype(np.float32)
    v0 = rng.uniform(*ddot_range, size=K)
    ddot = (v0[None, :] + rng.uniform(-1e-3, 1e-3, size=(n_rx, K))).astype(np.float32)
    return d, a, ddot


# --------------------------------------------------------------------------
# Workload presets (sizes of the hand-imaging workloads)
# --------------------------------------------------------------------------


def workload_tiny() -> Tuple[Radar, RayGrid, int]:
    """~2k-triangle hand at 0.30 m, 64x64 rays over +-30 deg, 1 TX 1 RX,
    one chirp of 64 samples, 60 -> 64 GHz in 64 us."""
    return (Radar(n_samples=64, n_chirps=1, rx=((0.0, 0.0, 0.0),)),
            RayGrid(64, 64, math.radians(30.0), math.radians(30.0)), 2000)


def workload_full_frame() -> Tuple[Radar, RayGrid, int]:
    """~20k-triangle hand at U(0.2, 0.6) m moving radially at U(-1, 1) m/s,
    512x512 rays over +-45 deg, 1 TX 3 RX (L, lambda/2), 64 chirps x 256
    samples, 60 -> 64 GHz in 64 us, chirp repetition 64 us."""
    return (Radar(n_samples=256, n_chirps=64, rx=rx_l_array()),
            RayGrid(512, 512, math.radians(45.0), math.radians(45.0)), 20000)


FULL_FRAME_RANGE = (0.2, 0.6)
FULL_FRAME_SPEED = (-1.0, 1.0)


# --------------------------------------------------------------------------
# Learned-surrogate workload: seeded hand parameters and their scenes
# --------------------------------------------------------------------------

# Training box of the surrogate's 32 inputs: 27 joint/pose angles (deg),
# hand centre x, y, z (m) and velocity (radial, lateral x) (m/s).
SURROGATE_LO = np.array([0.0] * N_ANGLES + [-0.05, -0.05, 0.20, -1.0, -1.0])
SURROGATE_HI = np.array([60.0] * N_ANGLES + [0.05, 0.05, 0.60, 1.0, 1.0])
SURROGATE_TRIANGLES = 2000


def surrogate_radar_grid() -> Tuple[Radar, RayGrid]:
    """Frames the surrogate learns: the tiny hand's 64 x 64 rays over
    +-30 deg, 1 TX 3 RX (L, lambda/2), 32 chirps x 32 samples, 60-64 GHz."""
    return (Radar(n_samples=32, n_chirps=32, rx=rx_l_array()),
            RayGrid(64, 64, math.radians(30.0), math.radians(30.0)))


def surrogate_inputs(seed: int, n: int, lo=None, hi=None) -> np.ndarray:
    """n seeded parameter vectors [n][32] (float64), uniform in the box."""
    rng = np.random.default_rng(seed)
    lo = SURROGATE_LO if lo is None else np.asarray(lo, np.float64)
    hi = SURROGATE_HI if hi is None else np.asarray(hi, np.float64)
    return lo + (hi - lo) * rng.random((n, lo.size))


def surrogate_features(raw: np.ndarray) -> np.ndarray:
    """Network inputs: each parameter mapped linearly from the training box
    to [-1, 1] (float32)."""
    return (2.0 * (np.asarray(raw) - SURROGATE_LO) / (SURROGATE_HI - SURROGATE_LO) - 1.0).astype(np.float32)


def surrogate_scene(raw_row: np.ndarray, n_tri_target: int = SURROGATE_TRIANGLES) -> Scene:
    """Hand scene of one parameter vector: posed by the 27 angles, centred
    at (x, y, z), moving with v_r along the unit vector from the radar to the
    centre plus v_x along x."""
    raw_row = np.asarray(raw_row, np.float64)
    center = raw_row[N_ANGLES:N_ANGLES + 3]
    vr, vx = raw_row[N_ANGLES + 3], raw_row[N_ANGLES + 4]
    chat = center / np.linalg.norm(center)
    vel = vr * chat + np.array([vx, 0.0, 0.0])
    V, F = hand_meshes(n_tri_target, raw_row[None, :N_ANGLES], center[None])
    return Scene(V=V[0], F=F, vel=vel.astype(np.float32), center=center, angles_deg=raw_row[:N_ANGLES])


def surrogate_scenes(raw: np.ndarray, n_tri_target: int = SURROGATE_TRIANGLES):
    """Vertices [P][nv][3], shared faces and velocities [P][3] of many
    parameter vectors at once (the batched form of surrogate_scene)."""
    raw = np.atleast_2d(np.asarray(raw, np.float64))
    center = raw[:, N_ANGLES:N_ANGLES + 3]
    chat = center / np.linalg.norm(center, axis=1, keepdims=True)
    vel = raw[:, N_ANGLES + 3:N_ANGLES + 4] * chat
    vel[:, 0] += raw[:, N_ANGLES + 4]
    V, F = hand_meshes(n_tri_target, raw[:, :N_ANGLES], center)
    return V, F, vel.astype(np.float32)


def surrogate_init_params(dims, seed: int) -> np.ndarray:
    """Seeded starting parameters of the surrogate network, packed FP32
    [W_1, b_1, W_2, b_2, ...] with W_l [out][in]: He-uniform weights
    (bound sqrt(6 / in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(len(dims) - 1):
        n_in, n_out = int(dims[i]), int(dims[i + 1])
        bound = math.sqrt(6.0 / n_in)
        parts.append(rng.uniform(-bound, bound, size=n_out * n_in))
        parts.append(np.zeros(n_out))
    return np.concatenate(parts).astype(np.float32)


# --------------------------------------------------------------------------
# Imaging workload (Sec. II and IV): square MIMO array, SFCW steps, volume
# --------------------------------------------------------------------------

IMAGING_F0 = 72e9            # first SFCW carrier (Hz)
IMAGING_DF = 10e9 / 128      # step: 10 GHz over 128 steps, the last below 82 GHz
IMAGING_NF = 128
IMAGING_RANGE = 0.315        # hand centre on the array's boresight (m)


def mimo_square_array(n_per_side: int = 47, pitch: float = 3e-3, z: float = 0.0):
    """Synthetic stand-in for the 94 TX / 94 RX square array (exact positions
    are not published): a square of side n_per_side * pitch (14.1 cm at 47 x
    3 mm), TX along its top and bottom edges, RX along its left and right
    edges, pitch apart, centred on the boresight in the plane z.  Returns
    (tx [2 n][3], rx [2 n][3]) float64."""
    half = 0.5 * n_per_side * pitch
    along = -half + pitch * (np.arange(n_per_side) + 0.5)
    zeros = np.zeros(n_per_side)
    tx = np.concatenate([np.stack([along, zeros + half, zeros + z], 1),
                         np.stack([along, zeros - half, zeros + z], 1)])
    rx = np.concatenate([np.stack([zeros - half, along, zeros + z], 1),
                         np.stack([zeros + half, along, zeros + z], 1)])
    return tx, rx


@dataclasses.dataclass
class Volume:
    """Voxel grid: centre of voxel (ix, iy, iz) = (x0 + ix dx, y0 + iy dy, z0 + iz dz)."""

    x0: float
    y0: float
    z0: float
    dx: float
    dy: float
    dz: float
    nx: int
    ny: int
    nz: int

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz


def imaging_volume() -> Volume:
    """x, y in [-10, 10] cm and z in [26, 34] cm at 1 mm: 201 x 201 x 81 voxels."""
    return Volume(-0.10, -0.10, 0.26, 1e-3, 1e-3, 1e-3, 201, 201, 81)


def workload_imaging() -> Tuple[RayGrid, int]:
    """Ray grid of each TX (512 x 512 over +-20 deg, covering a hand at
    0.315 m) and the hand's triangle count (~20k)."""
    return RayGrid(512, 512, math.radians(20.0), math.radians(20.0)), 20000
