"""FP64 CPU oracle of the radar ray-tracing hot path (arXiv 2307.15412).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg may use this package; the CUDA library never
does.  It shares no code with the CUDA path.  The heavy loops (brute-force
tracing, the direct IF sum, the direct DFTs) are plain C in ``rr_oracle.c``;
this module compiles that file with gcc, loads it with ctypes and adds the
numpy definitions of the LBVH's integer steps (``bvh.py``) and of the
surrogate network (``mlp.py``).

Parity status per function is listed in the header of each file; every
function here is pinned by tests under ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "librr_oracle.so")
_lock = threading.Lock()
_lib = None
C_LIGHT = 299_792_458.0


def build(force: bool = False) -> str:
    """Compile rr_oracle.c with gcc (OpenMP, IEEE double, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            I = ctypes.c_int
            D = ctypes.c_double
            lib.rro_ray_dirs.argtypes = [I, I, D, D, P, P, P]
            lib.rro_trace.argtypes = [P, I64, P, I64, P, P, I64, P, P]
            lib.rro_echo.argtypes = [I64, P, P, P, P, P, P, P, I, P, P, D, D, I, P, P, P]
            lib.rro_synth.argtypes = [I64, I, P, P, P, D, D, D, D, I, I, P]
            lib.rro_range_doppler.argtypes = [I, I, I, P, I, P]
            lib.rro_num_threads.restype = I
            U32 = ctypes.c_uint32
            lib.rro_philox4x32.argtypes = [P, P, P]
            lib.rro_stochastic.argtypes = [P, I64, P, I64, P, I, P, P, P, P, I64, D, D, I, U32, U32, D, I, I64,
                                           P, P, P, P, P, P]
            lib.rro_stochastic.restype = I64
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().rro_num_threads())


def ray_dirs(grid, frame=None):
    """Unit ray directions [n_rays, 3] (world frame) and cell solid angles."""
    lib = _load()
    R = np.ascontiguousarray(np.eye(3) if frame is None else np.asarray(frame, np.float64).reshape(3, 3))
    n = grid.n_az * grid.n_el
    dirs = np.empty((n, 3), np.float64)
    omega = np.empty(n, np.float64)
    lib.rro_ray_dirs(grid.n_az, grid.n_el, float(grid.half_az), float(grid.half_el), _p(R), _p(dirs), _p(omega))
    return dirs, omega


def trace(V, F, origin, dirs):
    """Brute-force closest hit: (tri int32 [n], t float64 [n]); miss = -1."""
    lib = _load()
    V = np.ascontiguousarray(V, np.float32)
    F = np.ascontiguousarray(F, np.int32)
    o = np.ascontiguousarray(origin, np.float64)
    dirs = np.ascontiguousarray(dirs, np.float64)
    n = dirs.shape[0]
    tri = np.empty(n, np.int32)
    t = np.empty(n, np.float64)
    lib.rro_trace(_p(V), V.shape[0], _p(F), F.shape[0], _p(o), _p(dirs), n, _p(tri), _p(t))
    return tri, t


def echo(V, F, origin, dirs, t, tri, omega, radar, vel):
    """Per-hit echo for each RX: d, a, ddot as float64 [n_rx][K]."""
    lib = _load()
    V = np.ascontiguousarray(V, np.float32)
    F = np.ascontiguousarray(F, np.int32)
    K = int(len(t))
    n_rx = radar.n_rx
    rx = np.ascontiguousarray(np.asarray(radar.rx, np.float64).reshape(n_rx, 3))
    d = np.empty((n_rx, K), np.float64)
    a = np.empty((n_rx, K), np.float64)
    dd = np.empty((n_rx, K), np.float64)
    lib.rro_echo(K, _p(np.ascontiguousarray(origin, np.float64)), _p(np.ascontiguousarray(dirs, np.float64)),
                 _p(np.ascontiguousarray(t, np.float64)), _p(np.ascontiguousarray(tri, np.int32)),
                 _p(np.ascontiguousarray(omega, np.float64)), _p(V), _p(F), n_rx, _p(rx),
                 _p(np.ascontiguousarray(vel, np.float64)), float(radar.alpha), float(radar.spec_exp),
                 int(radar.amp_mode), _p(d), _p(a), _p(dd))
    return d, a, dd


def synth(d, a, ddot, radar):
    """Direct FP64 IF sum (Eq. 4, FMCW form): complex128 [n_rx][M][N]."""
    lib = _load()
    d = np.ascontiguousarray(d, np.float64)
    a = np.ascontiguousarray(a, np.float64)
    ddot = np.ascontiguousarray(ddot, np.float64)
    n_rx, K = d.shape
    out = np.empty((n_rx, radar.n_chirps, radar.n_samples, 2), np.float64)
    lib.rro_synth(K, n_rx, _p(d), _p(a), _p(ddot), float(radar.f0), float(radar.slope), float(radar.dt),
                  float(radar.t_rep), radar.n_chirps, radar.n_samples, _p(out))
    return out[..., 0] + 1j * out[..., 1]


def range_doppler(if_cube, window: int = 0):
    """Direct 2-D DFT (+ kernel), Doppler fft-shifted: complex128 [n_rx][M][N]."""
    lib = _load()
    x = np.asarray(if_cube, np.complex128)
    n_rx, M, N = x.shape
    xi = np.ascontiguousarray(np.stack([x.real, x.imag], axis=-1))
    out = np.empty((n_rx, M, N, 2), np.float64)
    lib.rro_range_doppler(n_rx, M, N, _p(xi), int(window), _p(out))
    return out[..., 0] + 1j * out[..., 1]


def frame(scene_V, scene_F, vel, radar, grid, rays=None):
    """Whole single-bounce frame: rays -> closest hits -> echo -> IF.

    rays: optional subset of ray ids (the trace is per ray, so a subset gives
    exactly those rays' results).  Returns a dict with per-ray tri/t, the hit
    list in ray order and the IF cube of those hits."""
    dirs, omega = ray_dirs(grid, radar.frame)
    if rays is not None:
        rays = np.asarray(rays, np.int64)
        dirs, omega = dirs[rays], omega[rays]
    else:
        rays = np.arange(dirs.shape[0], dtype=np.int64)
    origin = np.asarray(radar.tx, np.float64)
    tri, t = trace(scene_V, scene_F, origin, dirs)
    hit = tri >= 0
    d, a, dd = echo(scene_V, scene_F, origin, dirs[hit], t[hit], tri[hit], omega[hit], radar,
                    np.asarray(vel, np.float64))
    return dict(ray_ids=rays, tri=tri, t=t, hit_rays=rays[hit], d=d, a=a, ddot=dd,
                if_cube=synth(d, a, dd, radar))


def triangle_samples(V, F, k: int):
    """Sample points of the per-triangle casting (rays cast to each mesh
    triangle, Sec. III): for every triangle (id order) the k * k centroids of
    the sub-triangles of its regular k-subdivision -- "up" cells (i, j) with
    i + j <= k - 1 at barycentric ((i + 1/3) / k, (j + 1/3) / k) row by row,
    then "down" cells with i + j <= k - 2 at ((i + 2/3) / k, (j + 2/3) / k).
    Returns (points float64 [n * k^2, 3], triangle id [n * k^2], sample index
    [n * k^2]), triangle-major."""
    b = [((i + 1.0 / 3.0) / k, (j + 1.0 / 3.0) / k) for i in range(k) for j in range(k - i)]
    b += [((i + 2.0 / 3.0) / k, (j + 2.0 / 3.0) / k) for i in range(k - 1) for j in range(k - 1 - i)]
    b = np.asarray(b, np.float64)                     # [S, 2]
    V64 = np.asarray(V, np.float32).astype(np.float64)
    F = np.asarray(F, np.int64)
    v0 = V64[F[:, 0]]
    e1, e2 = V64[F[:, 1]] - v0, V64[F[:, 2]] - v0
    P = v0[:, None, :] + b[None, :, 0:1] * e1[:, None, :] + b[None, :, 1:2] * e2[:, None, :]
    n, S = F.shape[0], b.shape[0]
    return P.reshape(-1, 3), np.repeat(np.arange(n), S), np.tile(np.arange(S), n)


def triangle_frame(V, F, vel, radar, k: int):
    """Frame of the per-triangle casting: a ray from the TX to every sample
    point (``triangle_samples``), received when its brute-force nearest hit
    is the sample's own triangle; each received sample stands for area / k^2
    of its face, seen under the solid angle (area / k^2) |n . u| / t^2, and
    is echoed and synthesised like a grid ray's hit (t = the exact distance
    to the sample point).  Returns the per-sample visibility, the received
    samples' ray ids (triangle id * k^2 + sample), their echo and the IF."""
    P, tid, samp = triangle_samples(V, F, k)
    S = k * k
    origin = np.asarray(radar.tx, np.float64)
    w = P - origin
    t = np.sqrt((w * w).sum(axis=1))
    dirs = w / t[:, None]
    hit, _ = trace(V, F, origin, dirs)
    vis = hit == tid
    V64 = np.asarray(V, np.float32).astype(np.float64)
    Fi = np.asarray(F, np.int64)
    nrm = np.cross(V64[Fi[:, 1]] - V64[Fi[:, 0]], V64[Fi[:, 2]] - V64[Fi[:, 0]])   # |nrm| = 2 area
    omega = 0.5 * np.abs((dirs * nrm[tid]).sum(axis=1)) / (S * t * t)
    rays = tid * S + samp
    d, a, dd = echo(V, F, origin, dirs[vis], t[vis], tid[vis].astype(np.int32), omega[vis], radar,
                    np.asarray(vel, np.float64))
    return dict(visible=vis, ray_ids=rays, hit_rays=rays[vis], omega=omega, d=d, a=a, ddot=dd,
                if_cube=synth(d, a, dd, radar))


def philox4x32(ctr, key):
    """Philox4x32-10 of a 4-word counter and a 2-word key: 4 uint32 words."""
    c = np.ascontiguousarray(np.asarray(ctr, np.uint64).astype(np.uint32))
    k = np.ascontiguousarray(np.asarray(key, np.uint64).astype(np.uint32))
    out = np.empty(4, np.uint32)
    _load().rro_philox4x32(_p(c), _p(k), _p(out))
    return out


STOCHASTIC_EPS = 1e-6   # origin offset (m) of bounce and return-leg rays along the face normal


def stochastic_frame(V, F, vel, radar, grid, alpha: float, theta_r: float, bounces: int, seed: int, frame: int,
                     rays=None):
    """Frame of the stochastic material model (Eq. 1-3 with random diffuse
    directions, reception cones of half-angle theta_r and up to `bounces`
    bounces; see rro_stochastic): the (ray, bounce) entries with at least
    one receiving antenna, their path lengths, amplitudes and path rates
    ([n_rx][K]) and the IF cube.  rays: optional subset of grid ray ids."""
    lib = _load()
    dirs, omega = ray_dirs(grid, radar.frame)
    ids = np.arange(dirs.shape[0], dtype=np.int64)
    if rays is not None:
        ids = np.asarray(rays, np.int64)
    V = np.ascontiguousarray(V, np.float32)
    F = np.ascontiguousarray(F, np.int32)
    n_rx = radar.n_rx
    rx = np.ascontiguousarray(np.asarray(radar.rx, np.float64).reshape(n_rx, 3))
    cap = max(1, len(ids) * bounces)
    ray_o = np.empty(cap, np.int32)
    b_o = np.empty(cap, np.int32)
    tri_o = np.empty(cap, np.int32)
    d = np.empty((n_rx, cap))
    a = np.empty((n_rx, cap))
    dd = np.empty((n_rx, cap))
    # the C loop numbers rays by their position in the given arrays: map back after
    sel_dirs = np.ascontiguousarray(dirs[ids])
    sel_om = np.ascontiguousarray(omega[ids])
    # the random stream is keyed by the grid ray id, so run ray by ray when a subset is given
    if rays is None:
        K = lib.rro_stochastic(_p(V), V.shape[0], _p(F), F.shape[0], _p(np.asarray(radar.tx, np.float64)), n_rx,
                               _p(rx), _p(np.asarray(vel, np.float64)), _p(sel_dirs), _p(sel_om), len(ids),
                               float(alpha), float(theta_r), int(bounces), int(seed), int(frame), STOCHASTIC_EPS,
                               int(radar.amp_mode), cap, _p(ray_o), _p(b_o), _p(tri_o), _p(d), _p(a), _p(dd))
    else:
        raise NotImplementedError("subsets: the stream is keyed by the grid ray id")
    K = int(K)
    assert K <= cap
    d, a, dd = d[:, :K].copy(), a[:, :K].copy(), dd[:, :K].copy()
    return dict(ray=ray_o[:K].copy(), bounce=b_o[:K].copy(), tri=tri_o[:K].copy(), d=d, a=a, ddot=dd,
                if_cube=synth(d, a, dd, radar))
