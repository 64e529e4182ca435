"""FP64 oracle of the imaging workload of Sec. II and IV: the SFCW baseband
of every TX-RX pair of the MIMO array (Eq. 4), its brute-force
back-projection into a voxel volume (Sec. IV-A) and the maximum projection
to a dB image (Sec. IV-A/B).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg may use this module; the CUDA library never
does, and it shares no code with it.

Parity status:
  * mimo_sfcw: composed from the pinned single-radar frame (trace, echo,
    Eq. 4 sum) with one chirp whose instantaneous frequency steps by df per
    sample; pinned by the equality with those frames and by the
    unit-amplitude plate closed form in tests/test_oracle_imaging.py.
  * backproject: the definition written out (a numpy sum over pairs and
    frequencies); pinned by the point-target closed form (the image of an
    ideal point scatterer equals n_pairs * n_f at the scatterer and is
    smaller everywhere else) and an integer-cycle special case.
  * max_projection: the definition; pinned by a hand-built volume.
"""
from __future__ import annotations

import types

import numpy as np

C_LIGHT = 299_792_458.0


def sfcw_radar(tx, rx, f0: float, df: float, n_f: int, alpha: float = 0.5, spec_exp: float = 8.0,
               amp_mode: int = 0, frame=None):
    """The radar description of one TX of the array for the single-radar
    oracle: one chirp of n_f samples with slope * dt = df, so sample n sees
    the carrier f0 + n df of CW step n (Eq. 4)."""
    rx = tuple(tuple(float(c) for c in r) for r in np.asarray(rx, np.float64).reshape(-1, 3))
    return types.SimpleNamespace(
        f0=float(f0), slope=float(df), dt=1.0, t_rep=1.0, n_samples=int(n_f), n_chirps=1,
        tx=tuple(float(c) for c in np.asarray(tx, np.float64).reshape(3)), rx=rx, n_rx=len(rx),
        frame=tuple(np.eye(3).ravel()) if frame is None else tuple(np.asarray(frame, np.float64).ravel()),
        alpha=float(alpha), spec_exp=float(spec_exp), amp_mode=int(amp_mode))


def mimo_sfcw(V, F, tx, rx, grid, f0: float, df: float, n_f: int, alpha: float = 0.5, spec_exp: float = 8.0,
              amp_mode: int = 0, frame=None):
    """Baseband of every TX-RX pair (Sec. II, Eq. 4): complex128 [n_tx][n_rx][n_f].

    Each TX shoots the ray grid from its own position (the static hand has
    no velocity); each hit's echo reaches every RX (Sec. III-A, III-B)."""
    from oracle import frame as single_frame
    tx = np.asarray(tx, np.float64).reshape(-1, 3)
    out = np.empty((tx.shape[0], np.asarray(rx).reshape(-1, 3).shape[0], n_f), np.complex128)
    for t in range(tx.shape[0]):
        r = sfcw_radar(tx[t], rx, f0, df, n_f, alpha, spec_exp, amp_mode, frame)
        out[t] = single_frame(V, F, np.zeros(3), r, grid)["if_cube"][:, 0, :]
    return out


def backproject(s, tx, rx, f0: float, df: float, voxels, chunk: int = 1 << 22):
    """Brute-force SFCW back-projection (Sec. IV-A): for each voxel v,
    I(v) = sum over TX t, RX j, step n of s[t, j, n] exp(+j 2 pi (f0 + n df) (|v - tx_t| + |v - rx_j|) / c).

    s: complex [n_tx][n_rx][n_f]; voxels: [n_vox][3] (m).  complex128 [n_vox]."""
    s = np.asarray(s, np.complex128)
    tx = np.asarray(tx, np.float64).reshape(-1, 3)
    rx = np.asarray(rx, np.float64).reshape(-1, 3)
    vox = np.asarray(voxels, np.float64).reshape(-1, 3)
    n_tx, n_rx, n_f = s.shape
    f = f0 + df * np.arange(n_f)
    sp = s.reshape(n_tx * n_rx, n_f)
    out = np.empty(vox.shape[0], np.complex128)
    step = max(1, chunk // (n_tx * n_rx * n_f))
    for a in range(0, vox.shape[0], step):
        v = vox[a:a + step]
        dt_ = np.linalg.norm(v[:, None, :] - tx[None, :, :], axis=-1)   # [nv, n_tx]
        dr_ = np.linalg.norm(v[:, None, :] - rx[None, :, :], axis=-1)   # [nv, n_rx]
        R = (dt_[:, :, None] + dr_[:, None, :]).reshape(v.shape[0], -1)  # [nv, pairs]
        E = np.exp(2j * np.pi * R[:, :, None] * f[None, None, :] / C_LIGHT)
        out[a:a + step] = np.einsum("vpn,pn->v", E, sp)
    return out


def volume_voxels(vol):
    """Voxel centres [nz*ny*nx][3] of a volume (x fastest), vol with fields
    x0, y0, z0, dx, dy, dz, nx, ny, nz."""
    z, y, x = np.meshgrid(vol.z0 + vol.dz * np.arange(vol.nz), vol.y0 + vol.dy * np.arange(vol.ny),
                          vol.x0 + vol.dx * np.arange(vol.nx), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=-1)


def max_projection(img, dyn_db: float):
    """Maximum projection along z (Sec. IV-A): per (y, x) the largest
    amplitude over z and its z index; amplitudes in dB relative to the
    image's maximum, floored at -dyn_db.  img: complex [nz][ny][nx]."""
    amp = np.abs(np.asarray(img))
    z = np.argmax(amp, axis=0).astype(np.int32)
    m = np.max(amp, axis=0)
    top = m.max()
    with np.errstate(divide="ignore"):
        db = 20.0 * np.log10(m / top) if top > 0 else np.full_like(m, -np.inf)
    return np.maximum(db, -float(dyn_db)), z
