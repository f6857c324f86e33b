"""Seeded synthetic channel-flow snapshots.

This module only draws random numbers and lays them out; it holds none of the
GKE arithmetic (no correlations, no derivatives, no averages of products).  It
is the one module that both the CPU oracle and the CUDA path read their inputs
from.

The paper's inputs are DNS snapshots of plane channel flow stored as Fourier
coefficients in the homogeneous directions x, z on a wall-normal grid y
(Sec. 4.1).  Those databases are not available, so every input here is a
seeded stand-in with the same shapes and structure:

* wall-normal grid: Chebyshev-Gauss-Lobatto points y_j = -cos(pi j/(ny-1))
  on [-1, 1] (walls at j = 0 and j = ny-1, no ghost nodes);
* box: L_x = 4 pi, L_z = 2 pi (the paper's DNS box, Sec. 4.1);
* four fields u, v, w, p.  For every (snapshot, field, y) a complex Gaussian
  half spectrum c(k) with amplitude (1 + |k|^2)^(-5/6), |k| the physical
  wavenumber (2 pi m_x / L_x, 2 pi m_z / L_z); the (0,0) mode and both
  Nyquist lines (m_x = n_x/2, m_z = n_z/2) are zeroed; the real field is
  irfft2 of it, multiplied by (1 - y^2) so it vanishes at the walls;
* the mean profile U(y) = 1 - y^2 is added to u (v, w, p have zero mean);
* the coefficients handed to the GPU path are rfft2 of the physical field
  with the forward normalisation a_hat(k) = (1/(n_x n_z)) sum_x a(x) e^{-i k.x},
  laid out [snapshot][field][y][m_z][m_x], m_x = 0..n_x/2 (torch/numpy rfft2
  layout).

Seed of snapshot s of a workload with id `wid`: 1910_06409 + 1000*wid + s,
drawn with numpy's PCG64 (numpy.random.default_rng).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FIELDS = ("u", "v", "w", "p")
SEED_BASE = 1910_06409


@dataclasses.dataclass(frozen=True)
class Workload:
    """Grid and sample sizes of one synthetic channel workload."""

    name: str
    wid: int          # workload id, enters the seed
    nx: int
    nz: int
    ny: int
    nsnap: int
    Lx: float = 4.0 * math.pi
    Lz: float = 2.0 * math.pi
    nu: float = 1.0 / 200.0

    @property
    def nxh(self) -> int:
        return self.nx // 2 + 1

    @property
    def npair(self) -> int:
        return self.ny * (self.ny + 1) // 2


# The workloads: a tiny one (the oracle finishes it in seconds), the
# Re_tau~200-shaped one, and the grouped / Re_tau~1000-shaped ones.
TINY = Workload("tiny_32x32x33_s4", 1, 32, 32, 33, 4)
RETAU200 = Workload("retau200_256x256x129_s16", 2, 256, 256, 129, 16)
GROUP_A = Workload("group_128x128x65_s32", 4, 128, 128, 65, 32)
GROUP_B = Workload("group_256x256x129_s16", 4, 256, 256, 129, 16)
GROUP_C = Workload("group_384x384x193_s8", 4, 384, 384, 193, 8)
RETAU1000 = Workload("retau1000_512x512x257_s32", 5, 512, 512, 257, 32, nu=1.0 / 1000.0)
# a narrow case with the Re_tau~200 wall-normal grid and snapshot count, small
# enough for multi-pass profiler captures (a few GB on the device)
PROFILE = Workload("profile_32x32x129_s16", 6, 32, 32, 129, 16)
# the Re_tau~200 plane size and snapshot count with few wall-normal points:
# the transform, combine and stencil kernels see production shapes
PROFILE_PLANE = Workload("profile_256x256x17_s16", 7, 256, 256, 17, 16)

WORKLOADS = {w.name: w for w in (TINY, RETAU200, GROUP_A, GROUP_B, GROUP_C, RETAU1000, PROFILE, PROFILE_PLANE)}


def small(nx: int, nz: int, ny: int, nsnap: int, wid: int = 90, nu: float = 1.0 / 200.0,
          Lx: float = 4.0 * math.pi, Lz: float = 2.0 * math.pi) -> Workload:
    """A custom (test-sized) workload with the same generator."""
    return Workload(f"custom_{nx}x{nz}x{ny}_s{nsnap}_w{wid}", wid, nx, nz, ny, nsnap, Lx, Lz, nu)


def cgl_grid(ny: int) -> np.ndarray:
    """Chebyshev-Gauss-Lobatto points -cos(pi j/(ny-1)), j = 0..ny-1 (increasing)."""
    j = np.arange(ny, dtype=np.float64)
    y = -np.cos(np.pi * j / (ny - 1))
    # make the grid exactly antisymmetric and hit the walls exactly
    y = 0.5 * (y - y[::-1])
    return y


def _amplitude(wl: Workload) -> np.ndarray:
    mx = np.arange(wl.nxh, dtype=np.float64)
    mz = np.fft.fftfreq(wl.nz, d=1.0 / wl.nz)          # signed integer index
    kx = 2.0 * np.pi * mx / wl.Lx
    kz = 2.0 * np.pi * mz / wl.Lz
    k2 = kz[:, None] ** 2 + kx[None, :] ** 2
    amp = (1.0 + k2) ** (-5.0 / 6.0)
    amp[0, 0] = 0.0
    amp[:, wl.nx // 2] = 0.0                            # x Nyquist line
    amp[wl.nz // 2, :] = 0.0                            # z Nyquist line
    return amp


def snapshot_physical(wl: Workload, s: int) -> np.ndarray:
    """Physical fields of snapshot s, float64 [4][ny][nz][nx] (u includes U(y))."""
    rng = np.random.default_rng(SEED_BASE + 1000 * wl.wid + s)
    amp = _amplitude(wl)
    y = cgl_grid(wl.ny)
    shape = (4, wl.ny, wl.nz, wl.nxh)
    c = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * amp
    # irfft2 with the forward convention: a(x) = sum_k c(k) e^{i k.x}
    phys = np.fft.irfft2(c, s=(wl.nz, wl.nx), axes=(-2, -1), norm="forward")
    phys *= (1.0 - y * y)[None, :, None, None]
    phys[0] += (1.0 - y * y)[:, None, None]
    return phys


def to_coefficients(phys: np.ndarray) -> np.ndarray:
    """rfft2 with forward normalisation over the last two axes (z, x)."""
    return np.fft.rfft2(phys, axes=(-2, -1), norm="forward")


def snapshot_coefficients(wl: Workload, s: int) -> np.ndarray:
    """complex128 [4][ny][nz][nx/2+1] coefficients of snapshot s."""
    return to_coefficients(snapshot_physical(wl, s))


def physical(wl: Workload, nsnap: int | None = None) -> np.ndarray:
    n = wl.nsnap if nsnap is None else nsnap
    return np.stack([snapshot_physical(wl, s) for s in range(n)])


def coefficients(wl: Workload, nsnap: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
    """complex128 [nsnap][4][ny][nz][nx/2+1]; `out` may be a preallocated (pinned) array."""
    n = wl.nsnap if nsnap is None else nsnap
    if out is None:
        out = np.empty((n, 4, wl.ny, wl.nz, wl.nxh), dtype=np.complex128)
    for s in range(n):
        out[s] = snapshot_coefficients(wl, s)
    return out


def snapshot_vorticity(wl: Workload, s: int):
    """Inputs of Step 1 for velocity-vorticity databases, snapshot s:
    (v_eta complex128 [2][ny][nz][nx/2+1], mean_uw float64 [2][ny]).

    v and eta are drawn like the fields above (random half spectra with the
    same amplitude, irfft2, then a wall envelope): v with (1 - y^2)^2 (v and
    dv/dy vanish at no-slip walls), eta with (1 - y^2).  The plane averages of
    u and w are (1 - y^2)(1 + 0.05 g_j) and 0.02 (1 - y^2) h_j with standard
    normal g_j, h_j.  Seed: 1910_06409 + 1000*wid + 500 + s."""
    rng = np.random.default_rng(SEED_BASE + 1000 * wl.wid + 500 + s)
    amp = _amplitude(wl)
    y = cgl_grid(wl.ny)
    shape = (2, wl.ny, wl.nz, wl.nxh)
    c = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * amp
    phys = np.fft.irfft2(c, s=(wl.nz, wl.nx), axes=(-2, -1), norm="forward")
    env = 1.0 - y * y
    phys[0] *= (env * env)[:, None, None]
    phys[1] *= env[:, None, None]
    mean_uw = np.stack([env * (1.0 + 0.05 * rng.standard_normal(wl.ny)),
                        0.02 * env * rng.standard_normal(wl.ny)])
    return to_coefficients(phys), mean_uw


def vorticity_inputs(wl: Workload, nsnap: int | None = None):
    """(v_eta [nsnap][2][ny][nz][nx/2+1], mean_uw [nsnap][2][ny]) of snapshots 0..nsnap-1."""
    n = wl.nsnap if nsnap is None else nsnap
    pairs = [snapshot_vorticity(wl, s) for s in range(n)]
    return np.stack([a for a, _ in pairs]), np.stack([b for _, b in pairs])


def single_mode_fields(nx: int, nz: int, ny: int, nsnap: int, modes, Lx: float, Lz: float,
                       mean_u=None) -> np.ndarray:
    """Physical fields built from a few Fourier modes with y-dependent amplitudes.

    `modes` is a list of (field_index, mx, mz, amp_fn, phase_per_snapshot)
    where amp_fn(y) gives the y profile and phase_per_snapshot[s] the phase.
    field(x, y, z) += amp_fn(y) * cos(2 pi mx x/Lx + 2 pi mz z/Lz + phase).
    Used by closed-form tests of the oracle.
    """
    y = cgl_grid(ny)
    x = np.arange(nx) * (Lx / nx)
    z = np.arange(nz) * (Lz / nz)
    out = np.zeros((nsnap, 4, ny, nz, nx))
    for (f, mx, mz, amp_fn, phases) in modes:
        a = amp_fn(y)
        for s in range(nsnap):
            arg = (2 * np.pi * mx / Lx) * x[None, :] + (2 * np.pi * mz / Lz) * z[:, None] + phases[s]
            out[s, f] += a[:, None, None] * np.cos(arg)[None, :, :]
    if mean_u is not None:
        out[:, 0] += mean_u(y)[None, :, None, None]
    return out


# ------------------------------------------------ one homogeneous direction
#
# Stand-ins for a flow homogeneous in x only (a straight duct): the cross
# section [-1, 1] x [-1, 1] is sampled on Chebyshev-Gauss-Lobatto grids in y
# and z (walls at both ends of each).  For every (snapshot, field, y, z) a
# complex Gaussian half spectrum in x with amplitude (1 + kx^2)^(-5/6),
# kx = 2 pi m_x / L_x; the m_x = 0 mode and the Nyquist mode are zeroed; the
# real field is irfft of it, times the wall envelope (1 - y^2)(1 - z^2).
# Mean flow: U = (1 - y^2)(1 - z^2) on u, and a weak cross-flow
# V = 0.02 z (1 - y^2)(1 - z^2), W = 0.02 y (1 - y^2)(1 - z^2) (so that every
# mean-flow term is exercised; the fields are not Navier-Stokes solutions).
# Coefficients for the GPU path: rfft over x with the forward normalisation,
# [snapshot][field][y][z][m_x].  Seed of snapshot s: 1910_06409 + 1000*wid +
# 700 + s (numpy PCG64).

@dataclasses.dataclass(frozen=True)
class DuctWorkload:
    """Grid and sample sizes of one synthetic flow homogeneous in x only."""

    name: str
    wid: int
    nx: int
    ny: int
    nz: int
    nsnap: int
    Lx: float = 4.0 * math.pi
    nu: float = 1.0 / 200.0

    @property
    def nxh(self) -> int:
        return self.nx // 2 + 1

    @property
    def npoint(self) -> int:
        return self.ny * self.nz

    @property
    def npair(self) -> int:
        return self.npoint * (self.npoint + 1) // 2


# a case the oracle finishes in seconds (several 32-point tiles of the
# cross-section pairs and a ragged tail), and the benchmark's duct
DUCT_TINY = DuctWorkload("duct_16x9x7_s4", 11, 16, 9, 7, 4)
DUCT = DuctWorkload("duct_256x33x33_s16", 12, 256, 33, 33, 16)
# the benchmark's x grid and snapshot count on a 17 x 17 cross section: the
# spectra (0.7 GB) exceed L2, small enough for multi-pass profiler captures
DUCT_PROFILE = DuctWorkload("duct_256x17x17_s16", 13, 256, 17, 17, 16)
DUCT_WORKLOADS = {w.name: w for w in (DUCT_TINY, DUCT, DUCT_PROFILE)}


def duct_small(nx: int, ny: int, nz: int, nsnap: int, wid: int = 91, Lx: float = 4.0 * math.pi,
               nu: float = 1.0 / 200.0) -> DuctWorkload:
    """A custom (test-sized) duct workload with the same generator."""
    return DuctWorkload(f"duct_{nx}x{ny}x{nz}_s{nsnap}_w{wid}", wid, nx, ny, nz, nsnap, Lx, nu)


def duct_snapshot_physical(wl: DuctWorkload, s: int) -> np.ndarray:
    """Physical fields of snapshot s, float64 [4][ny][nz][nx] (mean flow included)."""
    rng = np.random.default_rng(SEED_BASE + 1000 * wl.wid + 700 + s)
    kx = 2.0 * np.pi * np.arange(wl.nxh) / wl.Lx
    amp = (1.0 + kx * kx) ** (-5.0 / 6.0)
    amp[0] = 0.0
    amp[wl.nx // 2] = 0.0
    shape = (4, wl.ny, wl.nz, wl.nxh)
    c = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * amp
    phys = np.fft.irfft(c, n=wl.nx, axis=-1, norm="forward")
    y = cgl_grid(wl.ny)[:, None]
    z = cgl_grid(wl.nz)[None, :]
    env = (1.0 - y * y) * (1.0 - z * z)
    phys *= env[None, :, :, None]
    phys[0] += env[:, :, None]
    phys[1] += (0.02 * z * env)[:, :, None]
    phys[2] += (0.02 * y * env)[:, :, None]
    return phys


def duct_physical(wl: DuctWorkload, nsnap: int | None = None) -> np.ndarray:
    n = wl.nsnap if nsnap is None else nsnap
    return np.stack([duct_snapshot_physical(wl, s) for s in range(n)])


def duct_coefficients(wl: DuctWorkload, nsnap: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
    """complex128 [nsnap][4][ny][nz][nx/2+1]: rfft over x, forward normalisation."""
    n = wl.nsnap if nsnap is None else nsnap
    if out is None:
        out = np.empty((n, 4, wl.ny, wl.nz, wl.nxh), dtype=np.complex128)
    for s in range(n):
        out[s] = np.fft.rfft(duct_snapshot_physical(wl, s), axis=-1, norm="forward")
    return out
