"""CPU oracle of Step 1 for velocity-vorticity databases (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the product (CUDA) path never does.

Step 1 (Sec. 3.2) derives the fields the GKE needs from what the database
stores.  DNS solvers in velocity-vorticity form (Kim, Moin & Moser) store the
wall-normal velocity v and the wall-normal vorticity eta = du/dz - dw/dx as
Fourier coefficients in x, z, plus the plane averages of u and w; Step 1 then
recovers u, w and solves the Poisson equation for the pressure.  The paper
names these operations but not their discretisation; the readings taken here
(the same ones the CUDA path implements) are:

* wavenumbers: kx = 2 pi mx / Lx, kz = 2 pi mz / Lz with the signed index m
  (m - n above n/2) for odd derivatives, 0 on the Nyquist lines; even
  (second) derivatives use the true square (2 pi n/2 / L)^2 on the Nyquist
  lines;
* d/dy: the 5-point finite-difference weights of the Step-3 stencils
  (``oracle.fd_weights``: exact on polynomials of degree <= 4, one-sided next
  to the walls); d2/dy2: 5-point weights on the same nodes, also exact to
  degree 4 (``fd_weights2``);
* u, w: for kx^2 + kz^2 > 0 the unique solution of continuity,
  i kx u + dv/dy + i kz w = 0, and of the definition of the vorticity,
  eta = i kz u - i kx w; the (0, 0) modes are the stored plane averages; the
  other modes with kx^2 + kz^2 = 0 (Nyquist corners) are zero;
* pressure: lap p = -d_i d_j (u_i u_j) (incompressible flow, rho = 1), the
  products u_i u_j of the total velocity formed on the collocation grid (no
  dealiasing), with Neumann conditions from the wall-normal momentum
  equation at no-slip walls, dp/dy = nu d2v/dy2; the singular (0, 0) problem
  has its first row replaced by p(y_0) = 0.

Every function cites the relation it restates; numpy's FFT and dense solver
serve as library steps.
"""
from __future__ import annotations

import numpy as np

from . import fd_weights


def fd_weights2(y: np.ndarray, j: int):
    """(l0, w[5]): second-derivative weights at row j on nodes l0..l0+4.

    The weights make sum_l w_l f(y_{l0+l}) equal f''(y_j) for every
    polynomial f of degree <= 4 (moment conditions, solved in the scaled
    variable t = (y - y_j) / h)."""
    ny = len(y)
    l0 = min(max(j - 2, 0), ny - 5)
    t = np.asarray(y[l0:l0 + 5], dtype=np.float64) - y[j]
    h = np.max(np.abs(t))
    V = np.vander(t / h, 5, increasing=True).T          # V[p][l] = (t_l / h)^p
    rhs = np.zeros(5)
    rhs[2] = 2.0                                        # d2/dt2 of t^2
    return l0, np.linalg.solve(V, rhs) / (h * h)


def _dmat(y: np.ndarray, order: int) -> np.ndarray:
    """Dense matrix of the 5-point d/dy (order 1) or d2/dy2 (order 2)."""
    ny = len(y)
    D = np.zeros((ny, ny))
    for j in range(ny):
        l0, w = fd_weights(y, j) if order == 1 else fd_weights2(y, j)
        D[j, l0:l0 + 5] = w
    return D


def _signed(n: int, m: np.ndarray) -> np.ndarray:
    """Signed index of FFT bins m, 0 on the Nyquist bin."""
    s = np.where(m > n // 2, m - n, m).astype(np.float64)
    if n % 2 == 0:
        s[m == n // 2] = 0.0
    return s


def wavenumbers(nx: int, nz: int, Lx: float, Lz: float):
    """(kx, kz, kx2, kz2): odd-derivative wavenumbers of the half spectrum
    (Nyquist 0) and the true squares for second derivatives."""
    mx = np.arange(nx // 2 + 1)
    mz = np.arange(nz)
    kx = 2 * np.pi * _signed(nx, mx) / Lx
    kz = 2 * np.pi * _signed(nz, mz) / Lz
    kx_true = 2 * np.pi * np.where(mx > nx // 2, mx - nx, mx) / Lx
    kz_true = 2 * np.pi * np.where(mz > nz // 2, mz - nz, mz) / Lz
    return kx, kz, kx_true ** 2, kz_true ** 2


def velocity(v: np.ndarray, eta: np.ndarray, u00: np.ndarray, w00: np.ndarray, y: np.ndarray,
             Lx: float, Lz: float, nx: int):
    """u, w of one snapshot from v, eta ([ny][nz][nx/2+1]) and the plane averages
    u00, w00 ([ny]): per mode with kx^2 + kz^2 > 0, the 2 x 2 system
        i kx u + i kz w = -dv/dy        (continuity)
        i kz u - i kx w = eta           (eta = du/dz - dw/dx)
    solved by numpy."""
    ny, nz, nxh = v.shape
    kx, kz, _, _ = wavenumbers(nx, nz, Lx, Lz)
    Dv = np.einsum("jl,lzx->jzx", _dmat(y, 1), v)
    u = np.zeros_like(v)
    w = np.zeros_like(v)
    for iz in range(nz):
        for ix in range(nxh):
            if kx[ix] ** 2 + kz[iz] ** 2 == 0.0:
                continue
            M = np.array([[1j * kx[ix], 1j * kz[iz]], [1j * kz[iz], -1j * kx[ix]]])
            b = np.stack([-Dv[:, iz, ix], eta[:, iz, ix]])
            sol = np.linalg.solve(M, b)
            u[:, iz, ix] = sol[0]
            w[:, iz, ix] = sol[1]
    u[:, 0, 0] = u00
    w[:, 0, 0] = w00
    return u, w


def poisson_matrix(y: np.ndarray, k2: float, D1=None, D2=None) -> np.ndarray:
    """The discrete operator d2/dy2 - k^2 with its boundary rows: rows 0 and
    ny-1 are the Neumann rows d/dy (the right-hand side there carries
    nu d2v/dy2); for k^2 = 0 row 0 is the pin p(y_0) = 0 instead."""
    ny = len(y)
    D1 = _dmat(y, 1) if D1 is None else D1
    L = (_dmat(y, 2) if D2 is None else D2) - k2 * np.eye(ny)
    L[0] = D1[0]
    L[-1] = D1[-1]
    if k2 == 0.0:
        L[0] = 0.0
        L[0, 0] = 1.0
    return L


def solve_poisson(rhs: np.ndarray, dp_lo, dp_hi, y: np.ndarray, k2: float, D1=None, D2=None) -> np.ndarray:
    """p with (d2/dy2 - k^2) p = rhs inside, dp/dy = dp_lo at y_0 and dp_hi at
    y_{ny-1} (dp_lo unused when k^2 = 0: p(y_0) = 0)."""
    b = np.array(rhs, dtype=np.complex128)
    b[0] = 0.0 if k2 == 0.0 else dp_lo
    b[-1] = dp_hi
    return np.linalg.solve(poisson_matrix(y, k2, D1, D2), b)


def poisson_rhs(u: np.ndarray, v: np.ndarray, w: np.ndarray, y: np.ndarray, Lx: float, Lz: float, nx: int):
    """Fourier coefficients of -d_i d_j (u_i u_j) for one snapshot: the six
    products of the total velocity on the nx x nz grid (numpy irfft2 / rfft2,
    forward normalisation), then d/dx -> i kx, d/dz -> i kz, d2/dx2 -> -kx^2,
    d2/dz2 -> -kz^2, d/dy and d2/dy2 by the 5-point weights."""
    ny, nz, nxh = u.shape
    kx, kz, kx2, kz2 = wavenumbers(nx, nz, Lx, Lz)
    phys = [np.fft.irfft2(a, s=(nz, nx), axes=(-2, -1), norm="forward") for a in (u, v, w)]
    prod = {}
    for a, b in ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)):
        prod[(a, b)] = np.fft.rfft2(phys[a] * phys[b], axes=(-2, -1), norm="forward")
    D1, D2 = _dmat(y, 1), _dmat(y, 2)
    KX, KZ = kx[None, None, :], kz[None, :, None]
    KX2, KZ2 = kx2[None, None, :], kz2[None, :, None]
    dd = (-KX2 * prod[(0, 0)] - KZ2 * prod[(2, 2)] + np.einsum("jl,lzx->jzx", D2, prod[(1, 1)])
          + 2 * (-KX * KZ) * prod[(0, 2)]
          + 2 * 1j * KX * np.einsum("jl,lzx->jzx", D1, prod[(0, 1)])
          + 2 * 1j * KZ * np.einsum("jl,lzx->jzx", D1, prod[(1, 2)]))
    return -dd


def pressure(u: np.ndarray, v: np.ndarray, w: np.ndarray, y: np.ndarray, Lx: float, Lz: float, nu: float,
             nx: int) -> np.ndarray:
    """p of one snapshot: per mode, solve_poisson with the right-hand side of
    poisson_rhs and the wall values dp/dy = nu d2v/dy2 (y-momentum at a
    no-slip wall)."""
    ny, nz, nxh = u.shape
    _, _, kx2, kz2 = wavenumbers(nx, nz, Lx, Lz)
    rhs = poisson_rhs(u, v, w, y, Lx, Lz, nx)
    D1, D2 = _dmat(y, 1), _dmat(y, 2)
    d2v = np.einsum("jl,lzx->jzx", D2, v)
    p = np.zeros_like(u)
    for iz in range(nz):
        for ix in range(nxh):
            k2 = kx2[ix] + kz2[iz]
            p[:, iz, ix] = solve_poisson(rhs[:, iz, ix], nu * d2v[0, iz, ix], nu * d2v[-1, iz, ix], y, k2, D1, D2)
    return p


def step1(v_eta: np.ndarray, mean_uw: np.ndarray, y: np.ndarray, Lx: float, Lz: float, nu: float,
          nx: int) -> np.ndarray:
    """Fields [nsnap][4][ny][nz][nx/2+1] (u, v, w, p) from v_eta
    [nsnap][2][ny][nz][nx/2+1] (v, eta) and mean_uw [nsnap][2][ny] (plane
    averages of u and w)."""
    v_eta = np.asarray(v_eta, dtype=np.complex128)
    ns = v_eta.shape[0]
    out = np.zeros((ns, 4) + v_eta.shape[2:], dtype=np.complex128)
    for s in range(ns):
        v, eta = v_eta[s, 0], v_eta[s, 1]
        u, w = velocity(v, eta, mean_uw[s, 0], mean_uw[s, 1], y, Lx, Lz, nx)
        out[s, 0], out[s, 1], out[s, 2] = u, v, w
        out[s, 3] = pressure(u, v, w, y, Lx, Lz, nu, nx)
    return out
