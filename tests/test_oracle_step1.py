"""Pins of the Step-1 oracle for velocity-vorticity databases (Sec. 3.2, Step 1).

Each check compares the oracle with something other than itself: exact
derivatives of polynomials, the relations u, w must satisfy, a manufactured
solution of the Poisson problem, the closed-form pressure of the
Taylor-Green cell, and the gradient form of the Poisson source.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import fd_weights
from oracle import step1 as O

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _poly(coef, y, d=0):
    """Value of the d-th derivative of sum_p coef[p] y^p (coef along axis 0)."""
    c = np.asarray(coef)
    for _ in range(d):
        c = np.array([p * c[p] for p in range(1, len(c))]) if len(c) > 1 else np.zeros_like(c[:1])
    return sum(c[p] * y[(slice(None),) + (None,) * (c.ndim - 1)] ** p for p in range(len(c)))


@pytest.mark.parametrize("ny", [9, 17, 33])
def test_fd_weights2_exact_to_degree_four(ny):
    y = S.cgl_grid(ny)
    for j in range(ny):
        l0, w = O.fd_weights2(y, j)
        for p in range(5):
            f = y[l0:l0 + 5] ** p
            exact = p * (p - 1) * y[j] ** (p - 2) if p >= 2 else 0.0
            assert abs(w @ f - exact) <= 1e-9 * max(1.0, abs(exact)) * ny ** 2


def test_velocity_satisfies_continuity_and_vorticity():
    rng = np.random.default_rng(7)
    nx, nz, ny, Lx, Lz = 16, 12, 13, 4 * np.pi, 2 * np.pi
    nxh = nx // 2 + 1
    y = S.cgl_grid(ny)
    cv = rng.standard_normal((5, nz, nxh)) + 1j * rng.standard_normal((5, nz, nxh))
    ce = rng.standard_normal((5, nz, nxh)) + 1j * rng.standard_normal((5, nz, nxh))
    v, eta = _poly(cv, y), _poly(ce, y)
    dv = _poly(cv, y, 1)                     # exact dv/dy
    u00, w00 = rng.standard_normal(ny), rng.standard_normal(ny)
    u, w = O.velocity(v, eta, u00, w00, y, Lx, Lz, nx)
    kx, kz, _, _ = O.wavenumbers(nx, nz, Lx, Lz)
    KX, KZ = kx[None, None, :], kz[None, :, None]
    live = (KX ** 2 + KZ ** 2 > 0) & np.ones((ny, 1, 1), bool)
    scale = np.abs(dv).max()
    cont = 1j * KX * u + dv + 1j * KZ * w
    vort = 1j * KZ * u - 1j * KX * w - eta
    assert np.abs(cont[live]).max() < 1e-10 * scale
    assert np.abs(vort[live]).max() < 1e-10 * np.abs(eta).max()
    np.testing.assert_allclose(u[:, 0, 0], u00, rtol=0, atol=0)
    np.testing.assert_allclose(w[:, 0, 0], w00, rtol=0, atol=0)
    # Nyquist corners carry nothing
    assert np.all(u[:, nz // 2, nx // 2] == 0) and np.all(w[:, nz // 2, 0] == 0)


@pytest.mark.parametrize("k2", [0.0, 1.3, 40.0])
def test_poisson_manufactured_polynomial(k2):
    rng = np.random.default_rng(11)
    for ny in (9, 33):
        y = S.cgl_grid(ny)
        c = rng.standard_normal(5) + 1j * rng.standard_normal(5)
        p = _poly(c, y)
        rhs = _poly(c, y, 2) - k2 * p
        d1 = _poly(c, y, 1)
        sol = O.solve_poisson(rhs, d1[0], d1[-1], y, k2)
        want = p - p[0] if k2 == 0.0 else p
        assert np.abs(sol - want).max() < 1e-9 * np.abs(want).max() * ny


def test_taylor_green_pressure_closed_form():
    """u = g sin x cos z, w = -g cos x sin z, v = 0 (eta = -2 g sin x sin z):
    lap p = -d_i u_j d_j u_i = -g^2 (cos 2x + cos 2z), so p = g^2/4 (cos 2x + cos 2z)
    (the (0, 0) mode pinned to 0 at the first wall; dp/dy = 0 = nu d2v/dy2)."""
    nx = nz = 8
    ny, L, g, nu = 9, 2 * np.pi, 1.7, 0.01
    y = S.cgl_grid(ny)
    x = np.arange(nx) * L / nx
    z = np.arange(nz) * L / nz
    X, Z = np.meshgrid(x, z)                              # [nz][nx]
    eta = -2 * g * np.sin(X) * np.sin(Z)
    v_eta = np.zeros((1, 2, ny, nz, nx // 2 + 1), complex)
    v_eta[0, 1] = np.fft.rfft2(np.broadcast_to(eta, (ny, nz, nx)), axes=(-2, -1), norm="forward")
    mean_uw = np.zeros((1, 2, ny))
    out = O.step1(v_eta, mean_uw, y, L, L, nu, nx)
    phys = np.fft.irfft2(out[0], s=(nz, nx), axes=(-2, -1), norm="forward")
    np.testing.assert_allclose(phys[0], np.broadcast_to(g * np.sin(X) * np.cos(Z), phys[0].shape), atol=1e-12)
    np.testing.assert_allclose(phys[1], 0.0, atol=1e-14)
    np.testing.assert_allclose(phys[2], np.broadcast_to(-g * np.cos(X) * np.sin(Z), phys[2].shape), atol=1e-12)
    p_want = g * g / 4 * (np.cos(2 * X) + np.cos(2 * Z))
    np.testing.assert_allclose(phys[3], np.broadcast_to(p_want, phys[3].shape), atol=1e-11)


def test_poisson_source_equals_gradient_form():
    """For divergence-free fields whose y-profiles the 5-point stencils
    differentiate exactly (v, eta of degree <= 2, so u, w of degree <= 2 and
    their products of degree <= 4) and modes far from aliasing, the divergence
    form -d_i d_j (u_i u_j) equals the gradient form -d_i u_j d_j u_i."""
    rng = np.random.default_rng(3)
    nx, nz, ny, Lx, Lz = 16, 16, 11, 4 * np.pi, 2 * np.pi
    nxh = nx // 2 + 1
    y = S.cgl_grid(ny)
    mask = np.zeros((nz, nxh), bool)
    mask[:3, :3] = True
    mask[-2:, :3] = True
    cv = (rng.standard_normal((3, nz, nxh)) + 1j * rng.standard_normal((3, nz, nxh))) * mask
    ce = (rng.standard_normal((3, nz, nxh)) + 1j * rng.standard_normal((3, nz, nxh))) * mask
    # real fields: Hermitian kx = 0 column
    for c in (cv, ce):
        c[:, 1:, 0] = 0.5 * (c[:, 1:, 0] + np.conj(c[:, :0:-1, 0]))
        c[:, 0, 0] = c[:, 0, 0].real
    cv[1:, 0, 0] = 0.0                                    # continuity of the (0, 0) mode: v00 constant
    v, eta = _poly(cv, y), _poly(ce, y)
    u, w = O.velocity(v, eta, 0.3 + y * 0, 0.1 * y, y, Lx, Lz, nx)
    got = O.poisson_rhs(u, v, w, y, Lx, Lz, nx)
    kx, kz, _, _ = O.wavenumbers(nx, nz, Lx, Lz)
    KX, KZ = kx[None, None, :], kz[None, :, None]
    D1 = np.zeros((ny, ny))
    for j in range(ny):
        l0, wj = fd_weights(y, j)
        D1[j, l0:l0 + 5] = wj
    fields = (u, v, w)
    grads = {}                                            # grads[(i, j)] = d_i u_j, physical
    for jf, a in enumerate(fields):
        for i, da in enumerate((1j * KX * a, np.einsum("jl,lzx->jzx", D1, a), 1j * KZ * a)):
            grads[(i, jf)] = np.fft.irfft2(da, s=(nz, nx), axes=(-2, -1), norm="forward")
    q = sum(grads[(i, j)] * grads[(j, i)] for i in range(3) for j in range(3))
    want = -np.fft.rfft2(q, axes=(-2, -1), norm="forward")
    assert np.abs(got - want).max() < 1e-10 * np.abs(want).max()


def test_planted_mistakes_are_caught():
    """Each plausible slip in the Step-1 oracle fails one of the pins above."""
    rng = np.random.default_rng(5)
    nx, nz, ny, L = 8, 8, 9, 2 * np.pi
    y = S.cgl_grid(ny)
    # sign of eta in the vorticity relation
    v = np.zeros((ny, nz, nx // 2 + 1), complex)
    eta = rng.standard_normal(v.shape) + 1j * rng.standard_normal(v.shape)
    u, w = O.velocity(v, -eta, np.zeros(ny), np.zeros(ny), y, L, L, nx)
    kx, kz, _, _ = O.wavenumbers(nx, nz, L, L)
    vort = 1j * kz[None, :, None] * u - 1j * kx[None, None, :] * w - eta
    assert np.abs(vort[:, 1:, 1:]).max() > 1e-3
    # a Neumann row with the wrong sign breaks the manufactured solution
    c = rng.standard_normal(5)
    p = _poly(c, y)
    d1 = _poly(c, y, 1)
    bad = O.solve_poisson(_poly(c, y, 2) - 2.0 * p, -d1[0], d1[-1], y, 2.0)
    assert np.abs(bad - p).max() > 1e-3
