"""The synthetic channel inputs follow their stated recipe (no GKE arithmetic
here): Chebyshev-Gauss-Lobatto grid, vanishing fluctuations at the walls,
mean U(y) = 1 - y^2 carried by u only, zero (0,0) fluctuation mode and zero
Nyquist lines, coefficients of real fields, seeded reproducibility."""
import numpy as np
import pytest

import synthetic as S


@pytest.mark.parametrize("ny", [5, 9, 33, 129])
def test_cgl_grid(ny):
    y = S.cgl_grid(ny)
    j = np.arange(ny)
    assert y[0] == -1.0 and y[-1] == 1.0
    assert np.all(np.diff(y) > 0)
    assert np.array_equal(y, -y[::-1])                       # exactly symmetric
    assert np.allclose(y, -np.cos(np.pi * j / (ny - 1)), atol=1e-15)


def test_recipe_modes_mean_and_walls():
    wl = S.small(16, 8, 9, 2, wid=400)
    phys = S.physical(wl)
    coef = S.coefficients(wl)
    y = S.cgl_grid(wl.ny)
    assert coef.shape == (2, 4, 9, 8, 9) and coef.dtype == np.complex128
    # coefficients are those of the physical fields (forward-normalised rfft2)
    assert np.allclose(coef, np.fft.rfft2(phys, axes=(-2, -1), norm="forward"), atol=1e-15)
    # plane means: U(y) = 1 - y^2 on u, zero on v, w, p
    assert np.allclose(coef[:, 0, :, 0, 0].real, 1 - y * y, atol=1e-14)
    assert np.abs(coef[:, 1:, :, 0, 0]).max() < 1e-15
    # Nyquist lines empty
    assert np.abs(coef[..., wl.nz // 2, :]).max() < 1e-15
    assert np.abs(coef[..., wl.nx // 2]).max() < 1e-15
    # no-slip: every field vanishes at the walls (u = U = 0 there too)
    assert np.abs(phys[:, :, 0]).max() < 1e-15 and np.abs(phys[:, :, -1]).max() < 1e-15


def test_seeded_and_distinct():
    wl = S.small(8, 8, 5, 3, wid=401)
    a, b = S.coefficients(wl), S.coefficients(wl)
    assert np.array_equal(a, b)                              # reproducible
    assert not np.allclose(a[0], a[1])                       # snapshots differ
    other = S.coefficients(S.small(8, 8, 5, 3, wid=402))
    assert not np.allclose(a, other)                         # workload id enters the seed
    assert np.array_equal(S.snapshot_coefficients(wl, 2), a[2])
