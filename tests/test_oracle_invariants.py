"""Invariants of the GKE terms that hold for any field (checked on the oracle).

* zero increments: at r = 0 and Y1 = Y2 every increment vanishes, so every
  moment of increments is exactly zero (Sec. 2 definitions);
* r-inversion (Sec. 3.4): (Y1, Y2, r) -> (Y2, Y1, -r) swaps the two points,
  so <du^2>, <dp dv>, <du dv>, <v* du^2> are even and <du^2 du_j>, <du v*>,
  dA/dr are odd; hence Phi is odd and phi, xi even;
* r-average: with zero plane-mean fluctuations (the generator's), the mean
  over all separations of any two-point correlation vanishes, so the mean
  over r of <du^2> equals <u_i u_i>(Y1) + <u_i u_i>(Y2);
* the spot-check entry point reproduces the full evaluation;
* mirror sampling (Sec. 3.2 Step 2, Sec. 3.3): with each snapshot's mirror
  image added, the statistics are symmetric under the combined inversion of
  y and r, (Y1, Y2, r) -> (2h - Y2, 2h - Y1, -r), with the sign table the
  paper states: Phi_x, Phi_z and phi change sign, A, Phi_y and xi do not
  (nor does the residual, a sum of budget terms of one parity); U is even
  about the centreline and V odd.
"""
import numpy as np
import pytest

import oracle
import synthetic as S


@pytest.fixture(scope="module")
def case():
    wl = S.small(8, 6, 9, 2, wid=91)
    phys = S.physical(wl)
    y = S.cgl_grid(wl.ny)
    return wl, phys, y, oracle.full(phys, y, wl.Lx, wl.Lz, wl.nu)


def _neg(a):
    """index map r -> -r on the periodic separation grid (last two axes)."""
    return np.roll(a[..., ::-1, ::-1], shift=(1, 1), axis=(-2, -1))


def test_zero_increment(case):
    wl, phys, y, r = case
    c = r["comp"]
    name = {n: i for i, n in enumerate(oracle.COMPONENTS)}
    for n in ("A", "Bx", "By", "Bz", "C", "P", "Q", "R", "GxA", "GzA"):
        diag = np.array([c[name[n], j, j, 0, 0] for j in range(wl.ny)])
        assert np.abs(diag).max() < 1e-12 * max(1.0, np.abs(c[name[n]]).max()), n


def test_r_inversion(case):
    wl, phys, y, r = case
    c = r["comp"]
    t = r["terms"]
    name = {n: i for i, n in enumerate(oracle.COMPONENTS)}
    even = ("A", "C", "P", "Q")
    odd = ("Bx", "By", "Bz", "R", "GxA", "GzA")
    for n in even + odd:
        a = c[name[n]]
        swapped = _neg(np.swapaxes(a, 0, 1))
        sgn = 1.0 if n in even else -1.0
        assert np.abs(a - sgn * swapped).max() < 1e-12 * np.abs(a).max(), n
    for k, sgn in ((0, 1), (1, -1), (2, -1), (3, -1), (4, 1), (5, 1)):
        a = t[k]
        swapped = _neg(np.swapaxes(a, 0, 1))
        assert np.abs(a - sgn * swapped).max() < 1e-10 * np.abs(a).max(), oracle.TERMS[k]


def test_r_average_identity(case):
    wl, phys, y, r = case
    fl = phys - phys.mean(axis=(0, 3, 4), keepdims=True)
    q = (fl[:, :3] ** 2).sum(axis=1).mean(axis=(0, 2, 3))       # <u_i u_i>(y)
    A = r["comp"][0]
    mean_r = A.mean(axis=(2, 3))
    want = q[:, None] + q[None, :]
    assert np.abs(mean_r - want).max() < 1e-12 * want.max()


def test_points_match_full(case):
    wl, phys, y, r = case
    rng = np.random.default_rng(3)
    pts = np.stack([rng.integers(0, wl.ny, 20), rng.integers(0, wl.ny, 20),
                    rng.integers(0, wl.nz, 20), rng.integers(0, wl.nx, 20)], axis=1)
    p = oracle.points(phys, y, wl.Lx, wl.Lz, wl.nu, pts)
    for n, (i1, i2, mz, mx) in enumerate(pts):
        np.testing.assert_allclose(p["comp"][n], r["comp"][:, i1, i2, mz, mx], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(p["terms"][n], r["terms"][:6, i1, i2, mz, mx], rtol=1e-12, atol=1e-12)


SIGMA = (1, -1, 1, -1, -1, 1, 1)      # A, Phi_x, Phi_y, Phi_z, phi, xi, residual


def _combined_inversion(a):
    """T(-r; ny-1-i2, ny-1-i1) as an array over (i1, i2, m_z, m_x)."""
    return _neg(np.swapaxes(a[::-1, ::-1], 0, 1))


def test_mirror_sampling_symmetries(case):
    wl, phys, y, r = case
    m = oracle.full(phys, y, wl.Lx, wl.Lz, wl.nu, mirror=True)
    for k, sg in enumerate(SIGMA):
        a = m["terms"][k]
        assert np.abs(a - sg * _combined_inversion(a)).max() < 1e-10 * np.abs(a).max(), oracle.TERMS[k]
    prof = m["prof"]
    assert np.abs(prof[0] - prof[0][::-1]).max() < 1e-14        # U even
    assert np.abs(prof[1] + prof[1][::-1]).max() < 1e-14        # V odd
    assert np.abs(prof[5] - prof[5][::-1]).max() < 1e-12 * prof[5].max()
    # the synthetic sample alone is not symmetric: the check has teeth
    a = r["terms"][0]
    assert np.abs(a - _combined_inversion(a)).max() > 1e-3 * np.abs(a).max()


def test_mirror_of_mirrored_sample_is_plain(case):
    # a sample that already holds every snapshot's image is unchanged by mirror sampling
    wl, phys, y, r = case
    aug = oracle.mirror_augment(phys)
    a = oracle.full(aug, y, wl.Lx, wl.Lz, wl.nu)
    b = oracle.full(aug, y, wl.Lx, wl.Lz, wl.nu, mirror=True)
    for k in range(len(oracle.TERMS)):
        assert np.abs(a["terms"][k] - b["terms"][k]).max() <= 1e-12 * np.abs(a["terms"][k]).max()


def test_wedge_pairs():
    for ny in (5, 6, 9, 33):
        w = oracle.wedge_pairs(ny)
        assert len(w) == sum(ny - 2 * a for a in range((ny + 1) // 2))
        assert all(a <= b and a + b <= ny - 1 for a, b in w)
        assert w == sorted(w)
