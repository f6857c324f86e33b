"""Pins of the CPU oracle against what the mathematics fixes.

The oracle (oracle/gke_oracle.c) evaluates the GKE terms as direct averages of
increment products (Sec. 2, Eq. 1-6).  These tests check it against
results obtained by other routes:

* a single Fourier mode per field with polynomial wall-normal profiles: every
  second-order moment has a hand-derived closed form (averages of products of
  two cosines), the 5-point FD stencil is exact on the profiles involved, so
  every term -- and the budget residual of Eq. 3 -- is known exactly;
* a wavenumber triad (k_c = k_a + k_b) whose third-order moments are computed
  exactly by expanding the fields in complex exponentials and keeping the
  zero-wavenumber part of each product;
* the FD weights against polynomials of degree <= 4.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic as S

P = np.polynomial.Polynomial


# --------------------------------------------------------------------- FD
@pytest.mark.parametrize("ny", [5, 9, 33, 129])
def test_fd_weights_exact_on_quartics(ny):
    y = S.cgl_grid(ny)
    rng = np.random.default_rng(7)
    for _ in range(3):
        poly = P(rng.standard_normal(5))
        dpoly = poly.deriv()
        for j in range(ny):
            l0, w = oracle.fd_weights(y, j)
            assert l0 == min(max(j - 2, 0), ny - 5)
            approx = float(np.dot(w, poly(y[l0:l0 + 5])))
            scale = np.abs(w).sum() * np.abs(poly(y)).max()
            assert abs(approx - dpoly(y[j])) <= 1e-13 * scale


def test_fd_weights_not_exact_on_quintic():
    # a 5-point first-derivative formula cannot be exact for y^5 on a generic grid
    y = S.cgl_grid(17)
    l0, w = oracle.fd_weights(y, 8)
    assert abs(np.dot(w, y[l0:l0 + 5] ** 5) - 5 * y[8] ** 4) > 1e-8


# ----------------------------------------------------- single-mode closed form
class Closed:
    """Closed forms for one Fourier mode per field.

    u_f = g_s a_f(y) cos(k.x + phi_s + ph_f), ph = (0, alpha, beta, gamma).
    Every second-order moment is a sum of terms  amp * f1(Y1) * f2(Y2) * c(r),
    c(r) = cos(k.r + delta) or 1; derivatives act on the factors.
    """

    def __init__(self, a, ph, k, G2, nu):
        self.a, self.ph, self.k, self.G2, self.nu = a, ph, k, G2, nu
        one = P([1.0])
        al, ga = ph[1], ph[3]
        au, av, ap = a[0], a[1], a[3]
        h = 0.5 * G2
        # (amp, f1, f2, delta or None)
        self.A = []
        for i in range(3):
            self.A += [(h, a[i] * a[i], one, None), (h, one, a[i] * a[i], None), (-G2, a[i], a[i], 0.0)]
        self.Q = [(h * math.cos(al), au * av, one, None), (h * math.cos(al), one, au * av, None),
                  (-h, au, av, al), (-h, av, au, -al)]
        self.R = [(0.5 * h, av, au, -al), (0.5 * h * math.cos(al), one, au * av, None),
                  (-0.5 * h * math.cos(al), au * av, one, None), (-0.5 * h, au, av, al)]
        self.P = [(h * math.cos(al - ga), ap * av, one, None), (h * math.cos(al - ga), one, ap * av, None),
                  (-h, ap, av, al - ga), (-h, av, ap, ga - al)]
        self.U = P([1.0, 0.0, -1.0])
        self.eps = sum((0.5 * (k[0] ** 2 + k[1] ** 2) * a[i] * a[i] + 0.5 * a[i].deriv() ** 2 for i in range(3)),
                       P([0.0])) * (nu * G2)

    def ev(self, terms, Y1, Y2, rx, rz, d1=0, d2=0, nrx=0, nrz=0):
        kx, kz = self.k
        kr = kx * rx + kz * rz
        out = np.zeros(np.broadcast(Y1, Y2, rx, rz).shape)
        for amp, f1, f2, dl in terms:
            if dl is None:
                if nrx or nrz:
                    continue
                c = 1.0
            else:
                c = kx ** nrx * kz ** nrz * np.cos(kr + dl + (nrx + nrz) * math.pi / 2)
            out = out + amp * f1.deriv(d1)(Y1) * f2.deriv(d2)(Y2) * c
        return out


def single_mode_case(nx=8, nz=6, ny=9, ns=3, mx=1, mz=2):
    Lx, Lz, nu = 4 * math.pi, 2 * math.pi, 1.0 / 200.0
    a = [P([1.0, 0.0, -1.0]), P([0.5, 0.3, -0.2]), P([0.8, 0.0, -0.4]), P([0.3, 0.6, 0.1])]
    ph = [0.0, 0.7, -1.1, 2.0]
    g = np.array([1.0, 0.7, 1.3, 0.9][:ns])
    phase_s = np.array([0.3, 1.9, -2.2, 0.8][:ns])
    y = S.cgl_grid(ny)
    x = np.arange(nx) * Lx / nx
    z = np.arange(nz) * Lz / nz
    kx, kz = 2 * math.pi * mx / Lx, 2 * math.pi * mz / Lz
    th = kx * x[None, :] + kz * z[:, None]
    phys = np.zeros((ns, 4, ny, nz, nx))
    for s in range(ns):
        for f in range(4):
            phys[s, f] = g[s] * a[f](y)[:, None, None] * np.cos(th + phase_s[s] + ph[f])[None]
    phys[:, 0] += (1 - y * y)[None, :, None, None]
    cf = Closed(a, ph, (kx, kz), float(np.mean(g * g)), nu)
    return phys, y, (Lx, Lz, nu), cf


@pytest.fixture(scope="module")
def single_mode():
    phys, y, (Lx, Lz, nu), cf = single_mode_case()
    res = oracle.full(phys, y, Lx, Lz, nu)
    ns, _, ny, nz, nx = phys.shape
    Y1 = y[:, None, None, None]
    Y2 = y[None, :, None, None]
    rx = (np.arange(nx) * Lx / nx)[None, None, None, :]
    rz = (np.arange(nz) * Lz / nz)[None, None, :, None]
    return res, cf, (Y1, Y2, rx, rz), nu


def _close(got, want, rtol=1e-11):
    scale = max(np.abs(want).max(), 1e-300)
    err = np.abs(got - want).max() / scale
    assert err < rtol, f"max rel err {err:.3e}"


def test_single_mode_profiles(single_mode):
    res, cf, (Y1, Y2, rx, rz), nu = single_mode
    y = Y1[:, 0, 0, 0]
    _close(res["prof"][0], cf.U(y))
    _close(res["prof"][4], cf.U.deriv()(y))
    _close(res["prof"][5], cf.eps(y))
    for f in (1, 2, 3):
        assert np.abs(res["prof"][f]).max() < 1e-14


def test_single_mode_second_order(single_mode):
    res, cf, g, nu = single_mode
    c = res["comp"]
    name = {n: i for i, n in enumerate(oracle.COMPONENTS)}
    _close(c[name["A"]], cf.ev(cf.A, *g))
    _close(c[name["Q"]], cf.ev(cf.Q, *g))
    _close(c[name["R"]], cf.ev(cf.R, *g))
    _close(c[name["P"]], cf.ev(cf.P, *g))
    _close(c[name["GxA"]], cf.ev(cf.A, *g, nrx=1))
    _close(c[name["GzA"]], cf.ev(cf.A, *g, nrz=1))
    _close(c[name["dY1A"]], cf.ev(cf.A, *g, d1=1), 1e-10)
    _close(c[name["dY2A"]], cf.ev(cf.A, *g, d2=1), 1e-10)
    # a single mode has no third-order moments
    for n in ("Bx", "By", "Bz", "C"):
        assert np.abs(c[name[n]]).max() < 1e-13


def closed_terms(cf, g, nu):
    """The six terms and the Eq. 3 residual of a single-mode case, in closed form."""
    Y1, Y2 = g[0], g[1]
    A = cf.ev(cf.A, *g)
    dU = cf.U(Y2) - cf.U(Y1)
    dUp1, dUp2 = cf.U.deriv()(Y1), cf.U.deriv()(Y2)
    A1, A2 = cf.ev(cf.A, *g, d1=1), cf.ev(cf.A, *g, d2=1)
    Phix = A * dU - 2 * nu * cf.ev(cf.A, *g, nrx=1)
    Phiy = -2 * nu * 0.5 * (A2 - A1)
    Phiz = -2 * nu * cf.ev(cf.A, *g, nrz=1)
    phi = 2 * cf.ev(cf.P, *g) - 0.5 * nu * (A1 + A2)
    xi = (-2 * cf.ev(cf.Q, *g) * 0.5 * (dUp1 + dUp2) - 2 * cf.ev(cf.R, *g) * (dUp2 - dUp1)
          - 2 * (cf.eps(Y1) + cf.eps(Y2)))
    # Eq. 3 residual: d_rx Phi_x + d_rz Phi_z + d_ry Phi_y + d_Y phi - xi, all derivatives exact here
    A11 = cf.ev(cf.A, *g, d1=2)
    A22 = cf.ev(cf.A, *g, d2=2)
    A12 = cf.ev(cf.A, *g, d1=1, d2=1)
    dPhix = dU * cf.ev(cf.A, *g, nrx=1) - 2 * nu * cf.ev(cf.A, *g, nrx=2)
    dPhiz = -2 * nu * cf.ev(cf.A, *g, nrz=2)
    dPhiy = -0.5 * nu * (A22 - 2 * A12 + A11)
    dphi = 2 * (cf.ev(cf.P, *g, d1=1) + cf.ev(cf.P, *g, d2=1)) - 0.5 * nu * (A11 + 2 * A12 + A22)
    resid = dPhix + dPhiz + dPhiy + dphi - xi
    return [A, Phix, Phiy, Phiz, phi, xi, resid]


TERM_RTOL = (1e-11, 1e-11, 1e-10, 1e-11, 1e-10, 1e-11, 1e-9)


def test_single_mode_terms_and_residual(single_mode):
    res, cf, g, nu = single_mode
    for k, want in enumerate(closed_terms(cf, g, nu)):
        _close(res["terms"][k], want, TERM_RTOL[k])


def test_mirror_sampling_single_mode():
    # Mirror sampling (Sec. 3.2, Step 2) doubles the sample with each
    # snapshot's image about the centreline.  The image of the single-mode
    # field has the reflected profiles a_f(-y), v's with its sign changed; the
    # ensemble mean U = 1 - y^2 is already even, so every term is the average
    # of the closed forms of the two profile sets.
    phys, y, (Lx, Lz, nu), cf = single_mode_case()
    res = oracle.full(phys, y, Lx, Lz, nu, mirror=True)

    def reflect(q):
        return P(q.coef * (-1.0) ** np.arange(len(q.coef)))

    a_img = [reflect(cf.a[0]), -reflect(cf.a[1]), reflect(cf.a[2]), reflect(cf.a[3])]
    cf_img = Closed(a_img, cf.ph, cf.k, cf.G2, nu)
    ns, _, ny, nz, nx = phys.shape
    g = (y[:, None, None, None], y[None, :, None, None], (np.arange(nx) * Lx / nx)[None, None, None, :],
         (np.arange(nz) * Lz / nz)[None, None, :, None])
    for k, (w0, w1) in enumerate(zip(closed_terms(cf, g, nu), closed_terms(cf_img, g, nu))):
        _close(res["terms"][k], 0.5 * (w0 + w1), TERM_RTOL[k])
    _close(res["prof"][5], 0.5 * (cf.eps(y) + cf_img.eps(y)))
    # the plain evaluation differs: the pin has teeth
    plain = oracle.full(phys, y, Lx, Lz, nu)
    assert np.abs(plain["terms"][5] - res["terms"][5]).max() > 1e-3 * np.abs(res["terms"][5]).max()


# ------------------------------------------------------ triad: third order
class Trig:
    """Finite sum of complex exponentials sum_k c_k e^{i k.x} on the periodic box."""

    def __init__(self, d=None):
        self.d = dict(d or {})

    def __add__(self, o):
        d = dict(self.d)
        for k, v in o.d.items():
            d[k] = d.get(k, 0) + v
        return Trig(d)

    def __sub__(self, o):
        return self + o.scale(-1.0)

    def scale(self, s):
        return Trig({k: s * v for k, v in self.d.items()})

    def __mul__(self, o):
        d = {}
        for k1, v1 in self.d.items():
            for k2, v2 in o.d.items():
                k = (k1[0] + k2[0], k1[1] + k2[1])
                d[k] = d.get(k, 0) + v1 * v2
        return Trig(d)

    def shift(self, rx, rz, Lx, Lz):
        return Trig({k: v * np.exp(1j * (2 * math.pi * k[0] / Lx * rx + 2 * math.pi * k[1] / Lz * rz))
                     for k, v in self.d.items()})

    def mean(self):
        return self.d.get((0, 0), 0.0).real


def test_triad_third_order_and_mean_offsets():
    nx, nz, ny, ns = 6, 4, 5, 3
    Lx, Lz, nu = 4 * math.pi, 2 * math.pi, 1.0 / 200.0
    modes = [(1, 0), (0, 1), (1, 1)]     # k_c = k_a + k_b
    rng = np.random.default_rng(11)
    amp = rng.uniform(0.3, 1.0, size=(4, 3, 2))        # [field][mode][poly coef], linear in y
    phs = rng.uniform(-math.pi, math.pi, size=(ns, 4, 3))
    off = rng.standard_normal((ns, ny))                  # per-snapshot plane means of v ...
    off -= off.mean(axis=0, keepdims=True)               # ... that cancel in the ensemble mean
    y = S.cgl_grid(ny)
    x = np.arange(nx) * Lx / nx
    z = np.arange(nz) * Lz / nz
    phys = np.zeros((ns, 4, ny, nz, nx))
    trig = [[[None] * ny for _ in range(4)] for _ in range(ns)]
    for s in range(ns):
        for f in range(4):
            for j in range(ny):
                T = Trig()
                for m, (mx, mz) in enumerate(modes):
                    a = amp[f, m, 0] + amp[f, m, 1] * y[j]
                    th = 2 * math.pi * mx / Lx * x[None, :] + 2 * math.pi * mz / Lz * z[:, None]
                    phys[s, f, j] += a * np.cos(th + phs[s, f, m])
                    T = T + Trig({(mx, mz): 0.5 * a * np.exp(1j * phs[s, f, m]),
                                  (-mx, -mz): 0.5 * a * np.exp(-1j * phs[s, f, m])})
                if f == 1:
                    phys[s, f, j] += off[s, j]
                    T = T + Trig({(0, 0): off[s, j]})
                trig[s][f][j] = T
    res = oracle.full(phys, y, Lx, Lz, nu)
    comp = res["comp"]
    name = {n: i for i, n in enumerate(oracle.COMPONENTS)}
    want = {n: np.zeros((ny, ny, nz, nx)) for n in ("A", "Bx", "By", "Bz", "C", "P", "Q", "R")}
    for i1 in range(ny):
        for i2 in range(ny):
            for mz in range(nz):
                for mx in range(nx):
                    rx, rz = mx * Lx / nx, mz * Lz / nz
                    acc = dict.fromkeys(want, 0.0)
                    for s in range(ns):
                        f1 = [trig[s][f][i1] for f in range(4)]
                        f2 = [trig[s][f][i2].shift(rx, rz, Lx, Lz) for f in range(4)]
                        d = [f2[f] - f1[f] for f in range(4)]
                        vs = (f1[1] + f2[1]).scale(0.5)
                        q = d[0] * d[0] + d[1] * d[1] + d[2] * d[2]
                        acc["A"] += q.mean()
                        acc["Bx"] += (q * d[0]).mean()
                        acc["By"] += (q * d[1]).mean()
                        acc["Bz"] += (q * d[2]).mean()
                        acc["C"] += (vs * q).mean()
                        acc["P"] += (d[3] * d[1]).mean()
                        acc["Q"] += (d[0] * d[1]).mean()
                        acc["R"] += (d[0] * vs).mean()
                    for n in want:
                        want[n][i1, i2, mz, mx] = acc[n] / ns
    for n, w in want.items():
        _close(comp[name[n]], w, 1e-12)
    assert np.abs(want["Bx"]).max() > 1e-2 and np.abs(want["C"]).max() > 1e-2  # non-trivial case
