"""Pin of the oracle's assembled terms where the third-order moments enter.

The fluxes of the GKE carry third-order increment moments: the turbulent
scale flux <du^2 du_j> in Phi_j (Eq. 4) and the turbulent spatial flux
<v* du^2> in phi (Eq. 5), and the budget residual of Eq. 3 differentiates
both.  A single Fourier mode has no third-order moments, so the single-mode
closed forms cannot see how these enter the terms.  Here a wavenumber triad
(k_c = k_a + k_b) gives them non-zero values, and every moment is computed
exactly by another route: each field is a finite sum of complex
exponentials, a field at the second plane is shifted by r, so the average
over x and z of a product keeps the exponentials whose x-wavenumbers cancel
and leaves an exact trigonometric sum in r.  Derivatives in r_x, r_z then
multiply coefficients by i k; derivatives in Y1, Y2 follow from the product
rule, the wall-normal profiles being linear in y.  The terms are then
assembled from these exact moments by the paper's definitions (Eq. 3-6,
with d/dr_y = (d_Y2 - d_Y1)/2 and d/dY = d_Y1 + d_Y2, Eq. 10-11) and compared
with the oracle's terms and residual at every pair and separation.

All profiles are polynomials of low degree (linear amplitudes, a quadratic
mean U), so the oracle's 5-point stencil is exact on every quantity it
differentiates and the comparison is to rounding.

A second test plants mistakes in copies of the oracle's source (a weight on a
third-order moment, swapped flux components, a swapped derivative in the
residual) and checks that this pin catches each of them.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic as S

NX, NZ, NY, NS = 6, 4, 5, 3
LX, LZ, NU = 4 * math.pi, 2 * math.pi, 1.0 / 200.0
MODES = ((1, 0), (0, 1), (1, 1))          # k_c = k_a + k_b


# ------------------------------------------------- exact exponential sums
def _prod(X, Y):
    """Product of two exponential sums keyed (kx, kz, rkx, rkz)."""
    out = {}
    for (a, b, c, d), v in X.items():
        for (e, f, g, h), w in Y.items():
            k = (a + e, b + f, c + g, d + h)
            out[k] = out.get(k, 0) + v * w
    return out


def _add(*Xs, scale=None):
    out = {}
    for i, X in enumerate(Xs):
        s = 1.0 if scale is None else scale[i]
        for k, v in X.items():
            out[k] = out.get(k, 0) + s * v
    return out


def _mean(X, *Ys):
    """Average over x, z of X * Y1 * ...: an exponential sum in r keyed (rkx, rkz)."""
    P = X
    for Y in Ys:
        P = _prod(P, Y)
    out = {}
    for (a, b, c, d), v in P.items():
        if a == 0 and b == 0:
            out[(c, d)] = out.get((c, d), 0) + v
    return out


def _on_grid(R, nrx=0, nrz=0):
    """Value of an r-sum (optionally its nrx-th r_x and nrz-th r_z derivative)
    at the separations (m_z, m_x) of the grid, r = (m_x LX/NX, m_z LZ/NZ)."""
    mz = np.arange(NZ)[:, None]
    mx = np.arange(NX)[None, :]
    out = np.zeros((NZ, NX), dtype=complex)
    for (c, d), v in R.items():
        kx, kz = 2 * math.pi * c / LX, 2 * math.pi * d / LZ
        out += v * (1j * kx) ** nrx * (1j * kz) ** nrz * np.exp(2j * math.pi * (c * mx / NX + d * mz / NZ))
    assert np.abs(out.imag).max() < 1e-12 * max(1.0, np.abs(out.real).max())
    return out.real


class TriadCase:
    """u, v, w, p = sum over the triad of a(y) cos(k.x + phase), a(y) linear in
    y, plus per-snapshot plane means of v (linear in y, zero over the
    ensemble) and the mean flow U = 1 - y^2 in u."""

    def __init__(self, seed=11):
        rng = np.random.default_rng(seed)
        self.amp = rng.uniform(0.3, 1.0, size=(4, 3, 2))      # [field][mode][a0, a1]
        self.phs = rng.uniform(-math.pi, math.pi, size=(NS, 4, 3))
        off = rng.standard_normal((NS, 2))
        self.off = off - off.mean(axis=0, keepdims=True)      # v offsets o0 + o1 y, zero mean over snapshots
        self.y = S.cgl_grid(NY)
        self.U = lambda y: 1.0 - y * y
        self.dU = lambda y: -2.0 * y

    def physical(self):
        x = np.arange(NX) * LX / NX
        z = np.arange(NZ) * LZ / NZ
        phys = np.zeros((NS, 4, NY, NZ, NX))
        for s in range(NS):
            for f in range(4):
                for j, yj in enumerate(self.y):
                    for m, (mx, mz) in enumerate(MODES):
                        a = self.amp[f, m, 0] + self.amp[f, m, 1] * yj
                        th = 2 * math.pi * mx / LX * x[None, :] + 2 * math.pi * mz / LZ * z[:, None]
                        phys[s, f, j] += a * np.cos(th + self.phs[s, f, m])
                    if f == 1:
                        phys[s, f, j] += self.off[s, 0] + self.off[s, 1] * yj
        phys[:, 0] += self.U(self.y)[None, :, None, None]
        return phys

    def field(self, s, f, Y, second, dy=False, dx=0, dz=0):
        """Fluctuation f of snapshot s at wall-normal position Y as an
        exponential sum; second: at the second point (shifted by r); dy: its
        y-derivative; dx, dz: orders of x / z derivatives."""
        T = {}
        for m, (mx, mz) in enumerate(MODES):
            a = self.amp[f, m, 1] if dy else self.amp[f, m, 0] + self.amp[f, m, 1] * Y
            for sg in (1, -1):
                kx, kz = sg * mx, sg * mz
                c = 0.5 * a * np.exp(1j * sg * self.phs[s, f, m])
                c *= (1j * 2 * math.pi * kx / LX) ** dx * (1j * 2 * math.pi * kz / LZ) ** dz
                key = (kx, kz, kx, kz) if second else (kx, kz, 0, 0)
                T[key] = T.get(key, 0) + c
        if f == 1 and dx == 0 and dz == 0:
            o = self.off[s, 1] if dy else self.off[s, 0] + self.off[s, 1] * Y
            T[(0, 0, 0, 0)] = T.get((0, 0, 0, 0), 0) + o
        return T

    def eps(self, Y):
        """Pseudo-dissipation nu <d_j u_i d_j u_i> at Y, exactly."""
        acc = 0.0
        for s in range(NS):
            for i in range(3):
                for d in ({"dx": 1}, {"dz": 1}, {"dy": True}):
                    g = self.field(s, i, Y, False, **d)
                    acc += _mean(g, g).get((0, 0), 0).real
        return NU * acc / NS

    def moments(self, Y1, Y2):
        """Exact r-sums of the increment moments and their Y1 / Y2 derivatives."""
        acc = {}

        def put(name, R):
            acc[name] = _add(acc.get(name, {}), R)

        for s in range(NS):
            f1 = [self.field(s, f, Y1, False) for f in range(4)]
            f2 = [self.field(s, f, Y2, True) for f in range(4)]
            g1 = [self.field(s, f, Y1, False, dy=True) for f in range(4)]   # d/dY1 of f1
            g2 = [self.field(s, f, Y2, True, dy=True) for f in range(4)]    # d/dY2 of f2
            d = [_add(f2[f], f1[f], scale=(1.0, -1.0)) for f in range(4)]   # increments
            m1 = [{k: -v for k, v in g.items()} for g in g1]               # d/dY1 of the increments
            vs = _add(f1[1], f2[1], scale=(0.5, 0.5))                       # v*
            vs1, vs2 = {k: 0.5 * v for k, v in g1[1].items()}, {k: 0.5 * v for k, v in g2[1].items()}
            q = _add(*[_prod(d[i], d[i]) for i in range(3)])
            q1 = _add(*[_prod(d[i], m1[i]) for i in range(3)], scale=(2.0, 2.0, 2.0))   # dq/dY1
            q2 = _add(*[_prod(d[i], g2[i]) for i in range(3)], scale=(2.0, 2.0, 2.0))   # dq/dY2
            put("A", _mean(q))
            put("A_1", _mean(q1))
            put("A_2", _mean(q2))
            # second derivatives of A (the increments are linear in Y1 and Y2)
            put("A_11", _add(*[_mean(m1[i], m1[i]) for i in range(3)], scale=(2.0, 2.0, 2.0)))
            put("A_22", _add(*[_mean(g2[i], g2[i]) for i in range(3)], scale=(2.0, 2.0, 2.0)))
            put("A_12", _add(*[_mean(m1[i], g2[i]) for i in range(3)], scale=(2.0, 2.0, 2.0)))
            for j, nm in enumerate(("Bx", "By", "Bz")):
                put(nm, _mean(q, d[j]))
            put("By_1", _add(_mean(q1, d[1]), _mean(q, m1[1])))
            put("By_2", _add(_mean(q2, d[1]), _mean(q, g2[1])))
            put("C", _mean(vs, q))
            put("C_1", _add(_mean(vs1, q), _mean(vs, q1)))
            put("C_2", _add(_mean(vs2, q), _mean(vs, q2)))
            put("P", _mean(d[3], d[1]))
            put("P_1", _add(_mean(m1[3], d[1]), _mean(d[3], m1[1])))
            put("P_2", _add(_mean(g2[3], d[1]), _mean(d[3], g2[1])))
            put("Q", _mean(d[0], d[1]))
            put("R", _mean(d[0], vs))
        return {k: {kk: vv / NS for kk, vv in v.items()} for k, v in acc.items()}

    def terms(self, i1, i2):
        """A, Phi_x, Phi_y, Phi_z, phi, xi and the Eq. 3 residual at pair
        (i1, i2) on the separation grid, assembled from the exact moments by
        the paper's definitions."""
        Y1, Y2 = self.y[i1], self.y[i2]
        M = self.moments(Y1, Y2)
        g = lambda n, **kw: _on_grid(M[n], **kw)
        dU = self.U(Y2) - self.U(Y1)
        dUs, ddU = 0.5 * (self.dU(Y1) + self.dU(Y2)), self.dU(Y2) - self.dU(Y1)
        A = g("A")
        Phix = g("Bx") + A * dU - 2 * NU * g("A", nrx=1)                        # Eq. 4
        Phiy = g("By") - 2 * NU * 0.5 * (g("A_2") - g("A_1"))                   # Eq. 4, d/dr_y (Eq. 10)
        Phiz = g("Bz") - 2 * NU * g("A", nrz=1)                                 # Eq. 4
        phi = g("C") + 2 * g("P") - 0.5 * NU * (g("A_1") + g("A_2"))            # Eq. 5, d/dY (Eq. 11)
        xi = -2 * g("Q") * dUs - 2 * g("R") * ddU - 4 * 0.5 * (self.eps(Y1) + self.eps(Y2))   # Eq. 6
        # Eq. 3: d_rx Phi_x + d_ry Phi_y + d_rz Phi_z + d_Y phi - xi
        dPhix = g("Bx", nrx=1) + dU * g("A", nrx=1) - 2 * NU * g("A", nrx=2)
        dPhiz = g("Bz", nrz=1) - 2 * NU * g("A", nrz=2)
        dPhiy = 0.5 * (g("By_2") - g("By_1")) - 0.5 * NU * (g("A_22") - 2 * g("A_12") + g("A_11"))
        dphi = (g("C_1") + g("C_2") + 2 * (g("P_1") + g("P_2"))
                - 0.5 * NU * (g("A_11") + 2 * g("A_12") + g("A_22")))
        res = dPhix + dPhiy + dPhiz + dphi - xi
        return [A, Phix, Phiy, Phiz, phi, xi, res], {n: g(n) for n in ("Bx", "By", "Bz", "C")}


@pytest.fixture(scope="module")
def triad():
    case = TriadCase()
    want = np.zeros((7, NY, NY, NZ, NX))
    third = {n: np.zeros((NY, NY, NZ, NX)) for n in ("Bx", "By", "Bz", "C")}
    for i1 in range(NY):
        for i2 in range(NY):
            t, b = case.terms(i1, i2)
            for k in range(7):
                want[k, i1, i2] = t[k]
            for n in third:
                third[n][i1, i2] = b[n]
    return case, case.physical(), want, third


def _term_errors(got, want):
    return [float(np.abs(got[k] - want[k]).max() / np.abs(want[k]).max()) for k in range(7)]


def test_triad_terms_and_residual(triad):
    case, phys, want, third = triad
    res = oracle.full(phys, case.y, LX, LZ, NU)
    errs = _term_errors(res["terms"], want)
    assert max(errs) < 1e-11, dict(zip(oracle.TERMS, errs))
    # the third-order moments carry a sizeable share of each flux here, so a
    # wrong weight on one of them cannot hide under the other parts
    for n, t in (("Bx", 1), ("By", 2), ("Bz", 3), ("C", 4)):
        assert np.abs(third[n]).max() > 0.2 * np.abs(want[t]).max(), n
    # the oracle's own components agree with the exact moments
    name = {n: i for i, n in enumerate(oracle.COMPONENTS)}
    for n, v in third.items():
        assert np.abs(res["comp"][name[n]] - v).max() < 1e-12 * np.abs(v).max()


# Planted mistakes: (description, text in the oracle's source, replacement)
MUTATIONS = [
    ("half weight of B_x in Phi_x", "t[T_PHIX] = cm[C_BX] +", "t[T_PHIX] = 0.5 * cm[C_BX] +"),
    ("B_y in place of B_x in Phi_x", "t[T_PHIX] = cm[C_BX] +", "t[T_PHIX] = cm[C_BY] +"),
    ("B_x in place of B_y in Phi_y", "t[T_PHIY] = cm[C_BY] -", "t[T_PHIY] = cm[C_BX] -"),
    ("sign of B_z in Phi_z", "t[T_PHIZ] = cm[C_BZ] -", "t[T_PHIZ] = -cm[C_BZ] -"),
    ("half weight of C in phi", "t[T_PHI] = cm[C_C] +", "t[T_PHI] = 0.5 * cm[C_C] +"),
    ("weight 1 on P in phi", "cm[C_C] + 2.0 * cm[C_P]", "cm[C_C] + cm[C_P]"),
    ("r_z derivative of Phi_x in the residual",
     "naive_deriv(fx + (long)z * nx, res + (long)z * nx, nx, 1, Lx, cx, sx)",
     "naive_deriv(fz + (long)z * nx, res + (long)z * nx, nx, 1, Lx, cx, sx)"),
]


def test_planted_mistakes_are_caught(triad, tmp_path):
    case, phys, want, _ = triad
    src = oracle.source_text()
    for i, (what, old, new) in enumerate(MUTATIONS):
        assert src.count(old) == 1, f"mutation site not found: {what}"
        lib = oracle.load_library(oracle.compile_source(src.replace(old, new), str(tmp_path / f"mut{i}.so")))
        res = oracle.full(phys, case.y, LX, LZ, NU, lib=lib)
        assert max(_term_errors(res["terms"], want)) > 1e-3, f"planted mistake not caught: {what}"
