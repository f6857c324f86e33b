"""Pins of the CPU oracle for one homogeneous direction (oracle/gke1h_oracle.c).

Each check compares the oracle with something other than itself:
  * the channel: fields that do not depend on z, with the mean flow U(y) only,
    must give the channel oracle's terms (Sec. 2, Eq. 1-6) at every pair of
    cross-section points (pins x, y, the third-order moments, pressure,
    production by dU/dy and the dissipation);
  * the exchange of y and z (v <-> w, the y grid <-> the z grid) must map the
    terms onto each other (pins every z part against its y counterpart);
  * one x-mode with linear amplitudes and a linear mean flow in all three
    components: every moment is a closed form in r_x, Y1, Z1, Y2, Z2, hand
    derived from the mode's phase average; the terms and the residual follow
    from the definitions by exact differentiation (the stencils are exact on
    these polynomials) -- pins the mean-flow terms, the pressure term, the
    production by every mean gradient and the residual;
  * invariants: r-inversion parities, zero increments at coincident points;
  * planted mistakes in copies of the oracle's source each fail one of these.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic as S
from oracle import one_homog as O1

T = {n: i for i, n in enumerate(O1.TERMS)}


def _grid(n, seed):
    """a non-uniform increasing grid on [-1, 1]"""
    g = S.cgl_grid(n)
    rng = np.random.default_rng(seed)
    g[1:-1] += 0.1 * (g[2:] - g[:-2]) * (rng.random(n - 2) - 0.5)
    return g


def _random_fields(ns, nx, ny, nz, seed, mean=True):
    rng = np.random.default_rng(seed)
    phys = rng.standard_normal((ns, 4, ny, nz, nx))
    if mean:
        y = np.linspace(-1, 1, ny)[:, None]
        z = np.linspace(-1, 1, nz)[None, :]
        phys[:, 0] += ((1 - y * y) * (1 - z * z) * 3.0)[..., None]
        phys[:, 1] += (0.5 * y * z + 0.3 * z)[..., None]
        phys[:, 2] += (-0.4 * y + 0.2 * y * y + 0 * z)[..., None]
        phys[:, 3] += (y + z)[..., None]
    return phys


def _channel_case():
    ns, nx, ny, nzc = 3, 8, 7, 4
    rng = np.random.default_rng(2)
    g = rng.standard_normal((ns, 4, ny, nx))
    g[:, 1] -= g[:, 1].mean(axis=(0, 2), keepdims=True)      # no mean cross-flow
    g[:, 2] -= g[:, 2].mean(axis=(0, 2), keepdims=True)
    y = _grid(ny, 5)
    g[:, 0] += (1 - y * y)[None, :, None] * 2.0
    Lx, nu = 4 * math.pi, 0.01
    ch = oracle.full(np.repeat(g[:, :, :, None, :], nzc, axis=3), y, Lx, 2 * math.pi, nu)["terms"]
    return g, y, Lx, nu, ch


def _channel_errors(lib=None):
    """max relative difference per term between the one-direction oracle on
    z-independent fields (every pair of z positions) and the channel oracle"""
    g, y, Lx, nu, ch = _channel_case()
    ns, _, ny, nx = g.shape
    nz = 5
    z = _grid(nz, 6)
    one = O1.full(np.repeat(g[:, :, :, None, :], nz, axis=3), y, z, Lx, nu, lib=lib)["terms"]
    one = one.reshape(len(O1.TERMS), ny, nz, ny, nz, nx)
    pairs = {"A": "A", "Phi_x": "Phi_x", "Phi_y": "Phi_y", "Phi_z": "Phi_z", "phi": "psi_y", "xi": "xi",
             "residual": "residual"}
    errs = {}
    for cname, oname in pairs.items():
        want = ch[oracle.TERMS.index(cname)][:, :, 0, :]           # [i1][i2][mx], any m_z
        got = one[T[oname]].transpose(1, 3, 0, 2, 4)               # [iz1][iz2][i1][i2][mx]
        errs[cname] = float(np.abs(got - want[None, None]).max() / np.abs(want).max())
    return errs


def test_reduces_to_channel_for_z_independent_fields():
    for name, e in _channel_errors().items():
        assert e <= 1e-11, (name, e)


def _exchange_error(lib=None, terms=None):
    ns, nx, ny, nz = 3, 8, 7, 6
    phys = _random_fields(ns, nx, ny, nz, 9)
    y, z = _grid(ny, 1), _grid(nz, 2)
    Lx, nu = 3.0, 0.02
    a = O1.full(phys, y, z, Lx, nu, lib=lib)["terms"].reshape(8, ny, nz, ny, nz, nx)
    sw = phys[:, [0, 2, 1, 3]].transpose(0, 1, 3, 2, 4)        # u, w, v, p on (z, y)
    b = O1.full(sw, z, y, Lx, nu, lib=lib)["terms"].reshape(8, nz, ny, nz, ny, nx)
    b = b.transpose(0, 2, 1, 4, 3, 5)                           # back to (iy, iz) order
    swap = {"A": "A", "Phi_x": "Phi_x", "Phi_y": "Phi_z", "Phi_z": "Phi_y", "psi_y": "psi_z", "psi_z": "psi_y",
            "xi": "xi", "residual": "residual"}
    errs = {}
    for t, u in swap.items():
        scale = np.abs(a[T[t]]).max()
        assert scale > 0
        errs[t] = float(np.abs(b[T[u]] - a[T[t]]).max() / scale)
    return errs


def test_exchange_of_y_and_z():
    for name, e in _exchange_error().items():
        assert e <= 1e-11, (name, e)


# ------------------------------------------------------ single-mode closed form

def _closed_form_case():
    """One x-mode, amplitudes linear in (y, z), mean flow linear in (y, z)."""
    rng = np.random.default_rng(17)
    ns, nx, ny, nz = 4, 8, 6, 5
    Lx, nu, m = 2.5, 0.03, 1
    k = 2 * math.pi * m / Lx
    coef = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))   # a_f = c0 + c1 y + c2 z
    mean = rng.standard_normal((4, 3))                                      # U_f = m0 + m1 y + m2 z
    y, z = _grid(ny, 3), _grid(nz, 4)
    x = np.arange(nx) * Lx / nx
    Y, Z = np.meshgrid(y, z, indexing="ij")
    phys = np.zeros((ns, 4, ny, nz, nx))
    for s in range(ns):
        th = 2 * math.pi * s / ns
        for f in range(4):
            a = coef[f, 0] + coef[f, 1] * Y + coef[f, 2] * Z
            U = mean[f, 0] + mean[f, 1] * Y + mean[f, 2] * Z
            phys[s, f] = U[:, :, None] + np.real(a[:, :, None] * np.exp(1j * (k * x[None, None, :] + th)))
    return dict(phys=phys, y=y, z=z, Lx=Lx, nu=nu, k=k, coef=coef, mean=mean, nx=nx)


def _closed_form_terms(c):
    """The eight outputs of the closed form on every (p1, p2, m_x).

    With u_f = U_f + Re(a_f e^{i phi}), phi = k x + theta, the average over
    x and the snapshot phases of a product of two such waves is
    <Re(al e^{i phi}) Re(be e^{i phi})> = Re(al conj(be)) / 2, and of three
    waves 0.  With d_f = a_f(p2) e^{i k r} - a_f(p1) and s_f = a_f(p1) +
    a_f(p2) e^{i k r}: A = sum_i |d_i|^2 / 2, P_k = Re(d_p conj(d_k)) / 2,
    Q_ik = Re(d_i conj(d_k)) / 2, R_ik = Re(d_i conj(s_k)) / 4, B = C = 0,
    eps = nu sum_i (k^2 |a_i|^2 + |da_i/dy|^2 + |da_i/dz|^2) / 2.
    Derivatives are taken exactly (sympy)."""
    sp = pytest.importorskip("sympy")
    y1, z1, y2, z2, r = sp.symbols("y1 z1 y2 z2 r", real=True)
    k, nu, coef, mean = c["k"], c["nu"], c["coef"], c["mean"]
    E = sp.exp(sp.I * k * r)

    def amp(f, yy, zz):
        return sum(complex(coef[f, j]) * v for j, v in enumerate((1, yy, zz)))

    def U(f, yy, zz):
        return float(mean[f, 0]) + float(mean[f, 1]) * yy + float(mean[f, 2]) * zz

    d = [amp(f, y2, z2) * E - amp(f, y1, z1) for f in range(4)]
    s = [amp(f, y1, z1) + amp(f, y2, z2) * E for f in range(4)]

    def re_prod(a, b):
        return sp.re(sp.expand(a * sp.conjugate(b)))

    A = sum(re_prod(d[i], d[i]) for i in range(3)) / 2
    Pk = {kk: re_prod(d[3], d[kk]) / 2 for kk in (1, 2)}
    Q = {(i, kk): re_prod(d[i], d[kk]) / 2 for i in range(3) for kk in (1, 2)}
    R = {(i, kk): re_prod(d[i], s[kk]) / 4 for i in range(3) for kk in (1, 2)}
    grad = {(i, 1): float(mean[i, 1]) for i in range(3)}
    grad.update({(i, 2): float(mean[i, 2]) for i in range(3)})

    def eps_at(yy, zz):
        tot = 0
        for i in range(3):
            a = amp(i, yy, zz)
            tot += k * k * re_prod(a, a) + abs(complex(coef[i, 1])) ** 2 + abs(complex(coef[i, 2])) ** 2
        return nu * tot / 2

    dU = [U(f, y2, z2) - U(f, y1, z1) for f in range(3)]
    Us = [(U(f, y1, z1) + U(f, y2, z2)) / 2 for f in range(3)]
    dry = lambda f: (sp.diff(f, y2) - sp.diff(f, y1)) / 2
    drz = lambda f: (sp.diff(f, z2) - sp.diff(f, z1)) / 2
    dY = lambda f: sp.diff(f, y1) + sp.diff(f, y2)
    dZ = lambda f: sp.diff(f, z1) + sp.diff(f, z2)
    phix = A * dU[0] - 2 * nu * sp.diff(A, r)
    phiy = A * dU[1] - 2 * nu * dry(A)
    phiz = A * dU[2] - 2 * nu * drz(A)
    psiy = A * Us[1] + 2 * Pk[1] - nu / 2 * dY(A)
    psiz = A * Us[2] + 2 * Pk[2] - nu / 2 * dZ(A)
    xi = sum(-2 * Q[(i, kk)] * grad[(i, kk)] for i in range(3) for kk in (1, 2)) \
        - 4 * (eps_at(y1, z1) + eps_at(y2, z2)) / 2
    res = sp.diff(phix, r) + dry(phiy) + drz(phiz) + dY(psiy) + dZ(psiz) - xi
    exprs = [A, phix, phiy, phiz, psiy, psiz, xi, res]
    fns = [sp.lambdify((y1, z1, y2, z2, r), e, "numpy") for e in exprs]
    y, z, nx, Lx = c["y"], c["z"], c["nx"], c["Lx"]
    ny, nz = len(y), len(z)
    Y1, Z1, Y2, Z2, RR = np.meshgrid(y, z, y, z, np.arange(nx) * Lx / nx, indexing="ij")
    out = np.zeros((8, ny * nz, ny * nz, nx))
    for t, fn in enumerate(fns):
        out[t] = np.broadcast_to(fn(Y1, Z1, Y2, Z2, RR), Y1.shape).reshape(ny * nz, ny * nz, nx)
    return out


_CF = {}


def _cf():
    if not _CF:
        c = _closed_form_case()
        _CF["case"] = c
        _CF["want"] = _closed_form_terms(c)
    return _CF["case"], _CF["want"]


def _closed_form_errors(lib=None):
    c, want = _cf()
    got = O1.full(c["phys"], c["y"], c["z"], c["Lx"], c["nu"], lib=lib)["terms"]
    return [float(np.abs(got[t] - want[t]).max() / np.abs(want[t]).max()) for t in range(8)]


def test_single_mode_closed_form():
    errs = _closed_form_errors()
    for t, e in enumerate(errs):
        assert e < 1e-10, (O1.TERMS[t], e)


def test_inversion_parities_and_coincident_points():
    ns, nx, ny, nz = 3, 8, 6, 5
    phys = _random_fields(ns, nx, ny, nz, 21)
    r = O1.full(phys, _grid(ny, 7), _grid(nz, 8), 2.0, 0.01)
    t = r["terms"]
    flip = (-np.arange(nx)) % nx
    swapped = t.transpose(0, 2, 1, 3)[:, :, :, flip]               # T(p2, p1, -r)
    for name, sign in (("A", 1), ("Phi_x", -1), ("Phi_y", -1), ("Phi_z", -1), ("psi_y", 1), ("psi_z", 1),
                       ("xi", 1), ("residual", 1)):
        i = T[name]
        scale = np.abs(t[i]).max()
        assert np.abs(swapped[i] - sign * t[i]).max() <= 1e-12 * scale, name
    P = ny * nz
    diag = t[T["A"]][np.arange(P), np.arange(P), 0]
    assert np.abs(diag).max() == 0.0


# -------------------------------------------------------------- planted mistakes

MISTAKES = [
    # mean advection in the space of scales along z uses the wrong component
    ("t[T_PHIZ] = cm[C_BZ] + A * dU[2]", "t[T_PHIZ] = cm[C_BZ] + A * dU[1]"),
    # the jump of the mean gradient taken the wrong way round
    ("* (g2 - g1);", "* (g1 - g2);"),
    # the r_z derivative of A with the wrong sign
    ("0.5 * (cm[C_DZ2] - cm[C_DZ1])", "0.5 * (cm[C_DZ1] - cm[C_DZ2])"),
    # the turbulent z flux transported by v instead of w
    ("acc[C_CZ] += us[2] * q;", "acc[C_CZ] += us[1] * q;"),
    # the residual's r_z divergence without its 1/2
    ("0.5 * (fz2 - fz1)", "(fz2 - fz1)"),
    # dissipation without its z gradients
    ("acc += gx * gx + gy * gy + gz * gz;", "acc += gx * gx + gy * gy;"),
    # physical-space advection along z by the mean of V
    ("A * Us[2] + 2.0 * cm[C_PZ]", "A * Us[1] + 2.0 * cm[C_PZ]"),
]


@pytest.mark.parametrize("i", range(len(MISTAKES)))
def test_planted_mistakes_are_caught(tmp_path, i):
    old, new = MISTAKES[i]
    src = O1.source_text()
    assert src.count(old) == 1, old
    lib = O1.load_library(O1.compile_source(src.replace(old, new), str(tmp_path / f"bad{i}.so")))
    caught = (max(_closed_form_errors(lib)) > 1e-6 or max(_exchange_error(lib).values()) > 1e-6
              or max(_channel_errors(lib).values()) > 1e-6)
    assert caught, new


def test_points_equal_full():
    """The sampled mode (used by the full-size GPU test) gives the full
    mode's components and terms, including the stencil parts it evaluates
    from A at the neighbour pairs directly."""
    ns, nx, ny, nz = 2, 8, 6, 7
    phys = _random_fields(ns, nx, ny, nz, 31)
    y, z = _grid(ny, 11), _grid(nz, 12)
    ref = O1.full(phys, y, z, 2.0, 0.02)
    P = ny * nz
    rng = np.random.default_rng(4)
    pts = [(0, 0, 0), (P - 1, 0, 3), (5, 40, 7), (17, 17, 4)] + [
        (int(a), int(b), int(m)) for a, b, m in zip(rng.integers(0, P, 12), rng.integers(0, P, 12),
                                                       rng.integers(0, nx, 12))]
    got = O1.points(phys, y, z, 2.0, 0.02, pts)
    for q, (a, b, m) in enumerate(pts):
        np.testing.assert_allclose(got["comp"][q], ref["comp"][:, a, b, m], rtol=0, atol=1e-13)
        np.testing.assert_allclose(got["terms"][q], ref["terms"][:7, a, b, m], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(got["prof"], ref["prof"])
