"""Host-side checks of the C ABI library that need no GPU.

* libgke.so loads and exports every function include/gke.h and
  include/gke1h.h declare;
* the host FD weights (Fornberg's recursion) are exact on quartics on the
  wall-normal grids of the workloads, and agree with the oracle's independent
  moment-system solve;
* argument errors of the host utility are reported, not raised.
"""
import os
import re

import numpy as np
import pytest

import synthetic as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_1910_06409_gb300 import build as B
    B.build()
    import paper_1910_06409_gb300._native as N
    N.lib()
    return N


def declared_functions():
    """every function the headers under include/ declare"""
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(gke1?h?_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(native):
    decl = declared_functions()
    assert len(decl) >= 10
    L = native.lib()
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(native.EXPORTS) == decl


@pytest.mark.parametrize("ny", [5, 33, 129, 257])
def test_host_fd_weights_exact(native, ny):
    y = S.cgl_grid(ny)
    rng = np.random.default_rng(1)
    poly = np.polynomial.Polynomial(rng.standard_normal(5))
    for j in range(ny):
        l0, w = native.gke_fd_weights(y, j)
        assert l0 == min(max(j - 2, 0), ny - 5)
        got = np.dot(w, poly(y[l0:l0 + 5]))
        scale = np.abs(w).sum() * np.abs(poly(y)).max()
        assert abs(got - poly.deriv()(y[j])) < 1e-13 * scale


def test_host_fd_weights_match_oracle(native):
    import oracle
    y = S.cgl_grid(65)
    for j in range(65):
        l0a, wa = native.gke_fd_weights(y, j)
        l0b, wb = oracle.fd_weights(y, j)
        assert l0a == l0b
        np.testing.assert_allclose(wa, wb, rtol=1e-10, atol=1e-10 * np.abs(wb).max())


def test_host_fd_weights_bad_args(native):
    with pytest.raises(native.GkeError):
        native.gke_fd_weights(np.arange(4.0), 0)
    with pytest.raises(native.GkeError):
        native.gke_fd_weights(np.arange(8.0), 8)


def test_term_set_closure(native):
    """gke_term_set (host logic): Phi_y and phi bring A (their Step-3 FD
    parts, Eq. 10-11); the residual brings Phi_y, phi and A; 0 means all."""
    A, PX, PY, PZ, PH, XI, RES = (1 << t for t in range(7))
    f = native.gke_term_set
    assert f(0) == 127
    assert f(A) == A and f(PX) == PX and f(PZ) == PZ and f(XI) == XI
    assert f(PY) == PY | A and f(PH) == PH | A
    assert f(RES) == RES | PY | PH | A
    assert f(PX | XI) == PX | XI
    assert f(127) == 127 and f(1 << 9) == 127      # bits above the terms are ignored here


def test_one_homog_plan_argument_errors(native):
    """gke1h_plan validates its descriptor before touching the device."""
    y, z = S.cgl_grid(9), S.cgl_grid(7)
    bad = [dict(nx=16, ny=4, nz=7), dict(nx=16, ny=9, nz=3), dict(nx=10, ny=9, nz=7), dict(nx=1024, ny=9, nz=7)]
    codes = []
    for b in bad:
        with pytest.raises(native.GkeError) as e:
            native.gke1h_plan(b["nx"], b["ny"], b["nz"], 1.0, 0.01, S.cgl_grid(max(b["ny"], 1)),
                              S.cgl_grid(max(b["nz"], 1)), 2)
        codes.append(e.value.status)
    assert codes == [-1, -1, -7, -7]
    with pytest.raises(native.GkeError) as e:
        native.gke1h_plan(16, 9, 7, 1.0, 0.01, y[::-1].copy(), z, 2)
    assert e.value.status == -1 and "increasing" in str(e.value)


def test_one_homog_precision_errors(native):
    """Only GKE_PREC_F64 and GKE_PREC_F32 plans exist for one homogeneous
    direction; the descriptor is refused before the device is touched."""
    y, z = S.cgl_grid(9), S.cgl_grid(7)
    with pytest.raises(native.GkeError) as e:
        native.gke1h_plan(16, 9, 7, 1.0, 0.01, y, z, 2, precision=native.GKE_PREC_BF16X3)
    assert e.value.status == -7
    with pytest.raises(native.GkeError) as e:
        native.gke1h_plan(16, 9, 7, 1.0, 0.01, y, z, 2, precision=5)
    assert e.value.status == -1


def test_one_homog_pair_labels(native):
    """Output pair order of the one-direction path: p1 <= p2, row-major."""
    y, z = S.cgl_grid(6), S.cgl_grid(5)
    p1, p2, Y1, Z1, Y2, Z2 = native.gke1h_pair_labels(y, z)
    i1, i2 = np.triu_indices(30)
    np.testing.assert_array_equal(p1, i1)
    np.testing.assert_array_equal(p2, i2)
    np.testing.assert_array_equal(Y1, y[i1 // 5])
    np.testing.assert_array_equal(Z2, z[i2 % 5])
    np.testing.assert_array_equal(Z1, z[i1 % 5])
    np.testing.assert_array_equal(Y2, y[i2 // 5])
    assert native.lib().gke1h_pair_labels(0, 5, None, None, None, None, None, None, None, None) == -1
