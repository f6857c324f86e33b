"""The correlation expansion of the one-homogeneous-direction terms (Eq. 7
written for flows homogeneous in x only), restated in numpy and checked
against the direct-sum oracle (oracle/gke1h_oracle.c).

The GPU path evaluates the terms as snapshot sums of x-correlations between
the fluctuations u, v, w, p and their in-plane products (Parseval, Eq. 8-9),
plus one-point moments, then inverse transforms and stencils.  This test
writes that decomposition out with numpy FFTs and contractions: nine velocity
correlations <u_a u_b'>, for each k the four third-order groups
Q1 = <q u_k'>, Q2 = <u_k q'>, X1 = sum_i <(u_i u_k) u_i'>, X2 = sum_i
<u_i (u_i u_k)'>, and the pressure pair <p u_k'> + <u_k p'>, combined as

  A            = K(p1) + K(p2) - 2 sum_a <u_a u_a'>
  <du^2 du_k>  = S_k(p2) - S_k(p1) + Q1 + 2 X1 - Q2 - 2 X2
  <u_k* du^2>  = (S_k(p1) + S_k(p2) + Q1 + Q2) / 2 - X1 - X2
  <dp du_k>    = <p u_k>(p1) + <p u_k>(p2) - <p u_k'> - <u_k p'>
  xi (velocity part) = sum_ab [2 d_b U_a(p2) [b = y, z] + 2 d_a U_b(p1) [a = y, z]] <u_a u_b'>
                       + 2 (Pi - eps)(p1) + 2 (Pi - eps)(p2)

and compares every term with the oracle's direct averages.  It shares no
code with the oracle or with the CUDA path.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import fd_weights
from oracle import one_homog as O1


def _weights(g):
    n = len(g)
    w, l0 = np.zeros((n, 5)), np.zeros(n, int)
    for j in range(n):
        l0[j], w[j] = fd_weights(g, j)
    return w, l0


@pytest.mark.parametrize("dims", [(16, 6, 7, 3), (12, 5, 8, 2)])
def test_expansion_matches_direct_sums(dims):
    nx, ny, nz, ns = dims
    wl = S.duct_small(nx, ny, nz, ns, wid=35)
    y, z = S.cgl_grid(ny), S.cgl_grid(nz)
    nu, Lx = wl.nu, wl.Lx
    P, nxh = ny * nz, nx // 2 + 1
    phys = S.duct_physical(wl)
    ref = O1.full(phys, y, z, Lx, nu)

    f = np.fft.rfft(phys, axis=-1, norm="forward").reshape(ns, 4, P, nxh)
    U = f[:, :, :, 0].real.mean(axis=0)                          # [4][P]
    fl = f.copy()
    fl[:, :, :, 0] -= U[None]
    fl[:, :, :, 0] = fl[:, :, :, 0].real
    wy, ly = _weights(y)
    wz, lz = _weights(z)

    def stencil(F, first):
        """d_Y (first = 0) or d_Z (first = 1) of a per-point array along axis 0"""
        out = np.zeros_like(F)
        for p in range(P):
            iy, iz = divmod(p, nz)
            for l in range(5):
                q = (ly[iy] + l) * nz + iz if first == 0 else iy * nz + lz[iz] + l
                out[p] += (wy[iy, l] if first == 0 else wz[iz, l]) * F[q]
        return out

    g = {(i, k): stencil(U[i], k - 1) for i in range(3) for k in (1, 2)}   # d_k U_i
    ph = np.fft.irfft(fl, n=nx, axis=-1, norm="forward")                   # fluctuations [ns][4][P][nx]
    u = [ph[:, 0], ph[:, 1], ph[:, 2]]
    pp = ph[:, 3]
    q = u[0] ** 2 + u[1] ** 2 + u[2] ** 2
    prod = lambda i, k: u[i] * u[k]
    spec = lambda a: np.fft.rfft(a, axis=-1, norm="forward")

    def C(a, b):
        """<a(x, p1) b(x + r, p2)> as a [P][P][nx] array via Parseval"""
        S_ = np.einsum("spk,sqk->pqk", np.conj(spec(a)), spec(b)) / ns
        S_[..., 0] = S_[..., 0].real
        S_[..., -1] = S_[..., -1].real
        return np.fft.irfft(S_, n=nx, axis=-1, norm="forward")

    mean = lambda a: a.mean(axis=(0, 2))                                  # one-point, per point
    R = {(a, b): C(u[a], u[b]) for a in range(3) for b in range(3)}
    K = mean(q)
    A = K[:, None, None] + K[None, :, None] - 2 * (R[(0, 0)] + R[(1, 1)] + R[(2, 2)])
    B, Cs, Pk = {}, {}, {}
    for k in range(3):
        Sk = mean(q * u[k])
        Q1, Q2 = C(q, u[k]), C(u[k], q)
        X1 = sum(C(prod(i, k), u[i]) for i in range(3))
        X2 = sum(C(u[i], prod(i, k)) for i in range(3))
        B[k] = Sk[None, :, None] - Sk[:, None, None] + Q1 + 2 * X1 - Q2 - 2 * X2
        Cs[k] = 0.5 * (Sk[:, None, None] + Sk[None, :, None] + Q1 + Q2) - X1 - X2
        Spk = mean(pp * u[k])
        Pk[k] = Spk[:, None, None] + Spk[None, :, None] - C(pp, u[k]) - C(u[k], pp)
    # dissipation: spectral x derivative (Nyquist 0), stencils in y and z
    kx = 2 * np.pi * np.arange(nxh) / Lx
    kx[-1] = 0.0
    eps = np.zeros(P)
    for i in range(3):
        dx = np.fft.irfft(1j * kx * fl[:, i], n=nx, axis=-1, norm="forward")
        dy = np.stack([stencil(ph[s, i], 0) for s in range(ns)])
        dz = np.stack([stencil(ph[s, i], 1) for s in range(ns)])
        eps += nu * (dx ** 2 + dy ** 2 + dz ** 2).mean(axis=(0, 2))
    M = lambda i, k: mean(prod(i, k))
    Pi = -sum(M(i, k) * g[(i, k)] for i in range(3) for k in (1, 2))
    E0 = 2 * (Pi - eps)
    xi = E0[:, None, None] + E0[None, :, None]
    for a in range(3):
        for b in range(3):
            c = 0.0
            if b >= 1:
                c = c + 2 * g[(a, b)][None, :, None]
            if a >= 1:
                c = c + 2 * g[(b, a)][:, None, None]
            xi = xi + c * R[(a, b)]

    want = ref["terms"]
    comp = ref["comp"]
    names = O1.COMPONENTS
    scale = lambda x: np.abs(x).max()
    np.testing.assert_allclose(A, want[0], rtol=0, atol=1e-12 * scale(want[0]))
    for k, nm in ((0, "Bx"), (1, "By"), (2, "Bz")):
        c_ = comp[names.index(nm)]
        np.testing.assert_allclose(B[k], c_, rtol=0, atol=1e-12 * scale(c_))
    for k, nm in ((1, "Cy"), (2, "Cz")):
        c_ = comp[names.index(nm)]
        np.testing.assert_allclose(Cs[k], c_, rtol=0, atol=1e-12 * scale(c_))
    for k, nm in ((1, "Py"), (2, "Pz")):
        c_ = comp[names.index(nm)]
        np.testing.assert_allclose(Pk[k], c_, rtol=0, atol=1e-12 * scale(c_))
    np.testing.assert_allclose(xi, want[6], rtol=0, atol=1e-12 * scale(want[6]))
    np.testing.assert_allclose(eps, ref["prof"][O1.PROFILES.index("eps")], rtol=1e-12)
