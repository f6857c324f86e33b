"""Step 1 for velocity-vorticity databases on the GPU (gke_velocity_vorticity)
against the CPU oracle (oracle/step1.py), element by element.

Tolerances (relative to each field's largest coefficient): u, v, w come from
5-point sums and one division per coefficient in FP64 on both sides, 1e-13;
p is the solution of a banded system whose condition number grows like
ny^4 (the GPU factors it in band storage with partial pivoting, the oracle
with numpy's dense LU), 1e-10.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import step1 as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = (1e-13, 1e-13, 1e-13, 1e-10)


def _native():
    import paper_1910_06409_gb300._native as N
    return N


def _plan(wl, prec=0):
    N = _native()
    return N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), max(1, wl.nsnap), prec,
                      stream=torch.cuda.current_stream().cuda_stream)


def _errors(got, want):
    return [float(np.abs(got[:, f] - want[:, f]).max() / np.abs(want[:, f]).max()) for f in range(4)]


@pytest.mark.parametrize("shape", [(16, 12, 17, 2), (32, 32, 33, 2), (24, 16, 9, 1), (8, 48, 13, 1)])
def test_step1_matches_oracle(shape):
    N = _native()
    nx, nz, ny, ns = shape
    wl = S.small(nx, nz, ny, ns, wid=41)
    v_eta, mean_uw = S.vorticity_inputs(wl)
    want = O.step1(v_eta, mean_uw, S.cgl_grid(ny), wl.Lx, wl.Lz, wl.nu, nx)
    plan = _plan(wl)
    try:
        out = torch.empty(want.shape, dtype=torch.complex128, device="cuda")
        N.gke_velocity_vorticity(plan, torch.from_numpy(v_eta).cuda(), torch.from_numpy(mean_uw).cuda(), ns, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # host buffers in and out, on a split-precision plan (Step 1 is FP64 on every plan)
        got_h = np.zeros_like(want)
    finally:
        N.gke_destroy(plan)
    plan = _plan(wl, N.GKE_PREC_BF16X3)
    try:
        N.gke_velocity_vorticity(plan, v_eta, mean_uw, ns, got_h)
    finally:
        N.gke_destroy(plan)
    for f, (e, eh) in enumerate(zip(_errors(got, want), _errors(got_h, want))):
        assert e < TOL[f], (f, e)
        assert eh < TOL[f], (f, eh)


def test_step1_closed_form_taylor_green():
    """The Taylor-Green cell through the GPU path: p = g^2/4 (cos 2x + cos 2z)."""
    N = _native()
    nx = nz = 16
    ny, g = 9, 0.8
    wl = S.Workload("tg", 0, nx, nz, ny, 1, 2 * np.pi, 2 * np.pi, 0.01)
    x = np.arange(nx) * 2 * np.pi / nx
    X, Z = np.meshgrid(x, x)
    eta = -2 * g * np.sin(X) * np.sin(Z)
    v_eta = np.zeros((1, 2, ny, nz, nx // 2 + 1), complex)
    v_eta[0, 1] = np.fft.rfft2(np.broadcast_to(eta, (ny, nz, nx)), axes=(-2, -1), norm="forward")
    mean_uw = np.zeros((1, 2, ny))
    out = np.zeros((1, 4, ny, nz, nx // 2 + 1), complex)
    plan = _plan(wl)
    try:
        N.gke_velocity_vorticity(plan, v_eta, mean_uw, 1, out)
    finally:
        N.gke_destroy(plan)
    phys = np.fft.irfft2(out[0], s=(nz, nx), axes=(-2, -1), norm="forward")
    np.testing.assert_allclose(phys[0], np.broadcast_to(g * np.sin(X) * np.cos(Z), phys[0].shape), atol=1e-13)
    np.testing.assert_allclose(phys[2], np.broadcast_to(-g * np.cos(X) * np.sin(Z), phys[2].shape), atol=1e-13)
    np.testing.assert_allclose(phys[3], np.broadcast_to(g * g / 4 * (np.cos(2 * X) + np.cos(2 * Z)), phys[3].shape),
                               atol=1e-12)


def test_step1_full_size_sampled():
    """256 x 256 x 129 (the Re_tau ~ 200 grid), one snapshot: u, w at every
    mode; p at sampled modes, each solved alone by the oracle."""
    N = _native()
    wl = S.RETAU200
    v_eta, mean_uw = S.vorticity_inputs(wl, 1)
    y = S.cgl_grid(wl.ny)
    plan = _plan(S.Workload(wl.name, wl.wid, wl.nx, wl.nz, wl.ny, 1, wl.Lx, wl.Lz, wl.nu))
    try:
        out = torch.empty((1, 4) + v_eta.shape[2:], dtype=torch.complex128, device="cuda")
        N.gke_velocity_vorticity(plan, torch.from_numpy(v_eta).cuda(), torch.from_numpy(mean_uw).cuda(), 1, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()[0]
    finally:
        N.gke_destroy(plan)
    v = v_eta[0, 0]
    u, w = O.velocity(v, v_eta[0, 1], mean_uw[0, 0], mean_uw[0, 1], y, wl.Lx, wl.Lz, wl.nx)
    for f, want in ((0, u), (1, v), (2, w)):
        assert np.abs(got[f] - want).max() < TOL[f] * np.abs(want).max()
    rhs = O.poisson_rhs(u, v, w, y, wl.Lx, wl.Lz, wl.nx)
    _, _, kx2, kz2 = O.wavenumbers(wl.nx, wl.nz, wl.Lx, wl.Lz)
    D2 = O._dmat(y, 2)
    d2v = np.einsum("jl,lzx->jzx", D2, v)
    rng = np.random.default_rng(0)
    modes = [(0, 0), (0, 1), (1, 0), (wl.nz // 2, 0), (wl.nz - 1, wl.nxh - 1), (wl.nz // 2, wl.nx // 2)]
    modes += [(int(a), int(b)) for a, b in zip(rng.integers(0, wl.nz, 10), rng.integers(0, wl.nxh, 10))]
    scale = np.abs(got[3]).max()
    for iz, ix in modes:
        want = O.solve_poisson(rhs[:, iz, ix], wl.nu * d2v[0, iz, ix], wl.nu * d2v[-1, iz, ix], y,
                               kx2[ix] + kz2[iz])
        assert np.abs(got[3][:, iz, ix] - want).max() < TOL[3] * scale, (iz, ix)
