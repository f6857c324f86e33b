"""The one-homogeneous-direction path on the GPU (gke1h_compute) against the
CPU oracle (oracle/gke1h_oracle.c), element by element.

The oracle evaluates every term by direct sums over x and snapshots at every
ordered pair of cross-section points; the GPU forms the same terms from
x-correlations by Parseval (Eq. 7-9) on the pairs p1 <= p2.  Both run in
FP64; the tolerance, 1e-11 of each term's largest magnitude, covers the
different summation orders (direct sums of up to ns nx products against
FFTs of length nx and contractions over ns snapshots).
"""
import numpy as np
import pytest

import synthetic as S
from oracle import one_homog as O1

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11


def _native():
    import paper_1910_06409_gb300._native as N
    return N


def _run(wl, fields, host=False, f32=False):
    N = _native()
    y, z = S.cgl_grid(wl.ny), S.cgl_grid(wl.nz)
    plan = N.gke1h_plan(wl.nx, wl.ny, wl.nz, wl.Lx, wl.nu, y, z, wl.nsnap,
                        stream=torch.cuda.current_stream().cuda_stream,
                        precision=N.GKE_PREC_F32 if f32 else N.GKE_PREC_F64)
    try:
        npair = N.gke1h_npair(plan)
        assert npair == wl.npair
        if host:
            terms = np.zeros((N.GKE1H_NTERM, npair, wl.nx), dtype=np.float32 if f32 else np.float64)
            prof = np.zeros((N.GKE1H_NPROF, wl.npoint))
            N.gke1h_compute(plan, fields, wl.nsnap, terms, prof)
            terms = terms.astype(np.float64)
        else:
            t = torch.empty((N.GKE1H_NTERM, npair, wl.nx), dtype=torch.float32 if f32 else torch.float64,
                            device="cuda")
            pr = torch.empty((N.GKE1H_NPROF, wl.npoint), dtype=torch.float64, device="cuda")
            N.gke1h_compute(plan, torch.from_numpy(fields).cuda(), wl.nsnap, t, pr)
            torch.cuda.synchronize()
            terms, prof = t.cpu().numpy().astype(np.float64), pr.cpu().numpy()
    finally:
        N.gke1h_destroy(plan)
    return terms, prof


def _triangle(full):
    """[T][P][P][nx] -> [T][npair][nx] on the pairs p1 <= p2, row-major"""
    P = full.shape[1]
    i1, i2 = np.triu_indices(P)
    return full[:, i1, i2, :]


@pytest.mark.parametrize("dims,host", [((16, 9, 7, 4), False), ((24, 6, 11, 3), True), ((8, 5, 5, 1), False),
                                       ((12, 7, 10, 2), True), ((128, 5, 6, 2), False), ((512, 5, 5, 1), True)])
def test_full_parity_with_oracle(dims, host):
    nx, ny, nz, ns = dims
    wl = S.duct_small(nx, ny, nz, ns, wid=31)
    phys = S.duct_physical(wl)
    ref = O1.full(phys, S.cgl_grid(ny), S.cgl_grid(nz), wl.Lx, wl.nu)
    got, prof = _run(wl, S.duct_coefficients(wl), host=host)
    want = _triangle(ref["terms"])
    for t, name in enumerate(O1.TERMS):
        scale = np.abs(want[t]).max()
        err = np.abs(got[t] - want[t]).max() / scale
        assert err < TOL, (name, err)
    np.testing.assert_allclose(prof, ref["prof"], rtol=0, atol=TOL * np.abs(ref["prof"]).max())


def test_duct_tiny_workload():
    wl = S.DUCT_TINY
    ref = O1.full(S.duct_physical(wl), S.cgl_grid(wl.ny), S.cgl_grid(wl.nz), wl.Lx, wl.nu)
    got, _ = _run(wl, S.duct_coefficients(wl))
    want = _triangle(ref["terms"])
    for t, name in enumerate(O1.TERMS):
        assert np.abs(got[t] - want[t]).max() < TOL * np.abs(want[t]).max(), name


def test_duct_full_size_sampled():
    """The benchmark's 256 x 33 x 33 duct, 16 snapshots, in the launch
    configuration bench.py times: every term but the residual at sampled
    pairs and separations (tile edges, the diagonal, the last point)."""
    N = _native()
    wl = S.DUCT
    P = wl.npoint
    rng = np.random.default_rng(3)
    pts = [(0, 0, 0), (0, P - 1, 5), (31, 32, 17), (32, 32, 0), (P - 1, P - 1, wl.nx // 2), (100, 900, 128),
           (16 * 33, 16 * 33 + 1, 255), (33, 66, 1)]
    for _ in range(24):
        a, b = sorted(rng.integers(0, P, 2).tolist())
        pts.append((a, b, int(rng.integers(0, wl.nx))))
    ref = O1.points(S.duct_physical(wl), S.cgl_grid(wl.ny), S.cgl_grid(wl.nz), wl.Lx, wl.nu, pts)
    got, prof = _run(wl, S.duct_coefficients(wl))
    scale = np.abs(got[:7]).reshape(7, -1).max(axis=1)
    for q, (a, b, m) in enumerate(pts):
        pr = a * P - a * (a - 1) // 2 + (b - a)
        for t in range(7):
            assert abs(got[t, pr, m] - ref["terms"][q, t]) < TOL * scale[t], (a, b, m, O1.TERMS[t])
    np.testing.assert_allclose(prof, ref["prof"], rtol=0, atol=TOL * np.abs(ref["prof"]).max())
    # r-inversion at the diagonal: Phi odd, the rest even, so Phi_k(p, p, r) = -Phi_k(p, p, -r)
    idx = [p * P - p * (p - 1) // 2 for p in (0, 500, P - 1)]
    flip = (-np.arange(wl.nx)) % wl.nx
    for t in (1, 2, 3):
        v = got[t][idx]
        assert np.abs(v + v[:, flip]).max() < TOL * scale[t]
    assert N.GKE1H_NTERM == 8


def test_nonfinite_input_is_reported():
    N = _native()
    wl = S.duct_small(8, 5, 6, 2, wid=32)
    f = S.duct_coefficients(wl)
    f[1, 2, 3, 4, 1] = np.nan
    with pytest.raises(N.GkeError) as e:
        _run(wl, f)
    assert e.value.status == -5


# ------------------------------------------------------------ FP32 variant
# Operands, contractions, term spectra, transforms and stencils in FP32
# (means, products and one-point sums in FP64).  The bar is 1e-5 of each
# term's largest magnitude: FP32 rounding (6e-8) amplified by the
# contraction over snapshots and terms and by the stencils, whose weights
# grow like 1/dy near the walls; the errors measured on these grids are
# recorded in the assertion messages.
TOL32 = 1e-5


@pytest.mark.parametrize("dims,host", [((16, 9, 7, 4), False), ((24, 6, 11, 3), True), ((256, 8, 9, 4), False)])
def test_f32_parity_with_oracle(dims, host):
    nx, ny, nz, ns = dims
    wl = S.duct_small(nx, ny, nz, ns, wid=33)
    ref = O1.full(S.duct_physical(wl), S.cgl_grid(ny), S.cgl_grid(nz), wl.Lx, wl.nu)
    got, prof = _run(wl, S.duct_coefficients(wl), host=host, f32=True)
    want = _triangle(ref["terms"])
    for t, name in enumerate(O1.TERMS):
        err = np.abs(got[t] - want[t]).max() / np.abs(want[t]).max()
        assert err < TOL32, (name, err)


def test_f32_against_f64_full_size():
    """The benchmark's 256 x 33 x 33 duct: the FP32 variant against the FP64
    path on every output value."""
    wl = S.DUCT
    f = S.duct_coefficients(wl)
    ref, _ = _run(wl, f)
    got, _ = _run(wl, f, f32=True)
    errs = {}
    for t, name in enumerate(O1.TERMS):
        errs[name] = float(np.abs(got[t] - ref[t]).max() / np.abs(ref[t]).max())
    assert max(errs.values()) < TOL32, errs


def test_snapshot_count_errors():
    """nsnap outside [1, max_snap] and a missing output are refused before
    any launch (GKE_ERR_ARG), and the plan stays usable."""
    N = _native()
    wl = S.duct_small(8, 5, 6, 2, wid=34)
    f = torch.from_numpy(S.duct_coefficients(wl)).cuda()
    plan = N.gke1h_plan(wl.nx, wl.ny, wl.nz, wl.Lx, wl.nu, S.cgl_grid(wl.ny), S.cgl_grid(wl.nz), wl.nsnap)
    try:
        t = torch.empty((N.GKE1H_NTERM, wl.npair, wl.nx), dtype=torch.float64, device="cuda")
        for ns in (0, wl.nsnap + 1):
            with pytest.raises(N.GkeError) as e:
                N.gke1h_compute(plan, f, ns, t)
            assert e.value.status == -1
        with pytest.raises(N.GkeError) as e:
            N.gke1h_compute(plan, f, wl.nsnap, None)
        assert e.value.status == -1
        N.gke1h_compute(plan, f, wl.nsnap, t)
        torch.cuda.synchronize()
        assert torch.isfinite(t).all()
    finally:
        N.gke1h_destroy(plan)
