"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

The oracle evaluates the GKE terms as direct averages of increment products
(Sec. 2); the CUDA path uses the correlation expansion (Eq. 7) and Parseval
(Eq. 8-9).  Both are exact for grid sums, so in FP64 they agree to rounding:
the bar is max |gpu - oracle| <= TOL_F64 * max |oracle| per term.

TOL_F64 = 1e-12: the FP64 path sums O(10^2) snapshot-field products per
wavenumber and runs two radix-2 transforms of log2(n) <= 9 stages; the Step-3
stencils multiply rounding errors by at most sum |w| ~ 4/dy_min per
derivative, and the residual applies two of them, so the worst term stays a
few 1e-13 below the bar at these sizes.
"""
import os

import numpy as np
import pytest

import synthetic as S

TOL_F64 = 1e-12

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1910_06409_gb300 import build as B
    B.build()
    import paper_1910_06409_gb300._native as native
    return native


def run_gpu(N, wl, coef, precision=0, calls=None, host=False, domain=0):
    """All terms on the device through the C ABI; returns (terms, profiles) as numpy."""
    import torch
    y = S.cgl_grid(wl.ny)
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, coef.shape[0], precision, pair_domain=domain)
    tdt = torch.float64 if precision == N.GKE_PREC_F64 else torch.float32    # terms element type
    try:
        npair = N.gke_npair(plan)
        if host:
            f = torch.from_numpy(np.ascontiguousarray(coef))
            terms = torch.empty((N.GKE_NTERM, npair, wl.nz, wl.nx), dtype=tdt)
            prof = torch.empty((N.GKE_NPROF, wl.ny), dtype=torch.float64)
        else:
            f = torch.from_numpy(np.ascontiguousarray(coef)).cuda()
            terms = torch.empty((N.GKE_NTERM, npair, wl.nz, wl.nx), dtype=tdt, device="cuda")
            prof = torch.empty((N.GKE_NPROF, wl.ny), dtype=torch.float64, device="cuda")
        if calls is None:
            N.gke_compute(plan, f, coef.shape[0], terms, prof)
        else:
            N.gke_accumulate_mean(plan, f, coef.shape[0])
            s0 = 0
            for n in calls:
                N.gke_accumulate_snapshot(plan, f[s0:s0 + n], n)
                s0 += n
            N.gke_finalize_terms(plan, terms, prof)
        torch.cuda.synchronize()
        return terms.cpu().numpy().astype(np.float64), prof.cpu().numpy()
    finally:
        N.gke_destroy(plan)


def rel_err(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


def check_full(N, wl, got, prof, ref, tol):
    iu = np.triu_indices(wl.ny)
    for t in range(N.GKE_NTERM):
        e = rel_err(got[t], ref["terms"][t][iu])
        assert e <= tol, f"{N.TERMS[t]}: {e:.3e}"
    for k in (0, 4, 5):   # U, dU/dy, eps
        e = rel_err(prof[k], ref["prof"][k])
        assert e <= tol, f"profile {N.PROFILES[k]}: {e:.3e}"


@pytest.fixture(scope="module")
def tiny():
    import oracle
    wl = S.TINY
    phys = S.physical(wl)
    ref = oracle.full(phys, S.cgl_grid(wl.ny), wl.Lx, wl.Lz, wl.nu)
    return wl, S.to_coefficients(phys), ref


def test_tiny_f64_full_parity(N, tiny):
    wl, coef, ref = tiny
    got, prof = run_gpu(N, wl, coef)
    check_full(N, wl, got, prof, ref, TOL_F64)


@pytest.mark.parametrize("shape", [(16, 8, 7, 3), (8, 32, 11, 1), (64, 16, 6, 2), (24, 12, 9, 2), (48, 96, 7, 2)])
def test_ragged_f64_full_parity(N, shape):
    import oracle
    nx, nz, ny, ns = shape
    wl = S.small(nx, nz, ny, ns, wid=40 + nx + ny)
    phys = S.physical(wl)
    ref = oracle.full(phys, S.cgl_grid(ny), wl.Lx, wl.Lz, wl.nu)
    got, prof = run_gpu(N, wl, S.to_coefficients(phys))
    check_full(N, wl, got, prof, ref, TOL_F64)


def test_split_calls_match_single_call(N, tiny):
    wl, coef, ref = tiny
    a, pa = run_gpu(N, wl, coef)
    b, pb = run_gpu(N, wl, coef, calls=[1, 2, 1])
    assert rel_err(b, a) < 1e-13
    np.testing.assert_allclose(pb, pa, rtol=1e-13, atol=1e-15)


def test_host_pointers_match_device(N, tiny):
    wl, coef, ref = tiny
    a, pa = run_gpu(N, wl, coef)
    b, pb = run_gpu(N, wl, coef, host=True)
    assert np.array_equal(a, b)
    assert np.array_equal(pa, pb)


def test_pair_labels(N):
    wl = S.small(8, 8, 6, 1)
    y = S.cgl_grid(wl.ny)
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, 1)
    try:
        Y, ry, i1, i2 = N.gke_pair_labels(plan)
    finally:
        N.gke_destroy(plan)
    iu = np.triu_indices(wl.ny)
    assert np.array_equal(i1, iu[0]) and np.array_equal(i2, iu[1])
    assert np.array_equal(Y, 0.5 * (y[iu[0]] + y[iu[1]]))
    assert np.array_equal(ry, y[iu[1]] - y[iu[0]])


def test_error_codes(N):
    import torch
    wl = S.small(8, 8, 6, 2, wid=3)
    y = S.cgl_grid(wl.ny)
    coef = torch.from_numpy(S.coefficients(wl)).cuda()
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, 2)
    terms = torch.empty((N.GKE_NTERM, N.gke_npair(plan), wl.nz, wl.nx), dtype=torch.float64, device="cuda")
    try:
        with pytest.raises(N.GkeError) as e:
            N.gke_finalize_terms(plan, terms)
        assert e.value.status == -2
        with pytest.raises(N.GkeError) as e:
            N.gke_accumulate_snapshot(plan, coef, 2)          # no mean yet
        assert e.value.status == -2
        with pytest.raises(N.GkeError) as e:
            N.gke_accumulate_mean(plan, coef, 3)              # > max_snap
        assert e.value.status == -1
        with pytest.raises(N.GkeError) as e:
            N.gke_accumulate_mean(plan, coef, 0)              # empty batch
        assert e.value.status == -1
        N.gke_accumulate_mean(plan, coef, 2)
        bad = coef.clone()
        bad[1, 2, 3, 1, 1] = float("nan")
        N.gke_accumulate_snapshot(plan, bad, 2)
        with pytest.raises(N.GkeError) as e:
            N.gke_finalize_terms(plan, terms)
        assert e.value.status == -5
        with pytest.raises(N.GkeError) as e:
            N.gke_accumulate_snapshot(plan, coef, 2)          # finalized
        assert e.value.status == -2
        N.gke_reset(plan)
        N.gke_accumulate_mean(plan, coef, 2)
        N.gke_accumulate_snapshot(plan, coef, 2)
        N.gke_finalize_terms(plan, terms)
    finally:
        N.gke_destroy(plan)
    with pytest.raises(N.GkeError) as e:
        N.gke_plan(20, 8, 6, 1.0, 1.0, 0.1, S.cgl_grid(6), 1)   # nx neither 2^a nor 3 * 2^a
    assert e.value.status == -7
    with pytest.raises(N.GkeError) as e:
        N.gke_plan(8, 8, 6, 1.0, 1.0, 0.1, S.cgl_grid(6)[::-1], 1)
    assert e.value.status == -1


def test_checkpoint_merge_equals_single_pass(N, tiny, tmp_path):
    """Independent jobs on snapshot subsets, merged (Sec. 3.4), equal one pass."""
    import torch
    wl, coef, ref = tiny
    full, _ = run_gpu(N, wl, coef)
    y = S.cgl_grid(wl.ny)
    mean = np.ascontiguousarray(coef[:, :, :, 0, 0].real.mean(axis=0))   # Step 1 over all snapshots
    f = torch.from_numpy(coef).cuda()
    paths = []
    for part, (a, b) in enumerate([(0, 1), (1, 4)]):
        plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, wl.nsnap)
        try:
            N.gke_set_mean(plan, mean)
            N.gke_accumulate_snapshot(plan, f[a:b], b - a)
            p = str(tmp_path / f"part{part}.ckpt")
            N.gke_checkpoint(plan, p)
            paths.append(p)
        finally:
            N.gke_destroy(plan)
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, wl.nsnap)
    try:
        N.gke_restore(plan, paths[0])
        N.gke_merge(plan, paths[1])
        terms = torch.empty((N.GKE_NTERM, N.gke_npair(plan), wl.nz, wl.nx), dtype=torch.float64, device="cuda")
        N.gke_finalize_terms(plan, terms)
        got = terms.cpu().numpy()
    finally:
        N.gke_destroy(plan)
    assert rel_err(got, full) < 1e-13
    # the same merge done on the host by the checkpoint tool, then restored
    from paper_1910_06409_gb300 import merge as M
    merged = str(tmp_path / "merged.ckpt")
    M.merge(paths, merged)
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, wl.nsnap)
    try:
        N.gke_restore(plan, merged)
        terms = torch.empty((N.GKE_NTERM, N.gke_npair(plan), wl.nz, wl.nx), dtype=torch.float64, device="cuda")
        N.gke_finalize_terms(plan, terms)
        assert np.array_equal(terms.cpu().numpy(), got)
    finally:
        N.gke_destroy(plan)
    with open(paths[0], "r+b") as fp:          # truncated file -> IO error
        fp.truncate(200)
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, wl.nsnap)
    try:
        with pytest.raises(N.GkeError) as e:
            N.gke_restore(plan, paths[0])
        assert e.value.status == -6
    finally:
        N.gke_destroy(plan)


# ------------------------------------------------ full-size workload checks
@pytest.fixture(scope="module")
def retau200(N):
    """GPU terms at the Re_tau~200-shaped workload (256 x 256 x 129, 16 snapshots)."""
    wl = S.RETAU200
    phys = S.physical(wl)
    coef = S.to_coefficients(phys)
    got, prof = run_gpu(N, wl, coef)
    return wl, phys, got, prof


def _pidx(i1, i2, ny):
    return i1 * ny - i1 * (i1 - 1) // 2 + (i2 - i1)


def test_retau200_spot_checks_vs_oracle(N, retau200):
    import oracle
    wl, phys, got, prof = retau200
    rng = np.random.default_rng(2024)
    planes = [0, 1, 2, 37, 64, 100, 127, 128]
    pts = []
    for _ in range(40):
        a, b = sorted(rng.choice(planes, 2))
        pts.append((a, b, int(rng.integers(wl.nz)), int(rng.integers(wl.nx))))
    pts += [(64, 64, 0, 0), (0, 128, 5, 7), (2, 2, 128, 128)]
    ref = oracle.points(phys, S.cgl_grid(wl.ny), wl.Lx, wl.Lz, wl.nu, pts)
    scale = np.abs(got[:6]).reshape(6, -1).max(axis=1)
    for n, (a, b, mz, mx) in enumerate(pts):
        g = got[:6, _pidx(a, b, wl.ny), mz, mx]
        err = np.abs(g - ref["terms"][n]) / scale
        assert err.max() <= TOL_F64, (pts[n], err)


def test_retau200_split_spot_checks_vs_oracle(N, retau200):
    """The split-BF16 path at the full 256 x 256 x 129 x 16 size, as the bench
    runs it: sampled outputs against the oracle, 1e-6 of each term's largest
    magnitude."""
    import oracle
    wl, phys, got64, prof = retau200
    got, _ = run_gpu(N, wl, S.to_coefficients(phys), precision=N.GKE_PREC_BF16X3)
    rng = np.random.default_rng(2025)
    planes = [0, 1, 2, 40, 64, 90, 127, 128]
    pts = []
    for _ in range(30):
        a, b = sorted(rng.choice(planes, 2))
        pts.append((a, b, int(rng.integers(wl.nz)), int(rng.integers(wl.nx))))
    ref = oracle.points(phys, S.cgl_grid(wl.ny), wl.Lx, wl.Lz, wl.nu, pts)
    scale = np.abs(got64[:6]).reshape(6, -1).max(axis=1)
    for n, (a, b, mz, mx) in enumerate(pts):
        err = np.abs(got[:6, _pidx(a, b, wl.ny), mz, mx] - ref["terms"][n]) / scale
        assert err.max() <= 1e-6, (pts[n], err)


def test_largest_grid_spot_checks(N):
    """nx = nz = 1024 (the largest grid), the fewest wall-normal points (5) and
    one snapshot: sampled outputs against the oracle."""
    import oracle
    wl = S.small(1024, 1024, 5, 1, wid=45)
    phys = S.physical(wl)
    got, _ = run_gpu(N, wl, S.to_coefficients(phys))
    rng = np.random.default_rng(1024)
    pts = [(int(a), int(b), int(rng.integers(1024)), int(rng.integers(1024)))
           for a, b in [(0, 0), (0, 4), (1, 3), (2, 2), (3, 4), (0, 2)] for _ in range(3)]
    ref = oracle.points(phys, S.cgl_grid(wl.ny), wl.Lx, wl.Lz, wl.nu, pts)
    scale = np.abs(got[:6]).reshape(6, -1).max(axis=1)
    for n, (a, b, mz, mx) in enumerate(pts):
        err = np.abs(got[:6, _pidx(a, b, wl.ny), mz, mx] - ref["terms"][n]) / scale
        assert err.max() <= TOL_F64, (pts[n], err)


def test_retau200_invariants(N, retau200):
    wl, phys, got, prof = retau200
    ny, nz, nx = wl.ny, wl.nz, wl.nx
    diag = np.array([_pidx(j, j, ny) for j in range(ny)])
    A = got[0]
    scale = np.abs(A).max()
    # zero increment: r = 0, Y1 = Y2 -- A, and Phi_x, Phi_z (whose r-derivative
    # parts vanish at the minimum of A); Phi_y and phi carry FD parts
    for t in (0, 1, 3):
        assert np.abs(got[t, diag, 0, 0]).max() <= 1e-12 * np.abs(got[t]).max()
    # r-inversion on the diagonal pairs: A, phi, xi even; Phi odd
    neg = lambda a: np.roll(a[..., ::-1, ::-1], (1, 1), axis=(-2, -1))
    for t, sg in ((0, 1), (1, -1), (2, -1), (3, -1), (4, 1), (5, 1)):
        a = got[t, diag]
        assert np.abs(a - sg * neg(a)).max() <= 1e-12 * np.abs(got[t]).max(), t
    # r-average: mean over r of A = <u_i u_i>(Y1) + <u_i u_i>(Y2)
    fl = phys - phys.mean(axis=(0, 3, 4), keepdims=True)
    q = (fl[:, :3] ** 2).sum(axis=1).mean(axis=(0, 2, 3))
    iu = np.triu_indices(ny)
    mean_r = A.mean(axis=(1, 2))
    assert np.abs(mean_r - (q[iu[0]] + q[iu[1]])).max() <= 1e-12 * scale


@pytest.mark.parametrize("precision", [0, 1])
def test_pinned_host_output_matches_device(N, precision):
    """Pinned host outputs take the overlapped copy path (finished term rows go
    out per pair chunk on a second stream): bit-equal to device outputs."""
    import torch
    wl = S.small(16, 16, 33, 3, wid=44)
    coef = S.coefficients(wl)
    y = S.cgl_grid(wl.ny)
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, 3, precision)
    try:
        tdt = torch.float64 if precision == 0 else torch.float32
        shape = (N.GKE_NTERM, N.gke_npair(plan), wl.nz, wl.nx)
        dev = torch.empty(shape, dtype=tdt, device="cuda")
        pinned = torch.empty(shape, dtype=tdt).pin_memory()
        f = torch.from_numpy(coef).cuda()
        N.gke_compute(plan, f, 3, dev)
        N.gke_compute(plan, f, 3, pinned)
        torch.cuda.synchronize()
        assert torch.equal(dev.cpu(), pinned)
    finally:
        N.gke_destroy(plan)


@pytest.mark.parametrize("precision,shape", [(0, (16, 16, 33, 3)), (1, (16, 16, 33, 3)), (1, (256, 256, 9, 3))])
def test_pinned_host_input_matches_device(N, precision, shape):
    """Pinned host inputs are streamed (k = 0 coefficients for the mean, then
    snapshot by snapshot while the products of the earlier ones run):
    bit-equal to device inputs, also into pinned host outputs."""
    import torch
    nx, nz, ny, ns = shape
    wl = S.small(nx, nz, ny, ns, wid=45)
    coef = S.coefficients(wl)
    y = S.cgl_grid(wl.ny)
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, ns, precision)
    try:
        tdt = torch.float64 if precision == 0 else torch.float32
        shape_t = (N.GKE_NTERM, N.gke_npair(plan), wl.nz, wl.nx)
        dev = torch.empty(shape_t, dtype=tdt, device="cuda")
        out2 = torch.empty(shape_t, dtype=tdt, device="cuda")
        pinned_out = torch.empty(shape_t, dtype=tdt).pin_memory()
        f_dev = torch.from_numpy(coef).cuda()
        f_pin = torch.from_numpy(coef).pin_memory()
        prof_d, prof_h = np.zeros((N.GKE_NPROF, ny)), np.zeros((N.GKE_NPROF, ny))
        N.gke_compute(plan, f_dev, ns, dev, prof_d)
        N.gke_compute(plan, f_pin, ns, out2, prof_h)
        N.gke_compute(plan, f_pin, ns, pinned_out)
        torch.cuda.synchronize()
        assert torch.equal(dev, out2)
        assert torch.equal(dev.cpu(), pinned_out)
        assert np.array_equal(prof_d, prof_h)
    finally:
        N.gke_destroy(plan)
