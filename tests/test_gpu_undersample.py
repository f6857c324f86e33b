"""Undersampling of the separations (Sec. 3.4).

The paper keeps full resolution below a first threshold of |r|, one level of
undersampling between two thresholds and a coarser one beyond, and notes that
undersampling a posteriori loses no accuracy.  Thresholded undersampling
selects from the full-resolution result, so the kept values must be
bit-identical to the full-resolution output at those separations.  A uniform
stride (s | n in both directions) instead aliases the spectra onto the coarse
grid chunk by chunk and transforms there: the same values up to rounding.
Both must be within the FP64 bar of the oracle.  The kept set is computed
here from the rule documented in include/gke.h, independently of the
library's tables.
"""
import numpy as np
import pytest

import synthetic as S
from test_gpu_parity import TOL_F64, rel_err

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


def kept(n, u):
    t1, t2, s1, s2 = u
    if not any(u):
        return np.arange(n)
    d = np.minimum(np.arange(n), n - np.arange(n))
    keep = (d < t1) | ((d >= t1) & (d < t2) & (d % max(s1, 1) == 0)) | ((d >= t2) & (d % max(s2, 1) == 0))
    return np.nonzero(keep)[0]


def run(N, wl, coef, precision=0, domain=0, ux=(0, 0, 0, 0), uz=(0, 0, 0, 0)):
    import torch
    y = S.cgl_grid(wl.ny)
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, coef.shape[0], precision,
                      pair_domain=domain, under_x=ux, under_z=uz)
    try:
        mz, mx = N.gke_separation_labels(plan)
        tdt = torch.float64 if precision == 0 else torch.float32
        terms = torch.empty((N.GKE_NTERM, N.gke_npair(plan), len(mz), len(mx)), dtype=tdt, device="cuda")
        assert N.gke_terms_bytes(plan) == terms.numel() * terms.element_size()
        N.gke_compute(plan, torch.from_numpy(coef).cuda(), coef.shape[0], terms)
        torch.cuda.synchronize()
        return terms.cpu().numpy(), mz, mx
    finally:
        N.gke_destroy(plan)


def uniform(n, u):
    """True when the option keeps exactly the multiples of a stride dividing n."""
    return not any(u) or (u[0] == 0 and u[1] == 0 and u[3] >= 1 and n % u[3] == 0)


CASES = [((3, 6, 2, 4), (2, 5, 3, 5)), ((0, 0, 1, 4), (0, 0, 1, 4)), ((0, 0, 0, 0), (1, 1, 1, 8)),
         ((0, 0, 0, 2), (0, 0, 0, 4)), ((0, 0, 0, 0), (0, 0, 1, 8)), ((0, 0, 0, 4), (0, 0, 0, 0))]


@pytest.mark.parametrize("ux,uz", CASES)
def test_undersampled_equals_full_resolution_f64(N, ux, uz):
    import oracle
    wl = S.small(32, 32, 33, 3, wid=81)
    phys = S.physical(wl)
    coef = S.to_coefficients(phys)
    full, _, _ = run(N, wl, coef)
    got, mz, mx = run(N, wl, coef, ux=ux, uz=uz)
    assert np.array_equal(mz, kept(wl.nz, uz)) and np.array_equal(mx, kept(wl.nx, ux))
    sub = full[:, :, mz][:, :, :, mx]
    if uniform(wl.nz, uz) and uniform(wl.nx, ux):
        for t in range(N.GKE_NTERM):
            assert rel_err(got[t], sub[t]) <= TOL_F64, N.TERMS[t]
    else:
        assert np.array_equal(got, sub)
    ref = oracle.full(phys, S.cgl_grid(wl.ny), wl.Lx, wl.Lz, wl.nu)
    iu = np.triu_indices(wl.ny)
    for t in range(N.GKE_NTERM):
        want = ref["terms"][t][iu][:, mz][:, :, mx]
        assert rel_err(got[t], want) <= TOL_F64, N.TERMS[t]


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_stride_wedge_batches(N, precision):
    """Uniform strides on the wedge with several batches (the streaming mode):
    the oracle over snapshots and mirror images, read at the kept separations."""
    import oracle
    wl = S.small(32, 16, 17, 4, wid=83)
    phys = S.physical(wl)
    coef = S.to_coefficients(phys)
    ux, uz = (0, 0, 0, 4), (0, 0, 0, 2)
    import torch
    y = S.cgl_grid(wl.ny)
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, 2, precision,
                      pair_domain=N.GKE_DOMAIN_WEDGE, under_x=ux, under_z=uz)
    try:
        mz, mx = N.gke_separation_labels(plan)
        tdt = torch.float64 if precision == 0 else torch.float32
        terms = torch.empty((N.GKE_NTERM, N.gke_npair(plan), len(mz), len(mx)), dtype=tdt, device="cuda")
        f = torch.from_numpy(coef).cuda()
        N.gke_accumulate_mean(plan, f, 2)
        N.gke_accumulate_mean(plan, f[2:], 2)
        N.gke_accumulate_snapshot(plan, f[:2], 2)
        N.gke_accumulate_snapshot(plan, f[2:], 2)
        N.gke_finalize_terms(plan, terms)
        torch.cuda.synchronize()
        got = terms.cpu().numpy().astype(np.float64)
    finally:
        N.gke_destroy(plan)
    assert np.array_equal(mz, kept(wl.nz, uz)) and np.array_equal(mx, kept(wl.nx, ux))
    ref = oracle.full(phys, y, wl.Lx, wl.Lz, wl.nu, mirror=True)
    w = np.array(oracle.wedge_pairs(wl.ny))
    tol = TOL_F64 if precision == 0 else 1e-6
    for t in range(N.GKE_NTERM):
        want = ref["terms"][t][w[:, 0], w[:, 1]][:, mz][:, :, mx]
        assert rel_err(got[t], want) <= tol, (N.TERMS[t], rel_err(got[t], want))


def test_stride_checkpoint_merge(N, tmp_path):
    """Independent jobs (Sec. 3.4) on the coarse spectra merge to one pass."""
    wl = S.small(16, 16, 17, 4, wid=84)
    coef = S.coefficients(wl)
    ux = uz = (0, 0, 0, 2)
    one, _, _ = run(N, wl, coef, ux=ux, uz=uz)
    import torch
    y = S.cgl_grid(wl.ny)
    f = torch.from_numpy(coef).cuda()
    paths = []
    for part in ((0, 2), (2, 4)):
        plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, 4, under_x=ux, under_z=uz)
        try:
            N.gke_accumulate_mean(plan, f, 4)
            N.gke_accumulate_snapshot(plan, f[part[0]:part[1]], 2)
            path = str(tmp_path / f"part{part[0]}.ckpt")
            N.gke_checkpoint(plan, path)
            paths.append(path)
        finally:
            N.gke_destroy(plan)
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, 4, under_x=ux, under_z=uz)
    try:
        N.gke_restore(plan, paths[0])
        N.gke_merge(plan, paths[1])
        mz, mx = N.gke_separation_labels(plan)
        terms = torch.empty((N.GKE_NTERM, N.gke_npair(plan), len(mz), len(mx)), dtype=torch.float64, device="cuda")
        N.gke_finalize_terms(plan, terms)
        torch.cuda.synchronize()
        merged = terms.cpu().numpy()
    finally:
        N.gke_destroy(plan)
    assert rel_err(merged, one) <= TOL_F64


def test_undersampled_split_and_wedge(N):
    wl = S.small(32, 32, 33, 4, wid=82)
    coef = S.coefficients(wl)
    ux, uz = (4, 8, 2, 4), (0, 0, 1, 4)
    for precision in (0, 1):
        full, _, _ = run(N, wl, coef, precision, domain=N.GKE_DOMAIN_WEDGE)
        got, mz, mx = run(N, wl, coef, precision, domain=N.GKE_DOMAIN_WEDGE, ux=ux, uz=uz)
        assert np.array_equal(got, full[:, :, mz][:, :, :, mx]), precision


def test_undersampling_errors(N):
    wl = S.small(8, 8, 9, 1)
    y = S.cgl_grid(wl.ny)
    for bad in ((3, 2, 1, 1), (0, 2, 0, 1), (-1, 0, 1, 1)):
        with pytest.raises(N.GkeError) as e:
            N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, 1, under_x=bad)
        assert e.value.status == -1


# ------------------------------------ Re_tau~1000-shaped grid, streaming mode
def test_retau1000_grid_streaming_spot_checks(N):
    """512 x 512 x 257 (the Re_tau~1000-shaped grid) in the memory-bounded
    mode: mirror sampling on the wedge, separations every 4th grid step,
    snapshots streamed 2 at a time, split-BF16 contractions.  Sampled outputs
    against the oracle over the snapshots and their mirror images."""
    import oracle
    import torch
    base = S.RETAU1000
    wl = S.Workload(base.name, base.wid, base.nx, base.nz, base.ny, 4, base.Lx, base.Lz, base.nu)
    phys = S.physical(wl)
    coef = S.to_coefficients(phys)
    y = S.cgl_grid(wl.ny)
    st = (0, 0, 0, 4)
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, 2, N.GKE_PREC_BF16X3,
                      pair_domain=N.GKE_DOMAIN_WEDGE, under_x=st, under_z=st)
    try:
        mz, mx = N.gke_separation_labels(plan)
        assert len(mz) == 128 and len(mx) == 128
        terms = torch.empty((N.GKE_NTERM, N.gke_npair(plan), 128, 128), dtype=torch.float32, device="cuda")
        f = torch.from_numpy(coef).cuda()
        for b in (0, 2):
            N.gke_accumulate_mean(plan, f[b:b + 2], 2)
        for b in (0, 2):
            N.gke_accumulate_snapshot(plan, f[b:b + 2], 2)
        N.gke_finalize_terms(plan, terms)
        torch.cuda.synchronize()
        got = terms.cpu().numpy().astype(np.float64)
    finally:
        N.gke_destroy(plan)
    w = oracle.wedge_pairs(wl.ny)
    windex = {p: i for i, p in enumerate(w)}
    rng = np.random.default_rng(1000)
    planes = [0, 1, 2, 60, 128, 200, 254, 256]
    pts, idx = [], []
    while len(pts) < 24:
        a, b = sorted(rng.choice(planes, 2))
        if a + b > wl.ny - 1:
            continue
        jz, jx = int(rng.integers(128)), int(rng.integers(128))
        pts.append((a, b, int(mz[jz]), int(mx[jx])))
        idx.append((windex[(a, b)], jz, jx))
    ref = oracle.points(phys, y, wl.Lx, wl.Lz, wl.nu, pts, mirror=True)
    scale = np.abs(got[:6]).reshape(6, -1).max(axis=1)
    for n, (pw, jz, jx) in enumerate(idx):
        err = np.abs(got[:6, pw, jz, jx] - ref["terms"][n]) / scale
        assert err.max() <= 1e-6, (pts[n], err)


def test_stride_on_three_times_power_of_two_grid(N):
    """A 48 x 24 grid (radix-3 transforms) with stride 2 x 3 on the coarse 24 x 8 grid."""
    import oracle
    wl = S.small(24, 48, 9, 2, wid=85)
    phys = S.physical(wl)
    got, mz, mx = run(N, wl, S.to_coefficients(phys), ux=(0, 0, 0, 3), uz=(0, 0, 0, 2))
    assert np.array_equal(mz, np.arange(0, 48, 2)) and np.array_equal(mx, np.arange(0, 24, 3))
    ref = oracle.full(phys, S.cgl_grid(wl.ny), wl.Lx, wl.Lz, wl.nu)
    iu = np.triu_indices(wl.ny)
    for t in range(N.GKE_NTERM):
        assert rel_err(got[t], ref["terms"][t][iu][:, mz][:, :, mx]) <= TOL_F64, N.TERMS[t]


def test_grid_384_chunked_spot_checks(N):
    """The 384 x 384 x 193 grid of the grouped configuration (radix-3
    transforms; one batch's FP64 contractions would take 332 GB, so the plan
    runs in the chunked mode) at separation stride 2, two snapshots, FP64:
    sampled outputs against the oracle."""
    import oracle
    import torch
    base = S.GROUP_C
    wl = S.Workload(base.name, base.wid, base.nx, base.nz, base.ny, 2, base.Lx, base.Lz, base.nu)
    phys = S.physical(wl)
    coef = S.to_coefficients(phys)
    y = S.cgl_grid(wl.ny)
    st = (0, 0, 0, 2)
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, 2, under_x=st, under_z=st)
    try:
        mz, mx = N.gke_separation_labels(plan)
        terms = torch.empty((N.GKE_NTERM, N.gke_npair(plan), len(mz), len(mx)), dtype=torch.float64, device="cuda")
        N.gke_compute(plan, torch.from_numpy(coef).cuda(), 2, terms)
        torch.cuda.synchronize()
        got = terms.cpu().numpy()
    finally:
        N.gke_destroy(plan)
    rng = np.random.default_rng(384)
    planes = [0, 1, 2, 50, 96, 150, 191, 192]
    pts, idx = [], []
    for _ in range(24):
        a, b = sorted(rng.choice(planes, 2))
        jz, jx = int(rng.integers(len(mz))), int(rng.integers(len(mx)))
        pts.append((a, b, int(mz[jz]), int(mx[jx])))
        idx.append((a * wl.ny - a * (a - 1) // 2 + (b - a), jz, jx))
    ref = oracle.points(phys, y, wl.Lx, wl.Lz, wl.nu, pts)
    scale = np.abs(got[:6]).reshape(6, -1).max(axis=1)
    for n, (p, jz, jx) in enumerate(idx):
        err = np.abs(got[:6, p, jz, jx] - ref["terms"][n]) / scale
        assert err.max() <= TOL_F64, (pts[n], err)
