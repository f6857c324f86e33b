"""Mirror sampling on the half-channel wedge (Sec. 3.2 Step 2, Sec. 3.3).

With pair_domain = GKE_DOMAIN_WEDGE every snapshot also contributes its mirror
image about the centreline and the outputs are the wedge pairs i1 <= i2,
i1 + i2 <= ny - 1.  The oracle computes the same statistics by its definition:
the plain direct averages over the snapshot set doubled by the images
(oracle.mirror_augment), read at the wedge pairs.  The CUDA path instead folds
the spectra of each wedge pair with those of its image pair and fills the
Step-3 stencils across the wedge's edges by the inversion symmetries, so the
two routes share nothing but the definition.
"""
import numpy as np
import pytest

import synthetic as S
from test_gpu_parity import TOL_F64, rel_err, run_gpu

TOL_SPLIT = 1e-6

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


def wedge_ref(ref, ny):
    import oracle
    w = np.array(oracle.wedge_pairs(ny))
    return w, ref["terms"][:, w[:, 0], w[:, 1]]


def check_wedge(N, wl, got, prof, ref, tol):
    w, want = wedge_ref(ref, wl.ny)
    assert got.shape[1] == len(w)
    for t in range(N.GKE_NTERM):
        e = rel_err(got[t], want[t])
        assert e <= tol, f"{N.TERMS[t]}: {e:.3e}"
    for k in (0, 4, 5):   # U, dU/dy, eps
        e = rel_err(prof[k], ref["prof"][k])
        assert e <= tol, f"profile {N.PROFILES[k]}: {e:.3e}"
    assert np.abs(prof[1]).max() <= 1e-15            # V of snapshots and images vanishes


@pytest.mark.parametrize("shape", [(32, 32, 33, 4), (16, 8, 7, 3), (8, 16, 10, 2), (16, 16, 65, 2)])
def test_wedge_f64_parity(N, shape):
    import oracle
    nx, nz, ny, ns = shape
    wl = S.small(nx, nz, ny, ns, wid=60 + nx + ny)
    phys = S.physical(wl)
    ref = oracle.full(phys, S.cgl_grid(ny), wl.Lx, wl.Lz, wl.nu, mirror=True)
    got, prof = run_gpu(N, wl, S.to_coefficients(phys), domain=N.GKE_DOMAIN_WEDGE)
    check_wedge(N, wl, got, prof, ref, TOL_F64)


def test_wedge_split_parity(N):
    import oracle
    wl = S.small(32, 32, 33, 4, wid=71)
    phys = S.physical(wl)
    ref = oracle.full(phys, S.cgl_grid(wl.ny), wl.Lx, wl.Lz, wl.nu, mirror=True)
    got, prof = run_gpu(N, wl, S.to_coefficients(phys), precision=N.GKE_PREC_BF16X3, domain=N.GKE_DOMAIN_WEDGE)
    check_wedge(N, wl, got, prof, ref, TOL_SPLIT)


@pytest.mark.parametrize("precision", [0, 1])
def test_wedge_batches_match_single_call(N, precision):
    wl = S.small(16, 16, 129, 4, wid=72)
    coef = S.coefficients(wl)
    a, pa = run_gpu(N, wl, coef, precision=precision, domain=N.GKE_DOMAIN_WEDGE)
    b, pb = run_gpu(N, wl, coef, precision=precision, domain=N.GKE_DOMAIN_WEDGE, calls=[3, 1])
    assert rel_err(b, a) < (TOL_F64 if precision == 0 else TOL_SPLIT)


def test_wedge_split_matches_f64_at_129(N):
    wl = S.small(16, 16, 129, 3, wid=73)
    coef = S.coefficients(wl)
    a, _ = run_gpu(N, wl, coef, domain=N.GKE_DOMAIN_WEDGE)
    b, _ = run_gpu(N, wl, coef, precision=N.GKE_PREC_BF16X3, domain=N.GKE_DOMAIN_WEDGE)
    for t in range(N.GKE_NTERM):
        assert rel_err(b[t], a[t]) <= TOL_SPLIT, N.TERMS[t]


def test_wedge_labels_and_errors(N):
    import oracle
    wl = S.small(8, 8, 9, 1)
    y = S.cgl_grid(wl.ny)
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, 1, pair_domain=N.GKE_DOMAIN_WEDGE)
    try:
        assert N.gke_npair(plan) == len(oracle.wedge_pairs(wl.ny))
        Y, ry, i1, i2 = N.gke_pair_labels(plan)
    finally:
        N.gke_destroy(plan)
    w = np.array(oracle.wedge_pairs(wl.ny))
    assert np.array_equal(i1, w[:, 0]) and np.array_equal(i2, w[:, 1])
    assert np.array_equal(ry, y[w[:, 1]] - y[w[:, 0]])
    yb = y.copy()
    yb[2] += 1e-3                                            # not symmetric about the centre
    with pytest.raises(N.GkeError) as e:
        N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, yb, 1, pair_domain=N.GKE_DOMAIN_WEDGE)
    assert e.value.status == -1
    with pytest.raises(N.GkeError) as e:
        N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, 1, pair_domain=2)
    assert e.value.status == -1


def test_wedge_f32_thresholds_vs_oracle(N):
    """FP32 contractions, mirror sampling and thresholded undersampling together."""
    import oracle
    import torch
    wl = S.small(32, 16, 17, 3, wid=74)
    phys = S.physical(wl)
    y = S.cgl_grid(wl.ny)
    ux, uz = (3, 8, 2, 4), (2, 4, 2, 4)
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, 3, N.GKE_PREC_F32,
                      pair_domain=N.GKE_DOMAIN_WEDGE, under_x=ux, under_z=uz)
    try:
        mz, mx = N.gke_separation_labels(plan)
        terms = torch.empty((N.GKE_NTERM, N.gke_npair(plan), len(mz), len(mx)), dtype=torch.float32, device="cuda")
        N.gke_compute(plan, torch.from_numpy(S.to_coefficients(phys)).cuda(), 3, terms)
        torch.cuda.synchronize()
        got = terms.cpu().numpy().astype(np.float64)
    finally:
        N.gke_destroy(plan)
    ref = oracle.full(phys, y, wl.Lx, wl.Lz, wl.nu, mirror=True)
    w = np.array(oracle.wedge_pairs(wl.ny))
    for t in range(N.GKE_NTERM):
        want = ref["terms"][t][w[:, 0], w[:, 1]][:, mz][:, :, mx]
        assert rel_err(got[t], want) <= TOL_SPLIT, N.TERMS[t]
