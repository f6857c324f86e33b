"""Undersampling of the separations (Sec. 3.4).

The paper keeps full resolution below a first threshold of |r|, one level of
undersampling between two thresholds and a coarser one beyond, and notes that
undersampling a posteriori loses no accuracy: every transform and derivative
runs at full resolution and only the stored set shrinks.  So the kept values
must be bit-identical to the full-resolution output at those separations, and
within the FP64 bar of the oracle there.  The kept set is computed here from
the rule documented in include/gke.h, independently of the library's tables.
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


CASES = [((3, 6, 2, 4), (2, 5, 3, 5)), ((0, 0, 1, 4), (0, 0, 1, 4)), ((0, 0, 0, 0), (1, 1, 1, 8))]


@pytest.mark.parametrize("ux,uz", CASES)
def test_undersampled_equals_full_resolution_f64(N, ux, uz):
    import oracle
    wl = S.small(32, 32, 33, 3, wid=81)
    phys = S.physical(wl)
    coef = S.to_coefficients(phys)
    full, _, _ = run(N, wl, coef)
    got, mz, mx = run(N, wl, coef, ux=ux, uz=uz)
    assert np.array_equal(mz, kept(wl.nz, uz)) and np.array_equal(mx, kept(wl.nx, ux))
    assert np.array_equal(got, full[:, :, mz][:, :, :, mx])
    ref = oracle.full(phys, S.cgl_grid(wl.ny), wl.Lx, wl.Lz, wl.nu)
    iu = np.triu_indices(wl.ny)
    for t in range(N.GKE_NTERM):
        want = ref["terms"][t][iu][:, mz][:, :, mx]
        assert rel_err(got[t], want) <= TOL_F64, N.TERMS[t]


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
