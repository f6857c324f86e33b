"""term_mask: a plan computes the requested terms (and the terms they are
derived from) with only the contractions those need.

Each plane of the term set equals the full run's: bit-equal contractions and
combinations, and transforms whose packed partner plane is zero instead of a
computed one, which changes rounding only (the bar is the path's tolerance
relative to the term's largest magnitude).
"""
import numpy as np
import pytest

import synthetic as S
from test_gpu_parity import TOL_F64, rel_err
from test_gpu_split import TOL_SPLIT

pytestmark = pytest.mark.gpu

A, PX, PY, PZ, PH, XI, RES = (1 << t for t in range(7))


@pytest.fixture(scope="module")
def N():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1910_06409_gb300 import build as B
    B.build()
    import paper_1910_06409_gb300._native as native
    return native


def run(N, wl, coef, precision, mask, domain=0, calls=None, host=False):
    import torch
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), coef.shape[0], precision,
                      pair_domain=domain, term_mask=mask)
    try:
        tdt = torch.float64 if precision == N.GKE_PREC_F64 else torch.float32
        dev = "cpu" if host else "cuda"
        f = torch.from_numpy(np.ascontiguousarray(coef)).to(dev)
        terms = torch.full((N.GKE_NTERM, N.gke_npair(plan), wl.nz, wl.nx), float("nan"), dtype=tdt, device=dev)
        if calls is None:
            N.gke_compute(plan, f, coef.shape[0], terms)
        else:
            N.gke_accumulate_mean(plan, f, coef.shape[0])
            s0 = 0
            for n in calls:
                N.gke_accumulate_snapshot(plan, f[s0:s0 + n], n)
                s0 += n
            N.gke_finalize_terms(plan, terms)
        torch.cuda.synchronize()
        return terms.cpu().numpy().astype(np.float64)
    finally:
        N.gke_destroy(plan)


def check(N, got, full, mask, tol):
    tset = N.gke_term_set(mask)
    for t in range(N.GKE_NTERM):
        if (tset >> t) & 1:
            e = rel_err(got[t], full[t])
            assert e <= tol, (N.TERMS[t], mask, e)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_single_terms_match_full(N, precision):
    wl = S.small(32, 16, 17, 3, wid=300 + precision)
    coef = S.coefficients(wl)
    tol = TOL_F64 if precision == N.GKE_PREC_F64 else TOL_SPLIT
    full = run(N, wl, coef, precision, 0)
    for mask in (A, PX, PY, PZ, PH, XI, RES, PX | XI):
        got = run(N, wl, coef, precision, mask)
        check(N, got, full, mask, tol)
        # planes outside the set are not written
        tset = N.gke_term_set(mask)
        for t in range(N.GKE_NTERM):
            if not (tset >> t) & 1:
                assert np.isnan(got[t]).all(), (N.TERMS[t], mask)


@pytest.mark.parametrize("precision,domain,calls,host", [(0, 1, [2, 1], False), (1, 1, None, True),
                                                         (1, 0, [1, 2], True), (0, 0, None, True)])
def test_masks_with_wedge_batches_host_output(N, precision, domain, calls, host):
    wl = S.small(16, 16, 21, 3, wid=310 + domain)
    coef = S.coefficients(wl)
    tol = TOL_F64 if precision == N.GKE_PREC_F64 else TOL_SPLIT
    full = run(N, wl, coef, precision, 0, domain=domain)
    for mask in (PY | PZ, RES, A | XI):
        got = run(N, wl, coef, precision, mask, domain=domain, calls=calls, host=host)
        check(N, got, full, mask, tol)


def test_register_transforms_256(N):
    wl = S.small(256, 256, 9, 2, wid=320)
    coef = S.coefficients(wl)
    for precision in (0, 1):
        tol = TOL_F64 if precision == N.GKE_PREC_F64 else TOL_SPLIT
        full = run(N, wl, coef, precision, 0)
        for mask in (PH, PX | XI):
            check(N, run(N, wl, coef, precision, mask), full, mask, tol)


def test_checkpoint_needs_same_term_set(N, tmp_path):
    import torch
    wl = S.small(16, 8, 9, 2, wid=330)
    coef = torch.from_numpy(S.coefficients(wl)).cuda()
    y = S.cgl_grid(wl.ny)
    pa = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, 2, 0, term_mask=A)
    pb = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, 2, 0, term_mask=XI)
    pc = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, y, 2, 0, term_mask=A)
    try:
        N.gke_accumulate_mean(pa, coef, 2)
        N.gke_accumulate_snapshot(pa, coef, 2)
        path = str(tmp_path / "a.ckpt")
        N.gke_checkpoint(pa, path)
        with pytest.raises(N.GkeError) as ei:
            N.gke_restore(pb, path)
        assert ei.value.status == -1
        N.gke_restore(pc, path)                 # same set
    finally:
        for p in (pa, pb, pc):
            N.gke_destroy(p)


def test_bad_mask_rejected(N):
    wl = S.small(8, 8, 9, 1)
    with pytest.raises(N.GkeError) as ei:
        N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), 1, 0, term_mask=1 << 7)
    assert ei.value.status == -1


def test_noalloc_mask(N):
    import torch
    wl = S.small(16, 16, 9, 2, wid=340)
    coef = S.coefficients(wl)
    full = run(N, wl, coef, 0, 0)
    f = torch.from_numpy(coef).cuda()
    npair = wl.ny * (wl.ny + 1) // 2
    got = torch.full((N.GKE_NTERM, npair, wl.nz, wl.nx), float("nan"), dtype=torch.float64, device="cuda")
    N.gke_compute_noalloc(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), f, 2, got, term_mask=RES)
    torch.cuda.synchronize()
    check(N, got.cpu().numpy(), full, RES, TOL_F64)
