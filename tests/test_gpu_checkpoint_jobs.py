"""Checkpoints of independent jobs (Sec. 3.4): the split path's plane spectra,
the accumulator-layout check, and the Step-1 mean shared by merged jobs.

A job's spectra are sums of products of fluctuations about the Step-1 mean it
froze (Step 1 precedes Step 2, Sec. 3.2), so two jobs add exactly only when
they froze the same mean; gke_merge and the host merge tool refuse files whose
means differ.
"""
import numpy as np
import pytest

import synthetic as S
from test_gpu_parity import TOL_F64, rel_err, run_gpu
from test_gpu_split import TOL_SPLIT

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


def _job(N, wl, f, precision, part, path, mean=None, mean_from=None):
    """One job: its mean (given, or Step 1 over the snapshots mean_from), then
    its snapshot subset part = (a, b), saved to path."""
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), wl.nsnap, precision)
    try:
        if mean is not None:
            N.gke_set_mean(plan, mean)
        else:
            a, b = mean_from
            N.gke_accumulate_mean(plan, f[a:b], b - a)
        a, b = part
        N.gke_accumulate_snapshot(plan, f[a:b], b - a)
        N.gke_checkpoint(plan, path)
    finally:
        N.gke_destroy(plan)


def _finalize_from(N, wl, precision, paths):
    import torch
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), wl.nsnap, precision)
    try:
        N.gke_restore(plan, paths[0])
        for p in paths[1:]:
            N.gke_merge(plan, p)
        tdt = torch.float64 if precision == N.GKE_PREC_F64 else torch.float32
        terms = torch.empty((N.GKE_NTERM, N.gke_npair(plan), wl.nz, wl.nx), dtype=tdt, device="cuda")
        N.gke_finalize_terms(plan, terms)
        return terms.cpu().numpy().astype(np.float64)
    finally:
        N.gke_destroy(plan)


@pytest.mark.parametrize("shape", [(16, 16, 33, 5), (16, 8, 129, 4)])
def test_split_planes_checkpoint_merge(N, shape, tmp_path):
    """Split path on one 128-row tile: the plane spectra of two jobs, merged on
    the device and on the host, equal one pass within the split tolerance."""
    import torch
    nx, nz, ny, ns = shape
    wl = S.small(nx, nz, ny, ns, wid=140 + ny)
    coef = S.coefficients(wl)
    one, _ = run_gpu(N, wl, coef, precision=N.GKE_PREC_BF16X3)
    ref, _ = run_gpu(N, wl, coef, precision=N.GKE_PREC_F64)
    f = torch.from_numpy(coef).cuda()
    mean = np.ascontiguousarray(coef[:, :, :, 0, 0].real.mean(axis=0))
    paths = [str(tmp_path / f"j{i}.ckpt") for i in range(2)]
    _job(N, wl, f, N.GKE_PREC_BF16X3, (0, 2), paths[0], mean=mean)
    _job(N, wl, f, N.GKE_PREC_BF16X3, (2, ns), paths[1], mean=mean)
    got = _finalize_from(N, wl, N.GKE_PREC_BF16X3, paths)
    for t in range(N.GKE_NTERM):
        assert rel_err(got[t], one[t]) <= TOL_SPLIT, N.TERMS[t]
        assert rel_err(got[t], ref[t]) <= TOL_SPLIT, N.TERMS[t]
    from paper_1910_06409_gb300 import merge as M
    merged = str(tmp_path / "merged.ckpt")
    ck = M.merge(paths, merged)
    assert ck["header"]["acc_kind"] == 1            # plane spectra
    host = _finalize_from(N, wl, N.GKE_PREC_BF16X3, [merged])
    assert np.array_equal(host, got)
    # a plane-spectra file does not restore into a plan that combines per-pair term spectra
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), wl.nsnap, N.GKE_PREC_F64)
    try:
        with pytest.raises(N.GkeError) as e:
            N.gke_restore(plan, paths[0])
        assert e.value.status == -1
    finally:
        N.gke_destroy(plan)


def test_merge_refuses_jobs_with_their_own_means(N, tmp_path):
    """Each job froze the mean of its own snapshot subset: gke_merge and the
    host tool refuse; with a shared Step-1 mean the merge equals one pass."""
    import torch
    wl = S.small(16, 8, 9, 4, wid=150)
    coef = S.coefficients(wl)
    # per-snapshot plane means (the k = 0 coefficients), so that the mean of a
    # snapshot subset differs from the ensemble mean
    coef[:, :, :, 0, 0] += np.random.default_rng(3).standard_normal(coef.shape[:3]) * 0.1
    f = torch.from_numpy(coef).cuda()
    own = [str(tmp_path / f"own{i}.ckpt") for i in range(2)]
    _job(N, wl, f, N.GKE_PREC_F64, (0, 2), own[0], mean_from=(0, 2))
    _job(N, wl, f, N.GKE_PREC_F64, (2, 4), own[1], mean_from=(2, 4))
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), wl.nsnap)
    try:
        N.gke_restore(plan, own[0])
        with pytest.raises(N.GkeError) as e:
            N.gke_merge(plan, own[1])
        assert e.value.status == -1 and "mean" in str(e.value)
    finally:
        N.gke_destroy(plan)
    from paper_1910_06409_gb300 import merge as M
    with pytest.raises(M.CheckpointError, match="mean"):
        M.merge(own, str(tmp_path / "m.ckpt"))
    # Step 1 over all snapshots in each job (the same mean), Step 2 on subsets
    shared = [str(tmp_path / f"shared{i}.ckpt") for i in range(2)]
    _job(N, wl, f, N.GKE_PREC_F64, (0, 2), shared[0], mean_from=(0, 4))
    _job(N, wl, f, N.GKE_PREC_F64, (2, 4), shared[1], mean_from=(0, 4))
    got = _finalize_from(N, wl, N.GKE_PREC_F64, shared)
    one, _ = run_gpu(N, wl, coef)
    assert rel_err(got, one) <= TOL_F64
