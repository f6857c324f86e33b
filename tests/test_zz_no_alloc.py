"""gke_compute_noalloc: the FP64 path from a fixed device array, no allocation.

Some callers cannot call cudaMalloc (they run inside a memory pool or an
allocator they must not re-enter, or under a runtime that forbids device
allocation after start-up).  gke_compute_noalloc serves them: its workspaces
come from one file-scope device array, so its results must equal those of
the plan-based gke_compute on the same input, also on a second call that
reuses the array's stale contents.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

TOL = 1e-12   # same bar as the FP64 parity tests


def test_noalloc_matches_plan_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1910_06409_gb300 import build as B
    B.build()
    import paper_1910_06409_gb300._native as N

    outs = []
    for wid, shape in ((31, (16, 16, 17, 2)), (32, (16, 8, 13, 3)), (34, (24, 12, 9, 2))):
        nx, nz, ny, ns = shape
        wl = S.small(nx, nz, ny, ns, wid=wid)
        y = S.cgl_grid(ny)
        coef = torch.from_numpy(S.coefficients(wl)).cuda()
        plan = N.gke_plan(nx, nz, ny, wl.Lx, wl.Lz, wl.nu, y, ns, N.GKE_PREC_F64)
        try:
            npair = N.gke_npair(plan)
            ref = torch.empty((N.GKE_NTERM, npair, nz, nx), dtype=torch.float64, device="cuda")
            pref = torch.empty((N.GKE_NPROF, ny), dtype=torch.float64, device="cuda")
            N.gke_compute(plan, coef, ns, ref, pref)
        finally:
            N.gke_destroy(plan)
        for call in range(2):          # the second call reuses the array's previous contents
            got = torch.full((N.GKE_NTERM, npair, nz, nx), float("nan"), dtype=torch.float64, device="cuda")
            prof = torch.empty((N.GKE_NPROF, ny), dtype=torch.float64, device="cuda")
            N.gke_compute_noalloc(nx, nz, ny, wl.Lx, wl.Lz, wl.nu, y, coef, ns, got, prof)
            torch.cuda.synchronize()
            r, g = ref.cpu().numpy(), got.cpu().numpy()
            for t in range(N.GKE_NTERM):
                err = np.abs(g[t] - r[t]).max() / np.abs(r[t]).max()
                assert err <= TOL, (shape, call, N.TERMS[t], err)
            np.testing.assert_allclose(prof.cpu().numpy(), pref.cpu().numpy(), rtol=TOL, atol=1e-300)
            outs.append(g)
    # too large for the fixed array: a clear status, not a fault
    wl = S.small(64, 64, 65, 2, wid=33)
    coef = torch.from_numpy(S.coefficients(wl)).cuda()
    big = torch.empty((N.GKE_NTERM, wl.npair, 64, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(N.GkeError) as e:
        N.gke_compute_noalloc(64, 64, 65, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(65), coef, 2, big)
    assert e.value.status == -7
