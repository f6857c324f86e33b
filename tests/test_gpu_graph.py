"""gke_compute_graph: one pass captured into a CUDA graph and replayed.

The graph runs the same kernels as gke_compute on the same stream with the
same launch parameters, and the Step-1 mean is frozen by a device kernel
doing the same FP64 operations as the host freeze, so the results are
bit-equal to gke_compute's -- after a replay too, and after the input buffer
is overwritten in place (the graph reads the data again, not a copy).
"""
import numpy as np
import pytest

import synthetic as S

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


def _pass(N, fn, plan, f, ns, terms, prof):
    import torch
    fn(plan, f, ns, terms, prof)
    torch.cuda.synchronize()
    return terms.cpu().numpy().copy(), prof.cpu().numpy().copy()


@pytest.mark.parametrize("shape,precision,domain", [
    ((32, 16, 33, 5), 0, 0),
    ((32, 16, 33, 5), 1, 0),
    ((32, 16, 33, 5), 2, 0),
    ((16, 16, 21, 4), 0, 1),
    ((16, 16, 21, 4), 1, 1),
    ((256, 256, 17, 2), 1, 0),     # register transforms, several pair chunks
])
def test_graph_equals_compute(N, shape, precision, domain):
    import torch
    nx, nz, ny, ns = shape
    wl = S.small(nx, nz, ny, ns, wid=400 + ny + precision)
    coef = S.coefficients(wl)
    s = torch.cuda.Stream()
    plan = N.gke_plan(nx, nz, ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(ny), ns, precision,
                      stream=s.cuda_stream, pair_domain=domain)
    try:
        npair = N.gke_npair(plan)
        tdt = torch.float64 if precision == N.GKE_PREC_F64 else torch.float32
        f = torch.from_numpy(np.ascontiguousarray(coef)).cuda()
        terms = torch.empty((N.GKE_NTERM, npair, nz, nx), dtype=tdt, device="cuda")
        prof = torch.empty((N.GKE_NPROF, ny), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        want_t, want_p = _pass(N, N.gke_compute, plan, f, ns, terms, prof)
        l0 = N.gke_launch_count(plan)
        terms.fill_(float("nan"))
        got_t, got_p = _pass(N, N.gke_compute_graph, plan, f, ns, terms, prof)
        assert np.array_equal(got_t, want_t) and np.array_equal(got_p, want_p)
        l1 = N.gke_launch_count(plan)
        assert l1 > l0
        # replay
        terms.fill_(float("nan"))
        got_t, got_p = _pass(N, N.gke_compute_graph, plan, f, ns, terms, prof)
        assert np.array_equal(got_t, want_t) and np.array_equal(got_p, want_p)
        assert N.gke_launch_count(plan) - l1 == l1 - l0
        # new data in the same buffer: the replay reads it
        coef2 = S.coefficients(S.small(nx, nz, ny, ns, wid=500 + ny + precision))
        f.copy_(torch.from_numpy(np.ascontiguousarray(coef2)))
        g2_t, g2_p = _pass(N, N.gke_compute_graph, plan, f, ns, terms, prof)
        w2_t, w2_p = _pass(N, N.gke_compute, plan, f, ns, terms, prof)
        assert np.array_equal(g2_t, w2_t) and np.array_equal(g2_p, w2_p)
        assert not np.array_equal(g2_t, want_t)
        # another nsnap: captured again
        if ns > 1:
            g3_t, _ = _pass(N, N.gke_compute_graph, plan, f, ns - 1, terms, prof)
            w3_t, _ = _pass(N, N.gke_compute, plan, f, ns - 1, terms, prof)
            assert np.array_equal(g3_t, w3_t)
        # the plan still serves the incremental calls afterwards
        N.gke_compute_graph(plan, f, ns, terms, prof)
        N.gke_reset(plan)
        N.gke_accumulate_mean(plan, f, ns)
        N.gke_accumulate_snapshot(plan, f, ns)
        N.gke_finalize_terms(plan, terms, prof)
        torch.cuda.synchronize()
        assert np.array_equal(terms.cpu().numpy(), w2_t)
    finally:
        N.gke_destroy(plan)


def test_graph_rejects_host_pointers_and_default_stream(N):
    import torch
    wl = S.small(16, 16, 9, 2, wid=450)
    coef = S.coefficients(wl)
    f = torch.from_numpy(np.ascontiguousarray(coef))
    plan = N.gke_plan(16, 16, 9, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(9), 2, 0)
    try:
        npair = N.gke_npair(plan)
        terms = torch.empty((N.GKE_NTERM, npair, 16, 16), dtype=torch.float64, device="cuda")
        with pytest.raises(RuntimeError):
            N.gke_compute_graph(plan, f, 2, terms)               # host fields
        with pytest.raises(RuntimeError):
            N.gke_compute_graph(plan, f.cuda(), 2, terms)        # legacy-stream plan
    finally:
        N.gke_destroy(plan)
