"""tune_cache: the plan's schedule (transform pair-chunk size, combine
wavenumbers per CTA) measured on the device once per shape and kept in a
text file.  The knobs change no arithmetic, so tuned and untuned plans give
bit-equal results."""
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


def plan_and_run(N, wl, coef, precision, cache=None):
    import torch
    plan = N.gke_plan(wl.nx, wl.nz, wl.ny, wl.Lx, wl.Lz, wl.nu, S.cgl_grid(wl.ny), coef.shape[0], precision,
                      tune_cache=cache)
    try:
        knobs = N.gke_plan_knobs(plan)
        tdt = torch.float64 if precision == N.GKE_PREC_F64 else torch.float32
        terms = torch.empty((N.GKE_NTERM, N.gke_npair(plan), wl.nz, wl.nx), dtype=tdt, device="cuda")
        N.gke_compute(plan, torch.from_numpy(coef).cuda(), coef.shape[0], terms)
        torch.cuda.synchronize()
        return knobs, terms.cpu().numpy()
    finally:
        N.gke_destroy(plan)


@pytest.mark.parametrize("shape,precision", [((256, 256, 9, 2), 1), ((256, 256, 9, 2), 0), ((32, 16, 17, 3), 2)])
def test_tuned_plan_bit_equal_and_cached(N, tmp_path, shape, precision):
    nx, nz, ny, ns = shape
    wl = S.small(nx, nz, ny, ns, wid=350 + precision)
    coef = S.coefficients(wl)
    cache = tmp_path / "tune.txt"
    k0, ref = plan_and_run(N, wl, coef, precision)
    assert k0[2] == 0                                         # built-in schedule
    k1, got1 = plan_and_run(N, wl, coef, precision, cache)
    assert k1[2] == 2 and k1[0] in (48, 96, 192)              # measured now
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and f"nx{nx} nz{nz} ny{ny}" in lines[0]
    k2, got2 = plan_and_run(N, wl, coef, precision, cache)
    assert k2 == (k1[0], k1[1], 1)                            # from the file
    assert len(cache.read_text().splitlines()) == 1
    assert np.array_equal(got1, ref) and np.array_equal(got2, ref)


def test_cache_keys_and_bad_lines(N, tmp_path):
    cache = tmp_path / "tune.txt"
    cache.write_text("not a tuning line\ngke-tune-1 garbage : w_mib=7 comb_kc=3\n")
    a = S.small(16, 16, 9, 2, wid=360)
    b = S.small(32, 16, 9, 2, wid=361)
    ka, _ = plan_and_run(N, a, S.coefficients(a), 1, cache)
    kb, _ = plan_and_run(N, b, S.coefficients(b), 1, cache)
    assert ka[2] == 2 and kb[2] == 2
    assert len(cache.read_text().splitlines()) == 4           # two foreign lines kept, one line per shape
    # a line with values outside the candidates is not used
    lines = cache.read_text().splitlines()
    lines[-1] = lines[-1].split(" : ")[0] + " : w_mib=7 comb_kc=3"
    cache.write_text("\n".join(lines) + "\n")
    kb2, _ = plan_and_run(N, b, S.coefficients(b), 1, cache)
    assert kb2[2] == 2


def test_unwritable_cache_still_plans(N, tmp_path):
    wl = S.small(16, 16, 9, 2, wid=362)
    k, _ = plan_and_run(N, wl, S.coefficients(wl), 0, tmp_path / "missing_dir" / "tune.txt")
    assert k[2] == 2
