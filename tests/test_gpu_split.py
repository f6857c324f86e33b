"""Split-precision (BF16 x 3 slices, tcgen05) correlator against the FP64 path.

The bar (per term, relative to the term's largest magnitude) is
TOL_SPLIT = 1e-6: each real operand keeps ~24 significant bits in its three
BF16 slices, the six kept slice products drop terms of relative size 2^-24,
and the tensor cores accumulate in FP32, so a contraction over K <= 4 x 32
snapshot-field products carries ~1e-7 of the magnitude of its terms; the
transforms, the terms and the spectral parts of the Step-3 stencils are FP32
(the one-point parts are differenced in FP64), adding a few 1e-7.
"""
import numpy as np
import pytest

import synthetic as S
from test_gpu_parity import rel_err, run_gpu

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


@pytest.mark.parametrize("shape", [(32, 32, 33, 4), (16, 16, 129, 3), (8, 8, 257, 2), (16, 8, 65, 20)])
def test_split_matches_f64(N, shape):
    nx, nz, ny, ns = shape
    wl = S.small(nx, nz, ny, ns, wid=60 + ny)
    coef = S.coefficients(wl)
    ref, pref = run_gpu(N, wl, coef, precision=N.GKE_PREC_F64)
    got, pgot = run_gpu(N, wl, coef, precision=N.GKE_PREC_BF16X3)
    errs = [rel_err(got[t], ref[t]) for t in range(N.GKE_NTERM)]
    assert max(errs) <= TOL_SPLIT, dict(zip(N.TERMS, errs))
    assert max(errs) > 0.0          # the split path really ran (not the FP64 one)


def test_split_edge_row_with_nonzero_walls(N):
    """ny = 128 m + 1 leaves the last row / column to the CUDA-core edge kernel;
    give every field non-zero wall values so no edge term is skipped."""
    wl = S.small(16, 16, 129, 3, wid=78)
    coef = S.coefficients(wl)
    rng = np.random.default_rng(5)
    for j in (0, wl.ny - 1):
        noise = 0.05 * (rng.standard_normal(coef[:, :, j].shape) + 1j * rng.standard_normal(coef[:, :, j].shape))
        noise[..., 0] = noise[..., 0].real          # kx = 0 column of a real field stays real at kz = 0 ...
        coef[:, :, j] += noise
    # keep the fields real: rebuild the coefficients from their physical planes
    phys = np.fft.irfft2(coef, s=(wl.nz, wl.nx), axes=(-2, -1), norm="forward")
    coef = S.to_coefficients(phys)
    ref, _ = run_gpu(N, wl, coef, precision=N.GKE_PREC_F64)
    got, _ = run_gpu(N, wl, coef, precision=N.GKE_PREC_BF16X3)
    errs = [rel_err(got[t], ref[t]) for t in range(N.GKE_NTERM)]
    assert max(errs) <= TOL_SPLIT, dict(zip(N.TERMS, errs))


def test_split_multi_batch_promotes_to_fp64(N):
    """A second batch promotes the per-pair sums to FP64; the result matches one batch."""
    wl = S.small(16, 8, 33, 6, wid=77)
    coef = S.coefficients(wl)
    one, _ = run_gpu(N, wl, coef, precision=N.GKE_PREC_BF16X3)
    three, _ = run_gpu(N, wl, coef, precision=N.GKE_PREC_BF16X3, calls=[2, 3, 1])
    ref, _ = run_gpu(N, wl, coef, precision=N.GKE_PREC_F64)
    for t in range(N.GKE_NTERM):
        assert rel_err(three[t], ref[t]) <= TOL_SPLIT, N.TERMS[t]
        assert rel_err(three[t], one[t]) <= TOL_SPLIT, N.TERMS[t]


def test_split_tiny_vs_oracle(N):
    import oracle
    wl = S.TINY
    phys = S.physical(wl)
    ref = oracle.full(phys, S.cgl_grid(wl.ny), wl.Lx, wl.Lz, wl.nu)
    got, prof = run_gpu(N, wl, S.to_coefficients(phys), precision=N.GKE_PREC_BF16X3)
    iu = np.triu_indices(wl.ny)
    for t in range(N.GKE_NTERM):
        e = rel_err(got[t], ref["terms"][t][iu])
        assert e <= TOL_SPLIT, (N.TERMS[t], e)


# ------------------------------------------------------------ FP32 variant
# GKE_PREC_F32: the contractions in FP32 on the CUDA cores (FFMA, FP32
# accumulation over K <= 4 x 32 products), everything after them as on the
# split path.  Same bar as the split path.
@pytest.mark.parametrize("shape", [(32, 32, 33, 4), (16, 16, 129, 3), (16, 8, 65, 20), (16, 8, 7, 3)])
def test_f32_matches_f64(N, shape):
    nx, nz, ny, ns = shape
    wl = S.small(nx, nz, ny, ns, wid=90 + ny)
    coef = S.coefficients(wl)
    ref, _ = run_gpu(N, wl, coef, precision=N.GKE_PREC_F64)
    got, _ = run_gpu(N, wl, coef, precision=N.GKE_PREC_F32)
    errs = [rel_err(got[t], ref[t]) for t in range(N.GKE_NTERM)]
    assert max(errs) <= TOL_SPLIT, dict(zip(N.TERMS, errs))
    assert max(errs) > 0.0


def test_f32_tiny_vs_oracle(N):
    import oracle
    wl = S.TINY
    phys = S.physical(wl)
    ref = oracle.full(phys, S.cgl_grid(wl.ny), wl.Lx, wl.Lz, wl.nu)
    got, _ = run_gpu(N, wl, S.to_coefficients(phys), precision=N.GKE_PREC_F32, calls=[3, 1])
    iu = np.triu_indices(wl.ny)
    for t in range(N.GKE_NTERM):
        e = rel_err(got[t], ref["terms"][t][iu])
        assert e <= TOL_SPLIT, (N.TERMS[t], e)


# ------------------------------------------- 256 x 256: register transforms
# At nx = nz = 256 the split path runs the register-FFT column and row passes
# (two streams, pair chunks); these cases reach them with FP32 and FP64
# per-pair sums (one batch / two), the wedge and the a-posteriori separation
# selection.
@pytest.mark.parametrize("domain,calls", [(0, None), (0, [2, 1]), (1, None), (1, [1, 2])])
def test_split_256_matches_f64(N, domain, calls):
    wl = S.small(256, 256, 9, 3, wid=120 + domain)
    coef = S.coefficients(wl)
    ref, pref = run_gpu(N, wl, coef, precision=N.GKE_PREC_F64, domain=domain)
    got, pgot = run_gpu(N, wl, coef, precision=N.GKE_PREC_BF16X3, calls=calls, domain=domain)
    errs = [rel_err(got[t], ref[t]) for t in range(N.GKE_NTERM)]
    assert max(errs) <= TOL_SPLIT, dict(zip(N.TERMS, errs))
    assert max(errs) > 0.0


def test_split_256_selection_equals_full(N):
    from test_gpu_undersample import run
    wl = S.small(256, 256, 9, 2, wid=125)
    coef = S.coefficients(wl)
    full, _, _ = run(N, wl, coef, N.GKE_PREC_BF16X3)
    got, mz, mx = run(N, wl, coef, N.GKE_PREC_BF16X3, ux=(8, 64, 2, 8), uz=(4, 32, 4, 16))
    assert np.array_equal(got, full[:, :, mz][:, :, :, mx])


# --------------------------------------- plane mode over several row tiles
# ny = 193 (two tiles, the second partly empty) and 257 (two full tiles and
# the wall row): diagonal tile pairs by the shared-memory transposition,
# off-diagonal ones by the partner-free MMA order; the full triangle, the
# chunked mode at a uniform separation stride (plane chunks folded onto the
# coarse grid) and the wedge; against the FP64 path on the same inputs.
@pytest.mark.parametrize("ny,domain,stride,calls", [(257, 0, 1, None), (193, 0, 1, [2, 1]), (257, 0, 2, None),
                                                    (193, 1, 2, [1, 2]), (257, 1, 4, None), (65, 0, 2, None)])
def test_split_multi_tile_planes_match_f64(N, ny, domain, stride, calls):
    from test_gpu_undersample import run
    wl = S.small(16, 16, ny, 3, wid=140 + ny % 7 + domain)
    coef = S.coefficients(wl)
    u = (0, 0, 0, stride) if stride > 1 else (0, 0, 0, 0)
    if stride > 1:
        ref, _, _ = run(N, wl, coef, N.GKE_PREC_F64, domain=domain, ux=u, uz=u)
        got, _, _ = run(N, wl, coef, N.GKE_PREC_BF16X3, domain=domain, ux=u, uz=u)
    else:
        ref, _ = run_gpu(N, wl, coef, precision=N.GKE_PREC_F64, domain=domain)
        got, _ = run_gpu(N, wl, coef, precision=N.GKE_PREC_BF16X3, calls=calls, domain=domain)
    errs = [rel_err(got[t], ref[t]) for t in range(N.GKE_NTERM)]
    assert max(errs) <= TOL_SPLIT, dict(zip(N.TERMS, errs))
    assert max(errs) > 0.0
