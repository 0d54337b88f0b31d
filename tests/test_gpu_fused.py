"""GPU tests of the fused FP32 apply (trial y, x stage and test y in one kernel
per q3 plane and run of q2 lines, partials kept in shared memory).

Tolerance: the FP32 apply bound of the other FP32 tests, 1e-5 of the largest
oracle entry (operands rounded to 2^-24, a few hundred terms per output).  The
fused path sums the y contractions in another order than the staged path, so
the two agree to FP32 rounding, not bitwise: 2e-6 relative to the largest
entry.

Shapes: direction 1 long enough for a translation-invariant interior at
every degree, q2 counts that leave a partial last batch of 8 lines, enough q3 planes
for several q2 segments per plane (U rows shared by two segments are added
twice onto zero), a single-segment plane, every stencil degree 2..8, and
non-uniform knots in every direction (the fused kernel takes the bands of
directions 2 and 3 from tables, and the stencil x stage takes direction 1's
non-invariant rows from its band tables).""" 
import json

import numpy as np
import pytest

import oracle as O
from paper_1712_08565_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-5


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_08565_gb300 import build
    build.build()
    from paper_1712_08565_gb300 import mfwq
    return mfwq


def _patch(mf, ps, knots, seed):
    op = mf.Operator(ps, knots, mixed=True, device=DEV)
    tabs = [O.tables_1d(knots[l], ps[l]) for l in range(3)]
    C6 = O.coefficient_grid(tabs, "ring", inputs.fourier_modes(seed), 0.3)
    op.set_coeff(torch.from_numpy(np.ascontiguousarray(C6)).to(DEV))
    return op, tabs, C6


def _apply32(op, x):
    return op.apply_f32(torch.from_numpy(x).float().to(DEV)).double().cpu().numpy()


@pytest.mark.parametrize("p,nel", [(2, (12, 21, 6)), (3, (12, 18, 7)), (4, (13, 17, 6)), (5, (16, 20, 5)),
                                   (6, (18, 19, 5)), (7, (20, 22, 4)), (8, (22, 24, 4))])
def test_fused_apply_matches_oracle(mf, p, nel):
    knots = [inputs.open_uniform_knots(p, nel[l]) for l in range(3)]
    op, tabs, C6 = _patch(mf, (p, p, p), knots, 20 + p)
    assert op.fp32_path == "staged"  # the default; the autotuner may pick the fused path
    op.fp32_path = "fused"
    x = inputs.uniform_vector(op.shape, 30 + p)
    ref = O.apply_alg2(tabs, O.full_coeff(C6), x)
    y = _apply32(op, x)
    assert np.abs(y - ref).max() <= TOL * np.abs(ref).max()
    # twice in a row: the straddling rows are zeroed again, nothing carries over
    y2 = _apply32(op, x)
    assert np.array_equal(y, y2)
    op.close()


@pytest.mark.parametrize("ps,nel", [((3, 2, 4), (10, 4, 6)), ((4, 5, 3), (12, 30, 9)), ((6, 3, 2), (18, 25, 40))])
def test_fused_equals_staged(mf, ps, nel):
    """Mixed degrees; (3, 2, 4) with 4 elements in direction 2 has one segment per plane."""
    knots = [inputs.open_uniform_knots(ps[l], nel[l]) for l in range(3)]
    op, tabs, C6 = _patch(mf, ps, knots, 7)
    x = inputs.uniform_vector(op.shape, 8)
    op.fp32_path = "fused"
    yf = _apply32(op, x)
    op.fp32_path = "staged"
    ys = _apply32(op, x)
    ref = O.apply_alg2(tabs, O.full_coeff(C6), x)
    assert np.abs(ys - ref).max() <= TOL * np.abs(ref).max()
    assert np.abs(yf - ref).max() <= TOL * np.abs(ref).max()
    assert np.abs(yf - ys).max() <= 2e-6 * np.abs(ref).max()
    op.close()


def test_fused_with_graded_knots_in_directions_2_and_3(mf):
    p = 3
    knots = [inputs.open_uniform_knots(p, 12), inputs.jittered_knots(p, 16, seed=3), inputs.jittered_knots(p, 7, seed=5)]
    op, tabs, C6 = _patch(mf, (p, p, p), knots, 9)
    op.fp32_path = "fused"
    x = inputs.uniform_vector(op.shape, 10)
    ref = O.apply_alg2(tabs, O.full_coeff(C6), x)
    assert np.abs(_apply32(op, x) - ref).max() <= TOL * np.abs(ref).max()
    op.close()


def test_fused_unavailable_falls_back(mf):
    """Degree 9 in direction 1 is above the stencil forms (p <= 8): the staged
    path runs and asking for the fused one is refused with the reason.  Graded
    knots in direction 1 keep a one-pair interior, boundary rows from the band
    tables, and the fused apply still matches the oracle; a reaction term makes
    the apply take the staged kernels."""
    knots = [inputs.open_uniform_knots(9, 20), inputs.open_uniform_knots(2, 6), inputs.open_uniform_knots(2, 5)]
    op, tabs, C6 = _patch(mf, (9, 2, 2), knots, 2)
    assert op.fp32_path == "staged"
    with pytest.raises(mf.MfwqError) as e:
        op.fp32_path = "fused"
    assert "unavailable" in str(e.value)
    x = inputs.uniform_vector(op.shape, 3)
    ref = O.apply_alg2(tabs, O.full_coeff(C6), x)
    assert np.abs(_apply32(op, x) - ref).max() <= TOL * np.abs(ref).max()
    op.close()
    p = 3
    knots = [inputs.jittered_knots(p, 9, seed=4), inputs.open_uniform_knots(p, 6), inputs.open_uniform_knots(p, 5)]
    op, tabs, C6 = _patch(mf, (p, p, p), knots, 2)
    x = inputs.uniform_vector(op.shape, 5)
    ref = O.apply_alg2(tabs, O.full_coeff(C6), x)
    assert np.abs(_apply32(op, x) - ref).max() <= TOL * np.abs(ref).max()
    op.close()
    knots = [inputs.open_uniform_knots(p, n) for n in (8, 9, 5)]
    op, tabs, C6 = _patch(mf, (p, p, p), knots, 3)
    c = op.eval_mass_coeff("ring", 2.0)
    op.set_mass_coeff(c, fd_shift=2.0)
    x = inputs.uniform_vector(op.shape, 4)
    ref = O.apply_alg2(tabs, O.full_coeff(C6), x) + O.apply_mass_alg1(tabs, c.cpu().numpy(), x)
    assert np.abs(_apply32(op, x) - ref).max() <= TOL * np.abs(ref).max()
    op.close()


def test_autotune_picks_a_path_and_keeps_parity(mf, tmp_path):
    p, nel = 4, (14, 20, 9)
    knots = [inputs.open_uniform_knots(p, n) for n in nel]
    op, tabs, C6 = _patch(mf, (p, p, p), knots, 4)
    cache = str(tmp_path / "tune32.jsonl")
    op.autotune(cache)
    assert op.fp32_path in ("staged", "fused")
    codes = [json.loads(l)["xstage"] for l in open(cache) if "fp32" in l]
    assert len(codes) == 1 and ((codes[0] // 10000) % 10 == 1) == (op.fp32_path == "fused")
    x = inputs.uniform_vector(op.shape, 6)
    ref = O.apply_alg2(tabs, O.full_coeff(C6), x)
    assert np.abs(_apply32(op, x) - ref).max() <= TOL * np.abs(ref).max()
    op.close()


@pytest.mark.parametrize("ps,nel", [((4, 4, 4), (14, 20, 9)), ((3, 2, 5), (11, 7, 6)), ((2, 3, 2), (9, 13, 10))])
def test_slow_tiling_is_bitwise_the_same(mf, ps, nel):
    """Every (rows, cols) tiling of the FP32 slow stages sums each output in the
    same order: bitwise equal results on both FP32 paths.  (3, 2, 5) with 11
    elements gives an odd column count n1 = 14 for the y stages (n1 even: 2 columns
    run, 4 fall back to one column per thread), (2, 3, 2) n1 = 11 (all one column)."""
    knots = [inputs.open_uniform_knots(ps[l], nel[l]) for l in range(3)]
    op, tabs, C6 = _patch(mf, ps, knots, 11)
    x = inputs.uniform_vector(op.shape, 12)
    ref = O.apply_alg2(tabs, O.full_coeff(C6), x)
    for path in ("staged", "fused"):
        op.fp32_path = path
        op.set_slow_tiling(1, 1, fp32=True)
        base = _apply32(op, x)
        assert np.abs(base - ref).max() <= TOL * np.abs(ref).max()
        for rows in (1, 2, 4):
            for cols in (1, 2, 4):
                op.set_slow_tiling(rows, cols, fp32=True)
                assert op.slow_tiling(fp32=True) == (rows, cols)
                assert np.array_equal(_apply32(op, x), base), (path, rows, cols)
    with pytest.raises(mf.MfwqError):
        op.set_slow_tiling(2, 2, fp32=False)  # FP64 stages take one column per thread
    with pytest.raises(mf.MfwqError):
        op.set_slow_tiling(3, 1, fp32=True)
    op.close()
