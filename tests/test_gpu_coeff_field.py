"""GPU tests of the coefficient evaluated inside the FP32 operator
(mfwq_set_coeff_field with onthefly = 1), the memory-lean form of the paper's
remark on storing C (Section 3.2).

The FP32 operator then reads no stored coefficient: its x stage computes
C = kappa(x) G(xi1) at every quadrature point.  Tolerance: the FP32 apply
bound of the other FP32 tests, 1e-5 of the largest oracle entry.  kappa =
exp(0.3 g) with |g| <= 8 is evaluated in FP32 with the phase reduced modulo
one period before rounding (argument error about 1e-7 half-turns), so its
relative error is a few 1e-7, below the FP32 rounding of the apply itself.
The oracle evaluates C from the same definition in float64
(oracle.coefficient_points); nothing is shared with the library.

Fields: the Fourier field of the adjoint and batched workloads (8 modes,
|k| <= 3, amplitude scale 0.3) on the ring and on the cube."""
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


def _apply32(op, x):
    return op.apply_f32(torch.from_numpy(x).float().to(DEV)).double().cpu().numpy()


@pytest.mark.parametrize("geometry", ["ring", "cube"])
@pytest.mark.parametrize("ps,nel", [((3, 3, 3), (12, 9, 7)), ((6, 4, 5), (18, 11, 6)), ((2, 2, 2), (14, 20, 9))])
def test_field_apply_matches_oracle(mf, geometry, ps, nel):
    knots = [inputs.open_uniform_knots(ps[l], nel[l]) for l in range(3)]
    op = mf.Operator(ps, knots, mixed=True, device=DEV)
    modes = inputs.fourier_modes(3 + ps[0])
    op.set_coeff_field(geometry, modes, 0.3, onthefly=True)
    tabs = [O.tables_1d(knots[l], ps[l]) for l in range(3)]
    C6 = O.coefficient_grid(tabs, geometry, modes, 0.3)
    x = inputs.uniform_vector(op.shape, 17)
    ref = O.apply_alg2(tabs, O.full_coeff(C6), x)
    for path in ("staged", "fused"):
        op.fp32_path = path
        y = _apply32(op, x)
        assert np.abs(y - ref).max() <= TOL * np.abs(ref).max(), path
    # the FP64 operator keeps the stored coefficient of the same field
    y64 = op.apply(torch.from_numpy(x).to(DEV)).cpu().numpy()
    assert np.abs(y64 - ref).max() <= 1e-12 * np.abs(ref).max()
    op.close()


def test_field_equals_stored_and_set_coeff_turns_it_off(mf):
    p, nel = 4, (14, 10, 8)
    knots = [inputs.open_uniform_knots(p, n) for n in nel]
    op = mf.Operator(p, knots, mixed=True, device=DEV)
    modes = inputs.fourier_modes(12)
    x = inputs.uniform_vector(op.shape, 2)
    op.set_coeff_field("ring", modes, 0.3, onthefly=False)
    y_stored = _apply32(op, x)
    op.set_coeff_field("ring", modes, 0.3, onthefly=True)
    y_otf = _apply32(op, x)
    assert np.abs(y_otf - y_stored).max() <= 2e-6 * np.abs(y_stored).max()
    op.set_coeff(op.eval_coeff("ring", modes, 0.3))  # stored again
    assert np.array_equal(_apply32(op, x), y_stored)
    op.close()


def test_field_mixed_solve_reaches_fp64_residual(mf):
    """Adjoint-workload field on a small ring: the mixed refinement with the
    evaluated FP32 coefficient reaches ||f - K~ u|| <= 1e-8 ||f||, measured
    with the oracle's operator."""
    p, nel = 3, (10, 8, 7)
    knots = [inputs.open_uniform_knots(p, n) for n in nel]
    op = mf.Operator(p, knots, mixed=True, device=DEV)
    modes = inputs.fourier_modes(0)
    op.set_coeff_field("ring", modes, 0.3, onthefly=True)
    tabs = [O.tables_1d(knots[l], p) for l in range(3)]
    K = O.stiffness_wq(tabs, O.full_coeff(O.coefficient_grid(tabs, "ring", modes, 0.3)))
    f = op.load_vector("ring", "sines")
    u, info = op.solve(f, rtol=1e-8)
    assert info.converged and info.outer_iterations >= 1
    fn, un = f.cpu().numpy().ravel(), u.cpu().numpy().ravel()
    assert np.linalg.norm(fn - K @ un) <= 1.0001e-8 * np.linalg.norm(fn)
    op.close()


def test_field_batched_mixed_solve(mf):
    """Uneven patches of the batched workload's kind (degrees 2..6, 3..9
    elements per direction, each its own field), evaluated coefficient, mixed
    batched solve: every patch's FP64 residual <= 1e-8 with the oracle's K~."""
    specs = inputs.batch_patches(count=4, seed=7, p_range=(2, 6), nel_range=(3, 9))
    ops, fs, Ks = [], [], []
    for i, (p, nel) in enumerate(specs):
        nel = tuple(max(n, p + 4) for n in nel)  # a translation-invariant interior in direction 1
        knots = [inputs.open_uniform_knots(p, n) for n in nel]
        op = mf.Operator(p, knots, mixed=True, device=DEV)
        modes = inputs.fourier_modes(100 + i)
        op.set_coeff_field("ring", modes, 0.3, onthefly=True)
        tabs = [O.tables_1d(knots[l], p) for l in range(3)]
        Ks.append(O.stiffness_wq(tabs, O.full_coeff(O.coefficient_grid(tabs, "ring", modes, 0.3))))
        fs.append(op.load_vector("ring", "sines"))
        ops.append(op)
    batch = mf.Batch(ops)
    us, infos = batch.solve(fs, rtol=1e-8)
    for u, f, K, info in zip(us, fs, Ks, infos):
        assert info.converged
        fn, un = f.cpu().numpy().ravel(), u.cpu().numpy().ravel()
        assert np.linalg.norm(fn - K @ un) <= 1.0001e-8 * np.linalg.norm(fn)
    batch.close()
    for op in ops:
        op.close()


def test_field_refusals(mf):
    knots = [inputs.open_uniform_knots(3, n) for n in (10, 6, 5)]
    op = mf.Operator(3, knots, device=DEV)  # FP64 only
    with pytest.raises(mf.MfwqError):
        op.set_coeff_field("ring", inputs.fourier_modes(1), 0.3, onthefly=True)
    op.set_coeff_field("ring", inputs.fourier_modes(1), 0.3, onthefly=False)  # stores the FP64 fields
    op.close()
    knots = [inputs.open_uniform_knots(9, 20), inputs.open_uniform_knots(2, 6), inputs.open_uniform_knots(2, 5)]
    op = mf.Operator((9, 2, 2), knots, mixed=True, device=DEV)
    with pytest.raises(mf.MfwqError):
        op.set_coeff_field("ring", inputs.fourier_modes(1), 0.3, onthefly=True)
    op.close()
