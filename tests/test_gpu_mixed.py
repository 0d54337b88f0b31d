"""GPU tests of the mixed-precision path: FP32 operator, tensor-core (tcgen05)
FD preconditioner in TF32 and BF16, and the FP64 iterative refinement.

Tolerances (derived from the arithmetic, not from the paper, which is FP64):
* FP32 apply: operands rounded to FP32 (2^-24) and accumulated over a few
  hundred terms per output in five stages: normwise 1e-5 of the FP64 oracle.
* FD on tensor cores: each of the six passes rounds both operands to TF32
  (2^-11) or BF16 (2^-9) and accumulates in FP32, so the normwise error of
  one pass is about 2^-11 sqrt(2) (TF32) or 2^-9 sqrt(2) (BF16); six passes
  with random-sign errors give about sqrt(6) times that: 2e-3 (TF32) and
  7e-3 (BF16).  Asserted with a factor 5 margin: 1e-2 and 3.5e-2.
* Refinement: the FP64 residual ||f - K~ u|| / ||f|| <= 1e-8 is asserted
  with the oracle's operator, and the solution must agree with the FP64
  solve to the accuracy the two residuals buy:
  ||u - u64|| <= ||K~^-1||_2 (||f - K~ u|| + ||f - K~ u64||), with the
  smallest singular value of the oracle's dense K~ (1% for the rounding of
  the norms themselves).
"""
import numpy as np
import pytest

import oracle as O
from paper_1712_08565_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

FD_TOL = {"tf32": 1e-2, "bf16": 3.5e-2}


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_08565_gb300 import build
    build.build()
    from paper_1712_08565_gb300 import mfwq
    return mfwq


SHAPES = [((3, 3, 3), (5, 7, 9)), ((6, 6, 6), (10, 12, 8)), ((2, 4, 3), (30, 6, 5)), ((4, 4, 4), (125, 3, 4))]


def _setup(mf, ps, nel, fd):
    knots = [inputs.open_uniform_knots(ps[l], nel[l]) for l in range(3)]
    op = mf.Operator(ps, knots, mixed=True, fd_precision=fd, device=DEV)
    modes = inputs.fourier_modes(5)
    C = op.eval_coeff("ring", modes, 0.3)
    op.set_coeff(C)
    tabs = [O.tables_1d(knots[l], ps[l]) for l in range(3)]
    return op, tabs, O.coefficient_grid(tabs, "ring", modes, 0.3)


def _nrel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("fd", ["tf32", "bf16"])
@pytest.mark.parametrize("ps,nel", SHAPES)
def test_fd_tensor_core(mf, fd, ps, nel):
    op, tabs, _ = _setup(mf, ps, nel, fd)
    fdo = O.fd_setup(tabs)
    r = inputs.uniform_vector(op.shape, 11)
    z = op.fd_precond_f32(torch.from_numpy(r).float().to(DEV)).double().cpu().numpy()
    ref = O.fd_apply(fdo, r)
    err = _nrel(z, ref)
    assert err <= FD_TOL[fd], (fd, ps, nel, err)
    op.sync()
    op.close()


@pytest.mark.parametrize("ps,nel", SHAPES[:2])
def test_apply_fp32(mf, ps, nel):
    op, tabs, C6 = _setup(mf, ps, nel, "tf32")
    x = inputs.uniform_vector(op.shape, 12)
    y = op.apply_f32(torch.from_numpy(x).float().to(DEV)).double().cpu().numpy()
    ref = O.apply_alg2(tabs, O.full_coeff(C6), x)
    assert _nrel(y, ref) <= 1e-5
    op.close()


@pytest.mark.parametrize("fd", ["tf32", "bf16"])
def test_mixed_refinement_reaches_fp64_residual(mf, fd):
    ps, nel = (4, 4, 4), (10, 9, 11)
    op, tabs, C6 = _setup(mf, ps, nel, fd)
    f = op.load_vector("ring", "sines")
    u, info = op.solve(f, rtol=1e-8, maxit=50, inner_rtol=1e-4, history=True)
    assert info.converged, info
    assert info.outer_iterations >= 1 and info.rel_residual <= 1e-8
    K = O.stiffness_wq(tabs, O.full_coeff(C6))
    fn = f.cpu().numpy()
    res = np.linalg.norm(fn.ravel() - K @ u.cpu().numpy().ravel()) / np.linalg.norm(fn)
    assert res <= 1.01e-8
    u64, i64 = op.solve(f, rtol=1e-12, force_fp64=True)
    assert i64.converged
    un, u64n = u.cpu().numpy().ravel(), u64.cpu().numpy().ravel()
    Kd = K.toarray() if hasattr(K, "toarray") else np.asarray(K)
    smin = np.linalg.svd(Kd, compute_uv=False)[-1]
    bound = (np.linalg.norm(fn.ravel() - K @ un) + np.linalg.norm(fn.ravel() - K @ u64n)) / smin
    assert np.linalg.norm(un - u64n) <= 1.01 * bound, (np.linalg.norm(un - u64n), bound)
    op.sync()
    op.close()


@pytest.mark.parametrize("fd", ["tf32", "bf16"])
def test_fp64_solve_with_low_precision_fd(mf, fd):
    """FP64 BiCGStab with the tensor-core FD as preconditioner (fp64_low_fd):
    the iterate, the operator and the residual are FP64, so the FP64 tolerance
    holds with the oracle's operator, for K~ and for K~^T; the solution agrees
    with the plain FP64 solve to what the two residuals guarantee."""
    ps, nel = (4, 4, 4), (10, 9, 11)
    op, tabs, C6 = _setup(mf, ps, nel, fd)
    f = op.load_vector("ring", "sines")
    u, info = op.solve(f, rtol=1e-10, fp64_low_fd=True)
    assert info.converged and info.outer_iterations == 0 and info.rel_residual <= 1e-10, info
    K = O.stiffness_wq(tabs, O.full_coeff(C6))
    fn = f.cpu().numpy().ravel()
    un = u.cpu().numpy().ravel()
    assert np.linalg.norm(fn - K @ un) <= 1.01e-10 * np.linalg.norm(fn)
    u64, i64 = op.solve(f, rtol=1e-10, force_fp64=True)
    assert i64.converged
    u64n = u64.cpu().numpy().ravel()
    Kd = K.toarray() if hasattr(K, "toarray") else np.asarray(K)
    smin = np.linalg.svd(Kd, compute_uv=False)[-1]
    bound = (np.linalg.norm(fn - K @ un) + np.linalg.norm(fn - K @ u64n)) / smin
    assert np.linalg.norm(un - u64n) <= 1.01 * bound
    lam, il = op.solve_T(f, rtol=1e-10, fp64_low_fd=True)
    assert il.converged
    assert np.linalg.norm(fn - K.T @ lam.cpu().numpy().ravel()) <= 1.01e-10 * np.linalg.norm(fn)
    op.close()


def test_fp64_low_fd_needs_a_mixed_handle(mf):
    knots = [inputs.open_uniform_knots(3, n) for n in (5, 6, 7)]
    op = mf.Operator(3, knots, device=DEV)
    op.set_coeff(op.eval_coeff("ring"))
    f = op.load_vector("ring", "sines")
    with pytest.raises(mf.MfwqError):
        op.solve(f, fp64_low_fd=True)
    op.close()


def test_mixed_requires_small_directions(mf):
    knots = [inputs.open_uniform_knots(2, 300)] * 3
    with pytest.raises(mf.MfwqError) as e:
        mf.Operator(2, knots, mixed=True, device=DEV)
    assert e.value.status == -1
