"""GPU tests of the FP64 FD preconditioner on the BF16 tensor cores by operand
splitting (MFWQ_FD64_SPLIT, the default wherever every n_l <= 256) and of the
FP64-pipe kernels (MFWQ_FD64_PIPE) against the oracle's FD (O.fd_apply, the
FD method of Section 4 in float64).

Tolerance: 1e-12 of the largest oracle entry, the bar of the FP64 FD tests.
Each of the six mode products keeps 49 bits below the leading power of two of
every row of its operands, so one product is within about 2^-47 of
sum |U_ij| |x_j| (a few 1e-14 of it); the eigenvalue scaling and six passes
stay well inside 1e-12 of the result's largest entry.

Shapes: sizes below, at and above the 64-output tiles and the 32-element K
chunks (n = 7 .. 200 per direction, odd and even, unequal directions), graded
knots (no even/odd fold), several degrees, a zero right-hand side and one with
entries spread over 40 orders of magnitude, and an FD shift (reaction term)."""
import numpy as np
import pytest

import oracle as O
from paper_1712_08565_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-12


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_08565_gb300 import build
    build.build()
    from paper_1712_08565_gb300 import mfwq
    return mfwq


def _op(mf, ps, knots):
    op = mf.Operator(ps, knots, device=DEV)
    tabs = [O.tables_1d(knots[l], ps[l] if np.ndim(ps) else ps) for l in range(3)]
    return op, tabs


def _fd(op, r):
    return op.fd_precond(torch.from_numpy(r).to(DEV)).cpu().numpy()


@pytest.mark.parametrize("ps,nel", [((2, 2, 2), (5, 6, 7)), ((3, 3, 3), (30, 29, 12)), ((4, 3, 2), (61, 8, 40)),
                                    ((2, 5, 3), (62, 70, 33)), ((6, 4, 2), (130, 20, 9)), ((3, 3, 3), (197, 9, 6))])
def test_split_fd_matches_oracle(mf, ps, nel):
    knots = [inputs.open_uniform_knots(ps[l], nel[l]) for l in range(3)]
    op, tabs = _op(mf, ps, knots)
    assert op.fd64_path == "split"  # the default wherever every n_l <= 256
    r = inputs.uniform_vector(op.shape, sum(nel))
    ref = O.fd_apply(O.fd_setup(tabs), r)
    z = _fd(op, r)
    assert np.abs(z - ref).max() <= TOL * np.abs(ref).max()
    op.fd64_path = "pipe"
    zp = _fd(op, r)
    assert np.abs(zp - ref).max() <= TOL * np.abs(ref).max()
    op.close()


def test_split_fd_graded_knots_and_wide_range(mf):
    p = 3
    knots = [inputs.jittered_knots(p, 40, seed=1), inputs.jittered_knots(p, 25, seed=2), inputs.open_uniform_knots(p, 11)]
    op, tabs = _op(mf, p, knots)
    op.fd64_path = "split"
    fd = O.fd_setup(tabs)
    r = inputs.uniform_vector(op.shape, 3)
    g = inputs.rng(4)
    r = r * np.exp(g.uniform(-46.0, 46.0, size=r.shape))  # entries over 40 orders of magnitude
    ref = O.fd_apply(fd, r)
    z = _fd(op, r)
    assert np.abs(z - ref).max() <= TOL * np.abs(ref).max()
    z0 = _fd(op, np.zeros(op.shape))
    assert not np.any(z0)
    op.close()


def test_split_fd_with_shift_and_solve(mf):
    """The scaling table follows an FD shift set after the path; the FP64
    solve with the split FD reaches rtol 1e-10 (oracle residual) in the
    iterations of the FP64-pipe FD, give or take one."""
    p, nel = 3, (12, 10, 9)
    knots = [inputs.open_uniform_knots(p, n) for n in nel]
    op, tabs = _op(mf, p, knots)
    op.set_coeff(op.eval_coeff("ring"))
    f = op.load_vector("ring", "sines")
    op.fd64_path = "pipe"
    u0, i0 = op.solve(f, rtol=1e-10)
    op.fd64_path = "split"
    u1, i1 = op.solve(f, rtol=1e-10)
    assert i1.converged and abs(i1.iterations - i0.iterations) <= 1
    K = O.stiffness_wq(tabs, O.full_coeff(O.coefficient_grid(tabs, "ring", None, 0.0)))
    fn, un = f.cpu().numpy().ravel(), u1.cpu().numpy().ravel()
    assert np.linalg.norm(fn - K @ un) <= 1.0001e-10 * np.linalg.norm(fn)
    c = op.eval_mass_coeff("ring", 3.0)
    op.set_mass_coeff(c, fd_shift=3.0)
    r = inputs.uniform_vector(op.shape, 9)
    ref = O.fd_apply(O.fd_setup(tabs, shift=3.0), r)
    z = _fd(op, r)
    assert np.abs(z - ref).max() <= TOL * np.abs(ref).max()
    op.close()


def test_split_fd_in_a_batch(mf):
    """Patches with the split FD: the per-patch streams and the grouped sweep
    (one launch per stage over all patches, the split FD's slicing and product
    passes included) both match the separate solves bitwise."""
    specs = [(2, (6, 7, 5)), (3, (9, 8, 7)), (4, (10, 6, 6))]
    ops, fs = [], []
    for p, nel in specs:
        knots = [inputs.open_uniform_knots(p, n) for n in nel]
        op = mf.Operator(p, knots, device=DEV)
        op.set_coeff(op.eval_coeff("ring"))
        op.fd64_path = "split"
        ops.append(op)
        fs.append(op.load_vector("ring", "sines"))
    sep = [op.solve(f, rtol=1e-10)[0].cpu().numpy() for op, f in zip(ops, fs)]
    batch = mf.Batch(ops)
    us, infos = batch.solve(fs, rtol=1e-10)
    assert not batch.grouped
    for u, s_, info in zip(us, sep, infos):
        assert info.converged
        assert np.array_equal(u.cpu().numpy(), s_)
    for groups in (1, 2):
        batch.set_grouped(groups)
        ug, ig = batch.solve(fs, rtol=1e-10)
        assert batch.grouped
        for u, s_, info in zip(ug, sep, ig):
            assert info.converged
            assert np.array_equal(u.cpu().numpy(), s_)
    batch.close()
    for op in ops:
        op.close()


def test_split_fd_refuses_large_directions(mf):
    knots = [inputs.open_uniform_knots(2, 260), inputs.open_uniform_knots(2, 3), inputs.open_uniform_knots(2, 3)]
    op = mf.Operator(2, knots, device=DEV)
    assert op.fd64_path == "pipe"  # 262 DoFs in direction 1: the FP64-pipe FD
    with pytest.raises(mf.MfwqError):
        op.fd64_path = "split"
    assert op.fd64_path == "pipe"
    op.close()
