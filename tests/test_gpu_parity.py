"""GPU parity: the CUDA path (through the C ABI) against the oracle, element by
element, on the same seeded inputs.

Tolerances: FP64 operator apply (and its transpose, the gradient, the FD
preconditioner) within 1e-12 of the largest reference entry; solutions at a
1e-10 relative residual within 1e-9 (relative 2-norm) of a direct sparse
solve; coefficient and load vector within 1e-13 (they are evaluations with
CUDA's sin/cos/exp, whose error is a few ulp).
"""
import numpy as np
import pytest

import oracle as O
from paper_1712_08565_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

APPLY_TOL = 1e-12
SOLVE_TOL = 1e-9


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_08565_gb300 import build
    build.build()
    from paper_1712_08565_gb300 import mfwq
    return mfwq


DEV = "cuda:0"

# name, degrees, elements per direction, knot kind, geometry, K-field seed (None: K = I)
CASES = [
    ("cube-p2-16", (2, 2, 2), (16, 16, 16), "uniform", "cube", None),
    ("ring-p3-ragged", (3, 3, 3), (5, 7, 9), "uniform", "ring", 0),
    ("ring-p243", (2, 4, 3), (6, 4, 5), "uniform", "ring", 1),
    ("ring-p6", (6, 6, 6), (7, 6, 8), "uniform", "ring", 2),
    ("jitter-p5", (5, 5, 5), (8, 9, 7), "jitter", "ring", 3),
    ("min-p4", (4, 4, 4), (2, 3, 2), "uniform", "ring", None),
    ("min-p2", (2, 2, 2), (2, 2, 3), "uniform", "ring", 5),
    ("ring-p2-wide", (2, 2, 2), (40, 3, 4), "uniform", "ring", 4),
]


def _knots(p, nel, kind, l):
    if kind == "jitter":
        return inputs.jittered_knots(p, nel, seed=100 + l)
    return inputs.open_uniform_knots(p, nel)


class Case:
    def __init__(self, mf, spec, mixed=False):
        name, ps, nels, kind, geom, kseed = spec
        self.name, self.geom = name, geom
        self.knots = [_knots(ps[l], nels[l], kind, l) for l in range(3)]
        self.modes = inputs.fourier_modes(kseed) if kseed is not None else None
        self.kscale = 0.3 if kseed is not None else 0.0
        self.op = mf.Operator(ps, self.knots, mixed=mixed, device=DEV)
        self.tabs = [O.tables_1d(self.knots[l], ps[l]) for l in range(3)]
        self.C6 = O.coefficient_grid(self.tabs, geom, self.modes, self.kscale)
        self.Cd = self.op.eval_coeff(geom, self.modes, self.kscale)
        self.op.set_coeff(self.Cd)
        self.shape = self.op.shape


def _rel_max(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(mf, request):
    c = Case(mf, request.param)
    yield c
    c.op.close()


def test_shapes(case):
    assert case.shape == (case.tabs[2].n, case.tabs[1].n, case.tabs[0].n)
    for l in range(3):
        np.testing.assert_allclose(case.op.quad_points(l), case.tabs[l].xq, rtol=4e-16, atol=0)


def test_coefficient(case):
    assert _rel_max(case.Cd.cpu().numpy(), case.C6) <= 1e-13


def test_apply(case):
    K = O.stiffness_wq(case.tabs, O.full_coeff(case.C6))
    for seed in (1, 2):
        x = inputs.uniform_vector(case.shape, seed)
        y = case.op.apply(_dev(x)).cpu().numpy()
        ref = (K @ x.ravel()).reshape(case.shape)
        assert _rel_max(y, ref) <= APPLY_TOL, (case.name, _rel_max(y, ref))


def test_apply_transpose(case):
    K = O.stiffness_wq(case.tabs, O.full_coeff(case.C6))
    x = inputs.uniform_vector(case.shape, 3)
    y = case.op.apply_T(_dev(x)).cpu().numpy()
    ref = (K.T @ x.ravel()).reshape(case.shape)
    assert _rel_max(y, ref) <= APPLY_TOL, _rel_max(y, ref)


def test_fd_precond(case):
    fd = O.fd_setup(case.tabs)
    r = inputs.uniform_vector(case.shape, 4)
    z = case.op.fd_precond(_dev(r)).cpu().numpy()
    ref = O.fd_apply(fd, r)
    assert _rel_max(z, ref) <= APPLY_TOL, _rel_max(z, ref)


def test_grad_coeff(case):
    lam = inputs.uniform_vector(case.shape, 5)
    u = inputs.uniform_vector(case.shape, 6)
    g = case.op.grad_coeff(_dev(lam), _dev(u)).cpu().numpy()
    ref = O.grad_coeff(case.tabs, lam, u)
    assert _rel_max(g, ref) <= APPLY_TOL, _rel_max(g, ref)


def test_load_vector(case):
    f = case.op.load_vector(case.geom, "sines").cpu().numpy()
    ref = O.load_vector(case.tabs, case.geom, O.forcing_sines)
    assert _rel_max(f, ref) <= 1e-13, _rel_max(f, ref)


# Cases whose WQ matrix is so ill-conditioned that a relative residual of 1e-10
# bounds the solution error only to kappa_2 * 1e-10 > 1e-9 (kappa_2 measured by
# a dense SVD of the oracle's K~): there the 1e-10 solve must be as close to the
# direct solve as the oracle's own BiCGStab gets.  Every other case: 1e-9 flat.
WIDE_SOLVE_BOUND = {"ring-p6": 1.94e7}


def test_solve_matches_direct(case):
    """At rtol 1e-12 the solution is within 1e-9 of a direct sparse solve; at
    rtol 1e-10 too, except in the ill-conditioned cases listed above, where it
    is as close as the oracle's own BiCGStab gets at that tolerance; its true
    residual, measured by the oracle, is 1e-10."""
    import scipy.sparse.linalg as spla
    K = O.stiffness_wq(case.tabs, O.full_coeff(case.C6)).tocsc()
    F = O.load_vector(case.tabs, case.geom, O.forcing_sines)
    ref = spla.spsolve(K, F.ravel()).reshape(case.shape)
    patch = O.Patch(case.tabs, case.C6, O.fd_setup(case.tabs))
    u_or, _ = patch.solve(F, 1e-10, maxit=400)
    err_or = np.linalg.norm(u_or - ref) / np.linalg.norm(ref)
    u, info = case.op.solve(_dev(F), rtol=1e-10, maxit=400, history=True)
    assert info.converged, info
    assert info.rel_residual <= 1e-10
    un = u.cpu().numpy()
    err = np.linalg.norm(un - ref) / np.linalg.norm(ref)
    if case.name in WIDE_SOLVE_BOUND:
        assert err <= max(SOLVE_TOL, 5 * err_or), (err, err_or)
    else:
        assert err <= SOLVE_TOL, (case.name, err, err_or)
    res = np.linalg.norm(F.ravel() - K @ un.ravel()) / np.linalg.norm(F)
    assert res <= 2e-10, res
    assert info.history is not None and abs(info.history[-1] - info.rel_residual) <= 1e-12 + 1e-6 * info.rel_residual
    u12, info12 = case.op.solve(_dev(F), rtol=1e-12, maxit=600)
    assert info12.converged
    err12 = np.linalg.norm(u12.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err12 <= SOLVE_TOL, err12


def test_adjoint_solve(case):
    import scipy.sparse.linalg as spla
    K = O.stiffness_wq(case.tabs, O.full_coeff(case.C6)).tocsc()
    g = inputs.uniform_vector(case.shape, 7)
    ref = spla.spsolve(K.T.tocsc(), g.ravel()).reshape(case.shape)
    lam, info = case.op.solve_T(_dev(g), rtol=1e-12, maxit=600)
    assert info.converged, info
    err = np.linalg.norm(lam.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= SOLVE_TOL, err
    # the recursively updated residual drifts from the true one by about
    # kappa(K~) * 1e-16 (kappa up to 2e7 on the small p = 6 patch)
    res = np.linalg.norm(g.ravel() - K.T @ lam.cpu().numpy().ravel()) / np.linalg.norm(g)
    assert res <= 1e-10, res


# ---------------------------------------------------------------- specific properties
def test_cube_solve_takes_one_iteration(mf):
    """Unit cube, K = I: K~ equals the Kronecker Laplacian that FD inverts."""
    c = Case(mf, CASES[0])
    f = c.op.load_vector("cube", "sines")
    u, info = c.op.solve(f, rtol=1e-10)
    assert info.converged and info.iterations == 1
    c.op.close()


def test_solve_edge_cases(mf):
    c = Case(mf, CASES[1])
    z = torch.zeros(c.shape, dtype=torch.float64, device=DEV)
    u, info = c.op.solve(z, rtol=1e-10)
    assert info.converged and info.iterations == 0 and float(u.abs().max()) == 0.0
    f = c.op.load_vector("ring", "sines")
    u, info = c.op.solve(f, rtol=1e-14, maxit=1)
    assert info.status == -6 and info.iterations == 1
    # initial guess = converged solution: 0 iterations
    u, info = c.op.solve(f, rtol=1e-10)
    u2, info2 = c.op.solve(f, u=u.clone(), rtol=1e-9)
    assert info2.converged and info2.iterations == 0
    # NaN in the right-hand side is reported, not hidden
    fn = f.clone()
    fn.view(-1)[3] = float("nan")
    _, info3 = c.op.solve(fn, rtol=1e-10)
    assert info3.status == -8
    c.op.close()


def test_invalid_arguments(mf):
    c = Case(mf, CASES[1])
    import ctypes
    x = torch.zeros(c.shape, dtype=torch.float64, device=DEV)
    xp = ctypes.c_void_p(x.data_ptr())
    assert mf.lib().mfwq_apply(c.op._h, xp, xp) == -1  # aliasing input and output
    assert mf.lib().mfwq_apply(c.op._h, None, xp) == -1
    st = mf.lib().mfwq_apply_f32(c.op._h, xp, ctypes.c_void_p(x.data_ptr() + 8))
    assert st == -1  # not a mixed handle
    with pytest.raises(ValueError):
        c.op.apply(torch.zeros(5, dtype=torch.float64, device=DEV))
    with pytest.raises(TypeError):
        c.op.apply(x.float())
    c.op.close()


def test_solve_host_matches_device(mf):
    c = Case(mf, CASES[2])
    f = c.op.load_vector("ring", "sines")
    u, info = c.op.solve(f, rtol=1e-10)
    uh, infoh = c.op.solve_host(f.cpu().numpy(), rtol=1e-10)
    uh2, infoh2 = c.op.solve_host(f.cpu().numpy(), out=uh, rtol=1e-10)
    assert infoh2.iterations == info.iterations  # `out` is an output, not an initial guess
    assert infoh.converged and infoh.iterations == info.iterations
    assert np.abs(uh - u.cpu().numpy()).max() <= 1e-14 * float(u.abs().max())
    c.op.close()


def test_autograd_function_gradient(mf):
    """dJ/dC through the torch.autograd.Function against central differences."""
    c = Case(mf, CASES[2])
    from paper_1712_08565_gb300 import solve_fn
    f = c.op.load_vector("ring", "sines")
    C0 = c.Cd.clone()
    u_t = c.op.solve(f, rtol=1e-13)[0].detach()
    C = (C0 * 1.1).requires_grad_(True)
    u = solve_fn().apply(C, f, c.op, 1e-13)
    J = 0.5 * ((u - u_t) ** 2).sum()
    J.backward()
    g = C.grad.detach()

    def Jval(Cv):
        uu = solve_fn().apply(Cv, f, c.op, 1e-13)
        return float(0.5 * ((uu - u_t) ** 2).sum())

    gen = torch.Generator(device="cpu").manual_seed(0)
    for _ in range(3):
        d = (torch.rand(C0.shape, generator=gen, dtype=torch.float64) - 0.5).to(DEV) * C0.abs()
        h = 1e-6
        fd = (Jval((C0 * 1.1 + h * d)) - Jval((C0 * 1.1 - h * d))) / (2 * h)
        an = float((g * d).sum())
        assert abs(fd - an) <= 1e-5 * abs(an), (fd, an)
    c.op.close()


def test_graph_chunk_solve_is_the_same_solve(mf):
    """FP64 solve with BiCGStab iterations captured four at a time into a CUDA
    graph (operator on a stream of its own): the same kernels in the same
    order, so the same iterations and bits as the plain solve; a chunk larger
    than maxit runs uncaptured, and maxit is honoured."""
    p, nel = 3, (6, 7, 5)
    knots = [inputs.open_uniform_knots(p, n) for n in nel]
    s = torch.cuda.Stream()
    op = mf.Operator(p, knots, device=DEV, stream=s)
    op.set_coeff(op.eval_coeff("ring", inputs.fourier_modes(3), 0.3))
    f = op.load_vector("ring", "sines")
    u0, i0 = op.solve(f, rtol=1e-10)
    u4, i4 = op.solve(f, rtol=1e-10, graph_chunk=4)
    assert i0.converged and i4.converged and i4.iterations == i0.iterations
    assert torch.equal(u0, u4)
    u5, i5 = op.solve(f, rtol=1e-14, maxit=5, graph_chunk=4)
    assert i5.iterations == 5 and i5.status == -6
    op.close()
