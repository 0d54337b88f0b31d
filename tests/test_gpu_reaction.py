"""GPU parity of the reaction (mass) term alpha u of Eq. (poisson): the WQ mass
operator of Eq. (Mwq) applied by Algorithm 1 inside the library's apply,
transposed apply, FP32 apply, solves and batched solves, its coefficient
gradient, and the FD preconditioner with the reaction shift, all against the
oracle on the same seeded inputs.  Tolerances as in the other parity tests:
1e-12 of the largest reference entry for FP64 operators, 1e-5 for the FP32
apply, 1e-9 for solutions at rtol 1e-12."""
import numpy as np
import pytest

import oracle as O
from paper_1712_08565_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_08565_gb300 import build
    build.build()
    from paper_1712_08565_gb300 import mfwq
    return mfwq


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = {
    # name: (degrees, knots per direction, geometry, Fourier-mode seed, alpha)
    "ring-p3": ((3, 3, 3), lambda: [inputs.open_uniform_knots(3, n) for n in (5, 6, 7)], "ring", 2, 10.0),
    "ring-mixed-degree-jittered": ((2, 4, 3), lambda: [inputs.open_uniform_knots(2, 6),
                                                        inputs.jittered_knots(4, 5, seed=3),
                                                        inputs.open_uniform_knots(3, 4)], "ring", 3, 3.0),
    "cube-p2": ((2, 2, 2), lambda: [inputs.open_uniform_knots(2, n) for n in (6, 5, 4)], "cube", None, 25.0),
}


class Case:
    def __init__(self, mf, name, mixed=False):
        ps, kf, geom, seed, alpha = CASES[name]
        self.knots = kf()
        self.ps, self.geom, self.alpha = ps, geom, alpha
        self.modes = inputs.fourier_modes(seed) if seed is not None else None
        self.kscale = 0.3 if seed is not None else 0.0
        self.tabs = [O.tables_1d(self.knots[l], ps[l]) for l in range(3)]
        self.C6 = O.coefficient_grid(self.tabs, geom, self.modes, self.kscale)
        self.c = O.mass_coefficient_grid(self.tabs, geom, alpha)
        self.op = mf.Operator(ps, self.knots, mixed=mixed, device=DEV)
        self.op.set_coeff(self.op.eval_coeff(geom, self.modes, self.kscale))
        self.cd = self.op.eval_mass_coeff(geom, alpha)
        self.op.set_mass_coeff(self.cd, fd_shift=alpha)
        self.shape = self.op.shape

    def ref_apply(self, V):
        return O.apply_alg2(self.tabs, O.full_coeff(self.C6), V) + O.apply_mass_alg1(self.tabs, self.c, V)

    def ref_apply_T(self, Y):
        return O.apply_T_alg2(self.tabs, O.full_coeff(self.C6), Y) + O.apply_mass_T(self.tabs, self.c, Y)


@pytest.fixture(scope="module", params=list(CASES))
def case(mf, request):
    c = Case(mf, request.param)
    yield c
    c.op.close()


def test_mass_coefficient(case):
    assert _rel(case.cd.cpu().numpy(), case.c) <= 1e-13


def test_apply_with_reaction(case):
    V = inputs.uniform_vector(case.shape, 51)
    y = case.op.apply(_dev(V)).cpu().numpy()
    assert _rel(y, case.ref_apply(V)) <= 1e-12


def test_apply_T_with_reaction(case):
    Y = inputs.uniform_vector(case.shape, 52)
    y = case.op.apply_T(_dev(Y)).cpu().numpy()
    assert _rel(y, case.ref_apply_T(Y)) <= 1e-12


def test_grad_mass_coeff(case):
    lam = inputs.uniform_vector(case.shape, 53)
    u = inputs.uniform_vector(case.shape, 54)
    g = case.op.grad_mass_coeff(_dev(lam), _dev(u)).cpu().numpy()
    assert _rel(g, O.grad_mass_coeff(case.tabs, lam, u)) <= 1e-12


def test_fd_with_shift(case):
    R = inputs.uniform_vector(case.shape, 55)
    z = case.op.fd_precond(_dev(R)).cpu().numpy()
    assert _rel(z, O.fd_apply(O.fd_setup(case.tabs, shift=case.alpha), R)) <= 1e-12


def test_solve_with_reaction(case):
    F = O.load_vector(case.tabs, case.geom, O.forcing_sines)
    patch = O.Patch(case.tabs, case.C6, O.fd_setup(case.tabs, shift=case.alpha), case.c)
    ref, rinfo = patch.solve(F, 1e-13, maxit=600)
    assert rinfo.converged
    u, info = case.op.solve(_dev(F), rtol=1e-12, maxit=600)
    assert info.converged
    un = u.cpu().numpy()
    assert np.linalg.norm(un - ref) <= 1e-9 * np.linalg.norm(ref)
    if case.geom == "cube":  # K~ + M~ = P + alpha M(x)M(x)M: the shifted FD is its inverse
        assert info.iterations == 1


def test_reaction_off_restores_stiffness(mf):
    c = Case(mf, "ring-p3")
    V = inputs.uniform_vector(c.shape, 56)
    c.op.set_mass_coeff(None, fd_shift=0.0)
    y = c.op.apply(_dev(V)).cpu().numpy()
    assert _rel(y, O.apply_alg2(c.tabs, O.full_coeff(c.C6), V)) <= 1e-12
    R = inputs.uniform_vector(c.shape, 57)
    z = c.op.fd_precond(_dev(R)).cpu().numpy()
    assert _rel(z, O.fd_apply(O.fd_setup(c.tabs), R)) <= 1e-12
    with pytest.raises(mf.MfwqError):
        c.op.set_mass_coeff(c.cd, fd_shift=-1.0)
    with pytest.raises(mf.MfwqError):
        c.op.set_mass_coeff(c.cd, fd_shift=float("nan"))
    c.op.close()


def test_fp32_apply_tc_fd_and_mixed_solve_with_reaction(mf):
    c = Case(mf, "ring-mixed-degree-jittered", mixed=True)
    V = inputs.uniform_vector(c.shape, 58)
    y = c.op.apply_f32(_dev(V).float()).double().cpu().numpy()
    assert _rel(y, c.ref_apply(V)) <= 1e-5
    F = O.load_vector(c.tabs, c.geom, O.forcing_sines)
    u, info = c.op.solve(_dev(F), rtol=1e-10, inner_rtol=1e-4)
    assert info.converged and info.rel_residual <= 1e-10
    res = np.ravel(F) - np.ravel(c.ref_apply(u.cpu().numpy()))
    assert np.linalg.norm(res) <= 2e-10 * np.linalg.norm(F)
    c.op.close()


def test_batch_with_reaction_equals_separate(mf):
    a = Case(mf, "ring-p3")
    b = Case(mf, "cube-p2")
    fs = [a.op.load_vector("ring", "sines"), b.op.load_vector("cube", "sines")]
    sep = [a.op.solve(fs[0], rtol=1e-10)[0], b.op.solve(fs[1], rtol=1e-10)[0]]
    bt = mf.Batch([a.op, b.op])
    us, infos = bt.solve(fs, rtol=1e-10, force_fp64=True)
    assert all(i.converged for i in infos)
    for u, s in zip(us, sep):
        assert torch.equal(u, s)
    bt.close()
    a.op.close()
    b.op.close()


@pytest.mark.slow
def test_reaction_sampled_rows_at_130_cubed(mf):
    """The bench ring (p = 4, 128 elements, N = 130^3) with alpha = 10: sampled
    rows of (K~ + M~) v computed one by one by the oracle."""
    p, nel, alpha = 4, 128, 10.0
    knots = [inputs.open_uniform_knots(p, nel)] * 3
    op = mf.Operator(p, knots, device=DEV)
    op.set_coeff(op.eval_coeff("ring"))
    op.set_mass_coeff(op.eval_mass_coeff("ring", alpha), fd_shift=alpha)
    tabs = [O.tables_1d(knots[0], p)] * 3
    V = inputs.uniform_vector(op.shape, 59)
    y = op.apply(_dev(V)).cpu().numpy()
    g = inputs.rng(60)
    rows = [(0, 0, 0), (129, 129, 129), (64, 3, 127)] + [tuple(int(v) for v in g.integers(0, 130, 3)) for _ in range(20)]
    ref = (O.apply_rows(tabs, O.coefficient_box_fn(tabs, "ring"), V, rows)
           + O.mass_rows(tabs, O.mass_coefficient_box_fn(tabs, "ring", alpha), V, rows))
    got = np.array([y[r] for r in rows])
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    op.close()
