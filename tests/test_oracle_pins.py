"""Pins of the oracle to facts fixed by the paper or by mathematics (CPU only).

Each test checks the oracle against something other than itself: a library
routine (scipy's B-splines, sparse direct solve), an independent quadrature,
a closed form, an exact identity, or values printed in the paper.
"""
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse.linalg as spla
from scipy.interpolate import BSpline

import oracle as O
from paper_1712_08565_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _scipy_basis(knots, p, x, deriv):
    m = len(knots) - p - 1
    out = np.zeros((len(x), m))
    for i in range(m):
        c = np.zeros(m)
        c[i] = 1.0
        s = BSpline(knots, c, p)
        out[:, i] = (s.derivative() if deriv else s)(x)
    return out


def _nonuniform_knots(p, nel, seed):
    """Break points k/nel moved by up to 30% of a span (graded but well-conditioned)."""
    g = inputs.rng(seed)
    u = np.arange(1, nel) / nel + g.uniform(-0.3, 0.3, size=nel - 1) / nel
    return O.open_knots(p, np.concatenate([[0.0], u, [1.0]]))


def _independent_galerkin(knots, p, a, b):
    """int b_i^(a) b_j^(b) with scipy's B-splines and p+4 Gauss points per span."""
    xg, wg = O.gauss_rule(knots, p + 4)
    m = len(knots) - p - 1
    Fa = _scipy_basis(knots, p, xg, a)[:, 1:m - 1]
    Fb = _scipy_basis(knots, p, xg, b)[:, 1:m - 1]
    return Fa.T @ (wg[:, None] * Fb)


# ---------------------------------------------------------------- Section 2.1
@pytest.mark.parametrize("p", [2, 3, 5, 8])
def test_bspline_matches_scipy_and_partition_of_unity(p):
    for knots in (O.uniform_knots(p, 7), _nonuniform_knots(p, 9, seed=p)):
        x = np.concatenate([np.linspace(0, 1, 257), knots])
        val, der = O.bspline_basis(knots, p, x)
        assert np.abs(val.sum(axis=1) - 1).max() < 1e-14
        assert np.abs(der.sum(axis=1)).max() < 1e-11
        x_in = x[x < 1.0]
        v_in, d_in = O.bspline_basis(knots, p, x_in)
        assert np.abs(v_in - _scipy_basis(knots, p, x_in, 0)).max() < 1e-13
        assert np.abs(d_in - _scipy_basis(knots, p, x_in, 1)).max() < 1e-10


def test_bspline_derivative_central_difference():
    knots = _nonuniform_knots(4, 6, seed=1)
    x = np.linspace(0.013, 0.987, 61)
    h = 1e-6
    _, der = O.bspline_basis(knots, 4, x)
    vp, _ = O.bspline_basis(knots, 4, x + h)
    vm, _ = O.bspline_basis(knots, 4, x - h)
    assert np.abs(der - (vp - vm) / (2 * h)).max() < 1e-6


# ---------------------------------------------------------------- Section 2.2
@pytest.mark.parametrize("p,nel", [(2, 16), (3, 5), (4, 128), (6, 192), (10, 32), (5, 2)])
def test_point_count_rule(p, nel):
    xq = O.wq_points(O.uniform_knots(p, nel), p)
    assert len(xq) == 2 * nel + 2 * p - 1
    assert np.all(np.diff(xq) > 0) and xq[0] > 0 and xq[-1] < 1


def test_memory_figure_consistency():
    # Section 4: about 10 GB for the nine unsymmetrised stiffness coefficient
    # fields at 256^3 elements, nearly independent of p.
    for p in (2, 5, 8):
        nq = len(O.wq_points(O.uniform_knots(p, 256), p))
        gb = 9 * nq ** 3 * 8 / 1e9
        assert 9.0 < gb < 11.0


@pytest.mark.parametrize("p", list(range(2, 11)))
def test_weights_exactness_and_support(p):
    """Eq. (exactness1d) / Eq. (exactness_K) against integrals computed
    independently, Eq. (weights-support) on the open support, and the band
    width 2p+1 of rows whose support avoids the boundary spans."""
    for knots in (O.uniform_knots(p, max(2 * p + 3, 8)), _nonuniform_knots(p, 2 * p + 4, seed=10 + p)):
        tab = O.tables_1d(knots, p)
        m = len(knots) - p - 1
        for (a, b), W in tab.W.items():
            G = _independent_galerkin(knots, p, a, b)
            F = _scipy_basis(knots, p, tab.xq, b)[:, 1:m - 1]
            assert np.abs(W @ F - G).max() <= 1e-12 * np.abs(G).max()
            for i in range(tab.n):
                gi = i + 1
                outside = (tab.xq <= knots[gi]) | (tab.xq >= knots[gi + p + 1])
                assert np.all(W[i, outside] == 0.0)
                if p < i < tab.n - 1 - p:
                    assert np.count_nonzero(~outside) == 2 * p + 1


def _mp_basis(t, p, x, deriv):
    """B-spline values (deriv 0) or first derivatives (deriv 1) of all
    functions at x by de Boor's recursion in mpmath (this test's own
    evaluation, independent of the oracle's)."""
    import mpmath as mp
    m = len(t) - p - 1
    nb = len(t) - 1
    last = max(i for i in range(nb) if t[i] < t[i + 1])
    N = [mp.mpf(1) if (t[i] <= x < t[i + 1]) or (i == last and x == t[i + 1]) else mp.mpf(0) for i in range(nb)]
    for k in range(1, p + 1 - deriv):
        M = []
        for i in range(len(t) - k - 1):
            v = mp.mpf(0)
            if t[i + k] > t[i]:
                v += (x - t[i]) / (t[i + k] - t[i]) * N[i]
            if t[i + k + 1] > t[i + 1]:
                v += (t[i + k + 1] - x) / (t[i + k + 1] - t[i + 1]) * N[i + 1]
            M.append(v)
        N = M
    if not deriv:
        return N[:m]
    out = []
    for i in range(m):
        v = mp.mpf(0)
        if t[i + p] > t[i]:
            v += p * N[i] / (t[i + p] - t[i])
        if t[i + p + 1] > t[i + 1]:
            v -= p * N[i + 1] / (t[i + p + 1] - t[i + 1])
        out.append(v)
    return out


def _weight_systems(tab, knots, p):
    """(a, b, i, S, T) of every weight system: the row i's points S (open
    support, Eq. (weights-support)) and test functions T (|j - i| <= p)."""
    for (a, b) in tab.W:
        for i in range(tab.n):
            gi = i + 1
            S = np.nonzero((tab.xq > knots[gi]) & (tab.xq < knots[gi + p + 1]))[0]
            T = np.array([j for j in range(tab.n) if abs(j - i) <= p])
            yield a, b, i, S, T


def _nullspace_share_f64(A, w):
    """|P_null(A) w| / |w| and the condition number of A (float64 SVD)."""
    _, s, Vt = np.linalg.svd(A)
    rank = int(np.sum(s > s[0] * 1e-13))
    N = Vt[rank:]
    share = np.linalg.norm(N @ w) / np.linalg.norm(w) if N.shape[0] else 0.0
    return share, s[0] / s[rank - 1], rank


@pytest.mark.parametrize("p", list(range(2, 8)))
def test_weights_are_minimum_norm(p):
    """Reading R2: the under-determined weight systems take their
    minimum-2-norm solution, i.e. w_i lies in range(A_i^T), so its projection
    onto null(A_i) vanishes.  A_i (rows j in T, columns q in S) from scipy's
    B-splines; float64 resolves the null space to about eps * kappa(A_i), so
    the bound is 1e-14 kappa(A_i) (kappa <= 4e11 for p <= 7), against an O(1)
    share for any other solution (checked on a basic solution)."""
    for knots in (O.uniform_knots(p, max(2 * p + 3, 8)), _nonuniform_knots(p, 2 * p + 4, seed=10 + p)):
        tab = O.tables_1d(knots, p)
        m = len(knots) - p - 1
        F = {b: _scipy_basis(knots, p, tab.xq, b)[:, 1:m - 1] for b in (0, 1)}
        under = 0
        for a, b, i, S, T in _weight_systems(tab, knots, p):
            A = F[b][np.ix_(S, T)].T
            w = tab.W[(a, b)][i, S]
            share, kappa, rank = _nullspace_share_f64(A, w)
            if rank == len(S):
                continue
            under += 1
            assert share <= 1e-14 * kappa, (a, b, i, share, kappa)
            if under == 1:
                # a basic solution of the same system (nonzero on `rank` points only) is not minimum-norm
                piv = scipy.linalg.qr(A, pivoting=True)[2][:rank]
                wb = np.zeros(len(S))
                wb[piv] = np.linalg.lstsq(A[:, piv], A @ w, rcond=None)[0]
                assert np.abs(A @ wb - A @ w).max() <= 1e-9 * np.abs(A @ w).max()
                assert _nullspace_share_f64(A, wb)[0] > 1e-3
        assert under >= 2 * p  # the first and last p rows at least


@pytest.mark.slow
@pytest.mark.parametrize("p,kind", [(8, "uniform"), (10, "jittered")])
def test_weights_are_minimum_norm_high_degree(p, kind):
    """As test_weights_are_minimum_norm for p = 8, 10, where kappa(A_i) reaches
    1e13 and float64 cannot find null(A_i): A_i and its SVD in 50-digit
    mpmath (this test's own de Boor recursion); the float64 weights (the
    oracle's decimal solution rounded once) must then have a null-space share
    of rounding size."""
    import mpmath as mp
    knots = O.uniform_knots(p, max(2 * p + 3, 8)) if kind == "uniform" else _nonuniform_knots(p, 2 * p + 4, seed=10 + p)
    tab = O.tables_1d(knots, p)
    with mp.workdps(50):
        tm = [mp.mpf(float(v)) for v in knots]
        xm = [mp.mpf(float(v)) for v in tab.xq]
        vals = {b: [_mp_basis(tm, p, x, b) for x in xm] for b in (0, 1)}
        under = 0
        for a, b, i, S, T in _weight_systems(tab, knots, p):
            if len(S) == len(T):
                continue  # square systems of full rank have one solution
            A = mp.matrix([[vals[b][q][j + 1] for q in S] for j in T])
            _, s, V = mp.svd_r(A)
            smax = max(abs(v) for v in s)
            rank = sum(1 for v in s if abs(v) > smax * mp.mpf(10) ** -30)
            if rank == len(S):
                continue
            under += 1
            w = [mp.mpf(float(tab.W[(a, b)][i, q])) for q in S]
            share = mp.sqrt(sum(sum(V[r, k] * w[k] for k in range(len(S))) ** 2 for r in range(rank, V.rows)))
            assert float(share / mp.sqrt(sum(v * v for v in w))) <= 1e-14, (a, b, i)
        assert under >= 2 * p


def test_basis_tables_match_scipy():
    knots = _nonuniform_knots(3, 8, seed=3)
    tab = O.tables_1d(knots, 3)
    m = len(knots) - 3 - 1
    assert np.abs(tab.B0 - _scipy_basis(knots, 3, tab.xq, 0)[:, 1:m - 1]).max() < 1e-14
    assert np.abs(tab.B1 - _scipy_basis(knots, 3, tab.xq, 1)[:, 1:m - 1]).max() < 1e-11


# ---------------------------------------------------------------- Section 3.2
def _mixed_tables():
    return [O.tables_1d(O.uniform_knots(2, 3), 2),
            O.tables_1d(_nonuniform_knots(3, 4, seed=5), 3),
            O.tables_1d(O.uniform_knots(2, 4), 2)]


def test_constant_coefficient_equals_galerkin():
    """Identity map and a constant (here deliberately non-symmetric) C: every
    term of Eq. (stiffness_sum) is a tensor product of 1D integrals that the
    exactness conditions reproduce, so K~ equals the Galerkin stiffness
    sum_ab C_ab (G3 (x) G2 (x) G1) with G_l = int b^(a_l) b^(b_l)."""
    tabs = _mixed_tables()
    nq = int(np.prod([t.nq for t in tabs]))
    Cc = np.array([[2.0, 0.3, -0.2], [0.5, 1.5, 0.1], [0.4, -0.3, 1.2]])
    Cfull = [[np.full(nq, Cc[a, b]) for b in range(3)] for a in range(3)]
    K = O.stiffness_wq(tabs, Cfull).toarray()
    Kg = 0.0
    for a in range(3):
        for b in range(3):
            G = [_independent_galerkin(t.knots, t.p, int(l == a), int(l == b)) for l, t in enumerate(tabs)]
            Kg = Kg + Cc[a, b] * np.kron(G[2], np.kron(G[1], G[0]))
    assert np.abs(K - Kg).max() <= 1e-13 * np.abs(Kg).max()


def test_explicit_assembly_matches_entrywise_definition():
    """Kronecker assembly (Section 3.2) == K~_ij from Eq. (Kwq) term by term,
    variable non-symmetric coefficient."""
    tabs = _mixed_tables()
    nq = int(np.prod([t.nq for t in tabs]))
    g = inputs.rng(7)
    Cfull = [[g.uniform(0.5, 2.0, nq) for _ in range(3)] for _ in range(3)]
    K = O.stiffness_wq(tabs, Cfull).toarray()
    Kb = O.stiffness_wq_entries(tabs, Cfull)
    assert np.abs(K - Kb).max() <= 1e-13 * np.abs(K).max()


def test_algorithm2_and_rows_match_explicit():
    tabs = [O.tables_1d(O.uniform_knots(3, 5), 3), O.tables_1d(O.uniform_knots(2, 6), 2),
            O.tables_1d(_nonuniform_knots(4, 7, seed=2), 4)]
    C6 = O.coefficient_grid(tabs, "ring", inputs.fourier_modes(3), 0.3)
    Cfull = O.full_coeff(C6)
    K = O.stiffness_wq(tabs, Cfull)
    shape = (tabs[2].n, tabs[1].n, tabs[0].n)
    V = inputs.uniform_vector(shape, 11)
    Y = inputs.uniform_vector(shape, 12)
    ref = (K @ V.ravel()).reshape(shape)
    assert np.abs(O.apply_alg2(tabs, Cfull, V) - ref).max() <= 1e-13 * np.abs(ref).max()
    refT = (K.T @ Y.ravel()).reshape(shape)
    assert np.abs(O.apply_T_alg2(tabs, Cfull, Y) - refT).max() <= 1e-13 * np.abs(refT).max()
    rows = [(0, 0, 0), (shape[0] - 1, shape[1] - 1, shape[2] - 1), (3, 2, 4), (1, 5, 0)]
    got = O.apply_rows(tabs, O.coefficient_box_fn(tabs, "ring", inputs.fourier_modes(3), 0.3), V, rows)
    want = np.array([ref[r] for r in rows])
    assert np.abs(got - want).max() <= 1e-13 * np.abs(ref).max()


def test_symmetry_iff_constant_coefficient():
    tabs = [O.tables_1d(O.uniform_knots(3, 4), 3)] * 3
    nq = int(np.prod([t.nq for t in tabs]))
    Cs = O.full_coeff(np.stack([np.full(nq, v) for v in (1.0, 2.0, 3.0, 0.2, 0.1, -0.3)]))
    K = O.stiffness_wq(tabs, Cs).toarray()
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
    C6 = O.coefficient_grid(tabs, "ring")
    K = O.stiffness_wq(tabs, O.full_coeff(C6)).toarray()
    assert np.abs(K - K.T).max() > 1e-6 * np.abs(K).max()


# ---------------------------------------------------------------- Eq. (C)
def test_ring_coefficient_closed_form():
    """On the ring with K = I: det J = r pi/2 and C = diag(r pi/2, 2/(r pi), r pi/2)."""
    g = inputs.rng(4)
    xi = g.uniform(0, 1, size=(3, 200))
    C6 = O.coefficient_points("ring", xi[0], xi[1], xi[2])
    r = 1 + xi[0]
    np.testing.assert_allclose(C6[0], r * np.pi / 2, rtol=1e-14)
    np.testing.assert_allclose(C6[1], 2 / (r * np.pi), rtol=1e-14)
    np.testing.assert_allclose(C6[2], r * np.pi / 2, rtol=1e-14)
    assert np.abs(C6[3:]).max() < 1e-15
    modes = inputs.fourier_modes(9)
    C6k = O.coefficient_points("ring", xi[0], xi[1], xi[2], modes, 0.3)
    x1, x2, x3 = O.ring_map(xi[0], xi[1], xi[2])
    g_ = sum(a * np.cos(2 * np.pi * (k1 * x1 + k2 * x2 + k3 * x3) + ph) for a, k1, k2, k3, ph in modes)
    np.testing.assert_allclose(C6k[0], np.exp(0.3 * g_) * r * np.pi / 2, rtol=1e-13)


def test_exact_solution_forcing_is_minus_laplacian():
    g = inputs.rng(5)
    pts = g.uniform(0.2, 1.2, size=(3, 20))
    h = 1e-4
    lap = 0.0
    for d in range(3):
        e = np.zeros((3, 1))
        e[d] = h
        lap = lap + (O.exact_solution_ring(*(pts + e)) - 2 * O.exact_solution_ring(*pts)
                     + O.exact_solution_ring(*(pts - e))) / h ** 2
    f = O.exact_forcing_ring(*pts)
    assert np.abs(f + lap).max() < 1e-4 * np.abs(f).max()
    gr = O.exact_gradient_ring(*pts)
    for d in range(3):
        e = np.zeros((3, 1))
        e[d] = 1e-6
        fd = (O.exact_solution_ring(*(pts + e)) - O.exact_solution_ring(*(pts - e))) / 2e-6
        assert np.abs(gr[d] - fd).max() < 1e-6 * np.abs(gr[d]).max()


def test_load_vector_rows_match_full():
    tabs = O.uniform_tables(3, (4, 5, 6))
    F = O.load_vector(tabs, "ring", O.forcing_sines)
    rows = [(0, 0, 0), (2, 3, 1), (tabs[2].n - 1, tabs[1].n - 1, tabs[0].n - 1)]
    got = O.load_vector_rows(tabs, "ring", O.forcing_sines, rows)
    np.testing.assert_allclose(got, [F[r] for r in rows], rtol=1e-12, atol=1e-14)


def test_load_vector_of_constant_on_cube():
    """f = 1 on the unit cube: f_i = prod_l int b_{i_l}, and int b_i = (t_{i+p+1} - t_i)/(p+1)."""
    tabs = O.uniform_tables(3, 5)
    F = O.load_vector(tabs, "cube", lambda x, y, z: np.ones_like(x))
    t = tabs[0].knots
    p = 3
    ints = np.array([(t[i + p + 1] - t[i]) / (p + 1) for i in range(1, tabs[0].n + 1)])
    np.testing.assert_allclose(F, np.einsum("c,b,a->cba", ints, ints, ints), rtol=1e-13)


# ---------------------------------------------------------------- FD (Section 4)
def test_fd_is_exact_inverse_of_kronecker_laplacian():
    tabs = [O.tables_1d(O.uniform_knots(2, 5), 2), O.tables_1d(_nonuniform_knots(3, 4, 8), 3),
            O.tables_1d(O.uniform_knots(4, 3), 4)]
    fd = O.fd_setup(tabs)
    for l in range(3):
        n = tabs[l].n
        U = fd.U[l]
        assert np.abs(U.T @ fd.M[l] @ U - np.eye(n)).max() < 1e-12
        assert np.abs(U.T @ fd.K[l] @ U - np.diag(fd.lam[l])).max() < 1e-9 * fd.lam[l].max()
    P = O.fd_matrix(fd)
    shape = (tabs[2].n, tabs[1].n, tabs[0].n)
    R = inputs.uniform_vector(shape, 21)
    Z = O.fd_apply(fd, R)
    assert np.linalg.norm(P @ Z.ravel() - R.ravel()) <= 1e-12 * np.linalg.norm(R)
    np.testing.assert_allclose(Z.ravel(), O.fd_apply_explicit(fd, R.ravel()), rtol=0, atol=1e-12 * np.abs(Z).max())


def test_cube_identity_operator_is_fd_matrix_and_solve_takes_one_iteration():
    """Unit cube, K = I: C = I, so K~ equals the Kronecker Laplacian P exactly
    and FD-preconditioned BiCGStab converges in one iteration."""
    patch = O.make_patch(2, 6, "cube")
    K = O.stiffness_wq(patch.tabs, patch.Cfull)
    P = O.fd_matrix(patch.fd)
    assert abs(K - P).max() <= 1e-13 * abs(P).max()
    F = O.load_vector(patch.tabs, "cube", O.forcing_sines)
    U, info = patch.solve(F, 1e-10)
    assert info.converged and info.iterations == 1


# ---------------------------------------------------------------- BiCGStab
def test_bicgstab_matches_direct_solve():
    tabs = O.uniform_tables(3, (5, 4, 6))
    C6 = O.coefficient_grid(tabs, "ring", inputs.fourier_modes(1), 0.3)
    patch = O.Patch(tabs, C6, O.fd_setup(tabs))
    K = O.stiffness_wq(tabs, patch.Cfull).tocsc()
    F = O.load_vector(tabs, "ring", O.forcing_sines)
    ref = spla.spsolve(K, F.ravel())
    U, info = patch.solve(F, 1e-12)
    assert info.converged
    assert np.linalg.norm(U.ravel() - ref) <= 1e-10 * np.linalg.norm(ref)
    # transposed system
    UT, infoT = patch.solve(F, 1e-12, transpose=True)
    refT = spla.spsolve(K.T.tocsc(), F.ravel())
    assert infoT.converged and np.linalg.norm(UT.ravel() - refT) <= 1e-10 * np.linalg.norm(refT)


def test_bicgstab_breakdown_and_maxit_reported():
    patch = O.make_patch(2, 4, "ring")
    F = O.load_vector(patch.tabs, "ring", O.forcing_sines)
    _, info = patch.solve(F, 1e-14, maxit=1)
    assert not info.converged and info.iterations == 1
    _, info0 = patch.solve(np.zeros_like(F), 1e-10)
    assert info0.converged and info0.iterations == 0


# ---------------------------------------------------------------- adjoint
def test_gradient_euler_identity_and_central_differences():
    """K~ is linear in C, so sum_q sum_ab C_ab dJ/dC_ab = -lambda^T K~ u = -lambda^T f;
    and dJ/dC matches central differences of J(C) = 1/2 ||u(C) - u_t||^2."""
    tabs = O.uniform_tables(3, 4)
    modes = inputs.fourier_modes(2)
    C6 = O.coefficient_grid(tabs, "ring", modes, 0.3)
    F = O.load_vector(tabs, "ring", O.forcing_sines)
    shape = F.shape

    def solve(C6_, rhs, transpose=False):
        K = O.stiffness_wq(tabs, O.full_coeff(C6_)).tocsc()
        return spla.spsolve(K.T.tocsc() if transpose else K, rhs.ravel()).reshape(shape)

    u_t = solve(O.coefficient_grid(tabs, "ring"), F)
    u = solve(C6, F)
    lam = solve(C6, u - u_t, transpose=True)
    g = O.grad_coeff(tabs, lam, u)
    euler = np.sum(C6 * g)
    assert abs(euler + np.dot(lam.ravel(), F.ravel())) <= 1e-10 * abs(np.dot(lam.ravel(), F.ravel()))

    def J(C6_):
        d = solve(C6_, F) - u_t
        return 0.5 * np.dot(d.ravel(), d.ravel())

    gr = inputs.rng(3)
    h = 1e-6
    for _ in range(3):
        d = gr.uniform(-1, 1, size=C6.shape) * C6.std(axis=(1, 2, 3))[:, None, None, None]
        fd = (J(C6 + h * d) - J(C6 - h * d)) / (2 * h)
        an = np.sum(g * d)
        assert abs(fd - an) <= 1e-5 * abs(an)


# ---------------------------------------------------------------- reaction (mass) term
def test_constant_mass_equals_galerkin_mass():
    """Eq. (Mwq) with constant c: each direction's W^(00) B^(0) reproduces the 1D
    mass integrals (exactness), so M~ = c (G3 (x) G2 (x) G1) with G_l = int b_i b_j
    (computed here with scipy's B-splines and an independent Gauss rule)."""
    tabs = _mixed_tables()
    nq = int(np.prod([t.nq for t in tabs]))
    M = O.mass_wq(tabs, np.full(nq, 2.5)).toarray()
    G = [_independent_galerkin(t.knots, t.p, 0, 0) for t in tabs]
    Mg = 2.5 * np.kron(G[2], np.kron(G[1], G[0]))
    assert np.abs(M - Mg).max() <= 1e-13 * np.abs(Mg).max()
    assert np.abs(M - M.T).max() <= 1e-13 * np.abs(M).max()


def test_mass_assembly_algorithm1_rows_and_transpose():
    """Kronecker assembly of M~ == Eq. (Mwq) entry by entry (variable c on the
    ring); Algorithm 1, the transpose and the row-sampled form == the matrix."""
    tabs = _mixed_tables()
    c = O.mass_coefficient_grid(tabs, "ring", 3.0)
    M = O.mass_wq(tabs, c)
    Mb = O.mass_wq_entries(tabs, c)
    assert np.abs(M.toarray() - Mb).max() <= 1e-13 * np.abs(Mb).max()
    assert np.abs(M.toarray() - M.toarray().T).max() > 1e-6 * np.abs(Mb).max()  # non-constant c: not symmetric
    shape = (tabs[2].n, tabs[1].n, tabs[0].n)
    V = inputs.uniform_vector(shape, 31)
    ref = (M @ V.ravel()).reshape(shape)
    assert np.abs(O.apply_mass_alg1(tabs, c, V) - ref).max() <= 1e-13 * np.abs(ref).max()
    refT = (M.T @ V.ravel()).reshape(shape)
    assert np.abs(O.apply_mass_T(tabs, c, V) - refT).max() <= 1e-13 * np.abs(refT).max()
    rows = [(0, 0, 0), (shape[0] - 1, shape[1] - 1, shape[2] - 1), (1, 2, 1)]
    got = O.mass_rows(tabs, O.mass_coefficient_box_fn(tabs, "ring", 3.0), V, rows)
    assert np.abs(got - np.array([ref[r] for r in rows])).max() <= 1e-13 * np.abs(ref).max()


def test_ring_mass_coefficient_integrates_to_the_volume():
    """int c / alpha over the parameter cube = volume of the quarter ring shell,
    pi/4 (2^2 - 1^2) = 3 pi/4 (c = alpha det J, Eq. (M))."""
    xg, wg = O.gauss_rule(O.uniform_knots(2, 3), 3)
    X3, X2, X1 = np.meshgrid(xg, xg, xg, indexing="ij")
    c = O.mass_coefficient_points("ring", X1, X2, X3, 2.0)
    vol = np.einsum("c,b,a,cba->", wg, wg, wg, c) / 2.0
    assert abs(vol - 0.75 * np.pi) <= 1e-14


def test_cube_reaction_operator_is_shifted_fd_matrix():
    """Unit cube, K = I, constant alpha: K~ + M~ = P + alpha M3(x)M2(x)M1, the
    FD with shift alpha is its exact inverse, and the preconditioned solve
    converges in one iteration (reading R15)."""
    tabs = O.uniform_tables(2, (5, 4, 6))
    alpha = 7.0
    C6 = O.coefficient_grid(tabs, "cube")
    c = O.mass_coefficient_grid(tabs, "cube", alpha)
    A = O.stiffness_wq(tabs, O.full_coeff(C6)) + O.mass_wq(tabs, c)
    fd = O.fd_setup(tabs, shift=alpha)
    P = O.fd_matrix(fd)
    assert abs(A - P).max() <= 1e-13 * abs(P).max()
    shape = (tabs[2].n, tabs[1].n, tabs[0].n)
    R = inputs.uniform_vector(shape, 41)
    Z = O.fd_apply(fd, R)
    assert np.linalg.norm(P @ Z.ravel() - R.ravel()) <= 1e-12 * np.linalg.norm(R)
    patch = O.Patch(tabs, C6, fd, c)
    U, info = patch.solve(O.load_vector(tabs, "cube", O.forcing_sines), 1e-10)
    assert info.converged and info.iterations == 1


def test_reaction_gradient_euler_identity_and_central_differences():
    """K~(C) + M~(c) is linear in (C, c) jointly: sum C dJ/dC + sum c dJ/dc =
    -lambda^T f; dJ/dc matches central differences."""
    tabs = O.uniform_tables(2, (4, 3, 5))
    C6 = O.coefficient_grid(tabs, "ring", inputs.fourier_modes(5), 0.3)
    c = O.mass_coefficient_grid(tabs, "ring", 4.0)
    F = O.load_vector(tabs, "ring", O.forcing_sines)
    shape = F.shape

    def solve(cc, rhs, transpose=False):
        A = (O.stiffness_wq(tabs, O.full_coeff(C6)) + O.mass_wq(tabs, cc)).tocsc()
        return spla.spsolve(A.T.tocsc() if transpose else A, rhs.ravel()).reshape(shape)

    u_t = solve(0.0 * c, F)
    u = solve(c, F)
    lam = solve(c, u - u_t, transpose=True)
    gC, gc = O.grad_coeff(tabs, lam, u), O.grad_mass_coeff(tabs, lam, u)
    lf = np.dot(lam.ravel(), F.ravel())
    assert abs(np.sum(C6 * gC) + np.sum(c * gc) + lf) <= 1e-10 * abs(lf)

    def J(cc):
        d = solve(cc, F) - u_t
        return 0.5 * np.dot(d.ravel(), d.ravel())

    gr = inputs.rng(9)
    h = 1e-6
    for _ in range(3):
        d = gr.uniform(-1, 1, size=c.shape) * c
        fdv = (J(c + h * d) - J(c - h * d)) / (2 * h)
        an = np.sum(gc * d)
        assert abs(fdv - an) <= 1e-5 * abs(an)


# ---------------------------------------------------------------- Table 1
def _table1():
    rows = {}
    for line in open(os.path.join(GOLDEN, "table1_h1_errors.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = line.split()
        rows[int(v[0])] = [float(x) for x in v[1:]]
    return rows


@pytest.mark.slow
@pytest.mark.parametrize("p", [2, 3, 4])
def test_k_refinement_error_against_table1(p):
    """Section 4, Table 1: no approximation at h = 2^-4 (error ~ 0.5), and at
    h = 2^-5 the error agrees with the printed one within a factor 1.5 (the paper
    uses a NURBS ring, the oracle the exact polar map)."""
    table = _table1()
    errs = []
    for nel in (16, 32):
        tabs = O.uniform_tables(p, nel)
        patch = O.Patch(tabs, O.coefficient_grid(tabs, "ring"), O.fd_setup(tabs))
        F = O.load_vector(tabs, "ring", O.exact_forcing_ring)
        U, info = patch.solve(F, 1e-10)
        assert info.converged
        errs.append(O.h1_error(tabs, U, "ring", O.exact_solution_ring, O.exact_gradient_ring))
    assert 0.2 < errs[0] < 1.2
    assert table[p][1] / 1.5 < errs[1] < table[p][1] * 1.5
    assert errs[1] < errs[0] / 4
