"""MF-WQ oracle: plain float64 CPU implementation -- TEST INFRASTRUCTURE ONLY.

Imported only by tests/, __graft_entry__.smoke() and bench.py's cpu_baseline
and ``--impl reference`` legs.  It shares no code with the CUDA library.

Citations are to the paper's sections, equations and algorithms
(Sangalli & Tani, "Matrix-free weighted quadrature for a computationally
efficient isogeometric k-method"):

* Section 2.1  -- open knot vectors, B-splines, interior index set, ordering.
* Eq. (C), (A) -- stiffness coefficient C and Galerkin stiffness.
* Section 2.2  -- weighted quadrature: Eq. (exactness1d), Eq. (weights-support),
                  the point rule, Eq. (stiffness_sum), Eq. (Kwq), Eq. (exactness_K).
* Section 2.3  -- Kronecker products, Eq. (ordering), Eq. (sum-factorization).
* Eq. (M), (Mwq), (exactness_M) -- the mass (reaction) term c = alpha det J and
                  its WQ approximation M~_ij = sum_q w_iq c(x_q) b_j(x_q).
* Section 3.1  -- the factorisation M~ = W D B, Algorithm 1.
* Section 3.2  -- the factorisation K~ = sum_ab W^(ab) D^(ab) B^(b), Algorithm 2.
* Section 4    -- ring domain, Eq. (exact-solution), BiCGStab + FD preconditioner.

Readings of passages the paper leaves open (both implementations follow each one):

* R1  WQ points: all interior knots, the midpoints of the interior spans, and
      p+1 equispaced interior points in the first and in the last span
      (n_q = 2*nel + 2p - 1).
* R2  Boundary rows of the weight systems are under-determined; the weights
      are the minimum-2-norm solution.
* R3  "x_q not in supp" uses the open support.
* R4  The direction-l factor of W^(ab) is the 1D family W_l^(a_l,b_l) with
      a_l = [l = alpha], b_l = [l = beta], exact for
      int b_i^(a) b_j^(b) = sum_q w_iq b_j^(b)(x_q).
* R5  C = |det J| J^-1 K J^-T with J_ij = dF_i/dxi_j.
* R6  FD preconditioner: P = M3(x)M2(x)K1 + M3(x)K2(x)M1 + K3(x)M2(x)M1 built
      from exact 1D Galerkin K_l, M_l; P^-1 = U diag(1/(l1+l2+l3)) U^T with
      U_l^T M_l U_l = I, U_l^T K_l U_l = diag(l_l).
* R7  BiCGStab: right preconditioning, x0 given (default 0), r^_0 = r_0,
      convergence tested on the half step s and on the full step r.
* R8  Load vector: tensor Gauss with p_l+1 points per span in direction l, c = |det J|.
      The relative H1 error of Section 4 uses p_l+2 points per span in direction l.
* R14 Mass weights: the 1D family W^(00) of the stiffness (exactness for
      int b_i b_j, Eq. (exactness1d)) in every direction, so the mass term
      uses the same weights as the (alpha != l, beta != l) stiffness factors.
* R15 FD with a reaction term: P_sigma = P + sigma M3(x)M2(x)M1, whose inverse
      is U diag(1/(l1+l2+l3+sigma)) U^T with the same U (sigma >= 0 chosen by
      the caller; the paper gives no preconditioner for alpha > 0).

Boundary-row weights are pinned by exactness, support and the minimum-norm
property (w_i in range(A_i^T)); the paper prints no weight values.
Parity unpinned (nothing in the paper or in mathematics fixes them): BiCGStab
iteration counts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from decimal import Decimal, localcontext

import numpy as np
import scipy.linalg
import scipy.sparse as sp

# Storage order of the six symmetric coefficient fields (Section 3.2: only
# d(d+1)/2 of the C_ab need storing when C is symmetric).
SYM_PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


# ---------------------------------------------------------------------------
# Section 2.1: knots and B-splines
# ---------------------------------------------------------------------------
def open_knots(p: int, breaks) -> np.ndarray:
    """Open knot vector of degree p on the break points 0=u_0<...<u_nel=1,
    every interior knot of multiplicity 1 (maximum regularity, Section 2.1)."""
    u = np.asarray(breaks, dtype=np.float64)
    return np.concatenate([np.full(p, u[0]), u, np.full(p, u[-1])])


def uniform_knots(p: int, nel: int) -> np.ndarray:
    return open_knots(p, np.linspace(0.0, 1.0, nel + 1))


def num_functions(knots, p: int) -> int:
    """m: number of B-splines of degree p on the knot vector."""
    return len(knots) - p - 1


def bspline_basis(knots, p: int, x):
    """Values and first derivatives of all m B-splines at the points x.

    Cox-de Boor recursion from its definition: degree 0 are indicators of
    [t_i, t_{i+1}) (the point 1 belongs to the last non-empty span), degree k
    mixes degree k-1 with the usual ratios (0/0 taken as 0); the derivative
    of a degree-p B-spline is p times a difference of degree p-1 ones.
    Returns (val, der), each of shape (len(x), m).
    """
    t = np.asarray(knots, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    nb0 = len(t) - 1
    N = np.zeros((len(x), nb0))
    nonempty = [i for i in range(nb0) if t[i] < t[i + 1]]
    last = nonempty[-1]
    for i in nonempty:
        inside = (x >= t[i]) & (x < t[i + 1])
        if i == last:
            inside |= x == t[i + 1]
        N[:, i] = inside

    def raise_degree(Nprev, k):
        ncol = len(t) - k - 1
        out = np.zeros((len(x), ncol))
        for i in range(ncol):
            d1 = t[i + k] - t[i]
            d2 = t[i + k + 1] - t[i + 1]
            if d1 > 0:
                out[:, i] += (x - t[i]) / d1 * Nprev[:, i]
            if d2 > 0:
                out[:, i] += (t[i + k + 1] - x) / d2 * Nprev[:, i + 1]
        return out

    for k in range(1, p):
        N = raise_degree(N, k)
    Nlow = N  # degree p-1
    val = raise_degree(Nlow, p) if p >= 1 else N
    m = len(t) - p - 1
    der = np.zeros((len(x), m))
    for i in range(m):
        d1 = t[i + p] - t[i]
        d2 = t[i + p + 1] - t[i + 1]
        if d1 > 0:
            der[:, i] += p / d1 * Nlow[:, i]
        if d2 > 0:
            der[:, i] -= p / d2 * Nlow[:, i + 1]
    return val, der


def gauss_rule(knots, k: int):
    """Gauss-Legendre rule with k points in every knot span."""
    u = np.unique(np.asarray(knots, dtype=np.float64))
    g, w = np.polynomial.legendre.leggauss(k)
    xs, ws = [], []
    for s in range(len(u) - 1):
        a, b = u[s], u[s + 1]
        xs.append(0.5 * (a + b) + 0.5 * (b - a) * g)
        ws.append(0.5 * (b - a) * w)
    return np.concatenate(xs), np.concatenate(ws)


def galerkin_1d(knots, p: int, a: int, b: int) -> np.ndarray:
    """G[i, j] = int_0^1 b_i^(a) b_j^(b) over the interior functions
    i, j = 1..m-2 (Section 2.1), exact by Gauss with p+1 points per span."""
    xg, wg = gauss_rule(knots, p + 1)
    val, der = bspline_basis(knots, p, xg)
    m = val.shape[1]
    Fa = (der if a else val)[:, 1:m - 1]
    Fb = (der if b else val)[:, 1:m - 1]
    return Fa.T @ (wg[:, None] * Fb)


# ---------------------------------------------------------------------------
# Section 2.2: weighted quadrature in one direction
# ---------------------------------------------------------------------------
def wq_points(knots, p: int) -> np.ndarray:
    """Reading R1 of the point rule of Section 2.2."""
    u = np.unique(np.asarray(knots, dtype=np.float64))
    nel = len(u) - 1
    inner = np.arange(1, p + 2) / (p + 2)
    pts = list(u[0] + (u[1] - u[0]) * inner)
    for s in range(1, nel - 1):
        pts.append(u[s])
        pts.append(0.5 * (u[s] + u[s + 1]))
    if nel >= 2:
        pts.append(u[nel - 1])
        pts.extend(u[nel - 1] + (u[nel] - u[nel - 1]) * inner)
    return np.array(pts)


# The weight systems are ill-conditioned for larger p (condition numbers near
# 1e9 at p = 6 and 1e11 at p = 8 with the points of reading R1), so float64
# solves of them agree only to about kappa * 1e-16.  The oracle therefore
# computes the minimum-norm solution in 80-digit decimal arithmetic from the
# exact binary values of the knots, and rounds the result to float64 once.
_DPREC = 80


def _dec(x):
    return Decimal(float(x))


def _dec_points(tD, p):
    """Reading R1 in decimal arithmetic (same points as wq_points)."""
    u = sorted(set(tD))
    nel = len(u) - 1
    pts = [u[0] + (u[1] - u[0]) * k / (p + 2) for k in range(1, p + 2)]
    for s in range(1, nel - 1):
        pts.append(u[s])
        pts.append((u[s] + u[s + 1]) / 2)
    if nel >= 2:
        pts.append(u[nel - 1])
        pts.extend(u[nel - 1] + (u[nel] - u[nel - 1]) * k / (p + 2) for k in range(1, p + 2))
    return pts


def _dec_basis(tD, p, x):
    """All B-splines of degree p and their derivatives at one decimal point x,
    by the Cox-de Boor definition; returns dicts index -> value."""
    nb = len(tD) - 1
    nonempty = [i for i in range(nb) if tD[i] < tD[i + 1]]
    N = {}
    for i in nonempty:
        if tD[i] <= x < tD[i + 1] or (i == nonempty[-1] and x == tD[i + 1]):
            N[i] = Decimal(1)
    low = N
    for k in range(1, p + 1):
        M = {}
        for i in range(len(tD) - k - 1):
            v = Decimal(0)
            d1 = tD[i + k] - tD[i]
            d2 = tD[i + k + 1] - tD[i + 1]
            if d1 > 0 and i in N:
                v += (x - tD[i]) / d1 * N[i]
            if d2 > 0 and (i + 1) in N:
                v += (tD[i + k + 1] - x) / d2 * N[i + 1]
            if v != 0:
                M[i] = v
        if k == p:
            low = N
        N = M
    D = {}
    for i in range(len(tD) - p - 1):
        v = Decimal(0)
        d1 = tD[i + p] - tD[i]
        d2 = tD[i + p + 1] - tD[i + 1]
        if d1 > 0 and i in low:
            v += p * low[i] / d1
        if d2 > 0 and (i + 1) in low:
            v -= p * low[i + 1] / d2
        if v != 0:
            D[i] = v
    return N, D


def _dec_gauss(k):
    """Gauss-Legendre nodes/weights on [-1, 1], Newton's method in decimal."""
    g0, _ = np.polynomial.legendre.leggauss(k)
    nodes, weights = [], []
    for z0 in g0:
        z = Decimal(float(z0))
        for _ in range(8):
            p0, p1 = Decimal(1), z
            for j in range(2, k + 1):
                p0, p1 = p1, ((2 * j - 1) * z * p1 - (j - 1) * p0) / j
            dp = k * (z * p1 - p0) / (z * z - 1)
            z = z - p1 / dp
        p0, p1 = Decimal(1), z
        for j in range(2, k + 1):
            p0, p1 = p1, ((2 * j - 1) * z * p1 - (j - 1) * p0) / j
        dp = k * (z * p1 - p0) / (z * z - 1)
        nodes.append(z)
        weights.append(2 / ((1 - z * z) * dp * dp))
    return nodes, weights


def _dec_independent_rows(A):
    """Indices of rows of A that are not combinations of earlier kept rows
    (Gaussian elimination with column pivoting; a remaining row whose largest
    entry falls below 1e-40 of the largest entry of A is dependent)."""
    big = max(abs(v) for row in A for v in row)
    basis = []  # (pivot column, reduced row)
    keep = []
    for i, row in enumerate(A):
        r = list(row)
        for col, b in basis:
            f = r[col] / b[col]
            if f != 0:
                r = [x - f * y for x, y in zip(r, b)]
        col = max(range(len(r)), key=lambda k: abs(r[k]))
        if abs(r[col]) > big * Decimal("1e-40"):
            basis.append((col, r))
            keep.append(i)
    return keep


def _dec_min_norm(A, g):
    """Minimum-2-norm solution of the consistent system A w = g (A: list of
    rows): w = A_r^T (A_r A_r^T)^-1 g_r over the independent rows A_r (the
    dependent equations hold for every solution of the others)."""
    keep = _dec_independent_rows(A)
    Ar = [A[i] for i in keep]
    gr = [g[i] for i in keep]
    r = len(Ar)
    c = len(Ar[0])
    G = [[sum(Ar[i][k] * Ar[j][k] for k in range(c)) for j in range(r)] for i in range(r)]
    # Cholesky G = L L^T, then L L^T z = g_r
    L = [[Decimal(0)] * r for _ in range(r)]
    for j in range(r):
        d = G[j][j] - sum(L[j][k] * L[j][k] for k in range(j))
        L[j][j] = d.sqrt()
        for i in range(j + 1, r):
            L[i][j] = (G[i][j] - sum(L[i][k] * L[j][k] for k in range(j))) / L[j][j]
    y = [Decimal(0)] * r
    for i in range(r):
        y[i] = (gr[i] - sum(L[i][k] * y[k] for k in range(i))) / L[i][i]
    z = [Decimal(0)] * r
    for i in reversed(range(r)):
        z[i] = (y[i] - sum(L[k][i] * z[k] for k in range(i + 1, r))) / L[i][i]
    return [sum(Ar[i][k] * z[i] for i in range(r)) for k in range(c)]


def wq_weights_all(knots, p: int):
    """The four 1D weight families {(a, b): W (n x n_q)}.

    Row i solves Eq. (exactness1d) / the 1D form of Eq. (exactness_K),
    int b_i^(a) b_j^(b) = sum_q w_iq b_j^(b)(x_q) for every interior j, with
    w_iq = 0 unless x_q lies in the open support of b_i (Eq. (weights-support),
    reading R3).  Equations for |j - i| > p hold trivially (both sides vanish),
    the rest are solved in the minimum-2-norm sense (reading R2); the
    integrals use Gauss-Legendre with p+1 points per span (exact).
    """
    with localcontext() as ctx:
        ctx.prec = _DPREC
        tD = [_dec(v) for v in knots]
        m = len(tD) - p - 1
        n = m - 2
        xq = _dec_points(tD, p)
        nq = len(xq)
        at_q = [_dec_basis(tD, p, x) for x in xq]
        u = sorted(set(tD))
        gn, gw = _dec_gauss(p + 1)
        gauss = []  # (weight, (N, D)) over all spans
        for s in range(len(u) - 1):
            a0, b0 = u[s], u[s + 1]
            for z, w in zip(gn, gw):
                x = (a0 + b0) / 2 + (b0 - a0) / 2 * z
                gauss.append(((b0 - a0) / 2 * w, _dec_basis(tD, p, x)))

        def integral(i, a, j, b):
            tot = Decimal(0)
            for w, (N, D) in gauss:
                fa = (D if a else N).get(i)
                fb = (D if b else N).get(j)
                if fa is not None and fb is not None:
                    tot += w * fa * fb
            return tot

        out = {(a, b): np.zeros((n, nq)) for a in (0, 1) for b in (0, 1)}
        for i in range(n):
            gi = i + 1
            S = [q for q in range(nq) if tD[gi] < xq[q] < tD[gi + p + 1]]
            T = [j for j in range(n) if abs(j - i) <= p]
            for b in (0, 1):
                A = [[(at_q[q][1] if b else at_q[q][0]).get(j + 1, Decimal(0)) for q in S] for j in T]
                for a in (0, 1):
                    rhs = [integral(gi, a, j + 1, b) for j in T]
                    w = _dec_min_norm(A, rhs)
                    res = max(abs(sum(A[r][k] * w[k] for k in range(len(S))) - rhs[r]) for r in range(len(T)))
                    if res > Decimal("1e-40") * max(abs(v) for v in rhs):
                        raise ValueError(f"WQ system of row {i} is inconsistent")
                    out[(a, b)][i, S] = [float(v) for v in w]
    return out


def wq_weights(knots, p: int, xq, a: int, b: int) -> np.ndarray:
    """One weight family (a, b) (see wq_weights_all); xq must be wq_points(knots, p)."""
    W = wq_weights_all(knots, p)[(a, b)]
    assert W.shape[1] == len(xq)
    return W


def wq_weights_float64(knots, p: int, xq, a: int, b: int) -> np.ndarray:
    """Same systems solved in float64 by numpy's lstsq (a cross-check that is
    accurate only while the systems are well conditioned, p <= 4)."""
    t = np.asarray(knots, dtype=np.float64)
    xq = np.asarray(xq, dtype=np.float64)
    n = num_functions(t, p) - 2
    val, der = bspline_basis(t, p, xq)
    Fb = der if b else val
    G = galerkin_1d(t, p, a, b)
    W = np.zeros((n, len(xq)))
    for i in range(n):
        gi = i + 1
        S = np.nonzero((xq > t[gi]) & (xq < t[gi + p + 1]))[0]
        T = np.array([j for j in range(n) if abs(j - i) <= p])
        W[i, S] = np.linalg.lstsq(Fb[np.ix_(S, T + 1)].T, G[i, T], rcond=None)[0]
    return W


@dataclass
class Tables1D:
    """One direction's 1D data of Algorithm 2's setup: points, B0/B1 (values
    and derivatives of the interior B-splines at the points, Eq. (Bl)) and the
    four weight families W[(a, b)]."""
    p: int
    knots: np.ndarray
    xq: np.ndarray
    B0: np.ndarray
    B1: np.ndarray
    W: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.B0.shape[1]

    @property
    def nq(self) -> int:
        return len(self.xq)


def tables_1d(knots, p: int) -> Tables1D:
    t = np.asarray(knots, dtype=np.float64)
    xq = wq_points(t, p)
    val, der = bspline_basis(t, p, xq)
    m = val.shape[1]
    tab = Tables1D(p=p, knots=t, xq=xq, B0=val[:, 1:m - 1].copy(), B1=der[:, 1:m - 1].copy())
    key = (p, t.tobytes())
    if key not in _WEIGHT_CACHE:
        _WEIGHT_CACHE[key] = wq_weights_all(t, p)
    tab.W = {k: v.copy() for k, v in _WEIGHT_CACHE[key].items()}
    return tab


_WEIGHT_CACHE = {}


def uniform_tables(p, nel):
    """Three directions with open uniform knots; p, nel scalars or 3-tuples
    ordered (direction 1, direction 2, direction 3)."""
    ps = p if np.ndim(p) else (p, p, p)
    ns = nel if np.ndim(nel) else (nel, nel, nel)
    return [tables_1d(uniform_knots(ps[l], ns[l]), ps[l]) for l in range(3)]


# ---------------------------------------------------------------------------
# Section 2.3: Kronecker products, ordering with direction 1 fastest
# ---------------------------------------------------------------------------
def kron3(A3, A2, A1):
    """A3 (x) A2 (x) A1 as a sparse matrix; with the scalar ordering of
    Eq. (ordering) an index vector is the C-order flattening of [i3][i2][i1]."""
    return sp.kron(sp.csr_matrix(A3), sp.kron(sp.csr_matrix(A2), sp.csr_matrix(A1), "csr"), "csr")


def kron_action(A3, A2, A1, X):
    """(A3 (x) A2 (x) A1) x for x given as the tensor X[j3][j2][j1], evaluated
    by the nested sums of Eq. (sum-factorization)."""
    Y = np.tensordot(X, A1, axes=([2], [1]))            # [j3][j2][i1]
    Y = np.tensordot(Y, A2, axes=([1], [1]))            # [j3][i1][i2]
    Y = np.tensordot(Y, A3, axes=([0], [1]))            # [i1][i2][i3]
    return np.ascontiguousarray(Y.transpose(2, 1, 0))   # [i3][i2][i1]


def _pattern(l, alpha, beta):
    return (int(l == alpha), int(l == beta))


def w_factor(tab, l, alpha, beta):
    """Direction-l factor of W^(alpha,beta) (reading R4)."""
    return tab.W[_pattern(l, alpha, beta)]


def b_factor(tab, l, beta):
    """Direction-l factor of B^(beta): derivatives in direction beta, values elsewhere (Section 3.2)."""
    return tab.B1 if l == beta else tab.B0


def full_coeff(C6):
    """Expand the 6 symmetric fields (order 11,22,33,12,13,23) to a 3x3 nested list."""
    C = [[None] * 3 for _ in range(3)]
    for s, (a, b) in enumerate(SYM_PAIRS):
        C[a][b] = C6[s]
        C[b][a] = C6[s]
    return C


# ---------------------------------------------------------------------------
# Section 3.2: the WQ stiffness operator
# ---------------------------------------------------------------------------
def stiffness_wq(tabs, Cfull) -> sp.csr_matrix:
    """Explicit K~ = sum_{alpha,beta} W^(ab) D^(ab) B^(b) (Section 3.2, the
    factorisation preceding Algorithm 2).  Cfull[a][b] holds C_ab at the
    quadrature points flattened with direction 1 fastest."""
    K = None
    for al in range(3):
        for be in range(3):
            Wk = kron3(*[w_factor(tabs[l], l, al, be) for l in (2, 1, 0)])
            Bk = kron3(*[b_factor(tabs[l], l, be) for l in (2, 1, 0)])
            term = Wk @ sp.diags(np.ravel(Cfull[al][be])) @ Bk
            K = term if K is None else K + term
    return K.tocsr()


def stiffness_wq_entries(tabs, Cfull) -> np.ndarray:
    """Dense K~ entry by entry from Eq. (Kwq): K~_ij = sum_ab sum_q
    w^(ab)_{i,q} C_ab(x_q) d_b b_j(x_q), with the tensor weights
    w^(ab)_{i,q} = prod_l w^(ab)_{l,i_l,q_l} and tensor B-spline derivatives.
    For tiny grids only (N^2 * N_q work)."""
    n = [t.n for t in tabs]
    nq = [t.nq for t in tabs]
    N = n[0] * n[1] * n[2]
    K = np.zeros((N, N))
    Cg = [[np.reshape(Cfull[a][b], (nq[2], nq[1], nq[0])) for b in range(3)] for a in range(3)]
    for i in range(N):
        i3, rem = divmod(i, n[0] * n[1])
        i2, i1 = divmod(rem, n[0])
        ii = (i1, i2, i3)
        for j in range(N):
            j3, rem = divmod(j, n[0] * n[1])
            j2, j1 = divmod(rem, n[0])
            jj = (j1, j2, j3)
            s = 0.0
            for al in range(3):
                for be in range(3):
                    w = np.einsum("c,b,a->cba", *[w_factor(tabs[l], l, al, be)[ii[l]] for l in (2, 1, 0)])
                    d = np.einsum("c,b,a->cba", *[b_factor(tabs[l], l, be)[:, jj[l]] for l in (2, 1, 0)])
                    s += np.sum(w * Cg[al][be] * d)
            K[i, j] = s
    return K


def apply_alg2(tabs, Cfull, V):
    """w = K~ v by the steps of Algorithm 2 (MF-WQ product, stiffness), each
    Kronecker product applied through Eq. (sum-factorization).  V and the
    result are tensors [i3][i2][i1]; Cfull[a][b] are tensors [q3][q2][q1]."""
    W = np.zeros_like(V, dtype=np.float64)
    for be in range(3):
        vt = kron_action(*[b_factor(tabs[l], l, be) for l in (2, 1, 0)], V)
        for al in range(3):
            vtt = Cfull[al][be] * vt
            W += kron_action(*[w_factor(tabs[l], l, al, be) for l in (2, 1, 0)], vtt)
    return W


def apply_T_alg2(tabs, Cfull, Y):
    """K~^T y = sum_ab B^(b)^T D^(ab) W^(ab)^T y (transpose of Section 3.2's
    factorisation, taken term by term)."""
    out = np.zeros_like(Y, dtype=np.float64)
    for be in range(3):
        acc = None
        for al in range(3):
            s = kron_action(*[w_factor(tabs[l], l, al, be).T for l in (2, 1, 0)], Y)
            term = Cfull[al][be] * s
            acc = term if acc is None else acc + term
        out += kron_action(*[b_factor(tabs[l], l, be).T for l in (2, 1, 0)], acc)
    return out


def grad_coeff(tabs, LAM, U):
    """dJ/dC for J depending on C through K~(C) u = f, given the adjoint
    lambda (K~^T lambda = dJ/du): since K~ is linear in every C_ab(x_q)
    (Section 3.2), dJ/dC_ab(q) = -(W^(ab)^T lambda)_q (B^(b) u)_q.  The
    symmetric storage slot of an off-diagonal pair receives the sum of both
    orderings.  Returns shape (6, nq3, nq2, nq1)."""
    G = [kron_action(*[b_factor(tabs[l], l, be) for l in (2, 1, 0)], U) for be in range(3)]
    g = {}
    for al in range(3):
        for be in range(3):
            S = kron_action(*[w_factor(tabs[l], l, al, be).T for l in (2, 1, 0)], LAM)
            g[(al, be)] = -S * G[be]
    out = []
    for (a, b) in SYM_PAIRS:
        out.append(g[(a, b)] if a == b else g[(a, b)] + g[(b, a)])
    return np.stack(out)


def _row_supports(tab, i):
    return np.nonzero(np.any(np.stack([tab.W[k][i] != 0 for k in tab.W]), axis=0))[0]


def apply_rows(tabs, coef_box, V, rows):
    """Selected entries (K~ v)_i, each computed on its own from Eq. (Kwq):
    sum_ab sum_q w^(ab)_{i,q} C_ab(x_q) d_b v_h(x_q), q running over the points
    where the tensor weights of row i may be nonzero and d_b v_h(x_q) summed
    over the B-splines nonzero there.  coef_box(S3, S2, S1) returns the six
    symmetric C fields on that point box, shape (6, |S3|, |S2|, |S1|)."""
    out = np.empty(len(rows))
    for r, (i3, i2, i1) in enumerate(rows):
        ii = (i1, i2, i3)
        S = [_row_supports(tabs[l], ii[l]) for l in range(3)]
        J = [np.nonzero(np.any((tabs[l].B0[S[l]] != 0) | (tabs[l].B1[S[l]] != 0), axis=0))[0] for l in range(3)]
        vloc = V[np.ix_(J[2], J[1], J[0])]
        C = full_coeff(coef_box(S[2], S[1], S[0]))
        s = 0.0
        for be in range(3):
            Bl = [b_factor(tabs[l], l, be)[np.ix_(S[l], J[l])] for l in range(3)]
            g = np.einsum("ca,db,ef,abf->cde", Bl[2], Bl[1], Bl[0], vloc, optimize=True)
            for al in range(3):
                w = [w_factor(tabs[l], l, al, be)[ii[l], S[l]] for l in range(3)]
                s += np.einsum("c,d,e,cde,cde->", w[2], w[1], w[0], C[al][be], g, optimize=True)
        out[r] = s
    return out


# ---------------------------------------------------------------------------
# Section 3.1: the WQ mass operator (reaction term alpha u of Eq. (poisson))
# ---------------------------------------------------------------------------
def mass_wq(tabs, c) -> sp.csr_matrix:
    """Explicit M~ = W D B of Section 3.1: W = W3^(00) (x) W2^(00) (x) W1^(00)
    (reading R14), D = diag(c(x_q)), B = B3 (x) B2 (x) B1 (values).  c holds
    c = alpha det J at the quadrature points, direction 1 fastest."""
    Wk = kron3(*[tabs[l].W[(0, 0)] for l in (2, 1, 0)])
    Bk = kron3(*[tabs[l].B0 for l in (2, 1, 0)])
    return (Wk @ sp.diags(np.ravel(c)) @ Bk).tocsr()


def mass_wq_entries(tabs, c) -> np.ndarray:
    """Dense M~ entry by entry from Eq. (Mwq): M~_ij = sum_q w_{i,q} c(x_q)
    b_j(x_q), tensor weights w_{i,q} = prod_l w^(00)_{l,i_l,q_l}.  Tiny grids."""
    n = [t.n for t in tabs]
    nq = [t.nq for t in tabs]
    N = n[0] * n[1] * n[2]
    cg = np.reshape(c, (nq[2], nq[1], nq[0]))
    M = np.zeros((N, N))
    for i in range(N):
        i3, rem = divmod(i, n[0] * n[1])
        i2, i1 = divmod(rem, n[0])
        w = np.einsum("c,b,a->cba", tabs[2].W[(0, 0)][i3], tabs[1].W[(0, 0)][i2], tabs[0].W[(0, 0)][i1])
        for j in range(N):
            j3, rem = divmod(j, n[0] * n[1])
            j2, j1 = divmod(rem, n[0])
            b = np.einsum("c,b,a->cba", tabs[2].B0[:, j3], tabs[1].B0[:, j2], tabs[0].B0[:, j1])
            M[i, j] = np.sum(w * cg * b)
    return M


def apply_mass_alg1(tabs, c, V):
    """w = M~ v by the three steps of Algorithm 1: v~ = B v, then the pointwise
    product with c, then w = W v~~, each Kronecker product by Eq.
    (sum-factorization).  V, result [i3][i2][i1]; c [q3][q2][q1]."""
    vt = kron_action(tabs[2].B0, tabs[1].B0, tabs[0].B0, V)
    return kron_action(tabs[2].W[(0, 0)], tabs[1].W[(0, 0)], tabs[0].W[(0, 0)], c * vt)


def apply_mass_T(tabs, c, Y):
    """M~^T y = B^T D W^T y."""
    s = kron_action(tabs[2].W[(0, 0)].T, tabs[1].W[(0, 0)].T, tabs[0].W[(0, 0)].T, Y)
    return kron_action(tabs[2].B0.T, tabs[1].B0.T, tabs[0].B0.T, c * s)


def grad_mass_coeff(tabs, LAM, U):
    """dJ/dc(q) = -(W^T lambda)_q (B u)_q: M~ is linear in every c(x_q)."""
    S = kron_action(tabs[2].W[(0, 0)].T, tabs[1].W[(0, 0)].T, tabs[0].W[(0, 0)].T, LAM)
    return -S * kron_action(tabs[2].B0, tabs[1].B0, tabs[0].B0, U)


def mass_rows(tabs, c_box, V, rows):
    """Selected entries (M~ v)_i, each from Eq. (Mwq) on the points where the
    tensor weights of row i may be nonzero.  c_box(S3, S2, S1) returns c on
    that point box, shape (|S3|, |S2|, |S1|)."""
    out = np.empty(len(rows))
    for r, (i3, i2, i1) in enumerate(rows):
        ii = (i1, i2, i3)
        S = [np.nonzero(tabs[l].W[(0, 0)][ii[l]] != 0)[0] for l in range(3)]
        J = [np.nonzero(np.any(tabs[l].B0[S[l]] != 0, axis=0))[0] for l in range(3)]
        vloc = V[np.ix_(J[2], J[1], J[0])]
        B = [tabs[l].B0[np.ix_(S[l], J[l])] for l in range(3)]
        g = np.einsum("ca,db,ef,abf->cde", B[2], B[1], B[0], vloc, optimize=True)
        w = [tabs[l].W[(0, 0)][ii[l], S[l]] for l in range(3)]
        out[r] = np.einsum("c,d,e,cde,cde->", w[2], w[1], w[0], c_box(S[2], S[1], S[0]), g, optimize=True)
    return out


# ---------------------------------------------------------------------------
# Geometry and coefficient, Eq. (C) with reading R5
# ---------------------------------------------------------------------------
def ring_map(xi1, xi2, xi3):
    """Exact map of the thick quarter ring (Section 4): r = 1 + xi1 in [1, 2],
    theta = pi/2 xi2, z = xi3."""
    r = 1.0 + xi1
    th = 0.5 * np.pi * xi2
    return r * np.cos(th), r * np.sin(th), xi3


def ring_jacobian(xi1, xi2, xi3):
    """J[..., i, j] = dF_i / dxi_j of ring_map."""
    r = 1.0 + xi1
    th = 0.5 * np.pi * xi2
    J = np.zeros(np.shape(xi1) + (3, 3))
    J[..., 0, 0] = np.cos(th)
    J[..., 1, 0] = np.sin(th)
    J[..., 0, 1] = -r * 0.5 * np.pi * np.sin(th)
    J[..., 1, 1] = r * 0.5 * np.pi * np.cos(th)
    J[..., 2, 2] = 1.0
    return J


def kappa_field(x1, x2, x3, modes, scale):
    """K(x) = exp(scale * g(x)) I with g(x) = sum_m a_m cos(2 pi k_m . x + phi_m).
    modes is an array of rows (a, k1, k2, k3, phi); scale 0 gives K = I."""
    g = np.zeros(np.shape(x1))
    for a, k1, k2, k3, ph in np.atleast_2d(modes) if modes is not None and len(modes) else []:
        g = g + a * np.cos(2.0 * np.pi * (k1 * x1 + k2 * x2 + k3 * x3) + ph)
    return np.exp(scale * g)


def coefficient_points(geometry, xi1, xi2, xi3, modes=None, scale=0.0):
    """Six symmetric fields of C = |det J| J^-1 K J^-T (Eq. (C), reading R5)
    at the parametric points (xi1, xi2, xi3) (arrays of one shape)."""
    xi1, xi2, xi3 = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (xi1, xi2, xi3)))
    if geometry == "cube":
        J = np.zeros(xi1.shape + (3, 3))
        J[..., 0, 0] = J[..., 1, 1] = J[..., 2, 2] = 1.0
        x = (xi1, xi2, xi3)
    elif geometry == "ring":
        J = ring_jacobian(xi1, xi2, xi3)
        x = ring_map(xi1, xi2, xi3)
    else:
        raise ValueError(geometry)
    kap = kappa_field(*x, modes, scale)
    Jinv = np.linalg.inv(J)
    det = np.abs(np.linalg.det(J))
    C = det[..., None, None] * kap[..., None, None] * (Jinv @ np.swapaxes(Jinv, -1, -2))
    return np.stack([C[..., a, b] for (a, b) in SYM_PAIRS])


def coefficient_grid(tabs, geometry, modes=None, scale=0.0):
    """C6 on the full tensor grid of WQ points, shape (6, nq3, nq2, nq1)."""
    X3, X2, X1 = np.meshgrid(tabs[2].xq, tabs[1].xq, tabs[0].xq, indexing="ij")
    return coefficient_points(geometry, X1, X2, X3, modes, scale)


def coefficient_box_fn(tabs, geometry, modes=None, scale=0.0):
    def box(S3, S2, S1):
        X3, X2, X1 = np.meshgrid(tabs[2].xq[S3], tabs[1].xq[S2], tabs[0].xq[S1], indexing="ij")
        return coefficient_points(geometry, X1, X2, X3, modes, scale)
    return box


def mass_coefficient_points(geometry, xi1, xi2, xi3, alpha):
    """c = alpha |det J| (Eq. (M)) at parametric points, alpha a constant."""
    xi1, xi2, xi3 = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (xi1, xi2, xi3)))
    if geometry == "cube":
        return np.full(xi1.shape, float(alpha))
    if geometry == "ring":
        return alpha * np.abs(np.linalg.det(ring_jacobian(xi1, xi2, xi3)))
    raise ValueError(geometry)


def mass_coefficient_grid(tabs, geometry, alpha):
    """c on the full grid of WQ points, shape (nq3, nq2, nq1)."""
    X3, X2, X1 = np.meshgrid(tabs[2].xq, tabs[1].xq, tabs[0].xq, indexing="ij")
    return mass_coefficient_points(geometry, X1, X2, X3, alpha)


def mass_coefficient_box_fn(tabs, geometry, alpha):
    def box(S3, S2, S1):
        X3, X2, X1 = np.meshgrid(tabs[2].xq[S3], tabs[1].xq[S2], tabs[0].xq[S1], indexing="ij")
        return mass_coefficient_points(geometry, X1, X2, X3, alpha)
    return box


# ---------------------------------------------------------------------------
# Load vector (reading R8) and the manufactured solutions of Section 4
# ---------------------------------------------------------------------------
def forcing_sines(x1, x2, x3):
    """3 pi^2 sin(pi x) sin(pi y) sin(pi z): -Laplace of sin sin sin."""
    return 3.0 * np.pi ** 2 * np.sin(np.pi * x1) * np.sin(np.pi * x2) * np.sin(np.pi * x3)


def exact_solution_ring(x1, x2, x3):
    """Eq. (exact-solution)."""
    rho = x1 ** 2 + x2 ** 2
    return np.sin(5 * np.pi * x1) * np.sin(5 * np.pi * x2) * np.sin(5 * np.pi * x3) * (rho - 1) * (rho - 4)


def exact_gradient_ring(x1, x2, x3):
    k = 5 * np.pi
    s1, s2, s3 = np.sin(k * x1), np.sin(k * x2), np.sin(k * x3)
    c1, c2, c3 = np.cos(k * x1), np.cos(k * x2), np.cos(k * x3)
    rho = x1 ** 2 + x2 ** 2
    q = (rho - 1) * (rho - 4)
    dq = 2 * rho - 5  # dq/drho
    S = s1 * s2 * s3
    g1 = k * c1 * s2 * s3 * q + S * dq * 2 * x1
    g2 = k * s1 * c2 * s3 * q + S * dq * 2 * x2
    g3 = k * s1 * s2 * c3 * q
    return g1, g2, g3


def exact_forcing_ring(x1, x2, x3):
    """f = -Laplace u for Eq. (exact-solution) (K = I, alpha = 0)."""
    k = 5 * np.pi
    s1, s2, s3 = np.sin(k * x1), np.sin(k * x2), np.sin(k * x3)
    c1, c2 = np.cos(k * x1), np.cos(k * x2)
    rho = x1 ** 2 + x2 ** 2
    q = (rho - 1) * (rho - 4)
    S = s1 * s2 * s3
    lapS = -3 * k ** 2 * S
    gradS_dot_gradq = (2 * rho - 5) * 2 * (x1 * k * c1 * s2 * s3 + x2 * k * s1 * c2 * s3)
    lapq = 2 * 4 * rho + (2 * rho - 5) * 4
    return -(q * lapS + 2 * gradS_dot_gradq + S * lapq)


def exact_forcing_ring_reaction(alpha):
    """f = -Laplace u + alpha u for Eq. (exact-solution) (K = I, constant alpha)."""
    def f(x1, x2, x3):
        return exact_forcing_ring(x1, x2, x3) + alpha * exact_solution_ring(x1, x2, x3)
    return f


def _gauss_tables(tabs, k):
    """Gauss points, weights and interior basis values/derivatives per
    direction; k is a number of points per span or a list of one per direction."""
    ks = list(k) if np.ndim(k) else [k] * len(tabs)
    out = []
    for t, kl in zip(tabs, ks):
        xg, wg = gauss_rule(t.knots, kl)
        val, der = bspline_basis(t.knots, t.p, xg)
        m = val.shape[1]
        out.append((xg, wg, val[:, 1:m - 1], der[:, 1:m - 1]))
    return out


def _geom_at(geometry, X1, X2, X3):
    if geometry == "cube":
        return (X1, X2, X3), np.ones_like(X1), None
    J = ring_jacobian(X1, X2, X3)
    return ring_map(X1, X2, X3), np.abs(np.linalg.det(J)), J


def load_vector(tabs, geometry, forcing):
    """f_i = int |det J| b_i (f o F) dxi (Eq. (linearsystem) with reading R8),
    tensor Gauss with p_l+1 points per span in direction l; result [i3][i2][i1]."""
    gt = _gauss_tables(tabs, [t.p + 1 for t in tabs])
    X3, X2, X1 = np.meshgrid(gt[2][0], gt[1][0], gt[0][0], indexing="ij")
    x, det, _ = _geom_at(geometry, X1, X2, X3)
    wgt = np.einsum("c,b,a->cba", gt[2][1], gt[1][1], gt[0][1])
    integrand = wgt * det * forcing(*x)
    return kron_action(gt[2][2].T, gt[1][2].T, gt[0][2].T, integrand)


def load_vector_rows(tabs, geometry, forcing, rows):
    """Selected entries of load_vector, each from its own Gauss sum over the
    support of b_i."""
    gt = _gauss_tables(tabs, [t.p + 1 for t in tabs])
    out = np.empty(len(rows))
    for r, (i3, i2, i1) in enumerate(rows):
        ii = (i1, i2, i3)
        sel = [np.nonzero(gt[l][2][:, ii[l]] != 0)[0] for l in range(3)]
        X3, X2, X1 = np.meshgrid(gt[2][0][sel[2]], gt[1][0][sel[1]], gt[0][0][sel[0]], indexing="ij")
        x, det, _ = _geom_at(geometry, X1, X2, X3)
        b = [gt[l][2][sel[l], ii[l]] * gt[l][1][sel[l]] for l in range(3)]
        out[r] = np.einsum("c,d,e,cde->", b[2], b[1], b[0], det * forcing(*x))
    return out


def h1_error(tabs, U, geometry, exact_u, exact_grad):
    """Relative H1 error ||u - u_h||_H1 / ||u||_H1 (Section 4), tensor Gauss
    with p_l+2 points per span in direction l, gradients pulled back with J^-T."""
    gt = _gauss_tables(tabs, [t.p + 2 for t in tabs])
    X3, X2, X1 = np.meshgrid(gt[2][0], gt[1][0], gt[0][0], indexing="ij")
    x, det, J = _geom_at(geometry, X1, X2, X3)
    wgt = np.einsum("c,b,a->cba", gt[2][1], gt[1][1], gt[0][1]) * det
    uh = kron_action(gt[2][2], gt[1][2], gt[0][2], U)
    d1 = kron_action(gt[2][2], gt[1][2], gt[0][3], U)
    d2 = kron_action(gt[2][2], gt[1][3], gt[0][2], U)
    d3 = kron_action(gt[2][3], gt[1][2], gt[0][2], U)
    gref = np.stack([d1, d2, d3], axis=-1)
    if J is None:
        gphys = gref
    else:
        gphys = np.einsum("...ji,...j->...i", np.linalg.inv(J), gref)
    ue = exact_u(*x)
    ge = np.stack(exact_grad(*x), axis=-1)
    err = np.sum(wgt * ((ue - uh) ** 2 + np.sum((ge - gphys) ** 2, axis=-1)))
    nrm = np.sum(wgt * (ue ** 2 + np.sum(ge ** 2, axis=-1)))
    return math.sqrt(err / nrm)


# ---------------------------------------------------------------------------
# FD preconditioner (Section 4, reading R6)
# ---------------------------------------------------------------------------
@dataclass
class FD:
    lam: list
    U: list
    K: list
    M: list
    shift: float = 0.0


def fd_setup(tabs, shift: float = 0.0) -> FD:
    """FD factors (reading R6); shift sigma adds sigma M3(x)M2(x)M1 to P (reading R15)."""
    lam, U, K, M = [], [], [], []
    for t in tabs:
        Kl = galerkin_1d(t.knots, t.p, 1, 1)
        Ml = galerkin_1d(t.knots, t.p, 0, 0)
        ev, V = scipy.linalg.eigh(Kl, Ml)
        lam.append(ev)
        U.append(V)
        K.append(Kl)
        M.append(Ml)
    return FD(lam, U, K, M, float(shift))


def fd_diag(fd):
    """lambda1_i + lambda2_j + lambda3_k (+ sigma) as a tensor [k][j][i]."""
    return fd.lam[2][:, None, None] + fd.lam[1][None, :, None] + fd.lam[0][None, None, :] + fd.shift


def fd_apply(fd, R):
    """z = P^-1 r = (U3(x)U2(x)U1) diag(1/(l1+l2+l3)) (U3(x)U2(x)U1)^T r, the
    Kronecker actions by Eq. (sum-factorization).  R, z tensors [k][j][i]."""
    S = kron_action(fd.U[2].T, fd.U[1].T, fd.U[0].T, R) / fd_diag(fd)
    return kron_action(fd.U[2], fd.U[1], fd.U[0], S)


def fd_apply_explicit(fd, r):
    """Same as fd_apply with the Kronecker matrices formed densely (small N)."""
    Uk = np.kron(fd.U[2], np.kron(fd.U[1], fd.U[0]))
    return Uk @ ((Uk.T @ r) / fd_diag(fd).ravel())


def fd_matrix(fd) -> sp.csr_matrix:
    """P = M3(x)M2(x)K1 + M3(x)K2(x)M1 + K3(x)M2(x)M1 (+ sigma M3(x)M2(x)M1)."""
    K, M = fd.K, fd.M
    P = kron3(M[2], M[1], K[0]) + kron3(M[2], K[1], M[0]) + kron3(K[2], M[1], M[0])
    if fd.shift:
        P = P + fd.shift * kron3(M[2], M[1], M[0])
    return P.tocsr()


# ---------------------------------------------------------------------------
# BiCGStab with right preconditioning (Section 4, reading R7)
# ---------------------------------------------------------------------------
@dataclass
class SolveInfo:
    converged: bool
    iterations: int
    rel_residual: float
    history: list


def bicgstab(apply_A, apply_Pinv, f, rtol, maxit, x0=None):
    """Solve A x = f; vectors are flat float64 arrays; apply_A and apply_Pinv
    map flat arrays to flat arrays."""
    f = np.asarray(f, dtype=np.float64)
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64)
    fn = np.linalg.norm(f)
    if fn == 0.0:
        return np.zeros_like(f), SolveInfo(True, 0, 0.0, [])
    r = f - apply_A(x) if x0 is not None else f.copy()
    hist = [np.linalg.norm(r) / fn]
    if hist[-1] <= rtol:
        return x, SolveInfo(True, 0, hist[-1], hist)
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    p = np.zeros_like(f)
    v = np.zeros_like(f)
    for k in range(1, maxit + 1):
        rho = rhat @ r
        if rho == 0.0:
            break
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = apply_Pinv(p)
        v = apply_A(ph)
        alpha = rho / (rhat @ v)
        s = r - alpha * v
        sn = np.linalg.norm(s) / fn
        if sn <= rtol:
            x = x + alpha * ph
            hist.append(sn)
            return x, SolveInfo(True, k, sn, hist)
        sh = apply_Pinv(s)
        t = apply_A(sh)
        omega = (t @ s) / (t @ t)
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        rn = np.linalg.norm(r) / fn
        hist.append(rn)
        if rn <= rtol:
            return x, SolveInfo(True, k, rn, hist)
        if omega == 0.0:
            break
        rho_old = rho
    return x, SolveInfo(False, k, hist[-1], hist)


# ---------------------------------------------------------------------------
# Convenience: one patch
# ---------------------------------------------------------------------------
@dataclass
class Patch:
    tabs: list
    C6: np.ndarray          # (6, nq3, nq2, nq1)
    fd: FD
    cmass: np.ndarray = None  # c = alpha det J at the WQ points (nq3, nq2, nq1), or None

    @property
    def n(self):
        return [t.n for t in self.tabs]

    @property
    def shape(self):
        return (self.tabs[2].n, self.tabs[1].n, self.tabs[0].n)

    @property
    def Cfull(self):
        return full_coeff(self.C6)

    def apply(self, V):
        out = apply_alg2(self.tabs, self.Cfull, V)
        if self.cmass is not None:
            out = out + apply_mass_alg1(self.tabs, self.cmass, V)
        return out

    def apply_T(self, Y):
        out = apply_T_alg2(self.tabs, self.Cfull, Y)
        if self.cmass is not None:
            out = out + apply_mass_T(self.tabs, self.cmass, Y)
        return out

    def precond(self, R):
        return fd_apply(self.fd, R)

    def solve(self, F, rtol, maxit=500, transpose=False, x0=None):
        sh = self.shape
        A = (lambda v: self.apply_T(v.reshape(sh)).ravel()) if transpose else (lambda v: self.apply(v.reshape(sh)).ravel())
        P = lambda v: self.precond(v.reshape(sh)).ravel()
        x, info = bicgstab(A, P, np.ravel(F), rtol, maxit, None if x0 is None else np.ravel(x0))
        return x.reshape(sh), info


def make_patch(p, nel, geometry="cube", modes=None, scale=0.0) -> Patch:
    tabs = uniform_tables(p, nel)
    return Patch(tabs, coefficient_grid(tabs, geometry, modes, scale), fd_setup(tabs))
