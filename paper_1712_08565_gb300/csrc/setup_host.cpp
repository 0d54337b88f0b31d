// Host-side setup of the MF-WQ 1D tables (Algorithm 2's "Setup" line, Section
// 3.2; weights of Section 2.2; FD factors of the preconditioner of Section 4).
// Runs once per handle, O(n p^2) work per direction; not on the hot path.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <thread>

#include "mfwq_internal.h"

namespace mfwq {
namespace {

// ---------------------------------------------------------------- B-splines
// Span index k with t[k] <= x < t[k+1] among the non-empty spans p..m-1;
// the point 1 belongs to the last span.
int find_span(const std::vector<double>& t, int p, int m, double x) {
    if (x >= t[m]) return m - 1;
    int lo = p, hi = m;  // t[lo] <= x < t[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (x < t[mid]) hi = mid; else lo = mid;
    }
    return lo;
}

// Values N[j] = b_{k-p+j}(x) and derivatives D[j], j = 0..p, of the B-splines
// that may be nonzero on span k.  Degree-by-degree recurrence
// b_{i,d} = w_{i,d} b_{i,d-1} + (1 - w_{i+1,d}) b_{i+1,d-1},
// w_{i,d}(x) = (x - t_i)/(t_{i+d} - t_i), and the derivative formula
// b'_{i,p} = p b_{i,p-1}/(t_{i+p}-t_i) - p b_{i+1,p-1}/(t_{i+p+1}-t_{i+1}).
void local_basis(const std::vector<double>& t, int p, int k, double x, double* N, double* D) {
    double prev[kMaxDegree + 2], cur[kMaxDegree + 2];
    prev[0] = 1.0;
    double lowdeg[kMaxDegree + 2];  // degree p-1 values
    if (p == 0) lowdeg[0] = 1.0;
    for (int d = 1; d <= p; ++d) {
        for (int j = 0; j <= d; ++j) {
            int i = k - d + j;
            double v = 0.0;
            if (j >= 1) {  // b_{i,d-1} = prev[j-1]
                double den = t[i + d] - t[i];
                if (den > 0.0) v += (x - t[i]) / den * prev[j - 1];
            }
            if (j <= d - 1) {  // b_{i+1,d-1} = prev[j]
                double den = t[i + d + 1] - t[i + 1];
                if (den > 0.0) v += (t[i + d + 1] - x) / den * prev[j];
            }
            cur[j] = v;
        }
        if (d == p) {
            for (int j = 0; j < p; ++j) lowdeg[j] = prev[j];
        }
        for (int j = 0; j <= d; ++j) prev[j] = cur[j];
    }
    for (int j = 0; j <= p; ++j) N[j] = prev[j];
    for (int j = 0; j <= p; ++j) {
        int i = k - p + j;
        double v = 0.0;
        if (p >= 1) {
            if (j >= 1) {
                double den = t[i + p] - t[i];
                if (den > 0.0) v += p * lowdeg[j - 1] / den;
            }
            if (j <= p - 1) {
                double den = t[i + p + 1] - t[i + 1];
                if (den > 0.0) v -= p * lowdeg[j] / den;
            }
        }
        D[j] = v;
    }
}

// Value (deriv = 0) or derivative (deriv = 1) of the global B-spline g at x.
struct PointBasis {
    int span;
    double N[kMaxDegree + 1], D[kMaxDegree + 1];
};

PointBasis eval_point(const std::vector<double>& t, int p, int m, double x) {
    PointBasis pb;
    pb.span = find_span(t, p, m, x);
    local_basis(t, p, pb.span, x, pb.N, pb.D);
    return pb;
}

double basis_at(const PointBasis& pb, int p, int g, int deriv) {
    int j = g - (pb.span - p);
    if (j < 0 || j > p) return 0.0;
    return deriv ? pb.D[j] : pb.N[j];
}

// ---------------------------------------------------------------- double-double
// Unevaluated sums hi + lo of two doubles (about 106 significant bits), built
// on the error-free transformations of Dekker (split product) and Knuth
// (two-sum), as in Hida, Li & Bailey's double-double arithmetic.  The WQ
// weight systems are ill-conditioned for larger p (condition numbers near 1e9
// at p = 6), so they are assembled and solved in this arithmetic and rounded
// to double once.  This file is compiled without floating-point contraction.
struct dd {
    double hi, lo;
};
inline dd dd_from(double a) { return {a, 0.0}; }
inline dd two_sum(double a, double b) {
    double s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
inline dd quick_two_sum(double a, double b) {
    double s = a + b;
    return {s, b - (s - a)};
}
inline void split(double a, double& h, double& l) {
    double c = 134217729.0 * a;  // 2^27 + 1
    h = c - (c - a);
    l = a - h;
}
inline dd two_prod(double a, double b) {
    double p = a * b, ah, al, bh, bl;
    split(a, ah, al);
    split(b, bh, bl);
    return {p, ((ah * bh - p) + ah * bl + al * bh) + al * bl};
}
inline dd operator+(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
inline dd operator-(dd a) { return {-a.hi, -a.lo}; }
inline dd operator-(dd a, dd b) { return a + (-b); }
inline dd operator*(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}
inline dd operator*(dd a, double b) {
    dd p = two_prod(a.hi, b);
    p.lo += a.lo * b;
    return quick_two_sum(p.hi, p.lo);
}
inline dd operator/(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = a - b * q1;
    double q2 = r.hi / b.hi;
    r = r - b * q2;
    double q3 = r.hi / b.hi;
    return quick_two_sum(q1, q2) + dd_from(q3);
}
inline bool operator<(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
inline dd dd_sqrt(dd a) {
    if (a.hi <= 0) return dd_from(0.0);
    double x = 1.0 / std::sqrt(a.hi);
    double ax = a.hi * x;
    return two_sum(ax, (a - two_prod(ax, ax)).hi * (x * 0.5));
}
inline double to_d(dd a) { return a.hi + a.lo; }

// Local B-spline values/derivatives on span k in double-double (the
// recurrence of local_basis).
void local_basis_dd(const std::vector<double>& t, int p, int k, dd x, dd* N, dd* D) {
    dd prev[kMaxDegree + 2], cur[kMaxDegree + 2], low[kMaxDegree + 2];
    prev[0] = dd_from(1.0);
    for (int d = 1; d <= p; ++d) {
        for (int j = 0; j <= d; ++j) {
            int i = k - d + j;
            dd v = dd_from(0.0);
            if (j >= 1 && t[i + d] > t[i])
                v = v + (x - dd_from(t[i])) * prev[j - 1] / (dd_from(t[i + d]) - dd_from(t[i]));
            if (j <= d - 1 && t[i + d + 1] > t[i + 1])
                v = v + (dd_from(t[i + d + 1]) - x) * prev[j] / (dd_from(t[i + d + 1]) - dd_from(t[i + 1]));
            cur[j] = v;
        }
        if (d == p)
            for (int j = 0; j < p; ++j) low[j] = prev[j];
        for (int j = 0; j <= d; ++j) prev[j] = cur[j];
    }
    for (int j = 0; j <= p; ++j) N[j] = prev[j];
    for (int j = 0; j <= p; ++j) {
        int i = k - p + j;
        dd v = dd_from(0.0);
        if (j >= 1 && t[i + p] > t[i]) v = v + low[j - 1] * (double)p / (dd_from(t[i + p]) - dd_from(t[i]));
        if (j <= p - 1 && t[i + p + 1] > t[i + 1]) v = v - low[j] * (double)p / (dd_from(t[i + p + 1]) - dd_from(t[i + 1]));
        D[j] = v;
    }
}

struct PointBasisDD {
    int span;
    dd N[kMaxDegree + 1], D[kMaxDegree + 1];
};

dd basis_at_dd(const PointBasisDD& pb, int p, int g, int deriv) {
    int j = g - (pb.span - p);
    if (j < 0 || j > p) return dd_from(0.0);
    return deriv ? pb.D[j] : pb.N[j];
}

// Gauss-Legendre nodes and weights on [-1, 1] in double-double: Newton's
// method on P_k started from the double nodes x0.
void gauss_legendre_dd(int k, const std::vector<double>& x0, std::vector<dd>& x, std::vector<dd>& w) {
    x.resize(k);
    w.resize(k);
    for (int i = 0; i < k; ++i) {
        dd z = dd_from(x0[i]), dp = dd_from(1.0);
        for (int it = 0; it < 4; ++it) {
            dd p0 = dd_from(1.0), p1 = z;
            for (int j = 2; j <= k; ++j) {
                dd p2 = (z * p1 * (2.0 * j - 1.0) - p0 * (j - 1.0)) / dd_from((double)j);
                p0 = p1;
                p1 = p2;
            }
            dp = (z * p1 - p0) * (double)k / (z * z - dd_from(1.0));
            if (it < 3) z = z - p1 / dp;
        }
        x[i] = z;
        w[i] = dd_from(2.0) / ((dd_from(1.0) - z * z) * dp * dp);
    }
}
// ---------------------------------------------------------------- Gauss-Legendre
// Nodes and weights on [-1,1] by Newton's method on P_k (three-term recurrence).
void gauss_legendre(int k, std::vector<double>& x, std::vector<double>& w) {
    x.assign(k, 0.0);
    w.assign(k, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (k + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (k + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= k; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (k == 1) { p1 = z; p0 = 1.0; }
            dp = k * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // recompute derivative at the converged node
        double p0 = 1.0, p1 = z;
        for (int j = 2; j <= k; ++j) {
            double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        if (k == 1) { p1 = z; p0 = 1.0; }
        dp = k * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        x[k - 1 - i] = z;
        w[i] = w[k - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// ---------------------------------------------------------------- small dense linear algebra
// Minimum-2-norm solution of the consistent system A w = g (A: rows x cols,
// row-major, double-double) by Householder QR with column pivoting of A^T
// (cols x rows): A^T P = Q R; an equation whose pivot falls below 1e-26 of
// the first is a combination of the kept ones and is dropped (the system is
// consistent, so the solution set is unchanged); then w = Q_k R_k^-T (P^T g)_k.
// Returns false if no equation could be kept.
bool min_norm_solve_dd(std::vector<dd> M, int rows, int cols, const std::vector<dd>& g, std::vector<double>& w) {
    // M holds A^T column-major: column c (an equation) is row c of A, length cols.
    std::vector<int> perm(rows);
    for (int i = 0; i < rows; ++i) perm[i] = i;
    std::vector<std::vector<dd>> V;
    std::vector<dd> beta;
    int rank = 0;
    double first = 0.0;
    for (int k = 0; k < std::min(rows, cols); ++k) {
        int best = -1;
        dd bestn = dd_from(-1.0);
        for (int c = k; c < rows; ++c) {
            dd s = dd_from(0.0);
            for (int e = k; e < cols; ++e) s = s + M[(size_t)c * cols + e] * M[(size_t)c * cols + e];
            if (bestn < s) { bestn = s; best = c; }
        }
        double nrm = std::sqrt(std::max(bestn.hi, 0.0));
        if (k == 0) first = nrm;
        if (!(nrm > 1e-26 * first)) break;
        if (best != k) {
            for (int e = 0; e < cols; ++e) std::swap(M[(size_t)best * cols + e], M[(size_t)k * cols + e]);
            std::swap(perm[best], perm[k]);
        }
        dd* x = &M[(size_t)k * cols];
        dd alpha = dd_sqrt(bestn);
        if (x[k].hi > 0.0) alpha = -alpha;
        std::vector<dd> v(cols, dd_from(0.0));
        for (int e = k; e < cols; ++e) v[e] = x[e];
        v[k] = v[k] - alpha;
        dd vtv = dd_from(0.0);
        for (int e = k; e < cols; ++e) vtv = vtv + v[e] * v[e];
        dd b = vtv.hi > 0 ? dd_from(2.0) / vtv : dd_from(0.0);
        for (int c = k; c < rows; ++c) {
            dd* y = &M[(size_t)c * cols];
            dd s = dd_from(0.0);
            for (int e = k; e < cols; ++e) s = s + v[e] * y[e];
            s = s * b;
            for (int e = k; e < cols; ++e) y[e] = y[e] - s * v[e];
        }
        V.push_back(v);
        beta.push_back(b);
        ++rank;
    }
    if (rank == 0) return false;
    // R_k^T y = (P^T g)_k, R(i, j) = M[j*cols + i] for i <= j.
    std::vector<dd> y(cols, dd_from(0.0));
    for (int i = 0; i < rank; ++i) {
        dd s = g[perm[i]];
        for (int j = 0; j < i; ++j) s = s - M[(size_t)i * cols + j] * y[j];
        y[i] = s / M[(size_t)i * cols + i];
    }
    // w = H_0 H_1 ... H_{rank-1} [y; 0]
    for (int k = rank - 1; k >= 0; --k) {
        dd s = dd_from(0.0);
        for (int e = k; e < cols; ++e) s = s + V[k][e] * y[e];
        s = s * beta[k];
        for (int e = k; e < cols; ++e) y[e] = y[e] - s * V[k][e];
    }
    w.assign(cols, 0.0);
    for (int e = 0; e < cols; ++e) w[e] = to_d(y[e]);
    return true;
}

// Cholesky M = L L^T (row-major, lower).  Returns false if not SPD.
bool cholesky(std::vector<double>& L, const std::vector<double>& M, int n) {
    L.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double s = M[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(s > 0.0)) return false;
        double d = std::sqrt(s);
        L[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = M[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = v / d;
        }
    }
    return true;
}

// Cyclic Jacobi eigensolver for a symmetric matrix A (row-major, overwritten):
// A = V diag(ev) V^T, V row-major with eigenvectors in columns.
bool jacobi_eig(std::vector<double>& A, int n, std::vector<double>& ev, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
    double fro = 0;
    for (size_t i = 0; i < A.size(); ++i) fro += A[i] * A[i];
    fro = std::sqrt(fro);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += a(i, j) * a(i, j);
        if (std::sqrt(off) <= 1e-17 * fro) {
            ev.resize(n);
            for (int i = 0; i < n; ++i) ev[i] = a(i, i);
            return true;
        }
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = a(p, q);
                if (std::fabs(apq) <= 1e-300) continue;
                double app = a(p, p), aqq = a(q, q);
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(1.0 + theta * theta));
                double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    double akp = a(k, p), akq = a(k, q);
                    a(k, p) = c * akp - s * akq;
                    a(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    double apk = a(p, k), aqk = a(q, k);
                    a(p, k) = c * apk - s * aqk;
                    a(q, k) = s * apk + c * aqk;
                }
                a(p, q) = a(q, p) = 0.0;
                for (int k = 0; k < n; ++k) {
                    double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    return false;
}

// Generalized symmetric eigenproblem K U = M U diag(lam) with U^T M U = I:
// M = L L^T, L^-1 K L^-T = V diag(lam) V^T (cyclic Jacobi), U = L^-T V.
bool gen_eig(const std::vector<double>& K, const std::vector<double>& M, int n, std::vector<double>& lam,
             std::vector<double>& U, std::string& why) {
    std::vector<double> L;
    if (!cholesky(L, M, n)) { why = "1D mass matrix is not SPD"; return false; }
    std::vector<double> X((size_t)n * n), A((size_t)n * n);
    for (int c = 0; c < n; ++c)  // X = L^-1 K
        for (int i = 0; i < n; ++i) {
            double s = K[(size_t)i * n + c];
            for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * X[(size_t)k * n + c];
            X[(size_t)i * n + c] = s / L[(size_t)i * n + i];
        }
    for (int r = 0; r < n; ++r)  // A = X L^-T
        for (int i = 0; i < n; ++i) {
            double s = X[(size_t)r * n + i];
            for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * A[(size_t)r * n + k];
            A[(size_t)r * n + i] = s / L[(size_t)i * n + i];
        }
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double s = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
            A[(size_t)i * n + j] = A[(size_t)j * n + i] = s;
        }
    std::vector<double> V;
    if (!jacobi_eig(A, n, lam, V)) { why = "Jacobi eigensolver did not converge"; return false; }
    U.assign((size_t)n * n, 0.0);
    for (int c = 0; c < n; ++c)  // U = L^-T V
        for (int i = n - 1; i >= 0; --i) {
            double s = V[(size_t)i * n + c];
            for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * U[(size_t)k * n + c];
            U[(size_t)i * n + c] = s / L[(size_t)i * n + i];
        }
    for (int i = 0; i < n; ++i)
        if (!(lam[i] > 0.0)) { why = "FD eigenvalue not positive"; return false; }
    return true;
}

}  // namespace

int validate_knots(int p, int nknots, const double* t, std::string& why) {
    if (p < 2 || p > kMaxDegree) { why = "degree must be in [2, 12]"; return MFWQ_EINVAL; }
    if (!t) { why = "knots pointer is NULL"; return MFWQ_EINVAL; }
    int m = nknots - p - 1;
    int nel = m - p;
    if (nel < 2) { why = "need at least 2 elements per direction"; return MFWQ_EINVAL; }
    for (int i = 0; i <= p; ++i)
        if (t[i] != 0.0 || t[nknots - 1 - i] != 1.0) { why = "knot vector must be open on [0,1]"; return MFWQ_EINVAL; }
    for (int i = p; i < m; ++i)
        if (!(t[i] < t[i + 1])) { why = "interior knots must be strictly increasing (multiplicity 1)"; return MFWQ_EINVAL; }
    return MFWQ_OK;
}

// Builds every 1D table of one direction.
int build_dir(int p, int nknots, const double* knots, Dir1D& d, std::string& why) {
    int st = validate_knots(p, nknots, knots, why);
    if (st != MFWQ_OK) return st;
    d.p = p;
    d.t.assign(knots, knots + nknots);
    d.m = nknots - p - 1;
    d.nel = d.m - p;
    d.n = d.m - 2;
    const std::vector<double>& t = d.t;
    const int m = d.m, n = d.n, nel = d.nel;
    std::vector<double> u(nel + 1);
    for (int s = 0; s <= nel; ++s) u[s] = t[p + s];

    // WQ points: interior knots, interior-span midpoints, p+1 equispaced points
    // inside the first and the last span (n_q = 2 nel + 2p - 1).
    d.xq.clear();
    for (int k = 1; k <= p + 1; ++k) d.xq.push_back(u[0] + (u[1] - u[0]) * k / (p + 2.0));
    for (int s = 1; s < nel - 1; ++s) {
        d.xq.push_back(u[s]);
        d.xq.push_back(0.5 * (u[s] + u[s + 1]));
    }
    d.xq.push_back(u[nel - 1]);
    for (int k = 1; k <= p + 1; ++k) d.xq.push_back(u[nel - 1] + (u[nel] - u[nel - 1]) * k / (p + 2.0));
    const int nq = d.nq = (int)d.xq.size();

    std::vector<PointBasis> pb(nq);
    for (int q = 0; q < nq; ++q) pb[q] = eval_point(t, p, m, d.xq[q]);

    // Gauss rule with p+1 points per span, and the exact 1D Galerkin integrals
    // G^{ab}[i][j] = int b_i^(a) b_j^(b) (interior i, j; zero for |i-j| > p).
    std::vector<double> gx, gw;
    gauss_legendre(p + 1, gx, gw);
    d.xg.clear();
    d.wg.clear();
    for (int s = 0; s < nel; ++s) {
        double a = u[s], b = u[s + 1];
        for (int k = 0; k <= p; ++k) {
            d.xg.push_back(0.5 * (a + b) + 0.5 * (b - a) * gx[k]);
            d.wg.push_back(0.5 * (b - a) * gw[k]);
        }
    }
    const int ng = d.ng = (int)d.xg.size();
    std::vector<PointBasis> gb(ng);
    for (int g = 0; g < ng; ++g) gb[g] = eval_point(t, p, m, d.xg[g]);
    std::vector<double> Gal[4];  // dense [n][n], family 2a+b
    for (int f = 0; f < 4; ++f) Gal[f].assign((size_t)n * n, 0.0);
    for (int g = 0; g < ng; ++g) {
        int k = gb[g].span;
        for (int ja = 0; ja <= p; ++ja) {
            int gi = k - p + ja;
            if (gi < 1 || gi > m - 2) continue;
            for (int jb = 0; jb <= p; ++jb) {
                int gj = k - p + jb;
                if (gj < 1 || gj > m - 2) continue;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) {
                        double va = a ? gb[g].D[ja] : gb[g].N[ja];
                        double vb = b ? gb[g].D[jb] : gb[g].N[jb];
                        Gal[2 * a + b][(size_t)(gi - 1) * n + (gj - 1)] += d.wg[g] * va * vb;
                    }
            }
        }
    }

    // Trial band B: rows q, interior columns j whose value or derivative is
    // nonzero at x_q (exact zeros at the band ends are trimmed).
    {
        Band1D& B = d.B;
        B.rows = nq; B.cols = n; B.fams = 2; B.width = 0;
        B.start.assign(nq, 0); B.len.assign(nq, 0);
        for (int q = 0; q < nq; ++q) {
            int lo = n, hi = -1;
            for (int j = 0; j <= p; ++j) {
                int g = pb[q].span - p + j;
                if (g < 1 || g > m - 2) continue;
                if (pb[q].N[j] != 0.0 || pb[q].D[j] != 0.0) { lo = std::min(lo, g - 1); hi = std::max(hi, g - 1); }
            }
            if (hi < lo) { lo = 0; hi = -1; }
            B.start[q] = lo;
            B.len[q] = hi - lo + 1;
            B.width = std::max(B.width, B.len[q]);
        }
        B.val.assign((size_t)2 * nq * B.width, 0.0);
        for (int q = 0; q < nq; ++q)
            for (int tt = 0; tt < B.len[q]; ++tt) {
                int g = B.start[q] + tt + 1;
                B.at(0, q, tt) = basis_at(pb[q], p, g, 0);
                B.at(1, q, tt) = basis_at(pb[q], p, g, 1);
            }
    }

    // Weights: for each interior row i solve, in the minimum-norm sense,
    // sum_{q in S_i} w_iq b_j^(b)(x_q) = G^{ab}[i][j] for interior |j-i| <= p,
    // S_i = points in the open support (t_{i}, t_{i+p+1}) of b_i (global index
    // gi = i+1).  Eq. (exactness1d), Eq. (exactness_K), Eq. (weights-support).
    {
        Band1D& W = d.W;
        W.rows = n; W.cols = nq; W.fams = 4; W.width = 0;
        W.start.assign(n, 0); W.len.assign(n, 0);
        for (int i = 0; i < n; ++i) {
            int gi = i + 1;
            int lo = nq, hi = -1;
            for (int q = 0; q < nq; ++q)
                if (d.xq[q] > t[gi] && d.xq[q] < t[gi + p + 1]) { lo = std::min(lo, q); hi = std::max(hi, q); }
            if (hi < lo) { why = "empty weight support"; return MFWQ_ESETUP; }
            W.start[i] = lo;
            W.len[i] = hi - lo + 1;
            W.width = std::max(W.width, W.len[i]);
        }
        W.val.assign((size_t)4 * n * W.width, 0.0);
        // Points (the rule of d.xq), basis values at them, and the Gauss rule
        // of the exact integrals G^{ab}[i][j], all in double-double.
        std::vector<dd> xqd;
        for (int k = 1; k <= p + 1; ++k)
            xqd.push_back(dd_from(u[0]) + (dd_from(u[1]) - dd_from(u[0])) * (double)k / dd_from(p + 2.0));
        for (int s = 1; s < nel - 1; ++s) {
            xqd.push_back(dd_from(u[s]));
            xqd.push_back((dd_from(u[s]) + dd_from(u[s + 1])) * 0.5);
        }
        xqd.push_back(dd_from(u[nel - 1]));
        for (int k = 1; k <= p + 1; ++k)
            xqd.push_back(dd_from(u[nel - 1]) + (dd_from(u[nel]) - dd_from(u[nel - 1])) * (double)k / dd_from(p + 2.0));
        std::vector<PointBasisDD> pbd(nq);
        for (int q = 0; q < nq; ++q) {
            pbd[q].span = pb[q].span;
            local_basis_dd(t, p, pb[q].span, xqd[q], pbd[q].N, pbd[q].D);
        }
        std::vector<dd> gxd, gwd;
        gauss_legendre_dd(p + 1, gx, gxd, gwd);
        std::vector<dd> gw_span;                 // weights, [span][k]
        std::vector<PointBasisDD> gb_span;       // basis at the nodes, [span][k]
        for (int s = 0; s < nel; ++s) {
            dd a = dd_from(u[s]), b = dd_from(u[s + 1]);
            dd half = (b - a) * 0.5, mid = (a + b) * 0.5;
            for (int k = 0; k <= p; ++k) {
                PointBasisDD pbg;
                pbg.span = p + s;
                local_basis_dd(t, p, p + s, mid + half * gxd[k], pbg.N, pbg.D);
                gb_span.push_back(pbg);
                gw_span.push_back(half * gwd[k]);
            }
        }
        // int b_gi^(a) b_gj^(b) over the spans where both may be nonzero
        auto integral = [&](int gi, int a, int gj, int b) {
            dd tot = dd_from(0.0);
            int s_lo = std::max(gi, gj) - p, s_hi = std::min(gi, gj);  // spans k-p with k in [max, min+p]
            for (int s = std::max(0, s_lo); s <= std::min(nel - 1, s_hi); ++s)
                for (int k = 0; k <= p; ++k) {
                    const PointBasisDD& g = gb_span[(size_t)s * (p + 1) + k];
                    tot = tot + gw_span[(size_t)s * (p + 1) + k] * basis_at_dd(g, p, gi, a) * basis_at_dd(g, p, gj, b);
                }
            return tot;
        };
        // Rows are independent systems: solved on host threads, each row
        // written by one thread only, so the tables do not depend on the
        // thread count.
        std::mutex fail_mu;
        std::atomic<bool> failed{false};
        auto solve_row = [&](int i) {
            std::vector<int> T;
            for (int j = std::max(0, i - p); j <= std::min(n - 1, i + p); ++j) T.push_back(j);
            int rows = (int)T.size(), cols = W.len[i];
            for (int b = 0; b < 2; ++b) {
                std::vector<dd> A((size_t)rows * cols);
                for (int r = 0; r < rows; ++r)
                    for (int c = 0; c < cols; ++c)
                        A[(size_t)r * cols + c] = basis_at_dd(pbd[W.start[i] + c], p, T[r] + 1, b);
                for (int a = 0; a < 2; ++a) {
                    std::vector<dd> g(rows);
                    for (int r = 0; r < rows; ++r) g[r] = integral(i + 1, a, T[r] + 1, b);
                    std::vector<double> w;
                    bool ok = min_norm_solve_dd(A, rows, cols, g, w);
                    double res = 0.0, gn = 0.0;
                    for (int r = 0; ok && r < rows; ++r) {
                        dd s = -g[r];
                        for (int c = 0; c < cols; ++c) s = s + A[(size_t)r * cols + c] * dd_from(w[c]);
                        res = std::max(res, std::fabs(s.hi));
                        gn = std::max(gn, std::fabs(g[r].hi));
                    }
                    if (!ok || !(res <= 1e-12 * gn)) {
                        char buf[160];
                        std::snprintf(buf, sizeof buf, "weight system (a=%d,b=%d) of row %d inconsistent: residual %.3e",
                                      a, b, i, gn > 0 ? res / gn : res);
                        std::lock_guard<std::mutex> lk(fail_mu);
                        if (!failed.exchange(true)) why = buf;
                        return;
                    }
                    for (int c = 0; c < cols; ++c) W.at(2 * a + b, i, c) = w[c];
                }
            }
        };
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const int nth = (int)std::min<unsigned>(std::min(hw, 64u), (unsigned)std::max(1, n / 4));
        std::atomic<int> next{0};
        auto worker = [&]() {
            for (int i = next.fetch_add(1); i < n && !failed.load(); i = next.fetch_add(1)) solve_row(i);
        };
        std::vector<std::thread> pool;
        for (int k = 1; k < nth; ++k) pool.emplace_back(worker);
        worker();
        for (std::thread& t : pool) t.join();
        if (failed.load()) return MFWQ_ESETUP;
    }

    // Transposed bands.
    auto transpose_band = [](const Band1D& S, Band1D& T) {
        T.rows = S.cols; T.cols = S.rows; T.fams = S.fams; T.width = 0;
        T.start.assign(T.rows, 0); T.len.assign(T.rows, 0);
        std::vector<int> lo(T.rows, S.rows), hi(T.rows, -1);
        for (int r = 0; r < S.rows; ++r)
            for (int k = 0; k < S.len[r]; ++k) {
                int c = S.start[r] + k;
                lo[c] = std::min(lo[c], r);
                hi[c] = std::max(hi[c], r);
            }
        for (int c = 0; c < T.rows; ++c) {
            if (hi[c] < lo[c]) { lo[c] = 0; hi[c] = -1; }
            T.start[c] = lo[c];
            T.len[c] = hi[c] - lo[c] + 1;
            T.width = std::max(T.width, T.len[c]);
        }
        T.width = std::max(T.width, 1);
        T.val.assign((size_t)T.fams * T.rows * T.width, 0.0);
        for (int f = 0; f < S.fams; ++f)
            for (int r = 0; r < S.rows; ++r)
                for (int k = 0; k < S.len[r]; ++k) {
                    int c = S.start[r] + k;
                    T.at(f, c, r - T.start[c]) = S.at(f, r, k);
                }
    };
    transpose_band(d.B, d.BT);
    transpose_band(d.W, d.WT);

    // Load-vector band: rows j (interior) -> Gauss points, value b_j(x_g) w_g.
    {
        Band1D S;  // rows g -> columns j
        S.rows = ng; S.cols = n; S.fams = 1; S.width = p + 1;
        S.start.assign(ng, 0); S.len.assign(ng, 0);
        S.val.assign((size_t)ng * (p + 1), 0.0);
        for (int g = 0; g < ng; ++g) {
            int lo = std::max(1, gb[g].span - p), hi = std::min(m - 2, gb[g].span);
            S.start[g] = lo - 1;
            S.len[g] = std::max(0, hi - lo + 1);
            for (int k = 0; k < S.len[g]; ++k) S.at(0, g, k) = basis_at(gb[g], p, lo + k, 0) * d.wg[g];
        }
        transpose_band(S, d.GT);
    }

    // Error rule (relative H1 error, Section 4): Gauss with p+2 points per
    // span; band rows e -> interior columns j with values and derivatives.
    {
        std::vector<double> ex, ew;
        gauss_legendre(p + 2, ex, ew);
        d.xe.clear();
        d.we.clear();
        for (int s = 0; s < nel; ++s) {
            double a = u[s], b = u[s + 1];
            for (int k = 0; k < p + 2; ++k) {
                d.xe.push_back(0.5 * (a + b) + 0.5 * (b - a) * ex[k]);
                d.we.push_back(0.5 * (b - a) * ew[k]);
            }
        }
        const int ne = d.ne = (int)d.xe.size();
        Band1D& E = d.E;
        E.rows = ne; E.cols = n; E.fams = 2; E.width = p + 1;
        E.start.assign(ne, 0); E.len.assign(ne, 0);
        E.val.assign((size_t)2 * ne * (p + 1), 0.0);
        for (int g = 0; g < ne; ++g) {
            const PointBasis eb = eval_point(t, p, m, d.xe[g]);
            int lo = std::max(1, eb.span - p), hi = std::min(m - 2, eb.span);
            E.start[g] = lo - 1;
            E.len[g] = std::max(0, hi - lo + 1);
            for (int k = 0; k < E.len[g]; ++k) {
                E.at(0, g, k) = basis_at(eb, p, lo + k, 0);
                E.at(1, g, k) = basis_at(eb, p, lo + k, 1);
            }
        }
    }

    // FD factors: K_l = G^{11}, M_l = G^{00}; U^T M U = I, U^T K U = diag(lambda).
    if (!gen_eig(Gal[3], Gal[0], n, d.lam, d.U, why)) return MFWQ_ESETUP;
    d.UT.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) d.UT[(size_t)j * n + i] = d.U[(size_t)i * n + j];

    // Even/odd split for knot vectors symmetric about 1/2: then K_l and M_l
    // commute with the index reversal J, the eigenvectors can be taken even
    // (Ju = u) or odd (Ju = -u), and U^T x splits into two half-size products
    // on the folded vector x_j +- x_{n-1-j}.  Even basis: (e_j + e_{n-1-j})/sqrt2
    // (j < h) and e_h (odd n); odd basis: (e_j - e_{n-1-j})/sqrt2.
    d.sym = true;
    for (int i = 0; i < nknots; ++i)
        if (std::fabs(t[i] + t[nknots - 1 - i] - 1.0) > 1e-14) d.sym = false;
    if (d.sym) {
        const int h = n / 2, he = n - h, ho = h;
        d.he = he;
        d.ho = ho;
        const double r2 = std::sqrt(0.5);
        auto basis = [&](int parity, int col, int row) -> double {  // column col of E (parity 0) or O (1)
            if (parity == 0 && col == h) return row == h ? 1.0 : 0.0;  // middle (odd n)
            if (row == col) return r2;
            if (row == n - 1 - col) return parity == 0 ? r2 : -r2;
            return 0.0;
        };
        for (int parity = 0; parity < 2; ++parity) {
            const int m2 = parity == 0 ? he : ho;
            std::vector<double> Kh((size_t)m2 * m2, 0.0), Mh((size_t)m2 * m2, 0.0);
            for (int a = 0; a < m2; ++a)
                for (int b = 0; b < m2; ++b) {
                    double sk = 0.0, sm = 0.0;
                    for (int i = 0; i < n; ++i) {
                        const double ea = basis(parity, a, i);
                        if (ea == 0.0) continue;
                        for (int j = 0; j < n; ++j) {
                            const double eb = basis(parity, b, j);
                            if (eb == 0.0) continue;
                            sk += ea * Gal[3][(size_t)i * n + j] * eb;
                            sm += ea * Gal[0][(size_t)i * n + j] * eb;
                        }
                    }
                    Kh[(size_t)a * m2 + b] = sk;
                    Mh[(size_t)a * m2 + b] = sm;
                }
            std::vector<double> lh, Uh;
            if (!gen_eig(Kh, Mh, m2, lh, Uh, why)) return MFWQ_ESETUP;
            // V = D U with D the folding scale: 1/sqrt2 on paired rows, 1 on the middle row
            std::vector<double>& V = parity == 0 ? d.Ve : d.Vo;
            std::vector<double>& VT = parity == 0 ? d.VeT : d.VoT;
            V.assign((size_t)m2 * m2, 0.0);
            VT.assign((size_t)m2 * m2, 0.0);
            for (int i = 0; i < m2; ++i)
                for (int j = 0; j < m2; ++j) {
                    const double sc = (parity == 0 && i == h) ? 1.0 : r2;
                    V[(size_t)i * m2 + j] = sc * Uh[(size_t)i * m2 + j];
                    VT[(size_t)j * m2 + i] = V[(size_t)i * m2 + j];
                }
            for (int i = 0; i < m2; ++i) d.lam_split.push_back(lh[i]);
        }
    }
    return MFWQ_OK;
}

}  // namespace mfwq

extern "C" int mfwq_tables_1d(int degree, int nknots, const double* knots, int* n, int* nq, double* xq,
                              double* B0, double* B1, double* W, double* U, double* lam) {
    mfwq::Dir1D d;
    std::string why;
    int st = mfwq::build_dir(degree, nknots, knots, d, why);
    if (st != MFWQ_OK) return st;
    if (n) *n = d.n;
    if (nq) *nq = d.nq;
    if (xq) std::memcpy(xq, d.xq.data(), sizeof(double) * d.nq);
    if (B0 || B1) {
        for (int q = 0; q < d.nq; ++q)
            for (int j = 0; j < d.n; ++j) {
                if (B0) B0[(size_t)q * d.n + j] = 0.0;
                if (B1) B1[(size_t)q * d.n + j] = 0.0;
            }
        for (int q = 0; q < d.nq; ++q)
            for (int k = 0; k < d.B.len[q]; ++k) {
                int j = d.B.start[q] + k;
                if (B0) B0[(size_t)q * d.n + j] = d.B.at(0, q, k);
                if (B1) B1[(size_t)q * d.n + j] = d.B.at(1, q, k);
            }
    }
    if (W) {
        std::memset(W, 0, sizeof(double) * 4 * (size_t)d.n * d.nq);
        for (int f = 0; f < 4; ++f)
            for (int i = 0; i < d.n; ++i)
                for (int k = 0; k < d.W.len[i]; ++k)
                    W[((size_t)f * d.n + i) * d.nq + d.W.start[i] + k] = d.W.at(f, i, k);
    }
    if (U) std::memcpy(U, d.U.data(), sizeof(double) * (size_t)d.n * d.n);
    if (lam) std::memcpy(lam, d.lam.data(), sizeof(double) * d.n);
    return MFWQ_OK;
}
