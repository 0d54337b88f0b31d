// C ABI of the MF-WQ library (include/mfwq.h): handle, device memory, and the
// drivers that chain the kernels of Algorithm 2, the FD preconditioner and
// BiCGStab (Section 4).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <fstream>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "fd_oz.h"
#include "fused_apply.h"
#include "grouped.h"
#include "kernels.h"
#include "krylov.h"
#include "prof.h"

using namespace mfwq;

namespace {
thread_local std::string g_last_error;

int fail(int code, const std::string& why) {
    g_last_error = why;
    return code;
}

#define CU(x)                                                                                    \
    do {                                                                                         \
        cudaError_t _e = (x);                                                                    \
        if (_e != cudaSuccess) return fail(MFWQ_ECUDA, std::string(#x) + ": " + cudaGetErrorString(_e)); \
    } while (0)

#define ST(x)                          \
    do {                               \
        int _st = (x);                 \
        if (_st != MFWQ_OK) return _st; \
    } while (0)

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
}  // namespace

namespace mfwq {
void set_last_error(const std::string& why) { g_last_error = why; }
}  // namespace mfwq

namespace {

// Host staging of all device tables in one allocation.
struct Arena {
    std::vector<unsigned char> bytes;
    size_t add(const void* src, size_t n) {
        size_t off = (bytes.size() + 255) & ~(size_t)255;
        bytes.resize(off + (n ? n : 1));
        if (n) std::memcpy(bytes.data() + off, src, n);
        return off;
    }
    template <typename T>
    size_t add_vec(const std::vector<T>& v) {
        return add(v.data(), v.size() * sizeof(T));
    }
};

template <typename T>
std::vector<T> convert(const std::vector<double>& v) {
    return std::vector<T>(v.begin(), v.end());
}

struct BandOff {
    size_t start, len, v64, v32, t64, t32;
    int rows, width;
};

BandOff stage_band(Arena& a, const Band1D& b) {
    BandOff o;
    o.start = a.add_vec(b.start);
    o.len = a.add_vec(b.len);
    o.v64 = a.add_vec(b.val);
    o.v32 = a.add_vec(convert<float>(b.val));
    std::vector<double> t(b.val.size());  // lane-major copy [fams][width][rows]
    for (int f = 0; f < b.fams; ++f)
        for (int r = 0; r < b.rows; ++r)
            for (int k = 0; k < b.width; ++k) t[((size_t)f * b.width + k) * b.rows + r] = b.at(f, r, k);
    o.t64 = a.add_vec(t);
    o.t32 = a.add_vec(convert<float>(t));
    o.rows = b.rows;
    o.width = b.width;
    return o;
}

struct TileOff {
    size_t start, len, v64, v32;
    int ntile, width;
};

// Two-row tiles of a band (TileD): per tile the union window of rows 2k and
// 2k+1 and both rows' values on it, [fams][width][ntile][2].
TileOff stage_tiles(Arena& a, const Band1D& b) {
    const int nt = (b.rows + 1) / 2;
    std::vector<int> st(nt), ln(nt);
    int width = 1;
    for (int k = 0; k < nt; ++k) {
        int lo = 0x7fffffff, hi = 0;
        for (int r = 2 * k; r < std::min(2 * k + 2, b.rows); ++r)
            if (b.len[r] > 0) {
                lo = std::min(lo, b.start[r]);
                hi = std::max(hi, b.start[r] + b.len[r]);
            }
        st[k] = hi > 0 ? lo : 0;
        ln[k] = hi > 0 ? hi - lo : 0;
        width = std::max(width, ln[k]);
    }
    std::vector<double> v((size_t)b.fams * width * nt * 2, 0.0);
    for (int f = 0; f < b.fams; ++f)
        for (int k = 0; k < nt; ++k)
            for (int r = 2 * k; r < std::min(2 * k + 2, b.rows); ++r)
                for (int t = 0; t < b.len[r]; ++t) {
                    const int u = b.start[r] + t - st[k];
                    v[(((size_t)f * width + u) * nt + k) * 2 + (r - 2 * k)] = b.at(f, r, t);
                }
    TileOff o;
    o.start = a.add_vec(st);
    o.len = a.add_vec(ln);
    o.v64 = a.add_vec(v);
    o.v32 = a.add_vec(convert<float>(v));
    o.ntile = nt;
    o.width = width;
    return o;
}

// Translation-invariant interior of the direction's B and W bands (StencilD):
// the largest ranges around the middle rows whose rows equal the middle
// (phase) row shifted by one column per pair of points, or by two points
// per output, to 1e-12 relative, and whose fixed-size windows stay inside
// the band columns.  ok = 0 when the degree exceeds kStencilMaxP or no
// interior exists (e.g. non-uniform knots).
StencilD<double> detect_stencil(const Dir1D& d) {
    StencilD<double> S{};
    S.ok = 0;
    const int P = d.p;
    if (P < 2 || P > kStencilMaxP) return S;
    S.P = P;
    const Band1D& B = d.B;
    const Band1D& W = d.W;
    const int NB = P + 2, NW = 2 * P + 1;
    auto same_vals = [](const Band1D& b, int r, int r0, int fams) {
        if (b.len[r] != b.len[r0]) return false;
        double mx = 0.0;
        for (int f = 0; f < fams; ++f)
            for (int t = 0; t < b.len[r0]; ++t) mx = std::max(mx, std::fabs(b.at(f, r0, t)));
        for (int f = 0; f < fams; ++f)
            for (int t = 0; t < b.len[r0]; ++t)
                if (std::fabs(b.at(f, r, t) - b.at(f, r0, t)) > 1e-12 * mx) return false;
        return true;
    };
    // points: pairs (r0 + 2k, r0 + 2k + 1) around the middle
    const int nq = B.rows, n = B.cols;
    int r0 = nq / 2;
    if (r0 + 1 >= nq) return S;
    auto pair_ok = [&](int k) {  // pair starting at r0 + 2k
        const int a = r0 + 2 * k, b = a + 1;
        if (a < 0 || b >= nq) return false;
        if (B.start[a] != B.start[r0] + k || B.start[b] != B.start[r0 + 1] + k) return false;
        return same_vals(B, a, r0, 2) && same_vals(B, b, r0 + 1, 2);
    };
    if (!pair_ok(0)) return S;
    int klo = 0, khi = 1;  // pairs [klo, khi)
    while (pair_ok(klo - 1)) --klo;
    while (pair_ok(khi)) ++khi;
    const int jmin0 = std::min(B.start[r0], B.start[r0 + 1]);
    const int jmax0 = std::max(B.start[r0] + B.len[r0], B.start[r0 + 1] + B.len[r0 + 1]);
    if (jmax0 - jmin0 > NB) return S;
    // every pair's fixed window [jmin0 + k, jmin0 + k + NB) inside [0, n)
    while (klo < khi && jmin0 + klo < 0) ++klo;
    while (khi > klo && jmin0 + (khi - 1) + NB > n) --khi;
    if (khi - klo < 1) return S;
    S.q_lo = r0 + 2 * klo;
    S.q_hi = r0 + 2 * khi;
    S.jb = jmin0 + klo;
    for (int f = 0; f < 2; ++f)
        for (int ph = 0; ph < 2; ++ph) {
            const int r = r0 + ph, off = B.start[r] - jmin0;
            for (int t = 0; t < NB; ++t) S.bf[f][ph][t] = 0.0;
            for (int t = 0; t < B.len[r]; ++t) S.bf[f][ph][off + t] = B.at(f, r, t);
        }
    // outputs: rows i = w0 + m, start = start[w0] + 2m
    const int nr = W.rows, w0 = nr / 2;
    if (W.len[w0] > NW) return S;
    auto row_ok = [&](int m) {
        const int i = w0 + m;
        if (i < 0 || i >= nr) return false;
        return W.start[i] == W.start[w0] + 2 * m && same_vals(W, i, w0, 4);
    };
    int mlo = 0, mhi = 1;
    while (row_ok(mlo - 1)) --mlo;
    while (row_ok(mhi)) ++mhi;
    while (mlo < mhi && W.start[w0] + 2 * mlo < 0) ++mlo;
    while (mhi > mlo && W.start[w0] + 2 * (mhi - 1) + NW > d.nq) --mhi;
    if (mhi - mlo < 1) return S;
    S.i_lo = w0 + mlo;
    S.i_hi = w0 + mhi;
    S.qw = W.start[w0] + 2 * mlo;
    for (int f = 0; f < 4; ++f) {
        for (int t = 0; t < NW; ++t) S.wf[f][t] = 0.0;
        for (int t = 0; t < W.len[w0]; ++t) S.wf[f][t] = W.at(f, w0, t);
    }
    S.ok = 1;
    return S;
}

template <typename T>
StencilD<T> stencil_as(const StencilD<double>& a) {
    StencilD<T> b;
    b.ok = a.ok;
    b.P = a.P;
    b.q_lo = a.q_lo;
    b.q_hi = a.q_hi;
    b.jb = a.jb;
    b.i_lo = a.i_lo;
    b.i_hi = a.i_hi;
    b.qw = a.qw;
    for (int f = 0; f < 2; ++f)
        for (int ph = 0; ph < 2; ++ph)
            for (int t = 0; t < kStencilMaxP + 2; ++t) b.bf[f][ph][t] = (T)a.bf[f][ph][t];
    for (int f = 0; f < 4; ++f)
        for (int t = 0; t < 2 * kStencilMaxP + 1; ++t) b.wf[f][t] = (T)a.wf[f][t];
    return b;
}

template <typename T>
TileD<T> tiles_at(unsigned char* base, const TileOff& o) {
    TileD<T> t;
    t.start = reinterpret_cast<const int*>(base + o.start);
    t.len = reinterpret_cast<const int*>(base + o.len);
    t.val = reinterpret_cast<const T*>(base + (sizeof(T) == 8 ? o.v64 : o.v32));
    t.ntile = o.ntile;
    t.width = o.width;
    return t;
}

template <typename T>
BandD<T> band_at(unsigned char* base, const BandOff& o) {
    BandD<T> b;
    b.start = reinterpret_cast<const int*>(base + o.start);
    b.len = reinterpret_cast<const int*>(base + o.len);
    b.val = reinterpret_cast<const T*>(base + (sizeof(T) == 8 ? o.v64 : o.v32));
    b.valT = reinterpret_cast<const T*>(base + (sizeof(T) == 8 ? o.t64 : o.t32));
    b.rows = o.rows;
    b.width = o.width;
    return b;
}

}  // namespace

struct mfwq_handle_s {
    cudaStream_t stream = nullptr;
    int mixed = 0, fd_prec = MFWQ_FD_FP64;
    Dir1D dir[3];
    int n[3], nq[3], ng[3];
    size_t N = 0, Nq = 0;
    size_t cs = 0;  // field stride of C64 / C32: Nq rounded up to 32 (aligned bulk copies)
    unsigned char* d_tables = nullptr;
    DirD<double> d64[3];
    DirD<float> d32[3];
    double* C64 = nullptr;
    float* C32 = nullptr;
    double* Cm64 = nullptr;  // reaction coefficient (null: no reaction term)
    float* Cm32 = nullptr;
    double fd_shift = 0.0;
    void* scratch = nullptr;
    double* fd_tmp64 = nullptr;
    float* fd_tmp32 = nullptr;
    double* kv64 = nullptr;  // 8 N
    float* kv32 = nullptr;   // 10 N (8 Krylov + rhs + correction)
    double* part = nullptr;  // 2 kRedBlocks
    double* dnorm = nullptr; // 2 doubles
    int* derr = nullptr;     // device error word (bounded waits)
    int xlines = 4, max_xlines = 4;  // forward x-stage lines per block, FP64 (autotuned)
    int xmode = 0;                   // FP64 x-stage work mapping (autotuned)
    int xlines32 = 4, xmode32 = 1;   // the same for the FP32 operator
    int srows = 1, srows32 = 1;      // slow-dimension output rows per thread (autotuned)
    int svec32 = 1;                  // FP32 slow-dimension columns per thread (autotuned)
    int xcarve = 0, xcarve32 = 0;    // x stage with the reduced shared-memory carveout (autotuned)
    KScal* dsc = nullptr;
    KScal* hsc = nullptr;    // pinned
    Profiler prof;
    double* hnorm = nullptr; // pinned, 2 doubles
    double* host_io = nullptr;  // device f/u buffers of mfwq_solve_host (2 N), lazily
    OzPlan oz;                  // FP64 FD on the tensor cores by operand splitting (built on request)
    int fd64_path = MFWQ_FD64_PIPE;
    FusedPlan fplan;            // fused FP32 apply (mixed handles with a stencil direction 1)
    int fused32 = 0;            // 1: the FP32 apply runs the fused kernel
    int onthefly = 0;           // 1: the FP32 operator evaluates C in its x stage (C32 freed)
    CoeffField cf32;            // that coefficient field
    float* cf_tab = nullptr;    // its direction-1 tables: G [6][nq1], s [2][nq1]
};

namespace {

OpCtx<double> ctx64(mfwq_handle h) {
    OpCtx<double> c;
    for (int l = 0; l < 3; ++l) c.d[l] = h->d64[l];
    c.C = h->C64;
    c.Nq = h->Nq;
    c.cs = h->cs;
    c.err = h->derr;
    c.scratch = static_cast<double*>(h->scratch);
    c.stream = h->stream;
    c.xlines = h->xlines;
    c.xmode = h->xmode;
    c.srows = h->srows;
    c.xcarve = h->xcarve;
    c.cm = h->Cm64;
    return c;
}

OpCtx<float> ctx32(mfwq_handle h) {
    OpCtx<float> c;
    for (int l = 0; l < 3; ++l) c.d[l] = h->d32[l];
    c.C = h->C32;
    c.Nq = h->Nq;
    c.cs = h->cs;
    c.err = h->derr;
    c.scratch = static_cast<float*>(h->scratch);
    c.stream = h->stream;
    c.xlines = h->xlines32;
    c.xmode = h->xmode32;
    c.srows = h->srows32;
    c.svec = h->svec32;
    c.xcarve = h->xcarve32;
    c.cm = h->Cm32;
    c.fused = h->fused32 && h->fplan.ok ? &h->fplan : nullptr;
    c.cf = h->onthefly ? &h->cf32 : nullptr;
    return c;
}

// The FP64 FD preconditioner of the handle's FP64 path on stream s.
LinOp<double> fd64_linop(mfwq_handle h, cudaStream_t s) {
    double* tmp = h->fd_tmp64;
    if (h->fd64_path == MFWQ_FD64_SPLIT && h->oz.ok) {
        const OzPlan* p = &h->oz;
        int* err = h->derr;
        return [p, tmp, err, s](const double* in, double* out, const int* skip) {
            return run_fd_oz(*p, in, out, tmp, err, skip, s);
        };
    }
    DirD<double> d[3] = {h->d64[0], h->d64[1], h->d64[2]};
    return [d, tmp, s](const double* in, double* out, const int* skip) { return run_fd64(d, in, out, tmp, skip, s); };
}

void free_handle(mfwq_handle h) {
    if (!h) return;
    cudaFree(h->d_tables);
    cudaFree(h->C64);
    cudaFree(h->C32);
    cudaFree(h->Cm64);
    cudaFree(h->Cm32);
    cudaFree(h->scratch);
    cudaFree(h->fd_tmp64);
    cudaFree(h->fd_tmp32);
    cudaFree(h->kv64);
    cudaFree(h->kv32);
    cudaFree(h->part);
    cudaFree(h->dnorm);
    cudaFree(h->derr);
    cudaFree(h->dsc);
    cudaFree(h->host_io);
    fused_plan_free(h->fplan);
    oz_plan_free(h->oz);
    cudaFree(h->cf_tab);
    if (h->hsc) cudaFreeHost(h->hsc);
    if (h->hnorm) cudaFreeHost(h->hnorm);
    delete h;
}

int dmalloc(void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MFWQ_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    return MFWQ_OK;
}

// Builds the split FP64 FD of the handle (slices of U_l and U_l^T, scaling table) if not built yet.
int split_fd_enable(mfwq_handle h) {
    if (h->oz.ok) return MFWQ_OK;
    for (int l = 0; l < 3; ++l)
        if (h->n[l] > kOzMaxN) return fail(MFWQ_EINVAL, "the split FP64 FD needs at most 256 DoFs per direction");
    static std::once_flag once;
    static int conf = MFWQ_OK;
    std::call_once(once, [] { conf = configure_fd_oz(); });
    ST(conf);
    CU(cudaStreamSynchronize(h->stream));
    ST(oz_plan_build(h->dir, h->d64, h->stream, h->oz));
    CU(cudaStreamSynchronize(h->stream));
    return MFWQ_OK;
}

int setup_impl(const mfwq_setup_desc* desc, mfwq_handle h) {
    h->stream = static_cast<cudaStream_t>(desc->stream);
    h->mixed = desc->mixed ? 1 : 0;
    h->fd_prec = h->mixed ? desc->fd_precision : MFWQ_FD_FP64;
    if (h->mixed && h->fd_prec != MFWQ_FD_TF32 && h->fd_prec != MFWQ_FD_BF16)
        return fail(MFWQ_EINVAL, "fd_precision must be MFWQ_FD_TF32 or MFWQ_FD_BF16 when mixed = 1");
    for (int l = 0; l < 3; ++l) {
        std::string why;
        // a direction with the degree and knots of an earlier one reuses its tables
        int same = -1;
        for (int k = 0; k < l && same < 0; ++k)
            if (desc->degree[k] == desc->degree[l] && desc->nknots[k] == desc->nknots[l] &&
                std::memcmp(desc->knots[k], desc->knots[l], sizeof(double) * desc->nknots[l]) == 0)
                same = k;
        int st = MFWQ_OK;
        if (same >= 0) h->dir[l] = h->dir[same];
        else st = build_dir(desc->degree[l], desc->nknots[l], desc->knots[l], h->dir[l], why);
        if (st != MFWQ_OK) return fail(st, "direction " + std::to_string(l + 1) + ": " + why);
        h->n[l] = h->dir[l].n;
        h->nq[l] = h->dir[l].nq;
        h->ng[l] = h->dir[l].ng;
    }
    h->N = (size_t)h->n[0] * h->n[1] * h->n[2];
    h->Nq = (size_t)h->nq[0] * h->nq[1] * h->nq[2];
    h->cs = (h->Nq + 31) / 32 * 32;
    if (h->Nq * 9 >= ((size_t)1 << 40)) return fail(MFWQ_EINVAL, "problem too large");

    // ---- tables
    Arena a;
    BandOff bo[3][6];
    TileOff to[3][2];
    size_t U64[3], UT64[3], L64[3], U32[3], UT32[3], L32[3], XQ[3], XG[3], XE[3], WE[3];
    size_t VE[3] = {}, VET[3] = {}, VO[3] = {}, VOT[3] = {}, LS[3] = {}, QO[3], JO[3];
    for (int l = 0; l < 3; ++l) {
        const Dir1D& d = h->dir[l];
        {
            // item orders of the transposed and gradient x stages: rows by decreasing band
            // length, so that the lanes of a warp walk bands of one length
            auto by_len = [](const Band1D& b, std::vector<int> ord) {
                std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return b.len[x] > b.len[y]; });
                return ord;
            };
            std::vector<int> q(d.nq), j(d.n);
            const int half = (d.nq + 1) / 2;
            for (int r = 0; r < d.nq; ++r) q[r] = r < half ? 2 * r : 2 * (r - half) + 1;  // parity order
            for (int r = 0; r < d.n; ++r) j[r] = r;
            QO[l] = a.add_vec(by_len(d.WT, q));
            JO[l] = a.add_vec(by_len(d.BT, j));
        }
        bo[l][0] = stage_band(a, d.B);
        bo[l][1] = stage_band(a, d.BT);
        bo[l][2] = stage_band(a, d.W);
        bo[l][3] = stage_band(a, d.WT);
        bo[l][4] = stage_band(a, d.GT);
        bo[l][5] = stage_band(a, d.E);
        XE[l] = a.add_vec(d.xe);
        WE[l] = a.add_vec(d.we);
        to[l][0] = stage_tiles(a, d.B);
        to[l][1] = stage_tiles(a, d.W);
        U64[l] = a.add_vec(d.U);
        UT64[l] = a.add_vec(d.UT);
        L64[l] = a.add_vec(d.lam);
        U32[l] = a.add_vec(convert<float>(d.U));
        UT32[l] = a.add_vec(convert<float>(d.UT));
        L32[l] = a.add_vec(convert<float>(d.lam));
        XQ[l] = a.add_vec(d.xq);
        XG[l] = a.add_vec(d.xg);
        if (d.sym) {
            VE[l] = a.add_vec(d.Ve);
            VET[l] = a.add_vec(d.VeT);
            VO[l] = a.add_vec(d.Vo);
            VOT[l] = a.add_vec(d.VoT);
            LS[l] = a.add_vec(d.lam_split);
        }
    }
    ST(dmalloc((void**)&h->d_tables, a.bytes.size()));
    CU(cudaMemcpy(h->d_tables, a.bytes.data(), a.bytes.size(), cudaMemcpyHostToDevice));
    unsigned char* base = h->d_tables;
    for (int l = 0; l < 3; ++l) {
        DirD<double>& x = h->d64[l];
        DirD<float>& y = h->d32[l];
        x.n = y.n = h->n[l];
        x.nq = y.nq = h->nq[l];
        x.ng = y.ng = h->ng[l];
        x.B = band_at<double>(base, bo[l][0]);
        x.BT = band_at<double>(base, bo[l][1]);
        x.W = band_at<double>(base, bo[l][2]);
        x.WT = band_at<double>(base, bo[l][3]);
        x.GT = band_at<double>(base, bo[l][4]);
        y.B = band_at<float>(base, bo[l][0]);
        y.BT = band_at<float>(base, bo[l][1]);
        y.W = band_at<float>(base, bo[l][2]);
        y.WT = band_at<float>(base, bo[l][3]);
        y.GT = band_at<float>(base, bo[l][4]);
        x.E = band_at<double>(base, bo[l][5]);
        y.E = band_at<float>(base, bo[l][5]);
        x.ne = y.ne = h->dir[l].ne;
        x.xe = y.xe = reinterpret_cast<const double*>(base + XE[l]);
        x.we = y.we = reinterpret_cast<const double*>(base + WE[l]);
        x.BX = tiles_at<double>(base, to[l][0]);
        x.WX = tiles_at<double>(base, to[l][1]);
        {
            // W rows at each end whose band length differs from the middle row's, so
            // that the x stage can give the uniform rows warps of their own
            const Band1D& W = h->dir[l].W;
            const int nr = W.rows, lm = nr > 0 ? W.len[nr / 2] : 0;
            int nb = 0;
            for (int i = 0; i < nr; ++i)
                if (W.len[i] != lm) nb = std::max(nb, std::min(i + 1, nr - i));
            x.wnb = y.wnb = 2 * nb < nr ? nb : 0;
        }
        x.qord = y.qord = reinterpret_cast<const int*>(base + QO[l]);
        x.jord = y.jord = reinterpret_cast<const int*>(base + JO[l]);
        x.SX = detect_stencil(h->dir[l]);
        y.SX = stencil_as<float>(x.SX);
        y.BX = tiles_at<float>(base, to[l][0]);
        y.WX = tiles_at<float>(base, to[l][1]);
        x.U = reinterpret_cast<const double*>(base + U64[l]);
        x.UT = reinterpret_cast<const double*>(base + UT64[l]);
        x.lam = reinterpret_cast<const double*>(base + L64[l]);
        y.U = reinterpret_cast<const float*>(base + U32[l]);
        y.UT = reinterpret_cast<const float*>(base + UT32[l]);
        y.lam = reinterpret_cast<const float*>(base + L32[l]);
        x.xq = y.xq = reinterpret_cast<const double*>(base + XQ[l]);
        x.sym = h->dir[l].sym ? 1 : 0;
        y.sym = 0;
        x.he = y.he = h->dir[l].he;
        x.ho = y.ho = h->dir[l].ho;
        x.Ve = x.VeT = x.Vo = x.VoT = x.lam_split = nullptr;
        y.Ve = y.VeT = y.Vo = y.VoT = y.lam_split = nullptr;
        if (h->dir[l].sym) {
            x.Ve = reinterpret_cast<const double*>(base + VE[l]);
            x.VeT = reinterpret_cast<const double*>(base + VET[l]);
            x.Vo = reinterpret_cast<const double*>(base + VO[l]);
            x.VoT = reinterpret_cast<const double*>(base + VOT[l]);
            x.lam_split = reinterpret_cast<const double*>(base + LS[l]);
        }
        x.xg = y.xg = reinterpret_cast<const double*>(base + XG[l]);
    }

    // ---- coefficient, workspace
    ST(dmalloc((void**)&h->C64, sizeof(double) * 6 * h->cs));
    CU(cudaMemset(h->C64, 0, sizeof(double) * 6 * h->cs));
    if (h->mixed) {
        ST(dmalloc((void**)&h->C32, sizeof(float) * 6 * h->cs));
        CU(cudaMemset(h->C32, 0, sizeof(float) * 6 * h->cs));
    }
    size_t sc = apply_scratch_elems(h->n, h->nq);
    size_t sr = rhs_scratch_elems(h->n, h->ng);
    ST(dmalloc(&h->scratch, sizeof(double) * (sc > sr ? sc : sr)));
    ST(dmalloc((void**)&h->fd_tmp64, sizeof(double) * h->N));
    ST(dmalloc((void**)&h->kv64, sizeof(double) * 8 * h->N));
    if (h->mixed) {
        ST(dmalloc((void**)&h->fd_tmp32, sizeof(float) * h->N));
        ST(dmalloc((void**)&h->kv32, sizeof(float) * 10 * h->N));
    }
    ST(dmalloc((void**)&h->part, sizeof(double) * 2 * kRedBlocks));
    ST(dmalloc((void**)&h->dnorm, sizeof(double) * 2));
    ST(dmalloc((void**)&h->dsc, sizeof(KScal)));
    ST(dmalloc((void**)&h->derr, sizeof(int)));
    CU(cudaMemset(h->derr, 0, sizeof(int)));
    if (h->mixed) {
        int maxn = std::max(h->n[0], std::max(h->n[1], h->n[2]));
        if (maxn > 256) return fail(MFWQ_EINVAL, "the tensor-core FD needs at most 256 DoFs per direction");
        ST(configure_fd_tc(maxn));
    }
    CU(cudaMallocHost((void**)&h->hsc, sizeof(KScal)));
    CU(cudaMallocHost((void**)&h->hnorm, sizeof(double) * 2));

    int smem = std::max(xstage_smem_bytes(8, h->n[0], h->nq[0], 4, 0), xstage_aux_smem_bytes(8, h->n[0], h->nq[0]));
    if (smem > kXstageSmemMax) return fail(MFWQ_EINVAL, "direction-1 size too large for the x-stage tile");
    h->max_xlines = xstage_smem_bytes(8, h->n[0], h->nq[0], 8, 0) <= kXstageSmemMax ? 8 : 4;
    for (int es : {8, 4})
        for (int mode = 0; mode < 7; ++mode)
            for (int L : {2, 4, 8})
                if (xstage_mode_valid(es, h->n[0], h->nq[0], L, mode))
                    smem = std::max(smem, xstage_smem_bytes(es, h->n[0], h->nq[0], L, mode));
    ST(configure_xstage_smem(smem));
    if (h->mixed) {
        ST(configure_xstage_otf_smem(xstage_otf_smem_bytes(h->n[0], h->nq[0])));
        ST(fused_plan_build(h->dir[0], h->dir[1], h->d32[0].SX, h->d32[1].SX, h->nq[2], h->fplan));
        h->fused32 = 0;  // the staged kernels unless mfwq_autotune or mfwq_set_fp32_path picks the fused one
    }
    // the FP64 FD on the tensor cores by operand splitting wherever every direction allows it
    if (h->n[0] <= kOzMaxN && h->n[1] <= kOzMaxN && h->n[2] <= kOzMaxN) {
        ST(split_fd_enable(h));
        h->fd64_path = MFWQ_FD64_SPLIT;
    }
    CU(cudaDeviceSynchronize());
    return MFWQ_OK;
}

KrylovBufs<double> bufs64(mfwq_handle h) {
    double* v = h->kv64;
    size_t N = h->N;
    return KrylovBufs<double>{v, v + N, v + 2 * N, v + 3 * N, v + 4 * N, v + 5 * N, v + 6 * N, v + 7 * N};
}

KrylovBufs<float> bufs32(mfwq_handle h) {
    float* v = h->kv32;
    size_t N = h->N;
    return KrylovBufs<float>{v, v + N, v + 2 * N, v + 3 * N, v + 4 * N, v + 5 * N, v + 6 * N, v + 7 * N};
}

mfwq_solve_opts default_opts() {
    mfwq_solve_opts o;
    std::memset(&o, 0, sizeof o);
    o.rtol = 1e-10;
    o.maxit = 500;
    return o;
}

int solve64(mfwq_handle h, const double* f, double* u, const mfwq_solve_opts& o, mfwq_solve_info* info, bool transpose) {
    OpCtx<double> c = ctx64(h);
    LinOp<double> A = [c, transpose](const double* in, double* out, const int* skip) {
        return transpose ? run_apply_T<double>(c, in, out, skip) : run_apply<double>(c, in, out, skip);
    };
    cudaStream_t s = h->stream;
    LinOp<double> P = fd64_linop(h, s);
    if (o.fp64_low_fd) {
        // the FD in the handle's low precision: FP32 copies in the mixed refinement's
        // work vectors (unused by an FP64 solve), tensor-core mode products
        if (!h->mixed) return fail(MFWQ_EINVAL, "fp64_low_fd needs a handle set up with mixed = 1");
        const size_t N = h->N;
        float* x32 = h->kv32 + 8 * N;
        float* z32 = h->kv32 + 9 * N;
        DirD<float> d32[3] = {h->d32[0], h->d32[1], h->d32[2]};
        float* tmp32 = h->fd_tmp32;
        int* err = h->derr;
        const int prec = h->fd_prec;
        P = [=](const double* in, double* out, const int* skip) {
            int st = convert_into<double, float>(in, x32, N, skip, s);
            if (st == MFWQ_OK) st = run_fd_tc(d32, prec, x32, z32, tmp32, err, skip, s);
            if (st == MFWQ_OK) st = convert_into<float, double>(z32, out, N, skip, s);
            return st;
        };
    }
    int iters = 0, status = MFWQ_OK;
    double rel = 0.0;
    const int chunk = h->prof.on ? 0 : o.graph_chunk;  // profiling events cannot be captured
    ST(bicgstab<double>(A, P, f, u, o.use_initial_guess != 0, o.rtol, o.maxit, bufs64(h), h->dsc, h->hsc, h->part, h->N, s,
                        1, o.res_hist, &iters, &rel, &status, chunk));
    if (info) {
        info->status = status;
        info->iterations = iters;
        info->outer_iterations = 0;
        info->rel_residual = rel;
    }
    return status;
}

// FP64 iterative refinement around inner FP32 BiCGStab solves.
int solve_mixed(mfwq_handle h, const double* f, double* u, const mfwq_solve_opts& o, mfwq_solve_info* info) {
    const size_t N = h->N;
    cudaStream_t s = h->stream;
    OpCtx<double> c64 = ctx64(h);
    OpCtx<float> c32 = ctx32(h);
    double* w64 = h->kv64;       // K~ u
    double* r64 = h->kv64 + N;   // f - K~ u
    float* r32 = h->kv32 + 8 * N;
    float* d32 = h->kv32 + 9 * N;
    DirD<float> d[3] = {h->d32[0], h->d32[1], h->d32[2]};
    float* tmp = h->fd_tmp32;
    LinOp<float> A = [c32](const float* in, float* out, const int* skip) { return run_apply<float>(c32, in, out, skip); };
    int* err = h->derr;
    const int prec = h->fd_prec;
    LinOp<float> P = [d, tmp, s, err, prec](const float* in, float* out, const int* skip) {
        return run_fd_tc(d, prec, in, out, tmp, err, skip, s);
    };
    const double inner_rtol = o.inner_rtol > 0 ? o.inner_rtol : 1e-4;
    const int inner_maxit = o.inner_maxit > 0 ? o.inner_maxit : 200;
    if (!o.use_initial_guess) CU(cudaMemsetAsync(u, 0, sizeof(double) * N, s));
    ST(norm2_into(f, N, h->part, h->dnorm + 1, s));
    int outer = 0, inner_total = 0, status = MFWQ_ENOCONV;
    double rel = 1.0;
    for (;;) {
        if (outer == 0 && !o.use_initial_guess) {
            CU(cudaMemcpyAsync(r64, f, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));  // u = 0: r = f
        } else {
            ST(run_apply<double>(c64, u, w64, nullptr));
            ST(axpby_into<double>(f, w64, r64, N, s));
        }
        ST(norm2_into(r64, N, h->part, h->dnorm, s));
        CU(cudaMemcpyAsync(h->hnorm, h->dnorm, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        const double r2 = h->hnorm[0], f2 = h->hnorm[1];
        if (!std::isfinite(r2)) { status = MFWQ_ENAN; break; }
        rel = f2 > 0 ? std::sqrt(r2 / f2) : 0.0;
        if (o.res_hist) o.res_hist[outer] = rel;
        if (f2 == 0.0 || rel <= o.rtol) { status = MFWQ_OK; break; }
        if (outer >= o.maxit) break;
        ST(to_f32_scaled(r64, h->dnorm, r32, N, s));
        int it = 0, ist = MFWQ_OK;
        double irel = 0.0;
        ST(bicgstab<float>(A, P, r32, d32, false, inner_rtol, inner_maxit, bufs32(h), h->dsc, h->hsc, h->part, N, s, 4,
                           nullptr, &it, &irel, &ist));
        inner_total += it;
        if (ist == MFWQ_ENAN) { status = MFWQ_ENAN; break; }
        ST(add_f32_scaled(u, d32, h->dnorm, N, s));
        ++outer;
    }
    if (info) {
        info->status = status;
        info->iterations = inner_total;
        info->outer_iterations = outer;
        info->rel_residual = rel;
    }
    return status;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

const char* mfwq_status_string(int st) {
    switch (st) {
        case MFWQ_OK: return "ok";
        case MFWQ_EINVAL: return "invalid argument";
        case MFWQ_ENOMEM: return "out of memory";
        case MFWQ_ECUDA: return "CUDA error";
        case MFWQ_ESETUP: return "setup failed (weights or eigensolve)";
        case MFWQ_EBREAKDOWN: return "BiCGStab breakdown";
        case MFWQ_ENOCONV: return "not converged";
        case MFWQ_ETIMEOUT: return "device wait timed out";
        case MFWQ_ENAN: return "NaN or Inf encountered";
        case MFWQ_EINTERNAL: return "internal error";
        default: return "unknown status";
    }
}

const char* mfwq_last_error(void) { return g_last_error.c_str(); }

int mfwq_setup(const mfwq_setup_desc* desc, mfwq_handle* out) {
    if (!desc || !out) return fail(MFWQ_EINVAL, "NULL argument");
    *out = nullptr;
    mfwq_handle h = new (std::nothrow) mfwq_handle_s();
    if (!h) return fail(MFWQ_ENOMEM, "host allocation failed");
    int st = setup_impl(desc, h);
    if (st != MFWQ_OK) {
        free_handle(h);
        return st;
    }
    *out = h;
    return MFWQ_OK;
}

void mfwq_destroy(mfwq_handle h) {
    if (h && h->stream) cudaStreamSynchronize(h->stream);
    else if (h) cudaDeviceSynchronize();
    free_handle(h);
}

int mfwq_sizes(mfwq_handle h, int n[3], int nq[3]) {
    if (!h) return fail(MFWQ_EINVAL, "NULL handle");
    for (int l = 0; l < 3; ++l) {
        if (n) n[l] = h->n[l];
        if (nq) nq[l] = h->nq[l];
    }
    return MFWQ_OK;
}

int mfwq_quad_points(mfwq_handle h, int dir, double* xq_host) {
    if (!h || dir < 0 || dir > 2 || !xq_host) return fail(MFWQ_EINVAL, "bad argument");
    std::memcpy(xq_host, h->dir[dir].xq.data(), sizeof(double) * h->nq[dir]);
    return MFWQ_OK;
}

int mfwq_eval_coeff(mfwq_handle h, int geometry, const double* modes_host, int nmodes, double kscale, double* C_dev) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || !C_dev || nmodes < 0 || nmodes > 32 || (nmodes > 0 && !modes_host)) return fail(MFWQ_EINVAL, "bad argument");
    if (geometry != MFWQ_GEOM_CUBE && geometry != MFWQ_GEOM_RING) return fail(MFWQ_EINVAL, "unknown geometry");
    if (!aligned16(C_dev)) return fail(MFWQ_EINVAL, "C_dev must be 16-byte aligned");
    const double* xq[3] = {h->d64[0].xq, h->d64[1].xq, h->d64[2].xq};
    return run_eval_coeff(h->nq, xq, geometry, modes_host, nmodes, kscale, C_dev, h->stream);
}

namespace {
// y[s][cs] = x[s][n] for s < nf (coefficient fields into a padded FP32 copy)
__global__ void k_fields_to_f32(const double* __restrict__ x, size_t n, float* __restrict__ y, size_t cs, int nf) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf * n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t s = i / n, k = i - s * n;
        y[s * cs + k] = (float)x[i];
    }
}
}  // namespace

int mfwq_set_coeff(mfwq_handle h, const double* C_dev) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || !C_dev) return fail(MFWQ_EINVAL, "bad argument");
    h->onthefly = 0;
    if (h->mixed && !h->C32) ST(dmalloc((void**)&h->C32, sizeof(float) * 6 * h->cs));
    CU(cudaMemcpy2DAsync(h->C64, sizeof(double) * h->cs, C_dev, sizeof(double) * h->Nq, sizeof(double) * h->Nq, 6,
                         cudaMemcpyDeviceToDevice, h->stream));
    if (h->mixed) {
        launch_begin(S_SETUP, h->stream);
        k_fields_to_f32<<<1024, 256, 0, h->stream>>>(C_dev, h->Nq, h->C32, h->cs, 6);
        launch_end(S_SETUP, h->stream);
        CU(cudaGetLastError());
    }
    return MFWQ_OK;
}

namespace {
// |det J| J^-1 J^-T of the geometry at (xi1, xi2), K = I (Eq. (C), J_ij = dF_i/dxi_j),
// by the adjugate: J^-1 = adj(J) / det J, so the product is adj adj^T / |det|.
void geom_factor(int geom, double xi1, double xi2, double G[6]) {
    double J[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    if (geom == MFWQ_GEOM_RING) {
        const double hp = 1.5707963267948966, r = 1.0 + xi1;
        const double sn = std::sin(hp * xi2), cs = std::cos(hp * xi2);
        J[0][0] = cs;
        J[1][0] = sn;
        J[0][1] = -r * hp * sn;
        J[1][1] = r * hp * cs;
    }
    double A[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
            A[i][j] = J[i1][j1] * J[i2][j2] - J[i1][j2] * J[i2][j1];  // cofactor of J[j][i]
        }
    const double det = J[0][0] * A[0][0] + J[0][1] * A[1][0] + J[0][2] * A[2][0];
    const int pr[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int s = 0; s < 6; ++s) {
        const int i = pr[s][0], j = pr[s][1];
        G[s] = (A[i][0] * A[j][0] + A[i][1] * A[j][1] + A[i][2] * A[j][2]) / std::fabs(det);
    }
}
}  // namespace

int mfwq_set_coeff_field(mfwq_handle h, int geometry, const double* modes_host, int nmodes, double kscale, int onthefly) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || nmodes < 0 || nmodes > kMaxModes || (nmodes > 0 && !modes_host) || !std::isfinite(kscale))
        return fail(MFWQ_EINVAL, "bad argument");
    if (geometry != MFWQ_GEOM_CUBE && geometry != MFWQ_GEOM_RING) return fail(MFWQ_EINVAL, "unknown geometry");
    if (onthefly) {
        if (!h->mixed) return fail(MFWQ_EINVAL, "the coefficient is evaluated in the FP32 operator: needs mixed = 1");
        const StencilD<float>& S = h->d32[0].SX;
        if (!S.ok || S.P < 2 || S.P > kStencilMaxP)
            return fail(MFWQ_EINVAL, "evaluating the coefficient in the x stage needs the stencil form (p_1 <= 8)");
    }
    // the stored FP64 coefficient (the FP64 operator reads it) and, without on-the-fly, its FP32 copy
    double* tmp = nullptr;
    ST(dmalloc((void**)&tmp, sizeof(double) * 6 * h->Nq));
    const double* xq[3] = {h->d64[0].xq, h->d64[1].xq, h->d64[2].xq};
    int st = run_eval_coeff(h->nq, xq, geometry, modes_host, nmodes, kscale, tmp, h->stream);
    if (st == MFWQ_OK) st = mfwq_set_coeff(h, tmp);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) st = fail(MFWQ_ECUDA, "evaluating the coefficient failed");
    cudaFree(tmp);
    if (st != MFWQ_OK) return st;
    if (!onthefly) return MFWQ_OK;
    // direction-1 tables: G(xi1) (checked to be independent of xi2) and s = r or xi1 as a float pair
    const int nq1 = h->nq[0];
    std::vector<float> tab((size_t)8 * nq1);
    for (int q = 0; q < nq1; ++q) {
        const double xi1 = h->dir[0].xq[q];
        double G[6], G2[6];
        geom_factor(geometry, xi1, 0.0, G);
        for (double xi2 : {0.3, 0.7, 1.0}) {
            geom_factor(geometry, xi1, xi2, G2);
            for (int s = 0; s < 6; ++s)
                if (std::fabs(G2[s] - G[s]) > 1e-13 * (std::fabs(G[0]) + std::fabs(G[1]) + std::fabs(G[2])))
                    return fail(MFWQ_EINVAL, "the geometry factor of C depends on xi2: no direction-1 table");
        }
        for (int s = 0; s < 6; ++s) tab[(size_t)s * nq1 + q] = (float)G[s];
        const double sv = geometry == MFWQ_GEOM_RING ? 1.0 + xi1 : xi1;
        const float hi = (float)sv;
        tab[(size_t)6 * nq1 + q] = hi;
        tab[(size_t)7 * nq1 + q] = (float)(sv - (double)hi);
    }
    if (!h->cf_tab) ST(dmalloc((void**)&h->cf_tab, sizeof(float) * 8 * nq1));
    CU(cudaMemcpy(h->cf_tab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice));
    CoeffField& f = h->cf32;
    f.geom = geometry;
    f.nmodes = nmodes;
    f.kscale = (float)kscale;
    for (int m = 0; m < nmodes; ++m) {
        f.a[m] = (float)modes_host[5 * m];
        for (int d = 0; d < 3; ++d) f.k[m][d] = modes_host[5 * m + 1 + d];
        f.phi_pi[m] = modes_host[5 * m + 4] / 3.141592653589793;
    }
    f.g6 = h->cf_tab;
    f.s1 = h->cf_tab + (size_t)6 * nq1;
    f.xq2 = h->d64[1].xq;
    f.xq3 = h->d64[2].xq;
    cudaFree(h->C32);  // the FP32 operator no longer reads a stored coefficient
    h->C32 = nullptr;
    h->onthefly = 1;
    return MFWQ_OK;
}

int mfwq_eval_mass_coeff(mfwq_handle h, int geometry, double alpha, double* c_dev) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || !c_dev || !std::isfinite(alpha)) return fail(MFWQ_EINVAL, "bad argument");
    if (geometry != MFWQ_GEOM_CUBE && geometry != MFWQ_GEOM_RING) return fail(MFWQ_EINVAL, "unknown geometry");
    const double* xq[3] = {h->d64[0].xq, h->d64[1].xq, h->d64[2].xq};
    return run_eval_mass(h->nq, xq, geometry, alpha, c_dev, h->stream);
}

namespace {
// lambda_3 + shift into the device eigenvalue tables of direction 3 (all FD forms)
int upload_fd_shift(mfwq_handle h, double shift) {
    const Dir1D& d = h->dir[2];
    std::vector<double> l64(d.lam.size());
    std::vector<float> l32(d.lam.size());
    for (size_t k = 0; k < d.lam.size(); ++k) {
        l64[k] = d.lam[k] + shift;
        l32[k] = (float)l64[k];
    }
    CU(cudaMemcpy(const_cast<double*>(h->d64[2].lam), l64.data(), sizeof(double) * l64.size(), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(const_cast<float*>(h->d32[2].lam), l32.data(), sizeof(float) * l32.size(), cudaMemcpyHostToDevice));
    if (d.sym && h->d64[2].lam_split) {
        std::vector<double> ls(d.lam_split.size());
        for (size_t k = 0; k < ls.size(); ++k) ls[k] = d.lam_split[k] + shift;
        CU(cudaMemcpy(const_cast<double*>(h->d64[2].lam_split), ls.data(), sizeof(double) * ls.size(),
                      cudaMemcpyHostToDevice));
    }
    if (h->oz.ok) {
        ST(oz_update_dinv(h->d64, h->oz, h->stream));
        CU(cudaStreamSynchronize(h->stream));
    }
    return MFWQ_OK;
}
}  // namespace

int mfwq_set_mass_coeff(mfwq_handle h, const double* c_dev, double fd_shift) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h) return fail(MFWQ_EINVAL, "NULL handle");
    if (!std::isfinite(fd_shift) || fd_shift < 0.0) return fail(MFWQ_EINVAL, "fd_shift must be finite and >= 0");
    if (!c_dev) {
        CU(cudaStreamSynchronize(h->stream));
        cudaFree(h->Cm64);
        cudaFree(h->Cm32);
        h->Cm64 = nullptr;
        h->Cm32 = nullptr;
    } else {
        if (!h->Cm64) ST(dmalloc((void**)&h->Cm64, sizeof(double) * h->Nq));
        if (h->mixed && !h->Cm32) ST(dmalloc((void**)&h->Cm32, sizeof(float) * h->Nq));
        CU(cudaMemcpyAsync(h->Cm64, c_dev, sizeof(double) * h->Nq, cudaMemcpyDeviceToDevice, h->stream));
        if (h->mixed) {
            launch_begin(S_SETUP, h->stream);
            k_fields_to_f32<<<1024, 256, 0, h->stream>>>(c_dev, h->Nq, h->Cm32, h->Nq, 1);
            launch_end(S_SETUP, h->stream);
            CU(cudaGetLastError());
        }
    }
    if (fd_shift != h->fd_shift) {
        CU(cudaStreamSynchronize(h->stream));  // no FD of this handle may be reading the tables
        ST(upload_fd_shift(h, fd_shift));
        h->fd_shift = fd_shift;
    }
    return MFWQ_OK;
}

int mfwq_grad_mass_coeff(mfwq_handle h, const double* lambda_dev, const double* u_dev, double* gc_dev) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || !lambda_dev || !u_dev || !gc_dev) return fail(MFWQ_EINVAL, "bad argument");
    return run_grad_mass<double>(ctx64(h), lambda_dev, u_dev, gc_dev);
}

int mfwq_h1_error(mfwq_handle h, int geometry, int solution, const double* u_dev, double* rel_err) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || !u_dev || !rel_err) return fail(MFWQ_EINVAL, "bad argument");
    if (geometry != MFWQ_GEOM_CUBE && geometry != MFWQ_GEOM_RING) return fail(MFWQ_EINVAL, "unknown geometry");
    if (solution != MFWQ_EXACT_SINES && solution != MFWQ_EXACT_RING) return fail(MFWQ_EINVAL, "unknown exact solution");
    const int st = run_h1_error(h->d64, geometry, solution, u_dev, rel_err, h->stream);
    if (st == MFWQ_ENOMEM) return fail(st, "device allocation for the error evaluation failed");
    if (st != MFWQ_OK) return fail(st, "error evaluation failed");
    return MFWQ_OK;
}

int mfwq_load_vector(mfwq_handle h, int geometry, int forcing, double* f_dev) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || !f_dev) return fail(MFWQ_EINVAL, "bad argument");
    if (geometry != MFWQ_GEOM_CUBE && geometry != MFWQ_GEOM_RING) return fail(MFWQ_EINVAL, "unknown geometry");
    if (forcing != MFWQ_FORCING_SINES && forcing != MFWQ_FORCING_RING_EXACT) return fail(MFWQ_EINVAL, "unknown forcing");
    return run_load_vector(h->d64, geometry, forcing, static_cast<double*>(h->scratch), f_dev, h->stream);
}

int mfwq_apply(mfwq_handle h, const double* x_dev, double* y_dev) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || !x_dev || !y_dev || x_dev == y_dev) return fail(MFWQ_EINVAL, "bad argument");
    return run_apply<double>(ctx64(h), x_dev, y_dev, nullptr);
}

int mfwq_apply_T(mfwq_handle h, const double* x_dev, double* y_dev) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || !x_dev || !y_dev || x_dev == y_dev) return fail(MFWQ_EINVAL, "bad argument");
    return run_apply_T<double>(ctx64(h), x_dev, y_dev, nullptr);
}

int mfwq_apply_f32(mfwq_handle h, const float* x_dev, float* y_dev) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || !x_dev || !y_dev || x_dev == (const float*)y_dev) return fail(MFWQ_EINVAL, "bad argument");
    if (!h->mixed) return fail(MFWQ_EINVAL, "handle was set up without mixed = 1");
    return run_apply<float>(ctx32(h), x_dev, y_dev, nullptr);
}

int fd_precond(mfwq_handle h, const double* r_dev, double* z_dev) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || !r_dev || !z_dev || r_dev == z_dev) return fail(MFWQ_EINVAL, "bad argument");
    if (h->fd64_path == MFWQ_FD64_SPLIT && h->oz.ok)
        return run_fd_oz(h->oz, r_dev, z_dev, h->fd_tmp64, h->derr, nullptr, h->stream);
    return run_fd64(h->d64, r_dev, z_dev, h->fd_tmp64, nullptr, h->stream);
}

int fd_precond_f32(mfwq_handle h, const float* r_dev, float* z_dev) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || !r_dev || !z_dev || r_dev == (const float*)z_dev) return fail(MFWQ_EINVAL, "bad argument");
    if (!h->mixed) return fail(MFWQ_EINVAL, "handle was set up without mixed = 1");
    return run_fd_tc(h->d32, h->fd_prec, r_dev, z_dev, h->fd_tmp32, h->derr, nullptr, h->stream);
}

int mfwq_solve(mfwq_handle h, const double* f_dev, double* u_dev, const mfwq_solve_opts* opts, mfwq_solve_info* info) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || !f_dev || !u_dev || f_dev == u_dev) return fail(MFWQ_EINVAL, "bad argument");
    mfwq_solve_opts o = opts ? *opts : default_opts();
    if (!(o.rtol > 0) || o.maxit < 0) return fail(MFWQ_EINVAL, "rtol must be > 0 and maxit >= 0");
    if (h->mixed && !o.force_fp64 && !o.fp64_low_fd) return solve_mixed(h, f_dev, u_dev, o, info);
    return solve64(h, f_dev, u_dev, o, info, false);
}

int mfwq_solve_T(mfwq_handle h, const double* g_dev, double* lambda_dev, const mfwq_solve_opts* opts, mfwq_solve_info* info) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || !g_dev || !lambda_dev || g_dev == lambda_dev) return fail(MFWQ_EINVAL, "bad argument");
    mfwq_solve_opts o = opts ? *opts : default_opts();
    if (!(o.rtol > 0) || o.maxit < 0) return fail(MFWQ_EINVAL, "rtol must be > 0 and maxit >= 0");
    return solve64(h, g_dev, lambda_dev, o, info, true);
}

int mfwq_solve_host(mfwq_handle h, const double* f_host, double* u_host, const mfwq_solve_opts* opts, mfwq_solve_info* info) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || !f_host || !u_host) return fail(MFWQ_EINVAL, "bad argument");
    if (!h->host_io) ST(dmalloc((void**)&h->host_io, sizeof(double) * 2 * h->N));
    double* f = h->host_io;
    double* u = h->host_io + h->N;
    CU(cudaMemcpyAsync(f, f_host, sizeof(double) * h->N, cudaMemcpyHostToDevice, h->stream));
    mfwq_solve_opts o = opts ? *opts : default_opts();
    if (o.use_initial_guess) CU(cudaMemcpyAsync(u, u_host, sizeof(double) * h->N, cudaMemcpyHostToDevice, h->stream));
    int st = mfwq_solve(h, f, u, &o, info);
    if (st != MFWQ_OK && st != MFWQ_ENOCONV) return st;
    CU(cudaMemcpyAsync(u_host, u, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return st;
}

int mfwq_grad_coeff(mfwq_handle h, const double* lambda_dev, const double* u_dev, double* gC_dev) {
    ProfScope _ps(h ? &h->prof : nullptr);
    if (!h || !lambda_dev || !u_dev || !gC_dev) return fail(MFWQ_EINVAL, "bad argument");
    return run_grad<double>(ctx64(h), lambda_dev, u_dev, gC_dev);
}

static const char* kStageNames[S_NTAGS] = {
    "trial_z", "trial_y", "xstage", "test_y", "test_z", "test_zT", "test_yT", "xstage_T", "trial_yT", "trial_zT",
    "xstage_grad", "fd_dim1", "fd_dim23", "fd_tc", "krylov", "setup", "fd_fold", "mass", "h1_error", "fused_xy", "fd_oz"};

const char* mfwq_stage_name(int stage) { return stage >= 0 && stage < S_NTAGS ? kStageNames[stage] : ""; }

int mfwq_profile_enable(mfwq_handle h, int on) {
    if (!h) return fail(MFWQ_EINVAL, "NULL handle");
    h->prof.on = on != 0;
    return MFWQ_OK;
}

int mfwq_profile_stage_mask(mfwq_handle h, unsigned long long mask) {
    if (!h) return fail(MFWQ_EINVAL, "NULL handle");
    h->prof.mask = mask;
    return MFWQ_OK;
}

int mfwq_profile_read(mfwq_handle h, mfwq_profile_stats* out, int reset) {
    if (!h || !out) return fail(MFWQ_EINVAL, "bad argument");
    h->prof.drain();
    std::memset(out, 0, sizeof *out);
    for (int i = 0; i < S_NTAGS && i < MFWQ_NSTAGES; ++i) {
        out->ms[i] = h->prof.ms[i];
        out->launches[i] = h->prof.launches[i];
    }
    if (reset) {
        for (int i = 0; i < S_NTAGS; ++i) {
            h->prof.ms[i] = 0.0;
            h->prof.launches[i] = 0;
        }
    }
    return MFWQ_OK;
}

long long mfwq_kernel_launches(void) { return total_launches(); }

int mfwq_set_fp32_path(mfwq_handle h, int path) {
    if (!h) return fail(MFWQ_EINVAL, "NULL handle");
    if (path != MFWQ_PATH_STAGED && path != MFWQ_PATH_FUSED) return fail(MFWQ_EINVAL, "unknown FP32 apply path");
    if (path == MFWQ_PATH_FUSED && !h->mixed) return fail(MFWQ_EINVAL, "handle was set up without mixed = 1");
    if (path == MFWQ_PATH_FUSED && !h->fplan.ok) return fail(MFWQ_EINVAL, "fused FP32 apply unavailable: " + h->fplan.why);
    h->fused32 = path == MFWQ_PATH_FUSED ? 1 : 0;
    return MFWQ_OK;
}

int mfwq_fp32_path(mfwq_handle h) {
    if (!h) return fail(MFWQ_EINVAL, "NULL handle");
    return h->fused32 && h->fplan.ok ? MFWQ_PATH_FUSED : MFWQ_PATH_STAGED;
}

int mfwq_set_fd64_path(mfwq_handle h, int path) {
    if (!h) return fail(MFWQ_EINVAL, "NULL handle");
    if (path != MFWQ_FD64_PIPE && path != MFWQ_FD64_SPLIT) return fail(MFWQ_EINVAL, "unknown FP64 FD path");
    if (path == MFWQ_FD64_SPLIT) ST(split_fd_enable(h));
    h->fd64_path = path;
    return MFWQ_OK;
}

int mfwq_fd64_path(mfwq_handle h) {
    if (!h) return fail(MFWQ_EINVAL, "NULL handle");
    return h->fd64_path == MFWQ_FD64_SPLIT && h->oz.ok ? MFWQ_FD64_SPLIT : MFWQ_FD64_PIPE;
}

int mfwq_set_slow_tiling(mfwq_handle h, int fp32, int rows, int cols) {
    if (!h) return fail(MFWQ_EINVAL, "NULL handle");
    if (fp32 && !h->mixed) return fail(MFWQ_EINVAL, "set_slow_tiling: the handle has no FP32 operator");
    if ((rows != 1 && rows != 2 && rows != 4) || (cols != 1 && cols != 2 && cols != 4) || (!fp32 && cols != 1))
        return fail(MFWQ_EINVAL, "set_slow_tiling: rows 1, 2 or 4; cols 1, 2 or 4 (FP32 only)");
    if (fp32) {
        h->srows32 = rows;
        h->svec32 = cols;
    } else {
        h->srows = rows;
    }
    return MFWQ_OK;
}

int mfwq_slow_tiling(mfwq_handle h, int fp32, int* rows, int* cols) {
    if (!h || !rows || !cols) return fail(MFWQ_EINVAL, "NULL argument");
    *rows = fp32 ? h->srows32 : h->srows;
    *cols = fp32 ? h->svec32 : 1;
    return MFWQ_OK;
}

int mfwq_sync(mfwq_handle h) {
    if (!h) return fail(MFWQ_EINVAL, "NULL handle");
    CU(cudaStreamSynchronize(h->stream));
    CU(cudaGetLastError());
    int err = 0;
    CU(cudaMemcpy(&err, h->derr, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        CU(cudaMemset(h->derr, 0, sizeof(int)));
        return fail(MFWQ_ETIMEOUT, "a bounded device-side wait gave up");
    }
    return MFWQ_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- autotuner
namespace {
std::string tune_key(mfwq_handle h) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "xstage p=%d n1=%d nq1=%d nq2=%d nq3=%d", h->dir[0].p, h->n[0], h->nq[0], h->nq[1], h->nq[2]);
    return buf;
}

// Cache file: one JSON object per line, {"key": "...", "xstage": 10 * mode + lines}.
bool cache_lookup(const char* path, const std::string& key, int* val) {
    if (!path || !*path) return false;
    std::ifstream in(path);
    std::string line;
    const std::string k = "\"key\": \"" + key + "\"";
    while (std::getline(in, line)) {
        if (line.find(k) == std::string::npos) continue;
        size_t p = line.find("\"xstage\":");
        if (p == std::string::npos) continue;
        int v = std::atoi(line.c_str() + p + 9);
        if (v % 10 == 2 || v % 10 == 4 || v % 10 == 8) {
            *val = v;
            return true;
        }
    }
    return false;
}

void cache_store(const char* path, const std::string& key, int val) {
    if (!path || !*path) return;
    std::ofstream out(path, std::ios::app);
    out << "{\"key\": \"" << key << "\", \"xstage\": " << val << "}\n";
}
}  // namespace

namespace {
// Times the forward apply for every (lines, mode) pair in one precision and
// returns the fastest encoded as 10 * mode + lines.
template <typename T>
int tune_xstage(mfwq_handle h, bool f32, int* err) {
    T* x = reinterpret_cast<T*>(f32 ? (void*)h->kv32 : (void*)h->kv64);  // Krylov work vectors as timing buffers
    T* y = x + h->N;
    *err = MFWQ_OK;
    if (cudaMemsetAsync(x, 0, sizeof(T) * h->N, h->stream) != cudaSuccess) { *err = MFWQ_ECUDA; return 4; }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) { *err = MFWQ_ECUDA; return 4; }
    OpCtx<T> c;
    for (int l = 0; l < 3; ++l) c.d[l] = f32 ? *(DirD<T>*)&h->d32[l] : *(DirD<T>*)&h->d64[l];
    c.C = f32 ? (const T*)h->C32 : (const T*)h->C64;
    c.Nq = h->Nq;
    c.cs = h->cs;
    c.err = h->derr;
    c.cm = f32 ? (const T*)h->Cm32 : (const T*)h->Cm64;
    c.cf = f32 && h->onthefly ? &h->cf32 : nullptr;
    c.scratch = static_cast<T*>(h->scratch);
    c.stream = h->stream;
    // one untimed apply, then three timed ones
    auto time_apply = [&]() -> float {
        if (run_apply<T>(c, x, y, nullptr) != MFWQ_OK) { *err = MFWQ_ECUDA; return 1e30f; }
        cudaEventRecord(e0, h->stream);
        for (int r = 0; r < 3; ++r) run_apply<T>(c, x, y, nullptr);
        cudaEventRecord(e1, h->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    // the x stage first (slow stages one row per thread), then the slow stages' rows with that x stage
    float best_ms = 1e30f;
    int best_mode = 0, best_L = 4, best_R = 1, best_carve = 0;
    c.srows = 1;
    for (int carve = 0; carve < 2 && *err == MFWQ_OK; ++carve)
        for (int mode = 0; mode < 7 && *err == MFWQ_OK; ++mode)
            for (int L : {2, 4, 8}) {
                // modes 4-6 fix their lines per block; they are timed once (code digit 8)
                if (mode >= 4 && L != 8) continue;
                const int Lv = mode == 6 ? 8 : L;
                if ((mode < 4 && L > h->max_xlines) || !xstage_mode_valid((int)sizeof(T), h->n[0], h->nq[0], Lv, mode))
                    continue;
                if (mode == 6 && (carve || !(f32 ? h->d32[0].SX.ok : h->d64[0].SX.ok))) continue;
                if (c.cf && (mode != 6 || L != 8)) continue;  // the evaluated coefficient runs the stencil form
                c.xlines = L;
                c.xmode = mode;
                c.xcarve = carve;
                const float ms = time_apply();
                if (*err != MFWQ_OK) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best_mode = mode;
                    best_L = L;
                    best_carve = carve;
                }
            }
    c.xlines = best_L;
    c.xmode = best_mode;
    c.xcarve = best_carve;
    // the slow stages: rows per thread, and for FP32 columns per thread
    int best_V = 1;
    c.svec = 1;
    for (int V : {1, 2, 4}) {
        if (V > 1 && !f32) break;
        for (int R : {1, 2, 4}) {
            if (*err != MFWQ_OK || (V == 1 && R == 1)) continue;
            c.srows = R;
            c.svec = V;
            const float ms = time_apply();
            if (ms < best_ms) {
                best_ms = ms;
                best_R = R;
                best_V = V;
            }
        }
    }
    c.svec = best_V;
    // FP32: the fused trial-y / x / test-y kernel against the staged kernels
    int best_fused = 0;
    if (f32 && h->fplan.ok && !h->Cm32 && *err == MFWQ_OK) {
        c.srows = best_R;
        c.fused = &h->fplan;
        const float ms = time_apply();
        c.fused = nullptr;
        if (ms < best_ms) {
            best_ms = ms;
            best_fused = 1;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) *err = MFWQ_ECUDA;
    return (best_V > 1 ? 100000 * best_V : 0) + 10000 * best_fused + 1000 * best_carve + 100 * best_R + 10 * best_mode +
           best_L;
}
}  // namespace

extern "C" int mfwq_autotune(mfwq_handle h, const char* cache_path, int* xlines_out) {
    if (!h) return fail(MFWQ_EINVAL, "NULL handle");
    ProfScope _ps(nullptr);
    for (int prec = 0; prec < (h->mixed ? 2 : 1); ++prec) {
        const std::string key = tune_key(h) + (prec ? " fp32" : " fp64");
        int code = 0;
        if (!cache_lookup(cache_path, key, &code)) {
            int err = MFWQ_OK;
            code = prec ? tune_xstage<float>(h, true, &err) : tune_xstage<double>(h, false, &err);
            if (err != MFWQ_OK) return fail(err, "autotune: a timing launch failed");
            cache_store(cache_path, key, code);
        }
        int L = code % 10, mode = (code / 10) % 10, R = (code / 100) % 10, carve = (code / 1000) % 10 ? 1 : 0;
        const int fused = (code / 10000) % 10 ? 1 : 0;
        int V = (code / 100000) % 10;
        if (V != 2 && V != 4) V = 1;
        if (mode < 4 && L > h->max_xlines) L = h->max_xlines;
        if (R != 2 && R != 4) R = 1;
        if (prec) {
            h->fused32 = fused && h->fplan.ok ? 1 : 0;
            h->xlines32 = L;
            h->xmode32 = mode;
            h->srows32 = R;
            h->svec32 = V;
            h->xcarve32 = carve;
        } else {
            h->xlines = L;
            h->xmode = mode;
            h->srows = R;
            h->xcarve = carve;
        }
    }
    if (xlines_out) *xlines_out = 1000 * h->xcarve + 100 * h->srows + 10 * h->xmode + h->xlines;
    return MFWQ_OK;
}

// ---------------------------------------------------------------- batched solve
struct mfwq_batch_s {
    int grouped = 0;       // 1: FP64 sweeps as grouped launches where the patches allow it
    int groups = 4;        // concurrent groups (streams) of the grouped sweep
    int last_grouped = 0;  // the last FP64 solve ran grouped sweeps
    std::vector<mfwq_handle> h;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr;
    KScal* dsc = nullptr;
    KScal* hsc = nullptr;
};

namespace {
void free_batch(mfwq_batch b) {
    if (!b) return;
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    if (b->origin) cudaStreamDestroy(b->origin);
    if (b->fork) cudaEventDestroy(b->fork);
    cudaFree(b->dsc);
    if (b->hsc) cudaFreeHost(b->hsc);
    delete b;
}

// Operators of patch i on the batch's stream i.
struct PatchOps {
    LinOp<double> A, P;
};
PatchOps patch_ops(mfwq_handle h, cudaStream_t s) {
    OpCtx<double> c = ctx64(h);
    c.stream = s;
    PatchOps o;
    o.A = [c](const double* in, double* out, const int* skip) { return run_apply<double>(c, in, out, skip); };
    o.P = fd64_linop(h, s);
    return o;
}
}  // namespace

extern "C" int mfwq_batch_create(int count, const mfwq_handle* patches, mfwq_batch* out) {
    if (count < 1 || !patches || !out) return fail(MFWQ_EINVAL, "bad argument");
    *out = nullptr;
    mfwq_batch b = new (std::nothrow) mfwq_batch_s();
    if (!b) return fail(MFWQ_ENOMEM, "host allocation failed");
    int st = MFWQ_OK;
    for (int i = 0; i < count && st == MFWQ_OK; ++i) {
        if (!patches[i]) st = fail(MFWQ_EINVAL, "NULL patch handle");
        b->h.push_back(patches[i]);
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        if (st == MFWQ_OK && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) st = fail(MFWQ_ECUDA, "stream");
        if (st == MFWQ_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) st = fail(MFWQ_ECUDA, "event");
        if (s) b->streams.push_back(s);
        if (e) b->join.push_back(e);
    }
    if (st == MFWQ_OK && cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess) st = fail(MFWQ_ECUDA, "stream");
    if (st == MFWQ_OK && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) st = fail(MFWQ_ECUDA, "event");
    if (st == MFWQ_OK) st = dmalloc((void**)&b->dsc, sizeof(KScal) * count);
    if (st == MFWQ_OK && cudaMallocHost((void**)&b->hsc, sizeof(KScal) * count) != cudaSuccess) st = fail(MFWQ_ENOMEM, "pinned");
    if (st != MFWQ_OK) {
        cudaGetLastError();
        free_batch(b);
        return st;
    }
    *out = b;
    return MFWQ_OK;
}

extern "C" int mfwq_batch_set_grouped(mfwq_batch b, int grouped) {
    if (!b || grouped < 0) return fail(MFWQ_EINVAL, "bad argument");
    b->grouped = grouped ? 1 : 0;
    if (grouped > 0) b->groups = grouped;
    return MFWQ_OK;
}

extern "C" int mfwq_batch_last_grouped(mfwq_batch b) {
    if (!b) return fail(MFWQ_EINVAL, "NULL batch");
    return b->last_grouped;
}

extern "C" void mfwq_batch_destroy(mfwq_batch b) {
    if (b && b->origin) cudaStreamSynchronize(b->origin);
    free_batch(b);
}

namespace {
// Captures one BiCGStab iteration of the listed patches (each on its own
// stream, forked from and joined to the batch's origin stream) into a graph.
template <typename T>
int capture_sweep(mfwq_batch b, const std::vector<int>& list, const std::vector<LinOp<T>>& A, const std::vector<LinOp<T>>& P,
                  const std::vector<const T*>& f, const std::vector<T*>& x, const std::vector<KrylovBufs<T>>& bufs,
                  cudaGraphExec_t* exec) {
    cudaGraph_t graph = nullptr;
    *exec = nullptr;
    CU(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
    int cst = MFWQ_OK;
    if (cudaEventRecord(b->fork, b->origin) != cudaSuccess) cst = MFWQ_ECUDA;
    for (int i : list) {
        if (cst != MFWQ_OK) break;
        mfwq_handle h = b->h[i];
        if (cudaStreamWaitEvent(b->streams[i], b->fork, 0) != cudaSuccess) cst = MFWQ_ECUDA;
        if (cst == MFWQ_OK)
            cst = krylov_enqueue_iter<T>(A[i], P[i], f[i], x[i], bufs[i], &b->dsc[i], h->part, h->N, b->streams[i]);
        if (cst == MFWQ_OK && cudaEventRecord(b->join[i], b->streams[i]) != cudaSuccess) cst = MFWQ_ECUDA;
        if (cst == MFWQ_OK && cudaStreamWaitEvent(b->origin, b->join[i], 0) != cudaSuccess) cst = MFWQ_ECUDA;
    }
    cudaError_t ce = cudaStreamEndCapture(b->origin, &graph);
    if (cst != MFWQ_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(MFWQ_ECUDA, "capture of the batched iteration failed");
    }
    cudaError_t ie = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        cudaGetLastError();
        return fail(MFWQ_ECUDA, "cudaGraphInstantiate failed");
    }
    return MFWQ_OK;
}

// Runs sweeps of a captured iteration until every listed patch is done or
// maxit sweeps ran; returns the number of sweeps.
int run_sweeps(mfwq_batch b, const std::vector<int>& list, cudaGraphExec_t exec, int maxit, int* sweeps) {
    const int count = (int)b->h.size();
    *sweeps = 0;
    for (int k = 0; k < maxit; ++k) {
        CU(cudaGraphLaunch(exec, b->origin));
        CU(cudaMemcpyAsync(b->hsc, b->dsc, sizeof(KScal) * count, cudaMemcpyDeviceToHost, b->origin));
        CU(cudaStreamSynchronize(b->origin));
        *sweeps = k + 1;
        bool done = true;
        for (int i : list)
            if (!b->hsc[i].skip1) done = false;
        if (done) break;
    }
    return MFWQ_OK;
}

// Mixed form: FP64 refinement steps in lockstep over the patches still above
// rtol; each inner FP32 BiCGStab (FP32 operator, tensor-core FD) runs for all
// of them together, one graph launch per sweep.
int batch_solve_mixed(mfwq_batch b, const double* const* f_dev, double* const* u_dev, const mfwq_solve_opts& o,
                      mfwq_solve_info* infos) {
    const int count = (int)b->h.size();
    for (int i = 0; i < count; ++i)
        if (!b->h[i]->mixed) return fail(MFWQ_EINVAL, "every patch of a mixed batch solve needs mixed = 1");
    const double inner_rtol = o.inner_rtol > 0 ? o.inner_rtol : 1e-4;
    const int inner_maxit = o.inner_maxit > 0 ? o.inner_maxit : 200;
    std::vector<LinOp<float>> A(count), P(count);
    std::vector<const float*> r32(count);
    std::vector<float*> d32(count);
    std::vector<KrylovBufs<float>> bufs(count);
    for (int i = 0; i < count; ++i) {
        mfwq_handle h = b->h[i];
        OpCtx<float> c = ctx32(h);
        c.stream = b->streams[i];
        DirD<float> d[3] = {h->d32[0], h->d32[1], h->d32[2]};
        float* tmp = h->fd_tmp32;
        int* err = h->derr;
        const int prec = h->fd_prec;
        cudaStream_t s = b->streams[i];
        A[i] = [c](const float* in, float* out, const int* skip) { return run_apply<float>(c, in, out, skip); };
        P[i] = [d, tmp, s, err, prec](const float* in, float* out, const int* skip) {
            return run_fd_tc(d, prec, in, out, tmp, err, skip, s);
        };
        r32[i] = h->kv32 + 8 * h->N;
        d32[i] = h->kv32 + 9 * h->N;
        bufs[i] = bufs32(h);
    }
    std::vector<int> active(count), status(count, MFWQ_ENOCONV), outer(count, 0), inner(count, 0);
    std::vector<double> rel(count, 1.0);
    for (int i = 0; i < count; ++i) active[i] = i;
    for (int k = 0;; ++k) {
        // FP64 residuals (the first one is f when u starts at zero)
        for (int i : active) {
            mfwq_handle h = b->h[i];
            cudaStream_t s = b->streams[i];
            OpCtx<double> c = ctx64(h);
            c.stream = s;
            double* w64 = h->kv64;
            double* r64 = h->kv64 + h->N;
            if (k == 0 && !o.use_initial_guess) {
                CU(cudaMemsetAsync(u_dev[i], 0, sizeof(double) * h->N, s));
                CU(cudaMemcpyAsync(r64, f_dev[i], sizeof(double) * h->N, cudaMemcpyDeviceToDevice, s));
            } else {
                ST(run_apply<double>(c, u_dev[i], w64, nullptr));
                ST(axpby_into<double>(f_dev[i], w64, r64, h->N, s));
            }
            ST(norm2_into(r64, h->N, h->part, h->dnorm, s));
            if (k == 0) ST(norm2_into(f_dev[i], h->N, h->part, h->dnorm + 1, s));
            CU(cudaMemcpyAsync(h->hnorm, h->dnorm, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        }
        std::vector<int> next;
        for (int i : active) {
            mfwq_handle h = b->h[i];
            CU(cudaStreamSynchronize(b->streams[i]));
            const double r2 = h->hnorm[0], f2 = h->hnorm[1];
            if (!std::isfinite(r2)) {
                status[i] = MFWQ_ENAN;
                continue;
            }
            rel[i] = f2 > 0 ? std::sqrt(r2 / f2) : 0.0;
            if (f2 == 0.0 || rel[i] <= o.rtol) {
                status[i] = MFWQ_OK;
                continue;
            }
            if (outer[i] >= o.maxit) continue;
            next.push_back(i);
        }
        active = next;
        if (active.empty()) break;
        // inner solves of the active patches
        CU(cudaEventRecord(b->fork, b->origin));
        for (int i : active) {
            mfwq_handle h = b->h[i];
            cudaStream_t s = b->streams[i];
            CU(cudaStreamWaitEvent(s, b->fork, 0));
            ST(to_f32_scaled(h->kv64 + h->N, h->dnorm, const_cast<float*>(r32[i]), h->N, s));
            ST(krylov_enqueue_init<float>(A[i], r32[i], d32[i], false, inner_rtol, bufs[i], &b->dsc[i], h->part, h->N, s));
            CU(cudaEventRecord(b->join[i], s));
            CU(cudaStreamWaitEvent(b->origin, b->join[i], 0));
        }
        CU(cudaMemcpyAsync(b->hsc, b->dsc, sizeof(KScal) * count, cudaMemcpyDeviceToHost, b->origin));
        CU(cudaStreamSynchronize(b->origin));
        cudaGraphExec_t exec = nullptr;
        ST(capture_sweep<float>(b, active, A, P, r32, d32, bufs, &exec));
        int sweeps = 0;
        int st = run_sweeps(b, active, exec, inner_maxit, &sweeps);
        cudaGraphExecDestroy(exec);
        if (st != MFWQ_OK) return st;
        for (int i : active) {
            mfwq_handle h = b->h[i];
            inner[i] += b->hsc[i].iters;
            if (b->hsc[i].status == MFWQ_ENAN) {
                status[i] = MFWQ_ENAN;
                continue;
            }
            ST(add_f32_scaled(u_dev[i], d32[i], h->dnorm, h->N, b->streams[i]));
            ++outer[i];
        }
        std::vector<int> keep;
        for (int i : active)
            if (status[i] != MFWQ_ENAN) keep.push_back(i);
        active = keep;
        if (active.empty()) break;
    }
    int worst = MFWQ_OK;
    for (int i = 0; i < count; ++i) {
        CU(cudaStreamSynchronize(b->streams[i]));
        if (infos) {
            infos[i].status = status[i];
            infos[i].iterations = inner[i];
            infos[i].outer_iterations = outer[i];
            infos[i].rel_residual = rel[i];
        }
        if (status[i] != MFWQ_OK && worst == MFWQ_OK) worst = status[i];
    }
    return worst;
}
}  // namespace

namespace {
// One BiCGStab iteration of every patch as grouped launches: each patch's
// iteration is recorded (the kernels a separate solve launches, with its
// arguments), stage k of all patches becomes one launch over a device table.
// Returns MFWQ_OK with *exec = NULL when the patches' sequences differ or a
// kernel has no grouped form (the caller then captures per-patch streams).
struct GroupedSweep {
    void* dmem = nullptr;
    cudaGraphExec_t exec = nullptr;
    int stages = 0;
    ~GroupedSweep() {
        if (exec) cudaGraphExecDestroy(exec);
        if (dmem) cudaFree(dmem);
    }
};

int build_grouped_sweep(mfwq_batch b, const std::vector<PatchOps>& ops, const double* const* f_dev,
                        double* const* u_dev, GroupedSweep& gs) {
    const int count = (int)b->h.size();
    std::vector<Recorder> rec(count);
    for (int i = 0; i < count; ++i) {
        mfwq_handle h = b->h[i];
        RecScope rs(&rec[i]);
        const int st = krylov_enqueue_iter<double>(ops[i].A, ops[i].P, f_dev[i], u_dev[i], bufs64(h), &b->dsc[i],
                                                   h->part, h->N, b->streams[i]);
        if (st != MFWQ_OK || rec[i].unsupported) return MFWQ_OK;
    }
    const size_t nst = rec[0].recs.size();
    for (int i = 1; i < count; ++i) {
        if (rec[i].recs.size() != nst) return MFWQ_OK;
        for (size_t k = 0; k < nst; ++k)
            if (rec[i].recs[k].kind != rec[0].recs[k].kind || rec[i].recs[k].threads != rec[0].recs[k].threads)
                return MFWQ_OK;
    }
    // groups of patches (largest first, each to the group with the least work), one stream each
    const int G = std::max(1, std::min(b->groups, count));
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return b->h[x]->N > b->h[y]->N; });
    std::vector<std::vector<int>> grp(G);
    std::vector<double> load(G, 0.0);
    for (int i : order) {
        const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        grp[g].push_back(i);
        load[g] += (double)b->h[i]->N;
    }
    // tables: stage k of group g at off[g][k], slots of stride[k] bytes
    std::vector<int> stride(nst), smem(nst);
    for (size_t k = 0; k < nst; ++k) {
        size_t amax = 0;
        int sm = 0;
        for (int i = 0; i < count; ++i) {
            amax = std::max(amax, rec[i].recs[k].args.size());
            sm = std::max(sm, rec[i].recs[k].smem);
        }
        stride[k] = (int)((kSlotHeader + amax + 15) / 16 * 16);
        smem[k] = sm;
    }
    std::vector<std::vector<size_t>> off(G, std::vector<size_t>(nst));
    std::vector<std::vector<int>> grid(G, std::vector<int>(nst));
    size_t total = 0;
    for (int g = 0; g < G; ++g)
        for (size_t k = 0; k < nst; ++k) {
            long long items = 0;
            for (int i : grp[g]) items += rec[i].recs[k].items;
            grid[g][k] = (int)std::max<long long>(1, std::min<long long>(items, 152LL * 32 / G + 1));
            off[g][k] = total;
            total = (total + (size_t)stride[k] * grp[g].size() + 255) / 256 * 256;
        }
    std::vector<unsigned char> host(total, 0);
    for (int g = 0; g < G; ++g)
        for (size_t k = 0; k < nst; ++k)
            for (size_t q = 0; q < grp[g].size(); ++q) {
                const LaunchRec& r = rec[grp[g][q]].recs[k];
                unsigned char* slot = host.data() + off[g][k] + (size_t)stride[k] * q;
                std::memcpy(slot, &r.items, sizeof(int));
                std::memcpy(slot + 8, &r.skip, sizeof(const int*));
                std::memcpy(slot + kSlotHeader, r.args.data(), r.args.size());
            }
    ST(dmalloc(&gs.dmem, total));
    CU(cudaMemcpy(gs.dmem, host.data(), total, cudaMemcpyHostToDevice));
    int smax = 0;
    for (size_t k = 0; k < nst; ++k) smax = std::max(smax, smem[k]);
    if (smax > 48 * 1024) ST(configure_grouped_smem(smax));
    cudaGraph_t graph = nullptr;
    CU(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
    bool ok = cudaEventRecord(b->fork, b->origin) == cudaSuccess;
    for (int g = 0; g < G && ok; ++g) {
        cudaStream_t sg = b->streams[g];
        ok = cudaStreamWaitEvent(sg, b->fork, 0) == cudaSuccess;
        for (size_t k = 0; k < nst && ok; ++k) {
            const unsigned char* tab = static_cast<const unsigned char*>(gs.dmem) + off[g][k];
            const int kind = rec[0].recs[k].kind, n = (int)grp[g].size();
            ok = grouped_launch_krylov(kind, tab, stride[k], n, grid[g][k], smem[k], sg) ||
                 grouped_launch_fd(kind, tab, stride[k], n, grid[g][k], smem[k], sg) ||
                 grouped_launch_apply(kind, tab, stride[k], n, grid[g][k], smem[k], sg) ||
                 grouped_launch_xstage(kind, tab, stride[k], n, grid[g][k], smem[k], sg) ||
                 grouped_launch_oz(kind, tab, stride[k], n, grid[g][k], smem[k], sg);
        }
        if (ok) ok = cudaEventRecord(b->join[g], sg) == cudaSuccess && cudaStreamWaitEvent(b->origin, b->join[g], 0) == cudaSuccess;
    }
    cudaError_t ce = cudaStreamEndCapture(b->origin, &graph);
    if (!ok || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(MFWQ_ECUDA, "capture of the grouped sweep failed");
    }
    cudaError_t ie = cudaGraphInstantiate(&gs.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        gs.exec = nullptr;
        cudaGetLastError();
        return fail(MFWQ_ECUDA, "cudaGraphInstantiate of the grouped sweep failed");
    }
    gs.stages = (int)nst;
    return MFWQ_OK;
}
}  // namespace

extern "C" int mfwq_batch_solve(mfwq_batch b, const double* const* f_dev, double* const* u_dev, const mfwq_solve_opts* opts,
                                mfwq_solve_info* infos) {
    if (!b || !f_dev || !u_dev) return fail(MFWQ_EINVAL, "bad argument");
    ProfScope _ps(nullptr);
    const int count = (int)b->h.size();
    mfwq_solve_opts o = opts ? *opts : default_opts();
    if (!(o.rtol > 0) || o.maxit < 0) return fail(MFWQ_EINVAL, "rtol must be > 0 and maxit >= 0");
    if (o.fp64_low_fd) return fail(MFWQ_EINVAL, "fp64_low_fd is for single-patch solves");
    for (int i = 0; i < count; ++i)
        if (!f_dev[i] || !u_dev[i] || f_dev[i] == u_dev[i]) return fail(MFWQ_EINVAL, "bad patch vectors");
    if (!o.force_fp64) {
        bool all_mixed = true;
        for (int i = 0; i < count; ++i) all_mixed = all_mixed && b->h[i]->mixed;
        if (all_mixed) return batch_solve_mixed(b, f_dev, u_dev, o, infos);
    }
    std::vector<PatchOps> ops;
    for (int i = 0; i < count; ++i) ops.push_back(patch_ops(b->h[i], b->streams[i]));
    // initial residuals, every patch on its own stream
    CU(cudaEventRecord(b->fork, b->origin));
    for (int i = 0; i < count; ++i) {
        mfwq_handle h = b->h[i];
        CU(cudaStreamWaitEvent(b->streams[i], b->fork, 0));
        ST(krylov_enqueue_init<double>(ops[i].A, f_dev[i], u_dev[i], o.use_initial_guess != 0, o.rtol, bufs64(h), &b->dsc[i],
                                       h->part, h->N, b->streams[i]));
        CU(cudaEventRecord(b->join[i], b->streams[i]));
        CU(cudaStreamWaitEvent(b->origin, b->join[i], 0));
    }
    CU(cudaMemcpyAsync(b->hsc, b->dsc, sizeof(KScal) * count, cudaMemcpyDeviceToHost, b->origin));
    CU(cudaStreamSynchronize(b->origin));
    auto all_done = [&]() {
        for (int i = 0; i < count; ++i)
            if (!b->hsc[i].skip1) return false;
        return true;
    };
    int sweeps = 0;
    GroupedSweep gs;
    if (!all_done() && o.maxit > 0 && b->grouped && count <= 1024) ST(build_grouped_sweep(b, ops, f_dev, u_dev, gs));
    b->last_grouped = gs.exec ? 1 : 0;
    if (!all_done() && o.maxit > 0 && gs.exec) {
        // the grouped sweep: one launch per stage over every patch, one stream
        int st = MFWQ_OK;
        for (sweeps = 0; sweeps < o.maxit; ++sweeps) {
            if (cudaGraphLaunch(gs.exec, b->origin) != cudaSuccess ||
                cudaMemcpyAsync(b->hsc, b->dsc, sizeof(KScal) * count, cudaMemcpyDeviceToHost, b->origin) != cudaSuccess ||
                cudaStreamSynchronize(b->origin) != cudaSuccess) {
                st = fail(MFWQ_ECUDA, "grouped sweep failed");
                break;
            }
            if (all_done()) {
                ++sweeps;
                break;
            }
        }
        if (st != MFWQ_OK) return st;
    } else if (!all_done() && o.maxit > 0) {
        // one BiCGStab iteration of every patch, captured once into a graph
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        CU(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
        int cst = MFWQ_OK;
        if (cudaEventRecord(b->fork, b->origin) != cudaSuccess) cst = MFWQ_ECUDA;
        for (int i = 0; i < count && cst == MFWQ_OK; ++i) {
            mfwq_handle h = b->h[i];
            if (cudaStreamWaitEvent(b->streams[i], b->fork, 0) != cudaSuccess) cst = MFWQ_ECUDA;
            if (cst == MFWQ_OK)
                cst = krylov_enqueue_iter<double>(ops[i].A, ops[i].P, f_dev[i], u_dev[i], bufs64(h), &b->dsc[i], h->part, h->N,
                                                  b->streams[i]);
            if (cst == MFWQ_OK && cudaEventRecord(b->join[i], b->streams[i]) != cudaSuccess) cst = MFWQ_ECUDA;
            if (cst == MFWQ_OK && cudaStreamWaitEvent(b->origin, b->join[i], 0) != cudaSuccess) cst = MFWQ_ECUDA;
        }
        cudaError_t ce = cudaStreamEndCapture(b->origin, &graph);
        if (cst != MFWQ_OK || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return fail(MFWQ_ECUDA, "capture of the batched iteration failed");
        }
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
            cudaGraphDestroy(graph);
            cudaGetLastError();
            return fail(MFWQ_ECUDA, "cudaGraphInstantiate failed");
        }
        int st = MFWQ_OK;
        for (sweeps = 0; sweeps < o.maxit; ++sweeps) {
            if (cudaGraphLaunch(exec, b->origin) != cudaSuccess ||
                cudaMemcpyAsync(b->hsc, b->dsc, sizeof(KScal) * count, cudaMemcpyDeviceToHost, b->origin) != cudaSuccess ||
                cudaStreamSynchronize(b->origin) != cudaSuccess) {
                st = fail(MFWQ_ECUDA, "batched sweep failed");
                break;
            }
            if (all_done()) {
                ++sweeps;
                break;
            }
        }
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        if (st != MFWQ_OK) return st;
    }
    int worst = MFWQ_OK;
    for (int i = 0; i < count; ++i) {
        int it = 0, status = MFWQ_OK;
        double rel = 0.0;
        krylov_result(b->hsc[i], &it, &rel, &status);
        if (infos) {
            infos[i].status = status;
            infos[i].iterations = it;
            infos[i].outer_iterations = sweeps;
            infos[i].rel_residual = rel;
        }
        if (status != MFWQ_OK && worst == MFWQ_OK) worst = status;
    }
    return worst;
}
