// Internal declarations of the MF-WQ library (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mfwq.h"

#ifdef __CUDACC__
#define MFWQ_HD __host__ __device__
#else
#define MFWQ_HD
#endif

namespace mfwq {

constexpr int kMaxDegree = 12;

// One direction's 1D data (Section 2.2 and Algorithm 2's setup), host side.
// Bands store, for every row, the first column and the number of columns that
// may be nonzero; values are padded to the band width with zeros.
struct Band1D {
    int rows = 0, cols = 0, width = 0, fams = 0;
    std::vector<int> start, len;
    std::vector<double> val;  // [fams][rows][width]
    double& at(int f, int r, int t) { return val[((size_t)f * rows + r) * width + t]; }
    double at(int f, int r, int t) const { return val[((size_t)f * rows + r) * width + t]; }
};

struct Dir1D {
    int p = 0, nel = 0, m = 0, n = 0, nq = 0, ng = 0;
    std::vector<double> t;      // knots
    std::vector<double> xq;     // WQ points
    std::vector<double> xg, wg; // Gauss points / weights (p+1 per span), load vector
    Band1D B;    // rows q -> interior columns j, fams: 0 = values, 1 = derivatives
    Band1D BT;   // rows j -> points q, transposed B
    Band1D W;    // rows i -> points q, fams f = 2a+b
    Band1D WT;   // rows q -> rows i, transposed W
    Band1D GT;   // rows j -> Gauss points g, value b_j(x_g) * w_g
    std::vector<double> xe, we;  // error rule: Gauss, p+2 points per span
    int ne = 0;
    Band1D E;    // rows e (error points) -> columns j, fams: 0 = values, 1 = derivatives
    std::vector<double> U, UT, lam;  // FD: U [n][n] row-major, UT = U^T, lam[n]
    // FD even/odd split (knots symmetric about 1/2): he = n - n/2 even and
    // ho = n/2 odd modes; Ve [he][he], Vo [ho][ho] act on the folded vector
    // (x_j + x_{n-1-j}, middle; x_j - x_{n-1-j}); lam_split = (lam_even, lam_odd).
    bool sym = false;
    int he = 0, ho = 0;
    std::vector<double> Ve, VeT, Vo, VoT, lam_split;
};

// Host setup (setup_host.cpp).  Return MFWQ_* codes; `why` gets a message.
int validate_knots(int p, int nknots, const double* knots, std::string& why);
int build_dir(int p, int nknots, const double* knots, Dir1D& d, std::string& why);

// Device view of a band (values of type T).
template <typename T>
struct BandD {
    const int* start;
    const int* len;
    const T* val;      // [fams][rows][width]: a row's values contiguous (one row per block)
    const T* valT;     // [fams][width][rows]: the same values lane-major (consecutive rows per warp)
    int rows, width;
    MFWQ_HD const T* row(int f, int r) const {
        return val + ((size_t)f * rows + r) * width;
    }
    // value t of row r, family f, from the lane-major copy
    MFWQ_HD T lane(int f, int r, int t) const { return valT[((size_t)f * width + t) * rows + r]; }
};

// A band regrouped into tiles of two consecutive rows (rows 2k, 2k+1): tile
// k covers columns start[k] .. start[k] + len[k] - 1, the union of its rows'
// bands, and val holds both rows' values on that window, zero outside a
// row's own band: [fams][width][ntile][2], width = max len.
template <typename T>
struct TileD {
    const int* start;
    const int* len;
    const T* val;
    int ntile, width;
    // the two rows' values at window offset u of tile k, family f
    MFWQ_HD const T* pair(int f, int u, int k) const { return val + (((size_t)f * width + u) * ntile + k) * 2; }
};

// Translation-invariant interior of a direction's B and W bands (uniform
// knots): interior points q_lo <= q < q_hi come in pairs q_lo + 2k + phase
// whose rows are the phase's representative row shifted by k columns;
// interior outputs i_lo <= i < i_hi are the representative W row shifted by
// 2 points per output.  Filters are zero-padded to the fixed tap counts
// P + 2 (a pair's union window) and 2P + 1; the host guarantees that every
// fixed-size window stays inside the band's columns.
constexpr int kStencilMaxP = 8;

template <typename T>
struct StencilD {
    int ok;               // 1: the tables below are valid for degree P
    int P;
    int q_lo, q_hi;       // interior points, an even count
    int jb;               // first column of pair 0's union window
    int i_lo, i_hi;       // interior outputs
    int qw;               // first point of output i_lo's window
    T bf[2][2][kStencilMaxP + 2];  // [family][phase][t] on the pair's union window
    T wf[4][2 * kStencilMaxP + 1];  // [family][t]
};

template <typename T>
struct DirD {
    int n, nq, ng;
    BandD<T> B, BT, W, WT, GT;
    BandD<T> E;       // B-spline values and derivatives at the error points
    TileD<T> BX, WX;  // B and W in two-row tiles (the tiled x stage)
    StencilD<T> SX;   // translation-invariant interior of B and W (the stencil x stage)
    int wnb;          // W rows at each end whose band length differs from the middle row's (0: none split off)
    const int* qord;  // points q by decreasing length of their W^T band (ties in parity order): [nq]
    const int* jord;  // DoFs j by decreasing length of their B^T band (ties in index order): [n]
    int ne;           // error points
    const double* xe; // error points and weights (always FP64)
    const double* we;
    const T* U;     // [n][n]
    const T* UT;    // [n][n]
    const T* lam;   // [n]
    int sym, he, ho;   // FD even/odd split (FP64 only)
    const double* Ve;
    const double* VeT;
    const double* Vo;
    const double* VoT;
    const double* lam_split;
    const double* xq;  // points (always FP64)
    const double* xg;  // Gauss points (always FP64)
};

}  // namespace mfwq
