// Types and helpers shared by the operator kernels (apply_kernels.cu) and the
// forward x-stage kernels (xstage_kernels.cu).  Internal to the library.
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"

namespace mfwq {

constexpr int kThreads = 256;

__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T>
struct Ptr9 {
    T* p[9];
};

// Everything an x-stage kernel needs: direction-1 tables, sizes, coefficient.
template <typename T>
struct XArgs {
    BandD<T> B;    // rows q1 -> j1
    BandD<T> BT;   // rows j1 -> q1
    BandD<T> W;    // rows i1 -> q1
    BandD<T> WT;   // rows q1 -> i1
    TileD<T> BX;   // B in two-point tiles (tiled mapping)
    TileD<T> WX;   // W in two-output tiles (tiled mapping)
    int n1, nq1, nlines;
    int wnb;       // W rows at each end with a band length other than the middle row's
    const int* qord;  // points by decreasing W^T band length (the transposed and gradient x stages)
    const int* jord;  // DoFs by decreasing B^T band length
    size_t cs;     // element stride between the coefficient fields of C
    size_t gs;     // element stride between the fields of the gradient output
    const T* C;    // [6][cs], the first Nq of each field used
};

constexpr int kLines = 4;

template <typename T>
XArgs<T> xargs(const DirD<T>& d1, int nlines, size_t cs, const T* C) {
    XArgs<T> a;
    a.B = d1.B;
    a.BT = d1.BT;
    a.W = d1.W;
    a.WT = d1.WT;
    a.BX = d1.BX;
    a.WX = d1.WX;
    a.n1 = d1.n;
    a.nq1 = d1.nq;
    a.nlines = nlines;
    a.wnb = d1.wnb;
    a.qord = d1.qord;
    a.jord = d1.jord;
    a.cs = cs;
    a.gs = 0;
    a.C = C;
    return a;
}

// The forward x stage of Algorithm 2 (xstage_kernels.cu): T^(ab) for all
// (q3, q2) lines, in the launch shape c.xmode / c.xlines (falling back to
// mapping 0 when that shape does not fit these sizes).
template <typename T>
cudaError_t launch_forward_xstage(const OpCtx<T>& c, const XArgs<T>& a, const T* y0, const T* y1, const T* y2,
                                  T* tout, size_t tstride, const int* skip);

// Raises the dynamic shared-memory limit of every forward x-stage kernel.
cudaError_t configure_forward_xstage_smem(int bytes);

}  // namespace mfwq
