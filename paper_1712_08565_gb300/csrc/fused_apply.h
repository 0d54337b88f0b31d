// Fused FP32 apply of Algorithm 2 (internal): the trial y contraction, the
// x stage and the test y contraction in one kernel per (q3 plane, segment of
// q2 lines), so that the trial partials Y and the nine test partials T stay
// in shared memory.  Host plan and launcher.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "kernels.h"

namespace mfwq {

constexpr int kFusedLines = 8;    // q2 lines per batch (the stencil x stage's 8 lines)
constexpr int kFusedThreads = 256;

// Per-direction-2 plan of the fused apply, the same for every q3 plane.
// Batches are 8 consecutive q2 lines; a segment is a run of batches that one
// block sweeps.  Rows are held in rings (row r in slot r mod R).
struct FusedPlan {
    int ok = 0;
    std::string why;           // reason when ok = 0
    int P = 0;                 // stencil degree of direction 1
    int nbatch = 0, S = 0;     // batches per plane, segments per plane
    int KZ = 0, KU = 0;        // table widths: Z rows a batch reads, U rows it touches (kernel bounds P + 6)
    int RZ = 0, RU = 0;        // ring sizes (rows)
    int rY = 0, rG = 0, rT = 0;  // shared-memory row strides
    int smem = 0;              // dynamic shared memory per block
    int smem_onf = 0;          // the same with the coefficient evaluated in the block (CoeffField)
    int grid = 0;              // blocks per launch
    int nstraddle = 0;         // U rows that cross a segment boundary
    int nuniform = 0;          // batches that run the stencil taps of direction 2
    int phi = 0, psi = 0;      // their phases
    // device tables (one allocation, owned by the handle)
    void* dmem = nullptr;
    const int* batch = nullptr;   // [nbatch][8]: q2b, nl, zlo, zhi, ulo, uhi, rlo, rhi
    const float* Bd = nullptr;    // [nbatch][2][8][KZ]: B2 value/derivative rows of the batch's points on Z rows zlo..
    const float* Wd = nullptr;    // [nbatch][4][8][KU]: W2 families on the batch's points for U rows ulo..
    const int* fp = nullptr;      // [n2]: first point of U row i's weight band
    const int* lp = nullptr;      // [n2]: last point
    const int* seg = nullptr;     // [S][2]: first batch, end batch
    const int* straddle = nullptr;  // [nstraddle]
};

// Builds the plan for the FP32 operator of a patch (direction-2 tables d2,
// direction-1 stencil S1 and sizes); ok = 0 (with why) when the fused form
// does not apply.  Allocates the device tables.
int fused_plan_build(const Dir1D& d1, const Dir1D& d2, const StencilD<float>& S1, const StencilD<float>& S2, int nq3,
                     FusedPlan& plan);
void fused_plan_free(FusedPlan& plan);

// The fused stage: Z0, Z1 ([nq3][n2][n1], the trial z output) -> U_g
// ([nq3][n2][n1] at u + g * us, g = 2 a3 + b3 the z family), i.e. the trial y
// contraction, the x stage (direction-1 stencil form) and the test y
// contraction.  Zeroes the straddling U rows first (a second, small launch).
cudaError_t launch_fused(const OpCtx<float>& c, const FusedPlan& plan, const float* z0, const float* z1, float* u,
                         size_t us, const int* skip);
int configure_fused_smem(int bytes);

}  // namespace mfwq
