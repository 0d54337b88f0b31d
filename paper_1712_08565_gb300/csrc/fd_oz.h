// FP64-accurate FD preconditioner on the BF16 tensor cores by operand
// splitting (internal).  The six mode products of the FD method (Section 4)
// run as in fd_tc.cu (one rotation pass per product), with every FP64 operand
// split into kOzSlices integer slices of kOzBits bits under a power-of-two
// scale per row, after the error-free splitting of Ozaki, Ogita, Oishi and
// Rump (Numer. Algorithms 59, 2012).  Slice values are integers of magnitude
// below 2^7, exact in BF16; a product of two slices summed over K <= 256
// terms stays below 2^22, so the FP32 accumulation of the tensor cores is
// exact.  The slice pairs (s, j) with s + j <= kOzSlices + 1 are kept; pairs
// of one level L = s + j share a scale and accumulate in one TMEM block.  The
// epilogue adds the levels in a 128-bit integer and forms the FP64 result
// from its bits, so nothing but the final scaling runs on the FP64 pipe.
// Truncation: every operand keeps 56 bits below its row's leading power of
// two, and the dropped pairs weigh below 2^-56 of the row products.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "mfwq_internal.h"

namespace mfwq {

constexpr int kOzSlices = 8;   // slices per FP64 operand
constexpr int kOzBits = 7;     // bits per slice
constexpr int kOzFix = kOzSlices * kOzBits;  // fixed-point bits per operand (56)
constexpr int kOzLevels = 8;   // levels L = 2 .. kOzSlices + 1
constexpr int kOzNT = 64;      // output columns per tile (N of the MMA)
constexpr int kOzKC = 16;      // K elements per pipeline chunk (one MMA K step)
constexpr int kOzSBO = kOzKC / 8 * 128;  // bytes between 8-row groups of a slice tile
constexpr int kOzMaxN = 256;   // largest mode-matrix order

// A mode matrix Bm [n_out][n_in] (U_l^T or U_l) in slices, on the device.
struct OzMat {
    const uint16_t* sl = nullptr;  // [n_tiles][k_chunks] blocks of kOzSlices x (kOzNT rows x kOzKC) BF16 bits, each
                                   // slice in the shared-memory layout the MMA reads (8-row x 16-byte core matrices,
                                   // 128 B between K-neighbours, kOzSBO bytes between 8-row groups)
    const int* fexp = nullptr;     // [n_tiles * kOzNT]: biased exponent of each row's largest entry (0: zero row)
    int n_out = 0, n_in = 0, n_tiles = 0, k_chunks = 0;
};

struct OzPlan {
    int ok = 0;
    OzMat fwd[3], bwd[3];          // U_l^T (forward products) and U_l (backward products)
    double* dinv = nullptr;        // [n3][n2 n1]: 1 / (lam1[i] + lam2[j] + lam3[k]), the scaling pass's layout
    void* dmem = nullptr;          // slices and exponents (one allocation)
    uint16_t* asl = nullptr;       // slices of one pass's input, in the MMA layout (largest pass)
    int* aexp = nullptr;           // its row exponents
};

// 56-bit fixed-point magnitude of the FP64 value with bit pattern `bits`
// relative to a row whose largest biased exponent is emax: floor(|v| 2^(1078 -
// emax)), below 2^56.  Zeros and subnormals give 0.
MFWQ_HD inline uint64_t oz_fixed(uint64_t bits, int emax) {
    const int e = (int)((bits >> 52) & 0x7FF);
    if (e == 0) return 0;
    const uint64_t m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = emax - e - 3;
    if (sh < 0) return m << (-sh);
    return sh < 64 ? (m >> sh) : 0;
}

// Byte offset of element (r, k) of a slice tile (rows of kOzKC BF16 values)
// in the MMA's no-swizzle K-major layout.
MFWQ_HD inline int oz_off(int r, int k) { return (r >> 3) * kOzSBO + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

// Builds the slices of U_l, U_l^T from the host tables and the scaling table
// from the device eigenvalues (d64[l].lam, which include any FD shift).
int oz_plan_build(const Dir1D dir[3], const DirD<double> d64[3], cudaStream_t s, OzPlan& plan);
// Recomputes the scaling table (after the eigenvalues changed).
int oz_update_dinv(const DirD<double> d64[3], OzPlan& plan, cudaStream_t s);
void oz_plan_free(OzPlan& plan);
int configure_fd_oz();
// z = P^-1 r with FP64 input and output; tmp holds N doubles.  A bounded wait
// that times out sets *err = 1.
int run_fd_oz(const OzPlan& plan, const double* r, double* z, double* tmp, int* err, const int* skip, cudaStream_t s);

}  // namespace mfwq
