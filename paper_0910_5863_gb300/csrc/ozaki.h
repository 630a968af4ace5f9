// Trailing updates of the double-float partial Cholesky on the tensor cores (ozaki.cu).
//
// The block update C -= L L^T (L: rows of the factored block column, K <= 128 columns)
// is computed exactly enough for double-float by an error-free splitting of L into
// bf16 slices (Ozaki, Ogita, Oishi and Rump's scheme for accurate matrix products):
// every row r of L is scaled by a power of two 2^e_r >= max_k |L[r, k]| and written as
//     L[r, k] = 2^e_r sum_{p=1..7} d_p[r, k] 2^(-7p) + (remainder below 2^(e_r - 49)),
// with integer digits |d_1| <= 128 and |d_p| <= 64 (p >= 2), each exact in bf16.  The
// products of two digit matrices, summed over K <= 128, are integers below 2^24 and so
// exact in the FP32 accumulators of the tensor cores whatever the order of summation;
// all products with the same p + q = t share one accumulator (at most 7 of them:
// 9 x 2^12 x 128 < 2^24).  The seven accumulators t = 2..8 are then combined, t = 8 first
// (t = 8..6 in FP32, whose rounding stays below the dropped terms, t = 5..2 in
// double-float), scaled by 2^(e_r + e_c) and subtracted from C.  Terms with p + q > 8 are
// dropped: the result carries ~2^-49 of 2^(e_r + e_c) per product.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "common.cuh"
#include "ff.cuh"

namespace bddc {

constexpr int kOzSlices = 7;
constexpr int kOzK = 128;        // columns of a block (the slice rows are padded to this)
constexpr int kOzTileM = 128;    // output tile rows (TMEM lanes)
constexpr int kOzTileN = 32;     // output tile columns
constexpr int kOzKC = 32;        // K values per shared-memory stage (64-byte rows)

// Rows of a digit-plane block: padded to whole 128-row tiles, so that every tile's block
// is a contiguous, in-bounds copy.
__host__ __device__ inline int oz_rows_pad(int rows) { return (rows + 127) / 128 * 128; }

// Splitting of one matrix's block column: rows [0, rows) of L (double-float, ld ldl,
// k columns) into kOzSlices digit planes and the row exponents e_r.  Layout: for plane p
// and K chunk kc (32 columns; zero beyond k), rows_pad = oz_rows_pad(rows) rows of 64
// bytes at slices + ((p * 4 + kc) * rows_pad + r) * 32, the 16-byte chunk ch of row r at
// chunk ch ^ ((r / 2) mod 4) (the 64-byte swizzle of the tensor cores' shared-memory
// operands); rows past `rows` are zero.
struct OzSplitDesc {
    const ff *L;
    int ldl, rows, k;
    uint16_t *slices;   // bf16 bit patterns
    int *rexp;
};
// items: (descriptor, 256-row group)
void launch_oz_split(const OzSplitDesc *d, const int2 *items, int nitems, cudaStream_t s);

// Cholesky factorization of the w x w (w <= kOzK) diagonal block of a double-float matrix
// in place (lower triangle, column-major, ld) and the inverse of its factor, L^-1, written
// to Linv (column-major, ld kOzK, zero above the diagonal).  One CTA per block, in shared
// memory: right-looking, and at every pivot k the forward elimination of L Y = I takes the
// same column (Y = L^-1 kept transposed in the upper triangle).  A non-positive pivot is
// replaced by 1 and reported in *fail (non-NULL) or in the device status (item tag).
struct OzDiagDesc {
    ff *A;
    int ld, w;
    ff *Linv;
    int tag;
    int *fail;
};
void launch_oz_diag(const OzDiagDesc *d, int nd, DevStatus *st, cudaStream_t s);

// mode 0: C[i, j] -= sum_k L[i, k] L[j, k] for the lower triangle (i >= j) of an n x n
//         double-float block C (ld ldc), L split by launch_oz_split (rows = n); the B fields
//         repeat the A fields (nb = n);
// mode 1: C[i, j] = sum_k A[i, k] B[j, k] for all i < n, j < nb (C n x nb), A split with
//         rows = n into slices / rexp and B with rows = nb into slices_b / rexp_b.
struct OzSyrkDesc {
    ff *C;
    int ldc, n;
    const uint16_t *slices;
    const int *rexp;
    const uint16_t *slices_b;
    const int *rexp_b;
    int nb, mode;
};
// items: (descriptor, 128-row tile, 32-column tile, 0); mode 0: lower tiles only.  Persistent:
// one CTA per SM takes the items round robin.
void launch_oz_syrk(const OzSyrkDesc *d, const int4 *items, int nitems, DevStatus *st, double timeout_s,
                    cudaStream_t s);

}  // namespace bddc
