// Kernels of the mixed-precision interior elimination (mixed.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "common.cuh"

namespace bddc {

struct MixedSub {
    const double *A;   // dense local matrix (n x n, ld), FP64, unfactored
    int n, nI, ld;
    double *eq;        // (n) equilibration 1/sqrt(A_kk)
    int *ell_cnt;      // (n) entries kept per row
    int *ell_col;      // (ell_w x n): entry q of row r at q * n + r
    double *ell_val;   // (ell_w x n)
    int ell_w;
    float *eqf;        // (n) eq in FP32, or null
    double *ell_valf;  // (ell_w x n) the ELL values as double-float pairs (struct ff), or null
};

// out[r, c] = B[r, c] - sum_{interior cols} A[r0 + r, col] X[col, c], r < m, c < ncol
struct EllProduct {
    const int *ell_cnt, *ell_col;   // entry-major: entry q of row r at q * ell_n + r
    const double *ell_val;
    int ell_w, ell_n;
    int r0, m, ncol;
    const double *X;
    int ldx;
    const double *B;   // may be null (= 0)
    int ldb;
    double *out;
    int ldo;
    float *outf;       // optional FP32 copy of out (ldo), the operand of the tensor-core corrections
    // update form (update != 0): out = B - sum A dX accumulated in double-float from the
    // double-float ELL values and the FP32 correction dX (ldx), and Xu += dX (ldx) on the
    // same index space (r0 = 0, m = rows of X); B may alias out
    int update;
    const double *ell_valf;
    const float *dXf;
    double *Xu;
};

// X[r, c] += d[r] sum_k K[r, k] float(d[k] R[k, c]),  r, k < n, c < ncol
struct MixedUpdate {
    const float *K;
    int ldk;
    const double *d;
    const double *R;
    int ldr;
    double *X;
    int ldx;
    int n, ncol;
};

// ncol == 1 variant; items: (update, block of 32 rows); max_n = largest n (shared memory)
cudaError_t launch_mixed_update_vec(const MixedUpdate *us, const int2 *items, int nitems, int max_n, cudaStream_t s);

void launch_equilibrate(const MixedSub *subs, int nsub, cudaStream_t s);
// items: (sub, row), one warp each
void launch_ell_build(const MixedSub *subs, const int2 *items, int nitems, DevStatus *st, cudaStream_t s);
// all products of one call have the same form (update = p.update);
// items: (product, 256-row block, first of 8 columns, unused)
void launch_ell_product(const EllProduct *ps, const int4 *items, int nitems, int update, cudaStream_t s);
// out[2k] = |R_k|^2, out[2k+1] = |B_k|^2; colsums holds 2 doubles per column of all products,
// col_off (np + 1) the first column of each product
void launch_residual_norms(const EllProduct *ps, int np, int max_ncol, double *colsums, const int *col_off,
                           double *out, int with_b, cudaStream_t s);
void launch_symmetrize(double *const *S, const int *n, const int *ld, int ns, cudaStream_t s);

}  // namespace bddc
