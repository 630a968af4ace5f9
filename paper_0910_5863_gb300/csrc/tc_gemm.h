// Batched 3xTF32 GEMM on the fifth-generation tensor cores (tc_gemm.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "common.cuh"

namespace bddc {

// C[m, n] += alpha * cscale[m] * sum_k A[m, k] * bscale[k] * B[n, k]
// (bscale is applied in FP32 to the FP32 value of B, cscale and alpha in the
// output precision)
//   A: row m at A + m * lda, contiguous in k (FP32; a_f64 must be 0)
//   B: row n at B + n * ldb, contiguous in k (FP32; b_f64 must be 0)
//   C: column-major, C[m, n] at C[n * ldc + m], FP64 (or FP32 when c_f32)
// lda / ldb must keep every row 16-byte aligned (multiples of 4 floats).
struct TcGemm {
    const void *A;
    const void *B;
    void *C;
    const double *cscale;   // null = 1
    const float *bscale;    // null = 1
    int lda, ldb, ldc;
    int M, N, K;
    int a_f64, b_f64;
    double alpha;
    int c_f32;
    int store;              // 1: C[m, n] = (instead of +=) the product term
};

constexpr int kTcM = 128;   // rows of an output tile (one TMEM lane per row)
constexpr int kTcN = 128;   // columns of an output tile (TMEM columns)

// items: (job, 128-row tile, 128-column tile, unused)
void launch_tc_gemm(const TcGemm *jobs, const int4 *items, int nitems, DevStatus *st, double timeout_s,
                    cudaStream_t s);

}  // namespace bddc
