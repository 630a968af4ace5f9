// Descriptors and launchers of the batched dense kernels (dense.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include "common.cuh"

namespace bddc {

// One matrix of a batched partial Cholesky: eliminate columns [0, nstop).
template <typename T>
struct PcholDesc {
    T *A;
    int n;
    int ld;
    int nstop;
    int tag;    // batch tag reported with a failed pivot (item = tag * 100000 + matrix)
    T *diag;    // NB x NB scratch: the factored diagonal block of the current step
    int ncol;   // > 0: the trailing updates stop at column ncol (a block-column panel)
    // Rows [id0, id0 + nstop - idc) start as an identity block under the eliminated
    // columns: row id0 + q = e_{idc + q}^T (as in [[M, .], [I, 0]] with idc = 0; id0 = 0:
    // none).  Such a row stays zero in every column before idc + q, so at the step of
    // columns [kb, kb + nb) the rows with idc + q >= kb + nb take no part: their work
    // items are skipped.
    int id0;
    int idc;
    int *fail;  // non-NULL: a non-positive pivot sets *fail = 1 instead of the device status
};

// dst[p + dst_row_off, q + dst_col_off] (+)= scale * rscale[p] * cscale[q] * src(rmap[p], cmap[q])
struct GatherOp {
    const double *src;    // NULL = identity source (1 where the mapped row equals the mapped column)
    double *dst;
    const int *rmap;      // NULL = identity
    const int *cmap;      // NULL = identity
    const double *rscale; // NULL = 1
    const double *cscale; // NULL = 1
    int ld_src, ld_dst;
    int nr, nc;
    int dst_row_off, dst_col_off;
    int src_row_off, src_col_off;  // added to mapped indices
    double scale;
    int src_sym;          // src symmetric, lower triangle stored
    int dst_lower;        // write only dst rows >= cols
    int accumulate;
    int src_f32;          // src points to float
    int dst_f32;          // dst points to float
    int pad;
};

// A[r0 + p, c0 + q] = A[c0 + q, r0 + p] for p < nr, q < nc (FP32, column-major):
// copies a block of one triangle into the mirrored block of the other
struct TransposeOp {
    float *A;
    int ld;
    int r0, c0;
    int nr, nc;
};

struct DiagOp {
    double *dst;          // float * when f32
    int ld, row_off, col_off, n;
    double value;
    int f32;
    int pad;
};

struct GemmDesc {
    const double *A;
    const double *B;
    double *C;
    int lda, ldb, ldc;
    int m, n, k;
    int transA, transB;
    double alpha, beta;
};

template <typename T>
struct TrsvDesc {
    const T *L;
    double *x;
    int n, ld;
};

template <typename T>
void launch_pchol_panel(const PcholDesc<T> *descs, const int2 *items, int nitems, int kb, DevStatus *st,
                        cudaStream_t s);
// update items: (matrix, tile row, tile col); an item with tile row -1 copies the
// factored diagonal block of the step from the scratch into A
template <typename T>
void launch_pchol_update(const PcholDesc<T> *descs, const int4 *items, int nitems, int kb, cudaStream_t s);
// in-place conversion of the lower triangles between FP64 (to_ff = 0) and double-float
// (to_ff = 1; struct ff of ff.cuh); items = (matrix, first of kConvertCols columns)
constexpr int kConvertCols = 8;
void launch_ff_convert(const PcholDesc<double> *descs, const int2 *items, int nitems, int to_ff, cudaStream_t s);
void launch_gather(const GatherOp *ops, const int2 *items, int nitems, cudaStream_t s);
void launch_diag_set(const DiagOp *ops, int nops, cudaStream_t s);
// items: (op, 32-row tile, 32-column tile)
void launch_transpose_block(const TransposeOp *ops, const int4 *items, int nitems, cudaStream_t s);
void launch_zero(double *p, size_t n, cudaStream_t s);
// zero many buffers in one launch; items = (segment, 8192-element chunk)
void launch_zero_many(double *const *ptrs, const int64_t *sizes, const int2 *items, int nitems, cudaStream_t s);
// dst[idx[k]] = src[k] (scatter) or dst[k] = src[idx[k]] (gather), k < n
void launch_scatter(double *dst, const int64_t *idx, const double *src, int64_t n, cudaStream_t s);
void launch_gatherv(double *dst, const int64_t *idx, const double *src, int64_t n, cudaStream_t s);
// dst[k] += src[idx[k]]
void launch_gatherv_add(double *dst, const int64_t *idx, const double *src, int64_t n, cudaStream_t s);
// S_C[Rc[m], Rc[l]] += SCi[m, l], substructures added in order (deterministic)
struct CoarseAsmDesc {
    const double *SCi;
    const int *Rc;
    int nci, ld;
};
void launch_coarse_assemble(const CoarseAsmDesc *d, int nsub, double *SC, int nC, cudaStream_t s);
// use_ff: products accumulated in double-float on the FP32 pipe (C stays FP64)
void launch_gemm(const GemmDesc *descs, const int4 *items, int nitems, int use_ff, cudaStream_t s);
// descriptors with n == 1 and one transA value for the whole batch
void launch_gemv(const GemmDesc *descs, const int2 *items, int nitems, cudaStream_t s);
template <typename T>
void launch_trsv(const TrsvDesc<T> *descs, int nd, int backward, cudaStream_t s);

constexpr int kPanelNB = 32;
constexpr int kPanelRows = 128;
constexpr int kTile = 64;

}  // namespace bddc
