// Mixed-precision interior elimination: FP32 factorization, FP64 refinement.
//
// For each substructure, with the equilibration D = diag(A)^-1/2:
//   1. an FP32 partial Cholesky of [[D A_II D, .], [I, 0]] leaves -(D A_II D)^-1
//      in its trailing block (the explicit FP32 inverse K_s);
//   2. X = A_II^-1 A_IG is refined in FP64:  R = A_IG - A_II X  (FP64, the
//      sparse interior columns of A_i in ELL form; an FP32 copy of R feeds the
//      correction),  X += D K_s D R  (3xTF32 tensor-core product, tc_gemm.cu;
//      FP64 accumulation of X);
//   3. S_i = A_GG - A_GI X  in FP64 (the same sparse product over the
//      interface rows) -- the Schur complement of Section 2 of the paper.
// The same refinement solves A_II y = f_I for the condensed right-hand side
// and the interior recovery.
#include "common.cuh"
#include "mixed.h"
#include "ff.cuh"
#include <algorithm>

namespace bddc {

// eq[k] = 1 / sqrt(A_kk) for every local dof of every substructure
__global__ void equilibrate_kernel(const MixedSub *subs, int nsub) {
    const MixedSub s = subs[blockIdx.x];
    for (int k = threadIdx.x; k < s.n; k += blockDim.x) {
        const double e = rsqrt(s.A[(size_t)k * s.ld + k]);
        s.eq[k] = e;
        if (s.eqf) s.eqf[k] = (float)e;
    }
}

// ELL copy of the interior columns of A: row r keeps (c, a_rc) for c < nI and a_rc != 0.
// A is symmetric, so row r is read as column r (contiguous).  One warp per row.
__global__ void ell_build_kernel(const MixedSub *subs, const int2 *items, int nitems, DevStatus *st) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int it = blockIdx.x * (blockDim.x >> 5) + wid;
    if (it >= nitems) return;
    const int2 w = items[it];
    const MixedSub s = subs[w.x];
    const int r = w.y;
    const double *col = s.A + (size_t)r * s.ld;
    int cnt = 0;
    for (int c0 = 0; c0 < s.nI; c0 += 32) {
        const int c = c0 + lane;
        const double v = c < s.nI ? col[c] : 0.0;
        const unsigned m = __ballot_sync(0xffffffffu, v != 0.0);
        const int pos = cnt + __popc(m & ((1u << lane) - 1u));
        if (v != 0.0 && pos < s.ell_w) {  // entry-major: entry q of row r at q * n + r
            s.ell_col[(size_t)pos * s.n + r] = c;
            s.ell_val[(size_t)pos * s.n + r] = v;
            if (s.ell_valf) reinterpret_cast<ff *>(s.ell_valf)[(size_t)pos * s.n + r] = ff_from_double(v);
        }
        cnt += __popc(m);
    }
    if (cnt > s.ell_w) {
        if (lane == 0) dev_fail(st, BDDC_DEV_ERR_BOUNDS, w.x, r);
        cnt = s.ell_w;
    }
    if (lane == 0) s.ell_cnt[r] = cnt;
}

// Sparse products with the interior columns of A_i (ELL form), thread per (row,
// 8 consecutive columns), rows fastest: a row's ELL entries are read once for the
// 8 columns, and the gathers of the 8 X (or dX) columns, which neighbouring rows
// share, stay in L1.  items: (product, 256-row block, first column, unused).
//   FP64 form:   out[r, c] = B[r, c] - sum_q val[r, q] X[col[r, q], c]
//                for r in [r0, r0 + m), c < ncol (B may be null = 0).
//   Update form (UPDATE, p.update != 0, r0 = 0): out[r, c] = B[r, c] -
//                sum_q val[r, q] dX[col[r, q], c] and Xu[r, c] += dX[r, c].  The
//                correction is small, so its product is carried in double-float on
//                the FP32 pipe (FP64 accuracy relative to the correction); only the
//                update of out and of X uses the FP64 pipe.
// Each (r, c) sums its entries in row order, one accumulator, as a thread per
// (r, c) would.
constexpr int kEllCols = 8;
template <bool UPDATE>
__global__ void __launch_bounds__(256) ell_block_kernel(const EllProduct *ps, const int4 *items, int nitems) {
    const int it = blockIdx.x;
    if (it >= nitems) return;
    const int4 w = items[it];
    const EllProduct p = ps[w.x];
    const int i = w.y * 256 + threadIdx.x;
    if (i >= p.m) return;
    const int r = p.r0 + i, c0 = w.z;
    const int nc = min(kEllCols, p.ncol - c0);
    const int cnt = p.ell_cnt[r];
    const int *cols = p.ell_col + r;   // entry-major: consecutive rows are consecutive
    if (UPDATE) {
        const ff *vf = reinterpret_cast<const ff *>(p.ell_valf) + r;
        const float *dx = p.dXf + (size_t)c0 * p.ldx;
        ff acc[kEllCols];
#pragma unroll
        for (int u = 0; u < kEllCols; ++u) acc[u] = ff(0.f, 0.f);
        for (int q = 0; q < cnt; ++q) {
            const int k = cols[(size_t)q * p.ell_n];
            const ff a = vf[(size_t)q * p.ell_n];
#pragma unroll
            for (int u = 0; u < kEllCols; ++u)
                if (u < nc) ff_fma_acc_f(acc[u], a, __ldg(dx + (size_t)u * p.ldx + k));
        }
#pragma unroll
        for (int u = 0; u < kEllCols; ++u) {
            if (u >= nc) break;
            const int c = c0 + u;
            const double b = p.B ? p.B[(size_t)c * p.ldb + i] : 0.0;
            const double res = b - ff_to_double(ff_norm(acc[u]));
            p.out[(size_t)c * p.ldo + i] = res;
            if (p.outf) p.outf[(size_t)c * p.ldo + i] = (float)res;
            if (p.Xu) p.Xu[(size_t)c * p.ldx + r] += (double)dx[(size_t)u * p.ldx + r];
        }
    } else {
        const double *vals = p.ell_val + r;
        const double *x = p.X + (size_t)c0 * p.ldx;
        double acc[kEllCols];
#pragma unroll
        for (int u = 0; u < kEllCols; ++u) acc[u] = 0.0;
        for (int q = 0; q < cnt; ++q) {
            const int k = cols[(size_t)q * p.ell_n];
            const double a = vals[(size_t)q * p.ell_n];
#pragma unroll
            for (int u = 0; u < kEllCols; ++u)
                if (u < nc) acc[u] += a * __ldg(x + (size_t)u * p.ldx + k);
        }
#pragma unroll
        for (int u = 0; u < kEllCols; ++u) {
            if (u >= nc) break;
            const int c = c0 + u;
            const double b = p.B ? p.B[(size_t)c * p.ldb + i] : 0.0;
            p.out[(size_t)c * p.ldo + i] = b - acc[u];
            if (p.outf) p.outf[(size_t)c * p.ldo + i] = (float)(b - acc[u]);
        }
    }
}

// single right-hand side: x[r] += d[r] sum_k K[r, k] w[k], w = float(d o R).  A block
// takes 32 rows of one update: it forms w in shared memory (one FP64 product per
// entry of the vector, not per matrix entry), then every warp sums 4 rows with
// 16-byte loads of K, four in flight per lane (K is symmetric: row r is column r).
// items: (update, block of 32 rows); dynamic shared memory: max n floats.
__global__ void __launch_bounds__(256) mixed_update_vec_kernel(const MixedUpdate *us, const int2 *items, int nitems) {
    extern __shared__ float wsh[];
    const int it = blockIdx.x;
    if (it >= nitems) return;
    const int2 w = items[it];
    const MixedUpdate u = us[w.x];
    for (int k = threadIdx.x; k < u.n; k += blockDim.x) wsh[k] = (float)(u.d[k] * u.R[k]);
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n4 = u.n >> 2;   // full float4 chunks; K rows are 16-byte aligned (ldk % 8 == 0)
    const float4 *w4 = reinterpret_cast<const float4 *>(wsh);
    for (int q = 0; q < 4; ++q) {
        const int r = w.y * 32 + wid * 4 + q;
        if (r >= u.n) break;
        const float *kr = u.K + (size_t)r * u.ldk;
        const float4 *k4 = reinterpret_cast<const float4 *>(kr);
        float acc = 0.f;
        for (int c0 = lane; c0 < n4; c0 += 128) {
            float4 v[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) v[t] = (c0 + 32 * t < n4) ? __ldg(k4 + c0 + 32 * t) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (c0 + 32 * t < n4) {
                    const float4 x = w4[c0 + 32 * t];
                    acc += v[t].x * x.x + v[t].y * x.y + v[t].z * x.z + v[t].w * x.w;
                }
            }
        }
        for (int k = 4 * n4 + lane; k < u.n; k += 32) acc += kr[k] * wsh[k];   // the last n % 4 entries
        acc = warp_sum(acc);
        if (lane == 0) u.X[r] += u.d[r] * (double)acc;
    }
}

// per product: sums of R^2 and B^2 (for the refinement check).  One warp per
// column (eight loads in flight per lane), eight columns per block; the
// per-column sums are reduced in column order by residual_norms_finish_kernel, so
// the result is deterministic.  with_b = 0 keeps the B^2 sums of an earlier call
// (B does not change during a refinement).
__global__ void residual_norms_kernel(const EllProduct *ps, int np, double *colsums, const int *col_off, int with_b) {
    const int k = blockIdx.y;
    if (k >= np) return;
    const EllProduct p = ps[k];
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= p.ncol) return;
    auto sumsq = [&](const double *col) {
        double acc = 0.0;
        for (int i0 = lane; i0 < p.m; i0 += 256) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = (i0 + 32 * u < p.m) ? col[i0 + 32 * u] : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u) acc += v[u] * v[u];
        }
        return warp_sum(acc);
    };
    const double rr = sumsq(p.out + (size_t)c * p.ldo);
    const double bb = (with_b && p.B) ? sumsq(p.B + (size_t)c * p.ldb) : 0.0;
    if (lane == 0) {
        colsums[2 * (col_off[k] + c)] = rr;
        if (with_b) colsums[2 * (col_off[k] + c) + 1] = bb;
    }
}

// one warp per product: lane-strided column sums, then the fixed warp reduction
__global__ void residual_norms_finish_kernel(const double *colsums, const int *col_off, int np, double *out) {
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (k >= np) return;
    double rr = 0.0, bb = 0.0;
    for (int c = col_off[k] + lane; c < col_off[k + 1]; c += 32) {
        rr += colsums[2 * c];
        bb += colsums[2 * c + 1];
    }
    rr = warp_sum(rr);
    bb = warp_sum(bb);
    if (lane == 0) {
        out[2 * k] = rr;
        out[2 * k + 1] = bb;
    }
}

// S <- (S + S^T) / 2 for n x n column-major blocks
__global__ void symmetrize_kernel(double *const *S, const int *n, const int *ld, int ns) {
    const int s = blockIdx.y;
    if (s >= ns) return;
    double *A = S[s];
    const int nn = n[s], l = ld[s];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)nn * nn;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % nn), j = (int)(e / nn);
        if (i <= j) continue;
        const double v = 0.5 * (A[(size_t)j * l + i] + A[(size_t)i * l + j]);
        A[(size_t)j * l + i] = v;
        A[(size_t)i * l + j] = v;
    }
}

void launch_equilibrate(const MixedSub *subs, int nsub, cudaStream_t s) {
    if (nsub > 0) equilibrate_kernel<<<nsub, 256, 0, s>>>(subs, nsub);
}
void launch_ell_build(const MixedSub *subs, const int2 *items, int nitems, DevStatus *st, cudaStream_t s) {
    if (nitems > 0) ell_build_kernel<<<(nitems + 7) / 8, 256, 0, s>>>(subs, items, nitems, st);
}
void launch_ell_product(const EllProduct *ps, const int4 *items, int nitems, int update, cudaStream_t s) {
    if (nitems <= 0) return;
    if (update)
        ell_block_kernel<true><<<nitems, 256, 0, s>>>(ps, items, nitems);
    else
        ell_block_kernel<false><<<nitems, 256, 0, s>>>(ps, items, nitems);
}
cudaError_t launch_mixed_update_vec(const MixedUpdate *us, const int2 *items, int nitems, int max_n, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    const size_t smem = sizeof(float) * (size_t)std::max(max_n, 4);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(mixed_update_vec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    mixed_update_vec_kernel<<<nitems, 256, smem, s>>>(us, items, nitems);
    return cudaSuccess;
}
void launch_residual_norms(const EllProduct *ps, int np, int max_ncol, double *colsums, const int *col_off,
                           double *out, int with_b, cudaStream_t s) {
    if (np <= 0 || max_ncol <= 0) return;
    residual_norms_kernel<<<dim3((max_ncol + 7) / 8, np), 256, 0, s>>>(ps, np, colsums, col_off, with_b);
    residual_norms_finish_kernel<<<(np + 3) / 4, 128, 0, s>>>(colsums, col_off, np, out);
}
void launch_symmetrize(double *const *S, const int *n, const int *ld, int ns, cudaStream_t s) {
    if (ns > 0) symmetrize_kernel<<<dim3(64, ns), 256, 0, s>>>(S, n, ld, ns);
}

}  // namespace bddc
