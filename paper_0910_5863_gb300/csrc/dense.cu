// Batched variable-size dense kernels (FP64 and FP32) for the substructure
// and face-pair algebra of adaptive BDDC.
//
// The central operation is a *partial* right-looking blocked Cholesky: for a
// symmetric matrix stored column-major (lower triangle significant) it
// eliminates the first nstop columns.  Afterwards
//   A[0:n, 0:nstop]        holds L11 (lower) and L21 = A21 L11^-T,
//   A[nstop:n, nstop:n]    (lower) holds the Schur complement A22 - L21 L21^T,
//   the strict upper triangle keeps its original contents.
// With A = [[A_II, A_IG], [A_GI, A_GG]] and nstop = n_I this is the interior
// elimination of Section 2 of the paper (S_i = A_GG - A_GI A_II^{-1} A_IG),
// and with augmented matrices it also yields inverses and coarse operators.
#include "common.cuh"
#include "dense.h"
#include "ff.cuh"
#include <algorithm>
#include <type_traits>

namespace bddc {

constexpr int NB = 32;          // panel width
constexpr int PANEL_ROWS = 128; // rows of the panel solved per CTA
constexpr int TILE = 64;        // trailing-update tile

// ---------------------------------------------------------------------------
// panel: factor the nb x nb diagonal block in shared memory (redundantly per
// CTA) and solve the rows below it: A[r, kb:kb+nb] <- A[r, kb:kb+nb] L_kk^-T.
// Column j of the diagonal block is scaled after the loop, so each column
// costs one reciprocal square root and two block barriers.
template <typename T>
__global__ void __launch_bounds__(PANEL_ROWS) pchol_panel_kernel(const PcholDesc<T> *descs, const int2 *items,
                                                                 int nitems, int kb, DevStatus *st) {
    int it = blockIdx.x;
    if (it >= nitems) return;
    int2 w = items[it];
    const PcholDesc<T> d = descs[w.x];
    const int n = d.n, ld = d.ld;
    const int nb = min(NB, d.nstop - kb);
    T *A = d.A;
    __shared__ T Ld[NB][NB + 1];
    __shared__ T inv_d[NB];
    __shared__ int bad;
    const int tid = threadIdx.x;
    if (tid == 0) bad = 0;
    for (int e = tid; e < nb * nb; e += blockDim.x) {
        int i = e % nb, j = e / nb;
        Ld[i][j] = (i >= j) ? A[(size_t)(kb + j) * ld + kb + i] : T(0);
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (tid == 0) {
            T dj = Ld[j][j];
            if (!(dj > T(0))) {
                bad = 1;
                dj = T(1);
                Ld[j][j] = dj;
            } else if constexpr (std::is_same<T, float>::value) {
                if (w.y == 0) atomicMin(&st->minpiv, __float_as_uint(dj));  // positive floats order as unsigned
            }
            if constexpr (std::is_same<T, ff>::value)
                inv_d[j] = ff_rsqrt(dj);
            else
                inv_d[j] = ::rsqrt(dj);
        }
        __syncthreads();
        // trailing update with the unscaled column: a_ik -= a_ij a_kj / a_jj
        const T inv2 = inv_d[j] * inv_d[j];
        const int m = nb - j - 1;
        for (int e = tid; e < m * m; e += blockDim.x) {
            int i = j + 1 + e % m, k = j + 1 + e / m;
            if (i >= k) Ld[i][k] -= Ld[i][j] * Ld[k][j] * inv2;
        }
        __syncthreads();
    }
    for (int e = tid; e < nb * nb; e += blockDim.x) {
        int i = e % nb, j = e / nb;
        if (i > j) Ld[i][j] *= inv_d[j];
        else if (i == j) Ld[j][j] *= inv_d[j];  // a_jj / sqrt(a_jj)
    }
    __syncthreads();
    if (bad && tid == 0 && w.y == 0) {
        if (d.fail)
            *d.fail = 1;
        else
            dev_fail(st, BDDC_DEV_ERR_NOTSPD, d.tag * 100000 + w.x, kb);
    }
    // Every CTA of this matrix factors the diagonal block from A, so the factor
    // must not be written into A during this launch: CTA 0 leaves it in the
    // scratch and the update launch of the same step copies it into A.
    if (w.y == 0) {
        for (int e = tid; e < nb * nb; e += blockDim.x) {
            int i = e % nb, j = e / nb;
            if (i >= j) d.diag[j * NB + i] = Ld[i][j];
        }
    }
    int r = kb + nb + w.y * PANEL_ROWS + tid;
    if constexpr (std::is_same<T, ff>::value) {
        // Double-float: a fully unrolled solve would be ~10k instructions and thrash the
        // instruction cache, so the row lives in shared memory (x_c of this thread at
        // xs[c][tid], conflict-free) and the loops stay rolled; each x_c accumulates its
        // products without renormalising and is normalised once, as the trailing update does.
        __shared__ ff xs[NB][PANEL_ROWS];
        if (r < n) {
            for (int c = 0; c < nb; ++c) xs[c][tid] = A[(size_t)(kb + c) * ld + r];
            for (int c = 0; c < nb; ++c) {
                ff acc(0.f, 0.f);
#pragma unroll 4
                for (int k = 0; k < c; ++k) ff_fma_acc(acc, xs[k][tid], Ld[c][k]);
                const ff v = (xs[c][tid] - ff_norm(acc)) * inv_d[c];
                xs[c][tid] = v;
                A[(size_t)(kb + c) * ld + r] = v;
            }
        }
        return;
    }
    if (r < n) {
        T x[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c)
            if (c < nb) x[c] = A[(size_t)(kb + c) * ld + r];
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            if (c < nb) {
                T s0 = x[c], s1 = T(0);
#pragma unroll
                for (int k = 0; k < NB; k += 2) {
                    if (k < c) s0 -= x[k] * Ld[c][k];
                    if (k + 1 < c) s1 -= x[k + 1] * Ld[c][k + 1];
                }
                x[c] = (s0 + s1) * inv_d[c];
            }
        }
#pragma unroll
        for (int c = 0; c < NB; ++c)
            if (c < nb) A[(size_t)(kb + c) * ld + r] = x[c];
    }
}

// ---------------------------------------------------------------------------
// trailing update of one 64x64 lower tile: C -= P_i P_j^T with P = A[:, kb:kb+nb].
template <typename T>
__global__ void __launch_bounds__(256) pchol_update_kernel(const PcholDesc<T> *descs, const int4 *items,
                                                           int nitems, int kb) {
    int it = blockIdx.x;
    if (it >= nitems) return;
    int4 w = items[it];  // x = desc, y = tile row, z = tile col
    const PcholDesc<T> d = descs[w.x];
    const int n = d.n, ld = d.ld;
    const int nb = min(NB, d.nstop - kb);
    if (w.y < 0) {  // the factored diagonal block of this step, from the panel's scratch
        for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
            int i = e % nb, j = e / nb;
            if (i >= j) d.A[(size_t)(kb + j) * ld + kb + i] = d.diag[j * NB + i];
        }
        return;
    }
    const int t0 = kb + nb;
    const int i0 = t0 + w.y * TILE, j0 = t0 + w.z * TILE;
    const int cend = d.ncol > 0 ? min(d.ncol, n) : n;
    T *A = d.A;
    __shared__ T Pa[NB][TILE + 1];
    __shared__ T Pb[NB][TILE + 1];
    const int tid = threadIdx.x;
    for (int e = tid; e < NB * TILE; e += 256) {
        int r = e % TILE, k = e / TILE;
        T va = 0, vb = 0;
        if (k < nb) {
            if (i0 + r < n) va = A[(size_t)(kb + k) * ld + i0 + r];
            if (j0 + r < n) vb = A[(size_t)(kb + k) * ld + j0 + r];
        }
        Pa[k][r] = va;
        Pb[k][r] = vb;
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;
    for (int k = 0; k < nb; ++k) {
        T pa[4], pb[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) pa[a] = Pa[k][tx + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) pb[b] = Pb[k][ty + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if constexpr (std::is_same<T, ff>::value)
                    ff_fma_acc(acc[a][b], pa[a], pb[b]);
                else
                    acc[a][b] += pa[a] * pb[b];
            }
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        int c = j0 + ty + 16 * b;
        if (c >= cend) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            int r = i0 + tx + 16 * a;
            if (r < n && r >= c) {
                if constexpr (std::is_same<T, ff>::value)
                    A[(size_t)c * ld + r] -= ff_norm(acc[a][b]);
                else
                    A[(size_t)c * ld + r] -= acc[a][b];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// mirrored block copy through a 32 x 33 shared tile: reads along the source
// columns and writes along the destination columns, both coalesced.
__global__ void transpose_block_kernel(const TransposeOp *ops, const int4 *items, int nitems) {
    const int it = blockIdx.x;
    if (it >= nitems) return;
    const int4 w = items[it];
    const TransposeOp o = ops[w.x];
    const int p0 = w.y * 32, q0 = w.z * 32;
    __shared__ float t[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 256 threads: 8 rows of 32
    for (int j = ty; j < 32; j += 8) {
        const int p = p0 + j, q = q0 + tx;
        if (p < o.nr && q < o.nc) t[j][tx] = o.A[(size_t)(o.r0 + p) * o.ld + o.c0 + q];
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int q = q0 + j, p = p0 + tx;
        if (p < o.nr && q < o.nc) o.A[(size_t)(o.c0 + q) * o.ld + o.r0 + p] = t[tx][j];
    }
}

// ---------------------------------------------------------------------------
// generic gather: dst[p, q] (+)= scale * src(rmap[p], cmap[q]); maps < 0 give 0.
// src_sym: src holds a symmetric matrix in its lower triangle.
// dst_lower: only p >= q is written.
__global__ void gather_kernel(const GatherOp *ops, const int2 *items, int nitems) {
    int it = blockIdx.x;
    if (it >= nitems) return;
    int2 w = items[it];  // x = op, y = column block of 8
    const GatherOp o = ops[w.x];
    int q0 = w.y * 8;
    // a scale of +-1 (every caller's) is applied as a sign: exact, and no FP64 multiply
    const int sgn = o.scale == 1.0 ? 1 : (o.scale == -1.0 ? -1 : 0);
    for (int qq = 0; qq < 8; ++qq) {
        int q = q0 + qq;
        if (q >= o.nc) break;
        int cq = o.cmap ? o.cmap[q] : q;
        const double cs = o.cscale ? o.cscale[q] : 1.0;
        for (int p = threadIdx.x; p < o.nr; p += blockDim.x) {
            if (o.dst_lower && p + o.dst_row_off < q + o.dst_col_off) continue;
            int rp = o.rmap ? o.rmap[p] : p;
            double v = 0.0;
            if (rp >= 0 && cq >= 0) {
                if (!o.src) {
                    v = (rp == cq) ? 1.0 : 0.0;
                } else {
                    int a = rp + o.src_row_off, b = cq + o.src_col_off;
                    if (o.src_sym && a < b) {
                        int t = a;
                        a = b;
                        b = t;
                    }
                    v = o.src_f32 ? (double)reinterpret_cast<const float *>(o.src)[(size_t)b * o.ld_src + a]
                                  : o.src[(size_t)b * o.ld_src + a];
                }
                if (o.rscale) v *= o.rscale[p];
                if (o.cscale) v *= cs;
            }
            v = sgn == 1 ? v : (sgn == -1 ? -v : o.scale * v);
            const size_t di = (size_t)(q + o.dst_col_off) * o.ld_dst + p + o.dst_row_off;
            if (o.dst_f32) {
                float *dp = reinterpret_cast<float *>(o.dst) + di;
                if (o.accumulate)
                    *dp += (float)v;
                else
                    *dp = (float)v;
            } else {
                double *dp = o.dst + di;
                if (o.accumulate)
                    *dp += v;
                else
                    *dp = v;
            }
        }
    }
}

// dst[(off + k), (off2 + k)] = value for k < n (an identity block)
__global__ void diag_set_kernel(const DiagOp *ops, int nops) {
    int it = blockIdx.x;
    if (it >= nops) return;
    DiagOp o = ops[it];
    for (int k = threadIdx.x; k < o.n; k += blockDim.x) {
        const size_t di = (size_t)(o.col_off + k) * o.ld + o.row_off + k;
        if (o.f32)
            reinterpret_cast<float *>(o.dst)[di] = (float)o.value;
        else
            o.dst[di] = o.value;
    }
}

// zero many buffers in one launch: item = (segment, chunk of 8192 elements)
__global__ void zero_many_kernel(double *const *ptrs, const int64_t *sizes, const int2 *items, int nitems) {
    int it = blockIdx.x;
    if (it >= nitems) return;
    int2 w = items[it];
    double *p = ptrs[w.x];
    const int64_t n = sizes[w.x];
    const int64_t base = (int64_t)w.y * 8192;
    for (int64_t k = base + threadIdx.x; k < base + 8192 && k < n; k += blockDim.x) p[k] = 0.0;
}

__global__ void zero_kernel(double *p, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) p[i] = 0.0;
}

__global__ void scatter_kernel(double *dst, const int64_t *idx, const double *src, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dst[idx[k]] = src[k];
}
__global__ void gatherv_kernel(double *dst, const int64_t *idx, const double *src, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = src[idx[k]];
}
__global__ void gatherv_add_kernel(double *dst, const int64_t *idx, const double *src, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dst[k] += src[idx[k]];
}
__global__ void coarse_assemble_kernel(const CoarseAsmDesc *d, int nsub, double *SC, int nC) {
    for (int s = 0; s < nsub; ++s) {
        const CoarseAsmDesc c = d[s];
        for (int e = threadIdx.x; e < c.nci * c.nci; e += blockDim.x) {
            int m = e % c.nci, l = e / c.nci;
            SC[(size_t)c.Rc[l] * nC + c.Rc[m]] += c.SCi[(size_t)l * c.ld + m];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// batched GEMV (descriptors of GemmDesc with n == 1): y = alpha op(A) x + beta y
//   transA == 0: item = (desc, 32-row block); warps split k, lanes the rows
//   transA == 1: item = (desc, 8-row block);  one warp per row, lanes split k
__global__ void __launch_bounds__(256) gemv_kernel(const GemmDesc *descs, const int2 *items, int nitems) {
    int it = blockIdx.x;
    if (it >= nitems) return;
    int2 w = items[it];
    const GemmDesc d = descs[w.x];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ double red[8][32];
    if (!d.transA) {
        const int r = w.y * 32 + lane;
        double acc = 0.0;
        if (r < d.m) {
#pragma unroll 4
            for (int k = wid; k < d.k; k += 8) acc += d.A[(size_t)k * d.lda + r] * d.B[k];
        }
        red[wid][lane] = acc;
        __syncthreads();
        if (wid == 0 && r < d.m) {
            double s = 0.0;
            for (int q = 0; q < 8; ++q) s += red[q][lane];
            double *cp = d.C + r;
            *cp = d.alpha * s + (d.beta == 0.0 ? 0.0 : d.beta * *cp);
        }
    } else {
        const int r = w.y * 8 + wid;
        if (r >= d.m) return;
        const double *col = d.A + (size_t)r * d.lda;
        double acc = 0.0;
        for (int k = lane; k < d.k; k += 32) acc += col[k] * d.B[k];
        acc = warp_sum(acc);
        if (lane == 0) {
            double *cp = d.C + r;
            *cp = d.alpha * acc + (d.beta == 0.0 ? 0.0 : d.beta * *cp);
        }
    }
}

// ---------------------------------------------------------------------------
// batched GEMM: C = alpha op(A) op(B) + beta C, 64x64 tiles, k-step 16.  FP64, or
// with FF the tiles are converted to double-float as they are staged and the
// products accumulated in double-float on the FP32 pipe (C stays FP64).
template <bool FF>
__global__ void __launch_bounds__(256) gemm_kernel(const GemmDesc *descs, const int4 *items, int nitems) {
    using T = typename std::conditional<FF, ff, double>::type;
    int it = blockIdx.x;
    if (it >= nitems) return;
    int4 w = items[it];
    const GemmDesc d = descs[w.x];
    const int m0 = w.y * TILE, n0 = w.z * TILE;
    __shared__ T As[16][TILE + 1];
    __shared__ T Bs[16][TILE + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    // The next K step's tile entries are loaded into registers while the current one is
    // multiplied (8 of A and 8 of B per thread), then staged after the barrier.
    constexpr int PER = 16 * TILE / 256;
    double ra[PER], rb[PER];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = tid + q * 256;
            int r, k;
            // A tile: rows m0..m0+63, k0..k0+15
            if (!d.transA) {
                r = e % TILE;
                k = e / TILE;
            } else {
                k = e % 16;
                r = e / 16;
            }
            ra[q] = (m0 + r < d.m && k0 + k < d.k)
                        ? (d.transA ? d.A[(size_t)(m0 + r) * d.lda + k0 + k] : d.A[(size_t)(k0 + k) * d.lda + m0 + r])
                        : 0.0;
            int c;
            if (d.transB) {
                c = e % TILE;
                k = e / TILE;
            } else {
                k = e % 16;
                c = e / 16;
            }
            rb[q] = (n0 + c < d.n && k0 + k < d.k)
                        ? (d.transB ? d.B[(size_t)(k0 + k) * d.ldb + n0 + c] : d.B[(size_t)(n0 + c) * d.ldb + k0 + k])
                        : 0.0;
        }
    };
    auto stage = [&]() {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = tid + q * 256;
            const int ra_r = d.transA ? e / 16 : e % TILE, ra_k = d.transA ? e % 16 : e / TILE;
            const int rb_c = d.transB ? e % TILE : e / 16, rb_k = d.transB ? e / TILE : e % 16;
            if constexpr (FF) {
                As[ra_k][ra_r] = ff_from_double(ra[q]);
                Bs[rb_k][rb_c] = ff_from_double(rb[q]);
            } else {
                As[ra_k][ra_r] = ra[q];
                Bs[rb_k][rb_c] = rb[q];
            }
        }
    };
    fetch(0);
    for (int k0 = 0; k0 < d.k; k0 += 16) {
        stage();
        __syncthreads();
        if (k0 + 16 < d.k) fetch(k0 + 16);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if constexpr (FF)
                        ff_fma_acc(acc[i][j], a[i], b[j]);
                    else
                        acc[i][j] += a[i] * b[j];
                }
        }
        if constexpr (FF) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = ff_norm(acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int c = n0 + ty + 16 * j;
        if (c >= d.n) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int r = m0 + tx + 16 * i;
            if (r >= d.m) continue;
            double *cp = d.C + (size_t)c * d.ldc + r;
            double av;
            if constexpr (FF)
                av = ff_to_double(acc[i][j]);
            else
                av = acc[i][j];
            *cp = d.alpha * av + (d.beta == 0.0 ? 0.0 : d.beta * *cp);
        }
    }
}

// ---------------------------------------------------------------------------
// batched triangular solves with the factor of a partial Cholesky, one CTA
// per matrix, one right-hand side:
//   forward : y = L11^{-1} b        (b, y in x[0:nstop])
//   backward: x = L11^{-T} y
template <typename T>
__global__ void __launch_bounds__(256) trsv_kernel(const TrsvDesc<T> *descs, int nd, int backward) {
    int it = blockIdx.x;
    if (it >= nd) return;
    const TrsvDesc<T> d = descs[it];
    const int n = d.n, ld = d.ld;
    const T *L = d.L;
    double *x = d.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    __shared__ double part[8][32];
    if (!backward) {
        for (int jb = 0; jb < n; jb += 32) {
            int nb = min(32, n - jb);
            if (wid == 0) {
                double v = lane < nb ? x[jb + lane] : 0.0;
                const double rdiag = lane < nb ? 1.0 / (double)L[(size_t)(jb + lane) * ld + jb + lane] : 0.0;
                for (int c = 0; c < nb; ++c) {
                    if (lane == c) v *= rdiag;
                    double yc = __shfl_sync(0xffffffffu, v, c);
                    if (lane > c && lane < nb) v -= (double)L[(size_t)(jb + c) * ld + jb + lane] * yc;
                }
                if (lane < nb) x[jb + lane] = v;
            }
            __syncthreads();
            for (int r = jb + nb + tid; r < n; r += blockDim.x) {
                double s = 0.0;
                for (int c = 0; c < nb; ++c) s += (double)L[(size_t)(jb + c) * ld + r] * x[jb + c];
                x[r] -= s;
            }
            __syncthreads();
        }
    } else {
        int nblk = (n + 31) / 32;
        for (int bi = nblk - 1; bi >= 0; --bi) {
            int jb = bi * 32, nb = min(32, n - jb);
            // x[jb+c] -= sum_{r >= jb+nb} L[r, jb+c] x[r]
            for (int c = wid; c < nb; c += nw) {
                double s = 0.0;
                for (int r = jb + nb + lane; r < n; r += 32) s += (double)L[(size_t)(jb + c) * ld + r] * x[r];
                s = warp_sum(s);
                if (lane == 0) part[0][c] = s;
            }
            __syncthreads();
            if (wid == 0) {
                double v = lane < nb ? x[jb + lane] - part[0][lane] : 0.0;
                const double rdiag = lane < nb ? 1.0 / (double)L[(size_t)(jb + lane) * ld + jb + lane] : 0.0;
                for (int c = nb - 1; c >= 0; --c) {
                    if (lane == c) v *= rdiag;
                    double xc = __shfl_sync(0xffffffffu, v, c);
                    if (lane < c) v -= (double)L[(size_t)(jb + lane) * ld + jb + c] * xc;
                }
                if (lane < nb) x[jb + lane] = v;
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// host launchers
template <typename T>
void launch_pchol_panel(const PcholDesc<T> *descs, const int2 *items, int nitems, int kb, DevStatus *st,
                        cudaStream_t s) {
    if (nitems > 0) pchol_panel_kernel<T><<<nitems, PANEL_ROWS, 0, s>>>(descs, items, nitems, kb, st);
}
template <typename T>
void launch_pchol_update(const PcholDesc<T> *descs, const int4 *items, int nitems, int kb, cudaStream_t s) {
    if (nitems > 0) pchol_update_kernel<T><<<nitems, 256, 0, s>>>(descs, items, nitems, kb);
}
template void launch_pchol_panel<ff>(const PcholDesc<ff> *, const int2 *, int, int, DevStatus *, cudaStream_t);
template void launch_pchol_update<ff>(const PcholDesc<ff> *, const int4 *, int, int, cudaStream_t);

// In-place conversion of the lower triangle of every matrix between FP64 and
// double-float (both 8 bytes per entry); items = (matrix, column).
__global__ void ff_convert_kernel(const PcholDesc<double> *descs, const int2 *items, int nitems, int to_ff) {
    int it = blockIdx.x;
    if (it >= nitems) return;
    const int2 w = items[it];
    const PcholDesc<double> d = descs[w.x];
    const int nb = blockDim.x;
    // kConvertCols columns per block, four independent loads per thread in flight before any store
    for (int j = w.y; j < min(w.y + kConvertCols, d.n); ++j) {
        double *col = d.A + (size_t)j * d.ld;
        for (int i0 = j + threadIdx.x; i0 < d.n; i0 += 4 * nb) {
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = i0 + u * nb < d.n ? col[i0 + u * nb] : 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + u * nb;
                if (i >= d.n) break;
                if (to_ff) {
                    reinterpret_cast<ff *>(col)[i] = ff_from_double(v[u]);
                } else {
                    const long long b = __double_as_longlong(v[u]);   // the two words, h first in memory
                    col[i] = ff_to_double(
                        ff(__int_as_float((int)(b & 0xffffffffLL)), __int_as_float((int)(b >> 32))));
                }
            }
        }
    }
}
void launch_ff_convert(const PcholDesc<double> *descs, const int2 *items, int nitems, int to_ff, cudaStream_t s) {
    if (nitems > 0) ff_convert_kernel<<<nitems, 256, 0, s>>>(descs, items, nitems, to_ff);
}

template void launch_pchol_panel<double>(const PcholDesc<double> *, const int2 *, int, int, DevStatus *, cudaStream_t);
template void launch_pchol_panel<float>(const PcholDesc<float> *, const int2 *, int, int, DevStatus *, cudaStream_t);
template void launch_pchol_update<double>(const PcholDesc<double> *, const int4 *, int, int, cudaStream_t);
template void launch_pchol_update<float>(const PcholDesc<float> *, const int4 *, int, int, cudaStream_t);

void launch_gather(const GatherOp *ops, const int2 *items, int nitems, cudaStream_t s) {
    if (nitems > 0) gather_kernel<<<nitems, 256, 0, s>>>(ops, items, nitems);
}
void launch_transpose_block(const TransposeOp *ops, const int4 *items, int nitems, cudaStream_t s) {
    if (nitems > 0) transpose_block_kernel<<<nitems, 256, 0, s>>>(ops, items, nitems);
}
void launch_diag_set(const DiagOp *ops, int nops, cudaStream_t s) {
    if (nops > 0) diag_set_kernel<<<nops, 256, 0, s>>>(ops, nops);
}
void launch_zero(double *p, size_t n, cudaStream_t s) {
    if (n == 0) return;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    zero_kernel<<<blocks, 256, 0, s>>>(p, n);
}
void launch_zero_many(double *const *ptrs, const int64_t *sizes, const int2 *items, int nitems, cudaStream_t s) {
    if (nitems > 0) zero_many_kernel<<<nitems, 256, 0, s>>>(ptrs, sizes, items, nitems);
}
void launch_scatter(double *dst, const int64_t *idx, const double *src, int64_t n, cudaStream_t s) {
    if (n > 0) scatter_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(dst, idx, src, n);
}
void launch_gatherv(double *dst, const int64_t *idx, const double *src, int64_t n, cudaStream_t s) {
    if (n > 0) gatherv_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(dst, idx, src, n);
}
void launch_gatherv_add(double *dst, const int64_t *idx, const double *src, int64_t n, cudaStream_t s) {
    if (n > 0) gatherv_add_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(dst, idx, src, n);
}
void launch_coarse_assemble(const CoarseAsmDesc *d, int nsub, double *SC, int nC, cudaStream_t s) {
    if (nsub > 0) coarse_assemble_kernel<<<1, 1024, 0, s>>>(d, nsub, SC, nC);
}
void launch_gemv(const GemmDesc *descs, const int2 *items, int nitems, cudaStream_t s) {
    if (nitems > 0) gemv_kernel<<<nitems, 256, 0, s>>>(descs, items, nitems);
}
void launch_gemm(const GemmDesc *descs, const int4 *items, int nitems, int use_ff, cudaStream_t s) {
    if (nitems <= 0) return;
    if (use_ff)
        gemm_kernel<true><<<nitems, 256, 0, s>>>(descs, items, nitems);
    else
        gemm_kernel<false><<<nitems, 256, 0, s>>>(descs, items, nitems);
}
template <typename T>
void launch_trsv(const TrsvDesc<T> *descs, int nd, int backward, cudaStream_t s) {
    if (nd > 0) trsv_kernel<T><<<nd, 256, 0, s>>>(descs, nd, backward);
}
template void launch_trsv<double>(const TrsvDesc<double> *, int, int, cudaStream_t);
template void launch_trsv<float>(const TrsvDesc<float> *, int, int, cudaStream_t);

}  // namespace bddc
