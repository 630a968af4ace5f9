// Face-pair eigenproblems of adaptive BDDC (Section 3 of the paper).
//
// Each face pair's generalized problem has been reduced, exactly, to a
// symmetric standard problem C y = lambda y of order n_s (the number of
// shared non-corner dofs; see the adapt phase for the reduction).  One CTA
// per pair:
//   1. Householder reduction of C to tridiagonal T (reflectors kept),
//   2. Sturm-sequence counts give k = #{lambda > tau} exactly (Algorithm
//      3.1 selects the smallest k with lambda_{k+1} <= tau) and bisection
//      gives lambda_1..lambda_{k+1},
//   3. inverse iteration on T (LU with row interchanges) for the k vectors,
//      re-orthogonalised inside clusters, and back-transformation,
//   4. face rows d = (W1 y)|face (the face part of eq. (d-def); the edge
//      parts are dropped as in the paper's Remark, or kept by the edge-row
//      kernels further down), normalised and orthogonalised with row
//      pivoting; rows whose pivot is below drop_rel are dropped.
#include "common.cuh"
#include <algorithm>
#include "eig.h"
#include "ff.cuh"

namespace bddc {

constexpr int EIG_THREADS = 256;
static_assert(EIG_THREADS == 32 * kFaceVecWarps, "face_vec scratch is sized for kFaceVecWarps warps per CTA");

__device__ __forceinline__ int lane_of(int tid) { return tid & 31; }
// threads per row for a matrix-vector product of order m on nt threads: the largest
// power of two (at most 8) with m * tpr <= nt, so the rows still fit in one pass
__device__ __forceinline__ int rows_per_pass_split(int m, int nt) {
    int t = 1;
    while (t < 8 && m * t * 2 <= nt) t <<= 1;
    return t;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Number of eigenvalues of the symmetric tridiagonal T (diagonal d, squared
// off-diagonal e2) below x: the sign changes of the leading principal minors
// p_0 = 1, p_1 = d_0 - x, p_{i+1} = (d_i - x) p_i - e2_{i-1} p_{i-1}.  The product
// form needs three FP64 operations per step where the quotient form
// q_i = p_i / p_{i-1} needs a division (the FP64 pipe of this GPU retires ~2
// operations per clock and SM).  (p_{i-1}, p_i) is rescaled by a power of two
// when p_i leaves [2^-512, 2^512]; a zero minor counts as negative, like the
// quotient form's -pivmin.  Signs, zero tests and exponents use integer ops.
__device__ __forceinline__ bool dneg(double v) { return __double2hiint(v) < 0; }
__device__ __forceinline__ bool dzero(double v) { return ((__double2hiint(v) & 0x7fffffff) | __double2loint(v)) == 0; }

__device__ int sturm_less(const double *d, const double *e2, int n, double x) {
    double pm = 1.0, p = d[0] - x;
    if (dzero(p)) p = -0x1p-100;
    int cnt = dneg(p) ? 1 : 0;
    for (int i = 1; i < n; ++i) {
        double pn = fma(d[i] - x, p, -e2[i - 1] * pm);
        if (dzero(pn)) pn = -p * 0x1p-100;
        if ((__double2hiint(pn) ^ __double2hiint(p)) < 0) ++cnt;
        const int ex = (__double2hiint(pn) >> 20) & 0x7ff;
        if (ex > 1023 + 512 || ex < 1023 - 512) {
            const double sc = __hiloint2double((2046 - ex) << 20, 0);   // 2^(1023 - ex)
            pn *= sc;
            p *= sc;
        }
        pm = p;
        p = pn;
    }
    return cnt;
}

// Householder tridiagonalisation in double-float (the mixed modes): the same
// steps as the FP64 loop of face_eig_kernel, with the O(n^3) work (B x and the
// rank-2 update) on the FP32 pipe.  On entry A holds the matrix as doubles; it
// is converted to double-float in place, reduced, and the reflectors (below the
// subdiagonal) are converted back to doubles, so that everything after the
// reduction reads the same layout as in FP64 mode.  bet and ee are written as
// in the FP64 loop; the diagonal is returned in dd.
__device__ void householder_ff(double *A, int lda, int n, double *dd, double *ee, double *bet, double *Pw, double *Ww,
                               double *scratch) {
    const int tid = threadIdx.x, nt = blockDim.x;
    ff *F = reinterpret_cast<ff *>(A);
    ff *P = reinterpret_cast<ff *>(Pw);
    ff *W = reinterpret_cast<ff *>(Ww);
    for (int e = tid; e < n * n; e += nt) {
        const size_t o = (size_t)(e / n) * lda + e % n;
        F[o] = ff_from_double(A[o]);
    }
    __syncthreads();
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        ff *x = F + (size_t)k * lda + k + 1;
        ff acc(0.f, 0.f);
        for (int i = tid; i < m; i += nt) ff_fma_acc(acc, x[i], x[i]);
        const double s = block_sum(ff_to_double(ff_norm(acc)), scratch);
        const double x0 = ff_to_double(x[0]);
        const double rest = s - x0 * x0;
        if (rest <= 1e-300 * (s + 1e-300)) {
            if (tid == 0) {
                bet[k] = 0.0;
                ee[k] = x0;
            }
            __syncthreads();
            continue;
        }
        const double nrm = sqrt(s);
        const double alpha = x0 > 0 ? -nrm : nrm;
        const double v0 = x0 - alpha;
        const double beta = 2.0 / (rest + v0 * v0);
        __syncthreads();
        if (tid == 0) {
            x[0] = ff_from_double(v0);
            bet[k] = beta;
            ee[k] = alpha;
        }
        __syncthreads();
        ff *B = F + (size_t)(k + 1) * lda + k + 1;
        const ff fbeta = ff_from_double(beta);
        {   // tpr consecutive threads share a row (shorter dependency chains)
            const int tpr = rows_per_pass_split(m, nt), part = tid & (tpr - 1);
            for (int i0 = 0; i0 < m; i0 += nt / tpr) {
                const int i = i0 + tid / tpr;
                ff a(0.f, 0.f);
                if (i < m) {
                    int c = 0;
                    for (int j = part; j < m; j += tpr) {
                        ff_fma_acc(a, B[(size_t)j * lda + i], x[j]);
                        if ((++c & 15) == 0) a = ff_norm(a);
                    }
                }
                a = ff_norm(a);
                for (int o = tpr >> 1; o > 0; o >>= 1) {
                    const ff b(__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o));
                    a = a + b;
                }
                if (i < m && part == 0) P[i] = fbeta * a;
            }
        }
        __syncthreads();
        ff pa(0.f, 0.f);
        for (int i = tid; i < m; i += nt) ff_fma_acc(pa, P[i], x[i]);
        const double pv = block_sum(ff_to_double(ff_norm(pa)), scratch);
        const ff K = ff_from_double(0.5 * beta * pv);
        for (int i = tid; i < m; i += nt) W[i] = P[i] - K * x[i];
        __syncthreads();
        for (int e = tid; e < m * m; e += nt) {
            const int i = e % m, j = e / m;
            B[(size_t)j * lda + i] -= x[i] * W[j] + W[i] * x[j];
        }
        __syncthreads();
    }
    for (int i = tid; i < n; i += nt) dd[i] = ff_to_double(F[(size_t)i * lda + i]);
    if (tid == 0 && n >= 2) ee[n - 2] = ff_to_double(F[(size_t)(n - 2) * lda + n - 1]);
    __syncthreads();
    // reflectors back to doubles (column k, rows k + 1 .. n - 1)
    for (int e = tid; e < n * n; e += nt) {
        const int i = e % n, j = e / n;
        if (i > j) {
            const size_t o = (size_t)j * lda + i;
            A[o] = ff_to_double(F[o]);
        }
    }
    __syncthreads();
}

// Offset of column c of a packed lower triangle of order n (column-major, the
// diagonal first): column c holds rows c .. n-1.
__device__ __forceinline__ int pk_col(int c, int n) { return c * n - (c * (c - 1)) / 2; }

// The double-float Householder reduction of householder_ff on a packed lower
// triangle in shared memory F (n (n + 1) / 2 entries): the matrix is read from
// A (lower triangle), B x uses both triangles through the symmetry, and the
// rank-2 update touches the lower triangle only (half the work).  The
// reflectors are written back to A as doubles, with bet, ee and dd as in
// the FP64 loop.
__device__ void householder_ff_packed(double *A, int lda, int n, ff *F, double *dd, double *ee, double *bet,
                                      double *Pw, double *Ww, double *scratch) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    ff *P = reinterpret_cast<ff *>(Pw);
    ff *W = reinterpret_cast<ff *>(Ww);
    for (int j = wid; j < n; j += nw)
        for (int i = j + lane; i < n; i += 32) F[pk_col(j, n) + i - j] = ff_from_double(A[(size_t)j * lda + i]);
    __syncthreads();
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        ff *x = F + pk_col(k, n) + 1;   // column k below the diagonal
        ff acc(0.f, 0.f);
        for (int i = tid; i < m; i += nt) ff_fma_acc(acc, x[i], x[i]);
        const double s = block_sum(ff_to_double(ff_norm(acc)), scratch);
        const double x0 = ff_to_double(x[0]);
        const double rest = s - x0 * x0;
        if (rest <= 1e-300 * (s + 1e-300)) {
            if (tid == 0) {
                bet[k] = 0.0;
                ee[k] = x0;
            }
            __syncthreads();
            continue;
        }
        const double nrm = sqrt(s);
        const double alpha = x0 > 0 ? -nrm : nrm;
        const double v0 = x0 - alpha;
        const double beta = 2.0 / (rest + v0 * v0);
        __syncthreads();
        if (tid == 0) {
            x[0] = ff_from_double(v0);
            bet[k] = beta;
            ee[k] = alpha;
        }
        __syncthreads();
        const int k1 = k + 1;
        const ff fbeta = ff_from_double(beta);
        {   // P = beta B x, B(i, j) = A(k1 + i, k1 + j): tpr threads share a row
            const int tpr = rows_per_pass_split(m, nt), part = tid & (tpr - 1);
            for (int i0 = 0; i0 < m; i0 += nt / tpr) {
                const int i = i0 + tid / tpr;
                ff a(0.f, 0.f);
                if (i < m) {
                    int cnt = 0;
                    for (int j = part; j < i; j += tpr) {   // row i left of the diagonal: column j, row i
                        ff_fma_acc(a, F[pk_col(k1 + j, n) + (i - j)], x[j]);
                        if ((++cnt & 15) == 0) a = ff_norm(a);
                    }
                    const ff *col = F + pk_col(k1 + i, n);   // column i from the diagonal down
                    int j = i + ((part - i) % tpr + tpr) % tpr;
                    for (; j < m; j += tpr) {
                        ff_fma_acc(a, col[j - i], x[j]);
                        if ((++cnt & 15) == 0) a = ff_norm(a);
                    }
                }
                a = ff_norm(a);
                for (int o = tpr >> 1; o > 0; o >>= 1) {
                    const ff b(__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o));
                    a = a + b;
                }
                if (i < m && part == 0) P[i] = fbeta * a;
            }
        }
        __syncthreads();
        ff pa(0.f, 0.f);
        for (int i = tid; i < m; i += nt) ff_fma_acc(pa, P[i], x[i]);
        const double pv = block_sum(ff_to_double(ff_norm(pa)), scratch);
        const ff K = ff_from_double(0.5 * beta * pv);
        for (int i = tid; i < m; i += nt) W[i] = P[i] - K * x[i];
        __syncthreads();
        // rank-2 update of the lower triangle, one warp per column
        for (int j = wid; j < m; j += nw) {
            ff *col = F + pk_col(k1 + j, n);
            const ff xj = x[j], wj = W[j];
            for (int i = j + lane; i < m; i += 32) col[i - j] -= x[i] * wj + W[i] * xj;
        }
        __syncthreads();
    }
    for (int i = tid; i < n; i += nt) dd[i] = ff_to_double(F[pk_col(i, n)]);
    if (tid == 0 && n >= 2) ee[n - 2] = ff_to_double(F[pk_col(n - 2, n) + 1]);
    // reflectors back to A as doubles (column k, rows k + 1 .. n - 1)
    for (int j = wid; j < n; j += nw)
        for (int i = j + 1 + lane; i < n; i += 32) A[(size_t)j * lda + i] = ff_to_double(F[pk_col(j, n) + i - j]);
    __syncthreads();
}

// The per-eigenvalue steps of the face problem, one warp each, shared by face_eig_kernel and
// face_vec_kernel (bit-identical results whichever runs them).
// Eigenvalue j (ascending) of T by 32-way multisection: lanes 0..30 count at 31 interior points.
__device__ double tri_multisect(const double *dd, const double *e2, int n, int j, double tnorm) {
    const int lane = threadIdx.x & 31;
    double lo = -tnorm - 1.0, hi = tnorm + 1.0;
    for (int round = 0; round < 40; ++round) {
        const double w = hi - lo;
        if (w <= 1e-15 * fmax(fabs(lo), fabs(hi)) + 1e-300) break;
        const double x = lo + w * (double)(lane + 1) * (1.0 / 32.0);
        const bool above = lane < 31 && sturm_less(dd, e2, n, x) > j;
        const unsigned mask = __ballot_sync(0xffffffffu, above);
        const int first = mask ? __ffs(mask) - 1 : 31;
        const double nlo = first == 0 ? lo : lo + w * (double)first * (1.0 / 32.0);
        const double nhi = first == 31 ? hi : lo + w * (double)(first + 1) * (1.0 / 32.0);
        if (!(nlo > lo || nhi < hi)) break;
        lo = nlo;
        hi = nhi;
    }
    return 0.5 * (lo + hi);
}

// Inverse iteration on T - lm I (LU with row interchanges by lane 0, three solves), the
// normalised vector written to out.  wb: 6 n doubles of scratch for the warp.
__device__ void tri_inverse_iteration(const double *dd, const double *ee, int n, double lm, int mI, double tnorm,
                                      double *wb, double *out) {
    const int lane = threadIdx.x & 31;
    double *dl = wb, *du = dl + n, *dv = du + n, *du2 = dv + n, *xv = du2 + n;
    int *piv = (int *)(xv + n);
    if (lane == 0) {
        // LU with row interchanges of T - lm I; the reciprocals of the pivots are kept in dv
        const double small = 2.2e-16 * fmax(tnorm, 1e-300);
        for (int i = 0; i < n; ++i) {
            dv[i] = dd[i] - lm;
            du[i] = (i + 1 < n) ? ee[i] : 0.0;
            dl[i] = (i + 1 < n) ? ee[i] : 0.0;
            du2[i] = 0.0;
        }
        for (int i = 0; i + 1 < n; ++i) {
            if (fabs(dv[i]) >= fabs(dl[i])) {
                piv[i] = 0;
                if (dv[i] == 0.0) dv[i] = small;
                double f = dl[i] / dv[i];
                dl[i] = f;
                dv[i + 1] -= f * du[i];
            } else {
                piv[i] = 1;
                double f = dv[i] / dl[i];
                dv[i] = dl[i];
                dl[i] = f;
                double t = du[i];
                du[i] = dv[i + 1];
                dv[i + 1] = t - f * dv[i + 1];
                if (i + 2 < n) {
                    du2[i] = du[i + 1];
                    du[i + 1] = -f * du[i + 1];
                }
            }
        }
        if (dv[n - 1] == 0.0) dv[n - 1] = small;
        for (int i = 0; i < n; ++i) dv[i] = 1.0 / dv[i];
    }
    for (int i = lane; i < n; i += 32) xv[i] = 1.0 + 0.1 * (double)((i * 7919 + mI * 104729) % 17) / 17.0;
    __syncwarp();
    for (int itr = 0; itr < 3; ++itr) {
        if (lane == 0) {
            for (int i = 0; i + 1 < n; ++i) {
                if (piv[i] == 0) {
                    xv[i + 1] -= dl[i] * xv[i];
                } else {
                    double t = xv[i];
                    xv[i] = xv[i + 1];
                    xv[i + 1] = t - dl[i] * xv[i + 1];
                }
            }
            xv[n - 1] *= dv[n - 1];
            if (n >= 2) xv[n - 2] = (xv[n - 2] - du[n - 2] * xv[n - 1]) * dv[n - 2];
            for (int i = n - 3; i >= 0; --i) xv[i] = (xv[i] - du[i] * xv[i + 1] - du2[i] * xv[i + 2]) * dv[i];
        }
        __syncwarp();
        double s2 = 0.0;
        for (int i = lane; i < n; i += 32) s2 += xv[i] * xv[i];
        s2 = warp_sum(s2);
        const double inv = s2 > 0 ? 1.0 / sqrt(s2) : 0.0;
        for (int i = lane; i < n; i += 32) xv[i] *= inv;
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) out[i] = xv[i];
    __syncwarp();
}

// y = H_0 H_1 ... H_{n-3} y with the reflectors below the subdiagonal of A (read-only)
__device__ void tri_back_transform(const double *A, int lda, const double *bet, int n, double *y) {
    const int lane = threadIdx.x & 31;
    for (int k = n - 3; k >= 0; --k) {
        const double b = bet[k];
        if (b == 0.0) continue;
        const double *v = A + (size_t)k * lda + k + 1;
        double dot = 0.0;
        for (int i = lane; i < n - k - 1; i += 32) dot += v[i] * y[k + 1 + i];
        dot = warp_sum(dot) * b;
        for (int i = lane; i < n - k - 1; i += 32) y[k + 1 + i] -= dot * v[i];
        __syncwarp();
    }
}

__global__ void __launch_bounds__(EIG_THREADS) face_eig_kernel(const EigDesc *descs, int np, double tau,
                                                               double drop_rel, DevStatus *st, int use_smem,
                                                               int use_ff, int packed_off, int fixed_k) {
    extern __shared__ double sm[];
    __shared__ double scratch[32];
    __shared__ double sh_val[4];
    __shared__ int sh_int[4];
    if (blockIdx.x >= np) return;
    const EigDesc D = descs[blockIdx.x];
    const int n = D.n, tid = threadIdx.x, nt = blockDim.x;
    int *counts = D.counts;
    if (n <= 0) {
        if (tid == 0) counts[0] = counts[1] = counts[2] = counts[3] = counts[4] = 0;
        return;
    }
    double *A;
    int lda;
    double *work;
    if (D.given) {   // eigenpairs (1) or the tridiagonal form (2) supplied: C stays in place
        A = D.C;
        lda = D.ld;
        work = D.work;
    } else if (use_smem) {
        A = sm;
        lda = n;
        work = sm + (size_t)n * n;
        for (int e = tid; e < n * n; e += nt) A[e] = D.C[(size_t)(e / n) * D.ld + e % n];
    } else {
        A = D.C;
        lda = D.ld;
        work = D.work;
    }
    double *dd = work, *ee = work + n, *bet = work + 2 * n, *P = work + 3 * n, *Wv = work + 4 * n;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    __syncthreads();
    if (D.given == 1 || D.given == 3) {
        if (tid == 0) {
            sh_int[0] = counts[0];
            sh_int[1] = counts[3];
            sh_int[2] = counts[4];
            sh_int[3] = counts[2];
        }
        __syncthreads();
    } else {
    if (D.given != 2) {   // given == 2: the tridiagonal form comes from tridiag.cu
    // ---- 1. Householder tridiagonalisation: A = Q T Q^T ----
    if (use_ff && packed_off >= 0)
        householder_ff_packed(A, lda, n, reinterpret_cast<ff *>(reinterpret_cast<char *>(sm) + packed_off), dd, ee, bet,
                              P, Wv, scratch);
    else if (use_ff)
        householder_ff(A, lda, n, dd, ee, bet, P, Wv, scratch);
    for (int k = 0; !use_ff && k + 2 < n; ++k) {
        const int m = n - k - 1;
        double *x = A + (size_t)k * lda + k + 1;   // column k below the diagonal
        double s = 0.0;
        for (int i = tid; i < m; i += nt) s += x[i] * x[i];
        s = block_sum(s, scratch);
        const double x0 = x[0];
        const double rest = s - x0 * x0;
        if (rest <= 1e-300 * (s + 1e-300)) {
            if (tid == 0) {
                bet[k] = 0.0;
                ee[k] = x0;
            }
            __syncthreads();
            continue;
        }
        const double nrm = sqrt(s);
        const double alpha = x0 > 0 ? -nrm : nrm;
        const double v0 = x0 - alpha;
        const double beta = 2.0 / (rest + v0 * v0);
        __syncthreads();
        if (tid == 0) {
            x[0] = v0;
            bet[k] = beta;
            ee[k] = alpha;
        }
        __syncthreads();
        double *B = A + (size_t)(k + 1) * lda + k + 1;
        {   // P = beta B x: tpr consecutive threads share a row (shorter dependency chains)
            const int tpr = rows_per_pass_split(m, nt), part = tid & (tpr - 1);
            for (int i0 = 0; i0 < m; i0 += nt / tpr) {
                const int i = i0 + tid / tpr;
                double acc = 0.0;
                if (i < m)
                    for (int j = part; j < m; j += tpr) acc += B[(size_t)j * lda + i] * x[j];
                for (int o = tpr >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (i < m && part == 0) P[i] = beta * acc;
            }
        }
        __syncthreads();
        double pv = 0.0;
        for (int i = tid; i < m; i += nt) pv += P[i] * x[i];
        pv = block_sum(pv, scratch);
        const double K = 0.5 * beta * pv;
        for (int i = tid; i < m; i += nt) Wv[i] = P[i] - K * x[i];
        __syncthreads();
        for (int e = tid; e < m * m; e += nt) {
            int i = e % m, j = e / m;
            B[(size_t)j * lda + i] -= x[i] * Wv[j] + Wv[i] * x[j];
        }
        __syncthreads();
    }
    if (!use_ff)
        for (int i = tid; i < n; i += nt) dd[i] = A[(size_t)i * lda + i];
    if (tid == 0) {
        if (n >= 2) {
            if (!use_ff) ee[n - 2] = A[(size_t)(n - 2) * lda + n - 1];
            bet[n - 2] = 0.0;
        }
        bet[n - 1] = 0.0;
        ee[n - 1] = 0.0;
    }
    }   // D.given != 2
    __syncthreads();
    // ---- 2. counts and bisection ----
    double *e2 = work + 5 * n;
    double tn = 0.0;   // infinity norm of T (block max)
    for (int i = tid; i < n; i += nt) {
        const double a = i > 0 ? fabs(ee[i - 1]) : 0.0, b = i + 1 < n ? fabs(ee[i]) : 0.0;
        tn = fmax(tn, fabs(dd[i]) + a + b);
        if (i + 1 < n) e2[i] = ee[i] * ee[i];
    }
    tn = warp_max(tn);
    if (lane_of(tid) == 0) scratch[tid >> 5] = tn;
    __syncthreads();
    double tnorm = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) tnorm = fmax(tnorm, scratch[w]);
    __syncthreads();
    if (tid == 0) {
        int nsel, ties = 0;
        if (fixed_k > 0) {
            nsel = min(fixed_k, n);   // the fixed_k dominant eigenvalues (Section 7, "3eigv")
        } else {
            const int less = sturm_less(dd, e2, n, tau);
            nsel = n - less;
            ties = sturm_less(dd, e2, n, tau * (1 + 1e-6)) - sturm_less(dd, e2, n, tau * (1 - 1e-6));
        }
        int over = 0;   // > 0: the selected count when it exceeds the face's capacity
        if (nsel > D.cap) {
            over = nsel;
            nsel = D.cap;
        }
        sh_int[0] = nsel;
        sh_int[1] = ties;
        sh_int[2] = over;
        sh_int[3] = min(nsel + 1, n);
    }
    __syncthreads();
    const int nsel = sh_int[0], nval = sh_int[3];
    double *lam = D.lam;
    // 32-way multisection, one warp per eigenvalue
    for (int t = wid; t < nval; t += nw) {
        const double l = tri_multisect(dd, e2, n, n - 1 - t, tnorm);
        if (lane == 0) lam[t] = l;
    }
    __syncthreads();
    // fixed count: a boundary lambda_k ~ lambda_{k+1} leaves the selected subspace not unique
    if (fixed_k > 0 && tid == 0 && nsel > 0 && nsel < n && fabs(lam[nsel] / lam[nsel - 1] - 1.0) < 1e-6) sh_int[1] = 1;
    // ---- 3. inverse iteration on T (one warp per vector), back-transformation ----
    double *wbase = work + 10 * n;  // 6 n doubles per warp
    for (int mI = wid; mI < nsel; mI += nw)
        tri_inverse_iteration(dd, ee, n, lam[mI], mI, tnorm, wbase + (size_t)wid * 6 * n, D.vec + (size_t)mI * n);
    __syncthreads();
    // clusters (eigenvalues within 1e-5 relative): orthonormalise in order (rare)
    for (int mI = 1; mI < nsel; ++mI) {
        double *x = D.vec + (size_t)mI * n;
        bool any = false;
        for (int q = 0; q < mI; ++q) {
            if (fabs(lam[q] - lam[mI]) > 1e-5 * fabs(lam[mI])) continue;
            any = true;
            const double *vq = D.vec + (size_t)q * n;
            double dot = 0.0;
            for (int i = tid; i < n; i += nt) dot += vq[i] * x[i];
            dot = block_sum(dot, scratch);
            for (int i = tid; i < n; i += nt) x[i] -= dot * vq[i];
            __syncthreads();
        }
        if (any) {
            double s2 = 0.0;
            for (int i = tid; i < n; i += nt) s2 += x[i] * x[i];
            s2 = block_sum(s2, scratch);
            const double inv = s2 > 0 ? 1.0 / sqrt(s2) : 0.0;
            for (int i = tid; i < n; i += nt) x[i] *= inv;
            __syncthreads();
        }
    }
    // back-transformation y = H_0 H_1 ... H_{n-3} x, one warp per vector (reflectors are read-only)
    for (int mI = wid; mI < nsel; mI += nw) tri_back_transform(A, lda, bet, n, D.vec + (size_t)mI * n);
    __syncthreads();
    }   // !D.given
    const int nsel = sh_int[0], nval = sh_int[3];
    // ---- 4. face rows and their pivoted orthonormalisation ----
    const int nf = D.nface;
    double *R = D.rows;
    if (D.given != 3) {
        for (int e = tid; e < nsel * nf; e += nt) {
            int l = e / nf, f = e % nf;
            const double *y = D.vec + (size_t)l * n;
            const double *wr = D.W1 + D.face_pos[f];
            double acc = 0.0;
            for (int j = 0; j < n; ++j) acc += wr[(size_t)j * D.ldw] * y[j];
            R[(size_t)l * nf + f] = acc;
        }
    } else {
        // eigenpairs and rows from face_vec_kernel: the boundary test of the fixed count, and
        // clusters (eigenvalues within 1e-5 relative) orthonormalised in order, the rows with
        // the same combinations (they are linear in the vectors)
        const double *lam = D.lam;
        if (fixed_k > 0 && tid == 0 && nsel > 0 && nsel < n && fabs(lam[nsel] / lam[nsel - 1] - 1.0) < 1e-6)
            sh_int[1] = 1;
        for (int mI = 1; mI < nsel; ++mI) {
            double *x = D.vec + (size_t)mI * n;
            bool any = false;
            for (int q = 0; q < mI; ++q) {
                if (fabs(lam[q] - lam[mI]) > 1e-5 * fabs(lam[mI])) continue;
                any = true;
                const double *vq = D.vec + (size_t)q * n;
                double dot = 0.0;
                for (int i = tid; i < n; i += nt) dot += vq[i] * x[i];
                dot = block_sum(dot, scratch);
                for (int i = tid; i < n; i += nt) x[i] -= dot * vq[i];
                for (int f = tid; f < nf; f += nt) R[(size_t)mI * nf + f] -= dot * R[(size_t)q * nf + f];
                __syncthreads();
            }
            if (any) {
                double s2 = 0.0;
                for (int i = tid; i < n; i += nt) s2 += x[i] * x[i];
                s2 = block_sum(s2, scratch);
                const double inv = s2 > 0 ? 1.0 / sqrt(s2) : 0.0;
                for (int i = tid; i < n; i += nt) x[i] *= inv;
                for (int f = tid; f < nf; f += nt) R[(size_t)mI * nf + f] *= inv;
                __syncthreads();
            }
        }
    }
    __syncthreads();
    // normalise every row
    for (int l = wid; l < nsel; l += nw) {
        double s = 0.0;
        for (int f = lane; f < nf; f += 32) s += R[(size_t)l * nf + f] * R[(size_t)l * nf + f];
        s = warp_sum(s);
        double inv = s > 0 ? 1.0 / sqrt(s) : 0.0;
        for (int f = lane; f < nf; f += 32) R[(size_t)l * nf + f] *= inv;
    }
    __syncthreads();
    // Gram-Schmidt with row pivoting: rows [0, kept) are final
    int kept = 0;
    double first = -1.0;
    double *nrm = P;  // nsel <= n
    for (int step = 0; step < nsel; ++step) {
        for (int l = step + wid; l < nsel; l += nw) {
            double s = 0.0;
            for (int f = lane; f < nf; f += 32) s += R[(size_t)l * nf + f] * R[(size_t)l * nf + f];
            s = warp_sum(s);
            if (lane == 0) nrm[l] = sqrt(s);
        }
        __syncthreads();
        if (tid == 0) {
            int best = step;
            for (int l = step + 1; l < nsel; ++l)
                if (nrm[l] > nrm[best]) best = l;
            sh_int[0] = best;
            sh_val[0] = nrm[best];
        }
        __syncthreads();
        const int best = sh_int[0];
        const double pn = sh_val[0];
        if (first < 0) first = pn;
        if (!(pn > drop_rel * first) || pn == 0.0) break;
        // swap rows best <-> step and normalise (the normalised row is written last, so
        // best == step also leaves a unit row)
        for (int f = tid; f < nf; f += nt) {
            double a = R[(size_t)best * nf + f], b = R[(size_t)step * nf + f];
            R[(size_t)best * nf + f] = b;
            R[(size_t)step * nf + f] = a / pn;
        }
        __syncthreads();
        for (int l = step + 1 + wid; l < nsel; l += nw) {
            double s = 0.0;
            for (int f = lane; f < nf; f += 32) s += R[(size_t)l * nf + f] * R[(size_t)step * nf + f];
            s = warp_sum(s);
            for (int f = lane; f < nf; f += 32) R[(size_t)l * nf + f] -= s * R[(size_t)step * nf + f];
        }
        __syncthreads();
        kept = step + 1;
    }
    if (tid == 0) {
        counts[0] = nsel;
        counts[1] = kept;
        counts[2] = nval;
        counts[3] = sh_int[1];
        counts[4] = sh_int[2];
    }
}

// Eigenpairs and face rows of the faces whose Householder reduction is supplied (EigDesc::given
// == 2), several CTAs per face: item (face, g) of G; CTA g takes the eigenvalue indices g, g + G,
// ..., one warp each: multisection, and for the selected ones inverse iteration,
// back-transformation and the face row.  Every CTA forms the counts from the same Sturm counts;
// CTA 0 stores them.  The face kernel finishes these faces with given = 3.
__global__ void __launch_bounds__(EIG_THREADS) face_vec_kernel(const EigDesc *descs, const int2 *items, int G,
                                                               double tau, int fixed_k, double *const *scr) {
    extern __shared__ double fv_e2[];
    __shared__ double scratch[32];
    __shared__ int sh_int[4];
    const int2 it = items[blockIdx.x];
    const EigDesc D = descs[it.x];
    const int g = it.y, n = D.n, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    if (n <= 0) return;
    const double *dd = D.work, *ee = D.work + n, *bet = D.work + 2 * n;
    double tn = 0.0;
    for (int i = tid; i < n; i += nt) {
        const double a = i > 0 ? fabs(ee[i - 1]) : 0.0, b = i + 1 < n ? fabs(ee[i]) : 0.0;
        tn = fmax(tn, fabs(dd[i]) + a + b);
        if (i + 1 < n) fv_e2[i] = ee[i] * ee[i];
    }
    tn = warp_max(tn);
    if (lane == 0) scratch[wid] = tn;
    __syncthreads();
    double tnorm = 0.0;
    for (int w = 0; w < nw; ++w) tnorm = fmax(tnorm, scratch[w]);
    if (tid == 0) {
        int nsel, ties = 0;
        if (fixed_k > 0) {
            nsel = min(fixed_k, n);
        } else {
            const int less = sturm_less(dd, fv_e2, n, tau);
            nsel = n - less;
            ties = sturm_less(dd, fv_e2, n, tau * (1 + 1e-6)) - sturm_less(dd, fv_e2, n, tau * (1 - 1e-6));
        }
        int over = 0;
        if (nsel > D.cap) {
            over = nsel;
            nsel = D.cap;
        }
        sh_int[0] = nsel;
        sh_int[1] = ties;
        sh_int[2] = over;
        sh_int[3] = min(nsel + 1, n);
    }
    __syncthreads();
    const int nsel = sh_int[0], nval = sh_int[3], nf = D.nface;
    double *wb = scr[it.x] + (size_t)(g * nw + wid) * 6 * n;
    for (int t = g + G * wid; t < nval; t += G * nw) {
        const double l = tri_multisect(dd, fv_e2, n, n - 1 - t, tnorm);
        if (lane == 0) D.lam[t] = l;
        if (t >= nsel) continue;
        double *y = D.vec + (size_t)t * n;
        tri_inverse_iteration(dd, ee, n, l, t, tnorm, wb, y);
        tri_back_transform(D.C, D.ld, bet, n, y);
        for (int f = lane; f < nf; f += 32) {
            const double *wr = D.W1 + D.face_pos[f];
            double acc = 0.0;
            for (int j = 0; j < n; ++j) acc += wr[(size_t)j * D.ldw] * y[j];
            D.rows[(size_t)t * nf + f] = acc;
        }
    }
    if (g == 0 && tid == 0) {
        D.counts[0] = nsel;
        D.counts[1] = 0;
        D.counts[2] = nval;
        D.counts[3] = sh_int[1];
        D.counts[4] = sh_int[2];
    }
}

void launch_face_vec(const EigDesc *descs, const int2 *items, int nitems, int G, int nmax, double tau, int fixed_k,
                     double *const *scr, cudaStream_t s) {
    if (nitems <= 0) return;
    const size_t smem = sizeof(double) * (size_t)std::max(nmax, 1);
    if (smem > 48 * 1024) cudaFuncSetAttribute(face_vec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    face_vec_kernel<<<nitems, EIG_THREADS, smem, s>>>(descs, items, G, tau, fixed_k, scr);
}

void launch_face_eig_n(const EigDesc *descs, int npairs, int nmax, double tau, double drop_rel, int use_ff,
                       int fixed_k, DevStatus *st, cudaStream_t s) {
    if (npairs <= 0) return;
    size_t need = sizeof(double) * ((size_t)nmax * nmax + (10 + 6 * (EIG_THREADS / 32)) * (size_t)nmax + 16);
    int use_smem = need <= 200 * 1024;
    size_t smem = use_smem ? need : 0;
    // double-float reduction on a packed lower triangle in shared memory when it fits
    const size_t packed = sizeof(ff) * ((size_t)nmax * (nmax + 1) / 2);
    const size_t kMaxDyn = 224 * 1024;
    int packed_off = -1;
    if (use_ff && smem + packed <= kMaxDyn) {
        packed_off = (int)smem;
        smem += packed;
    }
    if (smem > 48 * 1024) cudaFuncSetAttribute(face_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    face_eig_kernel<<<npairs, EIG_THREADS, smem, s>>>(descs, npairs, tau, drop_rel, st, use_smem, use_ff, packed_off,
                                                      fixed_k);
}

// ---------------------------------------------------------------------------
// Kept adaptive edge rows (see eig.h).  Stage 1: the edge parts of every face pair's
// selected rows d, filtered and normalised, into the pair's slot of each edge.
__global__ void __launch_bounds__(EIG_THREADS) edge_parts_kernel(const EdgePartDesc *descs, int np, double drop_rel) {
    const EdgePartDesc D = descs[blockIdx.x];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    __shared__ double full[kEigCap], scl[kEigCap];
    int nsel = D.counts[0];
    nsel = nsel < 0 ? 0 : (nsel > kEigCap ? kEigCap : nsel);
    // |d_l| over all of s (side i), one warp per row
    for (int l = wid; l < nsel; l += nw) {
        const double *y = D.vec + (size_t)l * D.n;
        double s2 = 0.0;
        for (int p = lane; p < D.ns; p += 32) {
            double v = 0.0;
            for (int j = 0; j < D.n; ++j) v += D.W1[p + (size_t)j * D.ldw] * y[j];
            s2 += v * v;
        }
        s2 = warp_sum(s2);
        if (lane == 0) full[l] = sqrt(s2);
    }
    __syncthreads();
    for (int e = 0; e < D.nseg; ++e) {
        const int p0 = D.seg_ptr[e], len = D.seg_ptr[e + 1] - p0;
        double *R = D.slot[e];
        for (int idx = tid; idx < kEigCap * len; idx += nt) {
            const int l = idx / len, k = idx - l * len;
            double v = 0.0;
            if (l < nsel) {
                const int p = D.seg_pos[p0 + k];
                const double *y = D.vec + (size_t)l * D.n;
                for (int j = 0; j < D.n; ++j) v += D.W1[p + (size_t)j * D.ldw] * y[j];
            }
            R[idx] = v;
        }
        __syncthreads();
        for (int l = wid; l < nsel; l += nw) {
            double s2 = 0.0;
            for (int k = lane; k < len; k += 32) s2 += R[(size_t)l * len + k] * R[(size_t)l * len + k];
            s2 = warp_sum(s2);
            if (lane == 0) {
                const double nr = sqrt(s2);
                scl[l] = nr > drop_rel * 1.4142135623730951 * full[l] ? 1.0 / nr : 0.0;
            }
        }
        __syncthreads();
        for (int idx = tid; idx < nsel * len; idx += nt) R[idx] *= scl[idx / len];
        __syncthreads();
    }
}

// Stage 2: Gram-Schmidt with row pivoting over the stacked slots of one edge.
constexpr int kEdgeRowsMax = kMaxEdgeSlots * kEigCap;
__global__ void __launch_bounds__(EIG_THREADS) edge_globs_kernel(const EdgeGlobDesc *descs, int ne, double drop_rel) {
    const EdgeGlobDesc D = descs[blockIdx.x];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    __shared__ double nrm[kEdgeRowsMax];
    __shared__ int sh_best;
    __shared__ double sh_pn;
    const int nr = D.nrows < kEdgeRowsMax ? D.nrows : kEdgeRowsMax, len = D.len;
    double *R = D.R;
    int kept = 0;
    double first = -1.0;
    for (int step = 0; step < nr && step < len; ++step) {
        for (int l = step + wid; l < nr; l += nw) {
            double s2 = 0.0;
            for (int k = lane; k < len; k += 32) s2 += R[(size_t)l * len + k] * R[(size_t)l * len + k];
            s2 = warp_sum(s2);
            if (lane == 0) nrm[l] = sqrt(s2);
        }
        __syncthreads();
        if (tid == 0) {
            int best = step;
            for (int l = step + 1; l < nr; ++l)
                if (nrm[l] > nrm[best]) best = l;
            sh_best = best;
            sh_pn = nrm[best];
        }
        __syncthreads();
        const int best = sh_best;
        const double pn = sh_pn;
        if (first < 0) first = pn;
        if (!(pn > drop_rel * first) || pn == 0.0) break;
        for (int k = tid; k < len; k += nt) {
            const double a = R[(size_t)best * len + k], b = R[(size_t)step * len + k];
            R[(size_t)best * len + k] = b;
            R[(size_t)step * len + k] = a / pn;
        }
        __syncthreads();
        for (int l = step + 1 + wid; l < nr; l += nw) {
            double dot = 0.0;
            for (int k = lane; k < len; k += 32) dot += R[(size_t)l * len + k] * R[(size_t)step * len + k];
            dot = warp_sum(dot);
            for (int k = lane; k < len; k += 32) R[(size_t)l * len + k] -= dot * R[(size_t)step * len + k];
        }
        __syncthreads();
        kept = step + 1;
    }
    for (int idx = tid; idx < kept * len; idx += nt) {
        const int l = idx / len, k = idx - l * len;
        D.rowsT[(size_t)k * len + l] = R[(size_t)l * len + k];
    }
    if (tid == 0) *D.kept = kept;
}

void launch_edge_parts(const EdgePartDesc *d, int npairs, double drop_rel, cudaStream_t s) {
    if (npairs > 0) edge_parts_kernel<<<npairs, EIG_THREADS, 0, s>>>(d, npairs, drop_rel);
}
void launch_edge_globs(const EdgeGlobDesc *d, int nedges, double drop_rel, cudaStream_t s) {
    if (nedges > 0) edge_globs_kernel<<<nedges, EIG_THREADS, 0, s>>>(d, nedges, drop_rel);
}

// ---------------------------------------------------------------------------
__global__ void deflate_kernel(const DeflateDesc *dd, int np) {
    __shared__ double scratch[32];
    const DeflateDesc d = dd[blockIdx.x];
    const int ns = d.ns, tid = threadIdx.x;
    if (d.nnull == 0 || ns == 0) return;
    double mx = 0.0;
    for (int p = tid; p < 2 * ns; p += blockDim.x) mx = fmax(mx, d.Shat[(size_t)p * d.ld_s + p]);
    // block max via shared
    __syncthreads();
    double m = mx;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) scratch[tid >> 5] = m;
    __syncthreads();
    double sigma = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sigma = fmax(sigma, scratch[w]);
    for (int e = tid; e < ns * ns; e += blockDim.x) {
        int p = e % ns, q = e / ns;
        double v = 0.0;
        for (int l = 0; l < d.nnull; ++l) v += d.N0[(size_t)l * ns + p] * d.N0[(size_t)l * ns + q];
        v *= sigma;
        // blocks in order (w2, b, id): (w2,w2) += 4v (lower), (b,w2) += 2v, (b,b) += v (lower)
        if (p >= q) d.M3[(size_t)q * d.ld_m + p] += 4.0 * v;
        d.M3[(size_t)q * d.ld_m + ns + p] += 2.0 * v;
        if (p >= q) d.M3[(size_t)(ns + q) * d.ld_m + ns + p] += v;
    }
}

void launch_deflate(const DeflateDesc *d, int npairs, cudaStream_t s) {
    if (npairs > 0) deflate_kernel<<<npairs, 256, 0, s>>>(d, npairs);
}

// ---- pair problems with initial constraints (the projection of Section 3 onto
// the jumps that satisfy the initial glob constraints) ----
__device__ __forceinline__ double sym_lower(const double *M, int ld, int i, int j) {
    return i >= j ? M[(size_t)j * ld + i] : M[(size_t)i * ld + j];
}

// grid (pairs, row blocks): one thread per lower entry of a column strip
__global__ void pi_compress_kernel(const PiDesc *dd, int np) {
    const PiDesc d = dd[blockIdx.x];
    const int ns = d.ns, nsp = d.nsp, n = ns + 2 * nsp;
    if (nsp == 0) return;
    const int64_t total = (int64_t)n * n;
    for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.y * blockDim.x) {
        const int r = (int)(e % n), c = (int)(e / n);
        if (r < c) continue;
        double v = 0.0;
        if (r < ns) {                       // (w2, w2)
            v = sym_lower(d.M3, d.ld3, r, c);
        } else if (r < ns + nsp) {          // (u, w2) or (u, u)
            const int a = d.keep[r - ns], la = d.lead[a];
            if (c < ns) {
                v = d.M3[(size_t)c * d.ld3 + ns + a];
                if (la >= 0) v -= d.M3[(size_t)c * d.ld3 + ns + la];
            } else {
                const int b = d.keep[c - ns], lb = d.lead[b];
                v = sym_lower(d.M3, d.ld3, ns + a, ns + b);
                if (lb >= 0) v -= sym_lower(d.M3, d.ld3, ns + a, ns + lb);
                if (la >= 0) v -= sym_lower(d.M3, d.ld3, ns + la, ns + b);
                if (la >= 0 && lb >= 0) v += sym_lower(d.M3, d.ld3, ns + la, ns + lb);
            }
        } else {                            // identity row block
            v = (c >= ns && c < ns + nsp && r - ns - nsp == c - ns) ? 1.0 : 0.0;
        }
        d.M3c[(size_t)c * d.ldc + r] = v;
    }
}

void launch_pi_compress(const PiDesc *d, int npairs, int nmax, cudaStream_t s) {
    if (npairs <= 0) return;
    const int64_t n = 3 * (int64_t)nmax;
    const int ny = (int)std::min<int64_t>(64, (n * n + 255) / 256);
    pi_compress_kernel<<<dim3(npairs, std::max(ny, 1)), 256, 0, s>>>(d, npairs);
}

__global__ void pi_expand_kernel(const PiDesc *dd, int np) {
    const PiDesc d = dd[blockIdx.x];
    const int ns = d.ns, nsp = d.nsp;
    if (nsp == 0) return;
    const double *Xc = d.M3c + (size_t)ns * d.ldc + ns + nsp;   // X'(i, j) = Xc[j * ldc + i]
    const int64_t total = (int64_t)ns * nsp;
    for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.y * blockDim.x) {
        const int a = (int)(e % ns), j = (int)(e / ns);
        double v;
        if (d.newidx[a] >= 0) {
            v = Xc[(size_t)j * d.ldc + d.newidx[a]];
        } else {
            // a leads its group: minus the sum of the other members' rows
            v = 0.0;
            const int g = d.grp[a];
            for (int q = d.gptr[g] + 1; q < d.gptr[g + 1]; ++q) v -= Xc[(size_t)j * d.ldc + d.newidx[d.gidx[q]]];
        }
        d.Xg[(size_t)j * d.ldg + a] = v;
    }
}

void launch_pi_expand(const PiDesc *d, int npairs, int nmax, cudaStream_t s) {
    if (npairs <= 0) return;
    const int64_t n = nmax;
    const int ny = (int)std::min<int64_t>(64, (n * n + 255) / 256);
    pi_expand_kernel<<<dim3(npairs, std::max(ny, 1)), 256, 0, s>>>(d, npairs);
}

// one thread per (group, column)
__global__ void pi_project_kernel(const PiDesc *dd, int np) {
    const PiDesc d = dd[blockIdx.x];
    const int64_t total = (int64_t)d.ngroups * d.nsp;
    for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
        const int g = (int)(e % d.ngroups), j = (int)(e / d.ngroups);
        const int q0 = d.gptr[g], q1 = d.gptr[g + 1];
        double *col = d.W1 + (size_t)j * d.ldw;
        double m = 0.0;
        for (int q = q0; q < q1; ++q) m += col[d.gidx[q]];
        m /= (double)(q1 - q0);
        for (int q = q0; q < q1; ++q) col[d.gidx[q]] -= m;
    }
}

void launch_pi_project(const PiDesc *d, int npairs, cudaStream_t s) {
    if (npairs > 0) pi_project_kernel<<<npairs, 256, 0, s>>>(d, npairs);
}

__global__ void pair_weights_kernel(const PairWeightDesc *dd, int np) {
    const PairWeightDesc d = dd[blockIdx.x];
    for (int k = threadIdx.x; k < d.ns; k += blockDim.x) {
        double a = d.diag_i[d.pos_i[k]], b = d.diag_j[d.pos_j[k]];
        d.di[k] = a / (a + b);
        d.dj[k] = b / (a + b);
    }
}

void launch_pair_weights(const PairWeightDesc *d, int npairs, cudaStream_t s) {
    if (npairs > 0) pair_weights_kernel<<<npairs, 128, 0, s>>>(d, npairs);
}

}  // namespace bddc
