// Batched LOBPCG for the large face-pair eigenproblems (see lobpcg.h).
//
// One iteration over all large faces (the host loop in the adapt phase):
//   GEMM       C X for every face (batched FP64 GEMM, dense.cu), fresh each iteration;
//   lob_prep   (one CTA per face)  Rayleigh quotients theta_j = x_j^T (C x_j) of the
//              current block, residuals R = C X - X diag(theta), the convergence
//              test, and unit-norm columns of R and P (with C R, C P scaled alike);
//   GEMM       C R for every face (batched FP64 GEMM, dense.cu);
//   GEMM       Gram matrices S^T C S and S^T S of the trial space S = [X P R];
//   lob_rr     (one CTA per face)  Rayleigh-Ritz in FP64: S^T S = V diag(mu) V^T by
//              cyclic Jacobi, the numerically independent directions Z = V mu^-1/2
//              (mu > 1e-10 max mu), H = Z^T (S^T C S) Z by Jacobi again; the k largest
//              eigenpairs (theta, Y) give X_new = S Z Y and P_new = [0 P R] Z Y;
//   GEMM       [X_new | P_new] = S [cX | cP] and C P_new = (C S) cP.
// The trial space of the first iteration is [X, 0, C X].
#include <algorithm>
#include "common.cuh"
#include "lobpcg.h"

namespace bddc {

constexpr int LOB_THREADS = 256;

__device__ __forceinline__ double lob_block_sum(double v, double *scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double r = 0.0;
    for (int w = 0; w < nw; ++w) r += scratch[w];
    __syncthreads();
    return r;
}

// splitmix64 finaliser as a counter-based hash: a value in [-1, 1) per (i, j, seed)
__device__ __forceinline__ double lob_hash(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (double)(x >> 11) * 0x1p-52 - 1.0;
}

__global__ void lob_init_kernel(const LobDesc *descs, int nd, int cur) {
    const LobDesc d = descs[blockIdx.x];
    const int n = d.n, k = d.k;
    // both buffers fully defined: the update multiplies every column of S by its
    // coefficient (zeros included), so no column may hold a non-finite leftover
    for (int e = threadIdx.x; e < n * 3 * k; e += blockDim.x) {
        const int i = e % n, j = e / n;
        const size_t o = (size_t)j * d.lds + i;
        d.S[cur][o] = j < k ? lob_hash(((uint64_t)blockIdx.x << 40) ^ ((uint64_t)j << 20) ^ i) : 0.0;
        d.S[1 - cur][o] = 0.0;
        d.AS[0][o] = 0.0;
        d.AS[1][o] = 0.0;
    }
    for (int j = threadIdx.x; j < k; j += blockDim.x) d.theta[j] = 0.0;
    if (threadIdx.x == 0) d.state[0] = d.state[1] = d.state[2] = 0;
}

// Rayleigh quotients, residual block and convergence test; unit columns of R and P.
__global__ void __launch_bounds__(LOB_THREADS) lob_prep_kernel(const LobDesc *descs, int nd, int cur, double tau,
                                                               int fixed_k, double rtol, int final_check) {
    const LobDesc d = descs[blockIdx.x];
    if (final_check ? d.state[2] != 1 : d.state[0] != 0) return;
    const int n = d.n, k = d.k, tid = threadIdx.x;
    double *S = d.S[cur], *AS = d.AS[cur];
    const size_t ld = d.lds;
    __shared__ double scratch[32];
    __shared__ double th[kLobMaxK], rn[kLobMaxK];
    for (int j = 0; j < k; ++j) {
        const double *x = S + (size_t)j * ld, *ax = AS + (size_t)j * ld;
        double xx = 0.0, xax = 0.0;
        for (int i = tid; i < n; i += blockDim.x) {
            xx += x[i] * x[i];
            xax += x[i] * ax[i];
        }
        xx = lob_block_sum(xx, scratch);
        xax = lob_block_sum(xax, scratch);
        const double t = xx > 0.0 ? xax / xx : 0.0;
        double *r = S + (size_t)(2 * k + j) * ld;
        double rr = 0.0;
        for (int i = tid; i < n; i += blockDim.x) {
            const double v = ax[i] - t * x[i];
            r[i] = v;
            rr += v * v;
        }
        rr = lob_block_sum(rr, scratch);
        if (tid == 0) {
            th[j] = t;
            rn[j] = sqrt(rr / (xx > 0.0 ? xx : 1.0));
            d.rnorm[j] = rn[j];
        }
        __syncthreads();
    }
    // convergence: the selected pairs and the largest rejected one, residual small against
    // their Ritz value (with a floor at the rounding level of the largest)
    __shared__ int verdict;
    if (tid == 0) {
        double tmax = 0.0;
        for (int j = 0; j < k; ++j) tmax = fmax(tmax, fabs(th[j]));
        int nsel = 0;
        if (fixed_k > 0) {
            nsel = min(fixed_k, n);
        } else {
            for (int j = 0; j < k; ++j) nsel += th[j] > tau ? 1 : 0;
        }
        const int need = min(nsel + 1, n);
        int v = 1;   // converged
        if (!final_check && d.state[1] == 0) {
            v = 0;   // the start block has had no Rayleigh-Ritz step yet
        } else if (need > k) {
            v = 2;   // k Ritz values above tau bound k eigenvalues from below: block too small
        } else {
            for (int j = 0; j < need; ++j)
                if (!(rn[j] <= rtol * fabs(th[j]) + 1e-13 * tmax)) v = 0;
        }
        verdict = v;
        for (int j = 0; j < k; ++j) d.theta[j] = th[j];
        if (final_check) {
            if (v != 1) d.state[2] = 4;   // the fresh residuals do not pass
        } else {
            d.state[1] += 1;
            if (v) {
                d.state[0] = 1;
                d.state[2] = v;
            }
        }
    }
    __syncthreads();
    if (verdict || final_check) return;
    // unit columns of R (and of C R, recomputed by the caller's GEMM) and of P, C P
    for (int j = 0; j < 2 * k; ++j) {
        const int col = j < k ? 2 * k + j : j;   // R columns, then P columns (k .. 2k)
        double *v = S + (size_t)col * ld;
        double s2 = 0.0;
        for (int i = tid; i < n; i += blockDim.x) s2 += v[i] * v[i];
        s2 = lob_block_sum(s2, scratch);
        const double sc = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
        double *av = AS + (size_t)col * ld;
        for (int i = tid; i < n; i += blockDim.x) {
            v[i] *= sc;
            if (j >= k) av[i] *= sc;
        }
        __syncthreads();
    }
}

// Cyclic Jacobi on the symmetric m x m matrix A (shared memory, ld m, both triangles
// significant), accumulating the rotations into V (= I on entry).  Parallel ordering:
// in every round the index pairs of a round-robin tournament are disjoint, so their
// rotations are applied together (first to the columns of A and V, then to the rows).
// A rotation is skipped when |a_pq| is below 1e-15 sqrt(|a_pp a_qq|) or 1e-14 of the
// largest diagonal entry (the rounding level a rotation itself leaves behind, so the
// loop cannot go on rotating noise); a sweep without rotations ends the loop.
__device__ void lob_jacobi(double *A, double *V, int m, double *cs, double *scratch) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int mm = m + (m & 1), half = mm / 2;
    __shared__ int rotated;
    __shared__ double amax_sh;
    for (int sweep = 0; sweep < 30; ++sweep) {
        if (tid == 0) {
            double a = 0.0;
            for (int i = 0; i < m; ++i) a = fmax(a, fabs(A[(size_t)i * m + i]));
            amax_sh = a;
            rotated = 0;
        }
        __syncthreads();
        const double floor_abs = 1e-14 * amax_sh;
        for (int round = 0; round < mm - 1; ++round) {
            for (int t = tid; t < half; t += nt) {
                // circle method: player 0 fixed, the others rotate
                const int a = t == 0 ? 0 : 1 + (t - 1 + round) % (mm - 1);
                const int b = 1 + (mm - 2 - t + round) % (mm - 1);
                int p = min(a, b), q = max(a, b);
                double c = 1.0, s = 0.0;
                bool rot = false;
                if (q < m) {
                    const double apq = A[(size_t)q * m + p];
                    const double app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q];
                    if (fabs(apq) > floor_abs && fabs(apq) > 1e-15 * sqrt(fabs(app * aqq))) {
                        const double th = (aqq - app) / (2.0 * apq);
                        const double tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(tt * tt + 1.0);
                        s = tt * c;
                        rot = true;
                    }
                }
                if (!rot) p = q = -1;
                else rotated = 1;
                cs[4 * t] = c;
                cs[4 * t + 1] = s;
                reinterpret_cast<int *>(cs + 4 * t + 2)[0] = p;
                reinterpret_cast<int *>(cs + 4 * t + 2)[1] = q;
            }
            __syncthreads();
            // columns: A J and V J
            for (int e = tid; e < m * half; e += nt) {
                const int i = e % m, t = e / m;
                const int p = reinterpret_cast<const int *>(cs + 4 * t + 2)[0];
                const int q = reinterpret_cast<const int *>(cs + 4 * t + 2)[1];
                if (p < 0) continue;
                const double c = cs[4 * t], s = cs[4 * t + 1];
                const double aip = A[(size_t)p * m + i], aiq = A[(size_t)q * m + i];
                A[(size_t)p * m + i] = c * aip - s * aiq;
                A[(size_t)q * m + i] = s * aip + c * aiq;
                const double vip = V[(size_t)p * m + i], viq = V[(size_t)q * m + i];
                V[(size_t)p * m + i] = c * vip - s * viq;
                V[(size_t)q * m + i] = s * vip + c * viq;
            }
            __syncthreads();
            // rows: J^T (A J)
            for (int e = tid; e < m * half; e += nt) {
                const int j = e % m, t = e / m;
                const int p = reinterpret_cast<const int *>(cs + 4 * t + 2)[0];
                const int q = reinterpret_cast<const int *>(cs + 4 * t + 2)[1];
                if (p < 0) continue;
                const double c = cs[4 * t], s = cs[4 * t + 1];
                const double apj = A[(size_t)j * m + p], aqj = A[(size_t)j * m + q];
                A[(size_t)j * m + p] = c * apj - s * aqj;
                A[(size_t)j * m + q] = s * apj + c * aqj;
            }
            __syncthreads();
        }
        if (!rotated) break;
        __syncthreads();
    }
    (void)scratch;
}

// Rayleigh-Ritz on the trial space (see the file comment).  Shared memory: two m x m
// matrices (m = 3k <= 96) and the rotation table.
__global__ void __launch_bounds__(LOB_THREADS) lob_rr_kernel(const LobDesc *descs, int nd) {
    extern __shared__ double sm[];
    const LobDesc d = descs[blockIdx.x];
    const int k = d.k, m = 3 * k, tid = threadIdx.x, nt = blockDim.x;
    double *A = sm, *V = sm + (size_t)m * m, *cs = V + (size_t)m * m;
    __shared__ double scratch[32];
    __shared__ double mu[3 * kLobMaxK];
    __shared__ int idx[3 * kLobMaxK];
    __shared__ int r_sh;
    double *coef = d.coef;   // 3k x 2k, ld m
    if (d.state[0]) {   // converged: X and P stay (identity coefficients)
        for (int e = tid; e < m * 2 * k; e += nt) {
            const int i = e % m, j = e / m;
            coef[(size_t)j * m + i] = (i == j) ? 1.0 : 0.0;
        }
        return;
    }
    const double *GA = d.G, *GB = d.G + (size_t)m * m;
    double *Z = d.scratch, *T = d.scratch + (size_t)m * m;
    // 1. S^T S = V diag(mu) V^T
    for (int e = tid; e < m * m; e += nt) {
        const int i = e % m, j = e / m;
        A[e] = 0.5 * (GB[e] + GB[(size_t)i * m + j]);
        V[e] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    lob_jacobi(A, V, m, cs, scratch);
    if (tid == 0) {
        double mx = 0.0;
        for (int i = 0; i < m; ++i) mx = fmax(mx, A[(size_t)i * m + i]);
        int r = 0;
        for (int i = 0; i < m; ++i) {
            const double v = A[(size_t)i * m + i];
            if (v > 1e-10 * mx) {
                mu[r] = v;
                idx[r] = i;
                ++r;
            }
        }
        r_sh = r;
    }
    __syncthreads();
    const int r = r_sh;
    // 2. Z = V(:, kept) mu^-1/2 (m x r, ld m) into global scratch
    for (int e = tid; e < m * r; e += nt) {
        const int i = e % m, j = e / m;
        Z[(size_t)j * m + i] = V[(size_t)idx[j] * m + i] / sqrt(mu[j]);
    }
    __syncthreads();
    // 3. T = GA Z (m x r), then H = Z^T T (r x r) into A
    for (int e = tid; e < m * r; e += nt) {
        const int i = e % m, j = e / m;
        double acc = 0.0;
        for (int l = 0; l < m; ++l) acc += 0.5 * (GA[(size_t)l * m + i] + GA[(size_t)i * m + l]) * Z[(size_t)j * m + l];
        T[(size_t)j * m + i] = acc;
    }
    __syncthreads();
    for (int e = tid; e < r * r; e += nt) {
        const int i = e % r, j = e / r;
        double acc = 0.0;
        for (int l = 0; l < m; ++l) acc += Z[(size_t)i * m + l] * T[(size_t)j * m + l];
        A[(size_t)j * r + i] = acc;
    }
    __syncthreads();
    for (int e = tid; e < r * r; e += nt) {   // symmetrise
        const int i = e % r, j = e / r;
        if (i > j) {
            const double v = 0.5 * (A[(size_t)j * r + i] + A[(size_t)i * r + j]);
            A[(size_t)j * r + i] = v;
            A[(size_t)i * r + j] = v;
        }
        V[e] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    lob_jacobi(A, V, r, cs, scratch);
    // 4. the k largest: order by eigenvalue, descending
    if (tid == 0) {
        for (int i = 0; i < r; ++i) {
            mu[i] = A[(size_t)i * r + i];
            idx[i] = i;
        }
        for (int i = 1; i < r; ++i) {   // insertion sort (r <= 96)
            const double v = mu[i];
            const int id = idx[i];
            int j = i - 1;
            while (j >= 0 && mu[j] < v) {
                mu[j + 1] = mu[j];
                idx[j + 1] = idx[j];
                --j;
            }
            mu[j + 1] = v;
            idx[j + 1] = id;
        }
    }
    __syncthreads();
    // coefficients: cX = Z Y (m x k), cP = the same with the X rows zeroed
    for (int e = tid; e < m * k; e += nt) {
        const int i = e % m, j = e / m;
        double acc = 0.0;
        if (j < r)
            for (int l = 0; l < r; ++l) acc += Z[(size_t)l * m + i] * V[(size_t)idx[j] * r + l];
        coef[(size_t)j * m + i] = acc;
        coef[(size_t)(k + j) * m + i] = i < k ? 0.0 : acc;
    }
    for (int j = tid; j < k; j += nt) d.theta[j] = j < r ? mu[j] : 0.0;
    if (tid == 0 && r < k) {   // the trial space lost rank: give up on this face
        d.state[0] = 1;
        d.state[2] = 3;
    }
}

// Certificate matrix, lower triangle: M = sigma I - C + sum_{l < nsel} theta_l x_l x_l^T
// (x_l normalised).  items: one CTA per (matrix, 64-column block).
__global__ void __launch_bounds__(256) lob_cert_kernel(const LobCertDesc *descs, const int2 *items, int nitems) {
    const int2 w = items[blockIdx.x];
    const LobCertDesc d = descs[w.x];
    const int n = d.n, nsel = min(max(*d.nsel, 0), d.k - 1);
    __shared__ double xn[kLobMaxK];
    __shared__ double scratch[32];
    __shared__ double sigma_sh;
    // 1 / |x_l|^2 for the selected vectors, sigma from the largest rejected Ritz value
    for (int l = 0; l < nsel; ++l) {
        double s2 = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) s2 += d.X[(size_t)l * d.ldx + i] * d.X[(size_t)l * d.ldx + i];
        s2 = lob_block_sum(s2, scratch);
        if (threadIdx.x == 0) xn[l] = d.theta[l] / s2;
    }
    if (threadIdx.x == 0) {
        // the gap above the largest rejected value: relative to it, and at least 1e-9 of
        // the largest Ritz value (a Cholesky of M resolves that much against |C|)
        const double t = d.theta[nsel];
        sigma_sh = t + fmax(d.sigma_rel * fabs(t), fmax(1e-9 * fabs(d.theta[0]), 1e-300));
    }
    __syncthreads();
    const double sigma = sigma_sh;
    const int c0 = w.y * 64;
    for (int e = threadIdx.x; e < 64 * n; e += blockDim.x) {
        const int i = e % n, c = c0 + e / n;
        if (c >= n || i < c) continue;
        double v = -d.C[(size_t)c * d.ldc + i] + (i == c ? sigma : 0.0);
        for (int l = 0; l < nsel; ++l) v += xn[l] * d.X[(size_t)l * d.ldx + i] * d.X[(size_t)l * d.ldx + c];
        d.M[(size_t)c * d.ldm + i] = v;
    }
}

// Selection and outputs of converged faces (one CTA each).
__global__ void lob_select_kernel(const LobOutDesc *descs, int nd, double tau, int fixed_k) {
    const LobOutDesc d = descs[blockIdx.x];
    const int n = d.n, k = d.k;
    __shared__ int nsel_sh, ties_sh, over_sh, nval_sh;
    __shared__ double scratch[32];
    if (d.state[2] != 1) {   // not converged: the dense kernel solves this face
        if (threadIdx.x == 0)
            for (int c = 0; c < 5; ++c) d.counts[c] = 0;
        return;
    }
    if (threadIdx.x == 0) {
        int nsel = 0, ties = 0;
        if (fixed_k > 0) {
            nsel = min(fixed_k, n);
            if (nsel > 0 && nsel < k && fabs(d.theta[nsel] / d.theta[nsel - 1] - 1.0) < 1e-6) ties = 1;
        } else {
            for (int j = 0; j < k; ++j) {
                nsel += d.theta[j] > tau ? 1 : 0;
                ties += fabs(d.theta[j] / tau - 1.0) < 1e-6 ? 1 : 0;
            }
        }
        int over = 0;   // > 0: the selected count when it exceeds the capacity
        if (nsel > d.cap) {
            over = nsel;
            nsel = d.cap;
        }
        nsel_sh = nsel;
        ties_sh = ties;
        over_sh = over;
        nval_sh = min(nsel + 1, min(n, k));
    }
    __syncthreads();
    const int nsel = nsel_sh, nval = nval_sh;
    for (int j = threadIdx.x; j < nval; j += blockDim.x) d.lam[j] = d.theta[j];
    for (int l = 0; l < nsel; ++l) {
        const double *x = d.X + (size_t)l * d.ldx;
        double s2 = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) s2 += x[i] * x[i];
        s2 = lob_block_sum(s2, scratch);
        const double inv = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) d.vec[(size_t)l * n + i] = x[i] * inv;
    }
    if (threadIdx.x == 0) {
        d.counts[0] = nsel;
        d.counts[1] = 0;
        d.counts[2] = nval;
        d.counts[3] = ties_sh;
        d.counts[4] = over_sh;
    }
}

// C <- (C + C^T) / 2 (the reduction products are symmetric only to rounding; LOBPCG's
// residuals are measured against the symmetric matrix).  items: (descriptor, 64-column block).
__global__ void lob_symmetrize_kernel(const LobDesc *descs, const int2 *items, int nitems) {
    const int2 w = items[blockIdx.x];
    const LobDesc d = descs[w.x];
    double *C = const_cast<double *>(d.C);
    const int n = d.n, c0 = w.y * 64;
    for (int e = threadIdx.x; e < 64 * n; e += blockDim.x) {
        const int i = e % n, c = c0 + e / n;
        if (c >= n || i <= c) continue;
        const double v = 0.5 * (C[(size_t)c * d.ldc + i] + C[(size_t)i * d.ldc + c]);
        C[(size_t)c * d.ldc + i] = v;
        C[(size_t)i * d.ldc + c] = v;
    }
}

void launch_lob_symmetrize(const LobDesc *d, const int2 *items, int nitems, cudaStream_t s) {
    if (nitems > 0) lob_symmetrize_kernel<<<nitems, 256, 0, s>>>(d, items, nitems);
}
void launch_lob_init(const LobDesc *d, int nd, int cur, cudaStream_t s) {
    if (nd > 0) lob_init_kernel<<<nd, 256, 0, s>>>(d, nd, cur);
}
void launch_lob_prep(const LobDesc *d, int nd, int cur, double tau, int fixed_k, double rtol, int final_check,
                     cudaStream_t s) {
    if (nd > 0) lob_prep_kernel<<<nd, LOB_THREADS, 0, s>>>(d, nd, cur, tau, fixed_k, rtol, final_check);
}
void launch_lob_rr(const LobDesc *d, int nd, cudaStream_t s) {
    if (nd <= 0) return;
    const int m = 3 * kLobMaxK;
    const size_t smem = sizeof(double) * (2 * (size_t)m * m + 4 * (size_t)(m / 2 + 1));
    cudaFuncSetAttribute(lob_rr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    lob_rr_kernel<<<nd, LOB_THREADS, smem, s>>>(d, nd);
}
void launch_lob_cert(const LobCertDesc *d, const int2 *items, int nitems, cudaStream_t s) {
    if (nitems > 0) lob_cert_kernel<<<nitems, 256, 0, s>>>(d, items, nitems);
}
void launch_lob_select(const LobOutDesc *d, int nd, double tau, int fixed_k, cudaStream_t s) {
    if (nd > 0) lob_select_kernel<<<nd, 256, 0, s>>>(d, nd, tau, fixed_k);
}

}  // namespace bddc
