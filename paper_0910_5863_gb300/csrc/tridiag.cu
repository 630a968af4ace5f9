// Householder tridiagonalisation of the large face-pair matrices, several CTAs per
// face (step 1 of the face kernel in eig.cu, for matrices too large for one CTA).
//
// One CTA reduces a matrix of order n in n - 2 dependent steps, each a matrix-vector
// product and a symmetric rank-2 update of the trailing block: order n^3 memory
// traffic through a single SM.  Here the G CTAs of a face share every step, and each
// step costs one pass over the trailing block and one barrier of the face's CTAs:
//   * CTA g owns the columns c = g, g + G, ... for the whole reduction;
//   * step k starts with P = beta B x complete (B the trailing block after step k - 1,
//     x the reflector of column k).  Every CTA reads all of P and forms W = P - K x,
//     then column k + 1 after this step's update, x' (the next reflector's column),
//     and its Householder scalars: the same operands in the same order in every CTA,
//     so all CTAs take the same decisions.  Column k + 1 itself is never written in
//     step k, so reading it needs no extra barrier;
//   * each CTA then updates its columns c >= k + 2, B -= x W^T + W x^T, and in the same
//     pass dots them with x' (the next step's P entries), and all CTAs meet once.
// Each step's reflector is written into its column by all CTAs (a share each) at the
// start of the next step, after every CTA has read that column (column 0's, one entry,
// after the barrier that follows P_0).  Both triangles of the
// trailing block are kept below row k + 1 (the row of the current pivot is not updated:
// nothing reads it again).  The grid is one cooperative launch (all CTAs co-resident);
// the barrier of a face spins with a bound and records BDDC_DEV_ERR_TIMEOUT instead of
// hanging.
//
// Output, as the face kernel's step 1 leaves it: the reflectors below the
// subdiagonal of C (as doubles), and in the face's work array dd (diagonal),
// ee (off-diagonal, ee[n-1] = 0) and bet (reflector coefficients, bet[n-2] =
// bet[n-1] = 0).  T = double (FP64 path) or ff (double-float, the mixed paths).
#include <type_traits>
#include "common.cuh"
#include "eig.h"
#include "ff.cuh"

namespace bddc {

constexpr int TRI_THREADS = 256;

template <typename T> __device__ __forceinline__ T tri_from(double x);
template <> __device__ __forceinline__ double tri_from<double>(double x) { return x; }
template <> __device__ __forceinline__ ff tri_from<ff>(double x) { return ff_from_double(x); }
__device__ __forceinline__ double tri_to(double x) { return x; }
__device__ __forceinline__ double tri_to(ff x) { return ff_to_double(x); }
__device__ __forceinline__ void tri_fma(double &acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void tri_fma(ff &acc, ff a, ff b) { ff_fma_acc(acc, a, b); }
__device__ __forceinline__ double tri_norm(double a) { return a; }
__device__ __forceinline__ ff tri_norm(ff a) { return ff_norm(a); }
// c - (a b + d e): two accumulated products, one renormalisation (double-float)
__device__ __forceinline__ double tri_sub2(double c, double a, double b, double d, double e) {
    return fma(-d, e, fma(-a, b, c));
}
__device__ __forceinline__ ff tri_sub2(ff c, ff a, ff b, ff d, ff e) {
    ff_fma_acc(c, -a, b);
    ff_fma_acc(c, -d, e);
    return ff_norm(c);
}

// Loads of data that other CTAs of the face write during the launch bypass L1 (.cg):
// the SMs' L1 caches are not coherent with each other, and a column changes owner as
// the trailing block shrinks, so a line read in an earlier step may be stale.
__device__ __forceinline__ double tri_ld(const double *p) { return __ldcg(p); }
__device__ __forceinline__ ff tri_ld(const ff *p) {
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return ff(v.x, v.y);
}

__device__ __forceinline__ double tri_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ ff tri_warp_sum(ff v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const ff b(__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o));
        v = v + b;
    }
    return v;
}

__device__ __forceinline__ double tri_block_sum(double v, double *scratch) {
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

// Barrier of the G CTAs of one face: bar[0] counts arrivals, bar[1] is the generation.
__device__ __forceinline__ bool face_barrier(unsigned *bar, unsigned G, DevStatus *st, uint64_t timeout_ns) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *vgen = bar + 1;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == G - 1) {
            bar[0] = 0;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            unsigned spins = 0;
            while (*vgen == g) {
                __nanosleep(32);
                if ((++spins & 255u) == 0) {
                    if (globaltimer_ns() - t0 > timeout_ns) {
                        dev_fail(st, BDDC_DEV_ERR_TIMEOUT, -2, -2);
                        ok = 0;
                        break;
                    }
                    if (*(volatile int *)&st->code != 0) {
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Householder scalars of the vector v (length len >= 2, shared memory, every thread):
// alpha (the new off-diagonal), v0 (the reflector's leading entry) and beta = 2 / |v|^2;
// beta = 0 (and v0 = alpha = x0) when v is already reduced.
struct TriHh {
    double alpha, v0, beta;
};
template <typename T>
__device__ TriHh tri_householder(const T *v, int len, double *scratch) {
    T acc = tri_from<T>(0.0);
    int cnt = 0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const T x = v[i];
        tri_fma(acc, x, x);
        if ((++cnt & 15) == 0) acc = tri_norm(acc);
    }
    const double s = tri_block_sum(tri_to(tri_norm(acc)), scratch);
    const double x0 = tri_to(v[0]);
    const double rest = s - x0 * x0;
    if (rest <= 1e-300 * (s + 1e-300)) return TriHh{x0, x0, 0.0};
    const double nrm = sqrt(s);
    const double alpha = x0 > 0 ? -nrm : nrm;
    const double v0 = x0 - alpha;
    return TriHh{alpha, v0, 2.0 / (rest + v0 * v0)};
}

template <typename T>
__global__ void __launch_bounds__(TRI_THREADS) tridiag_multi_kernel(const TridiagDesc *descs, const int2 *items,
                                                                    DevStatus *st, uint64_t timeout_ns) {
    extern __shared__ double tri_sm[];
    __shared__ double scratch[32];
    const int2 w = items[blockIdx.x];
    const TridiagDesc D = descs[w.x];
    const int n = D.n, G = D.G, g = w.y, tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    const size_t lda = D.lda;
    double *Ad = D.A;
    T *F = reinterpret_cast<T *>(Ad);   // ff: a double slot holds one double-float
    T *xs = reinterpret_cast<T *>(tri_sm), *Ws = xs + n, *xn = Ws + n;
    double *dd = D.work, *ee = D.work + n, *bet = D.work + 2 * n;
    T *Pbuf = reinterpret_cast<T *>(D.work + 3 * n);   // P of the even / odd steps, n each, shared by the face
    unsigned *bar = D.bar;
    auto first_own = [&](int c0) { return c0 + ((g - c0) % G + G) % G; };   // first c >= c0 with c = g mod G
    if constexpr (std::is_same<T, ff>::value) {   // to double-float in place, this CTA's columns
        for (int c = g; c < n; c += G)
            for (int i = tid; i < n; i += nt) F[(size_t)c * lda + i] = ff_from_double(Ad[(size_t)c * lda + i]);
    }
    if (!face_barrier(bar, G, st, timeout_ns)) return;
    // step 0's reflector (column 0 below the diagonal) and P_0 over the original columns 1..
    for (int i = tid; i < n - 1; i += nt) xs[i] = tri_ld(F + 1 + i);
    __syncthreads();
    const TriHh h0 = tri_householder(xs, n - 1, scratch);
    if (tid == 0) xs[0] = tri_from<T>(h0.v0);
    __syncthreads();
    if (g == 0 && tid == 0) dd[0] = tri_to(tri_ld(F));
    double beta = h0.beta, alpha = h0.alpha;
    {
        const T fb = tri_from<T>(beta);
        for (int c = first_own(1) + wid * G; c < n; c += nw * G) {
            const T *col = F + (size_t)c * lda + 1;
            T a = tri_from<T>(0.0);
            int cnt = 0;
            for (int i = lane; i < n - 1; i += 32) {
                tri_fma(a, col[i], xs[i]);
                if ((++cnt & 15) == 0) a = tri_norm(a);
            }
            a = tri_warp_sum(tri_norm(a));
            if (lane == 0) Pbuf[c - 1] = fb * a;
        }
    }
    if (!face_barrier(bar, G, st, timeout_ns)) return;
    // column 0's reflector: only its leading entry differs from the column, and it is stored
    // only now, when every CTA of the face has read column 0 (a store before this barrier could
    // reach a CTA still loading the column)
    if (g == 0 && tid == 0) F[1] = tri_from<T>(h0.v0);
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;   // trailing rows / columns k + 1 .. n - 1, local index 0 .. m - 1
        const T *Pk = Pbuf + (size_t)(k & 1) * n;
        T *Pn = Pbuf + (size_t)((k + 1) & 1) * n;
        if (k > 0)   // step k's reflector into column k (every CTA has read that column in step k - 1)
            for (int i = g * nt + tid; i < m; i += G * nt) F[(size_t)k * lda + k + 1 + i] = xs[i];
        // (a) W = P - K x, K = beta (P . x) / 2
        T pa = tri_from<T>(0.0);
        int cnt = 0;
        for (int i = tid; i < m; i += nt) {
            tri_fma(pa, tri_ld(Pk + i), xs[i]);
            if ((++cnt & 15) == 0) pa = tri_norm(pa);
        }
        const double pv = tri_block_sum(tri_to(tri_norm(pa)), scratch);
        const T K = tri_from<T>(0.5 * beta * pv);
        for (int i = tid; i < m; i += nt) Ws[i] = tri_ld(Pk + i) - K * xs[i];
        __syncthreads();
        // (b) column k + 1 after this step: its diagonal and, below, the next reflector's column
        const T *cn = F + (size_t)(k + 1) * lda + (k + 1);
        for (int t = tid; t < m - 1; t += nt) xn[t] = tri_sub2(tri_ld(cn + 1 + t), xs[1 + t], Ws[0], Ws[1 + t], xs[0]);
        if (g == 0 && tid == 0) dd[k + 1] = tri_to(tri_sub2(tri_ld(cn), xs[0], Ws[0], Ws[0], xs[0]));
        __syncthreads();
        const bool more = k + 3 < n;   // a step k + 1 follows
        TriHh hn{0.0, 0.0, 0.0};
        if (more) {
            hn = tri_householder(xn, m - 1, scratch);
            if (tid == 0) xn[0] = tri_from<T>(hn.v0);
            __syncthreads();
        }
        if (g == 0 && tid == 0) {
            bet[k] = beta;
            ee[k] = alpha;
            if (!more) {   // k + 1 = n - 2: the last off-diagonal, no reflection
                ee[k + 1] = tri_to(xn[0]);
                bet[k + 1] = 0.0;
            }
        }
        // (c) own columns c >= k + 2: B -= x W^T + W x^T below row k + 1, and the next P entries.
        // A warp takes two of its columns at a time, so x, W and x' are read from shared memory
        // once for both.
        const T fbn = tri_from<T>(more ? hn.beta : 0.0);
        const int cstep = nw * G;
        for (int c = first_own(k + 2) + wid * G; c < n; c += 2 * cstep) {
            const int c2 = c + cstep;
            const bool two = c2 < n;
            const int j = c - (k + 1), j2 = two ? c2 - (k + 1) : j;
            T *col = F + (size_t)c * lda + (k + 1);
            T *col2 = F + (size_t)(two ? c2 : c) * lda + (k + 1);
            const T wj = Ws[j], xj = xs[j], wj2 = Ws[j2], xj2 = xs[j2];
            T a = tri_from<T>(0.0), a2 = tri_from<T>(0.0);
            cnt = 0;
            for (int i = 1 + lane; i < m; i += 32) {
                const T xi = xs[i], wi = Ws[i];
                const T v = tri_sub2(col[i], xi, wj, wi, xj);
                col[i] = v;
                T v2 = v;
                if (two) {
                    v2 = tri_sub2(col2[i], xi, wj2, wi, xj2);
                    col2[i] = v2;
                }
                if (more) {
                    const T xni = xn[i - 1];
                    tri_fma(a, v, xni);
                    tri_fma(a2, v2, xni);
                    if ((++cnt & 15) == 0) {
                        a = tri_norm(a);
                        a2 = tri_norm(a2);
                    }
                }
            }
            if (more) {
                a = tri_warp_sum(tri_norm(a));
                a2 = tri_warp_sum(tri_norm(a2));
                if (lane == 0) {
                    Pn[c - (k + 2)] = fbn * a;
                    if (two) Pn[c2 - (k + 2)] = fbn * a2;
                }
            }
        }
        beta = more ? hn.beta : 0.0;
        alpha = hn.alpha;
        __syncthreads();   // xs, Ws and xn read by every warp
        for (int t = tid; t < m - 1; t += nt) xs[t] = xn[t];
        if (!face_barrier(bar, G, st, timeout_ns)) return;
    }
    // the last diagonal entry (updated by its owner in the last step)
    if (g == 0 && tid == 0) {
        dd[n - 1] = tri_to(tri_ld(F + (size_t)(n - 1) * lda + n - 1));
        bet[n - 1] = 0.0;
        ee[n - 1] = 0.0;
    }
    if constexpr (std::is_same<T, ff>::value) {   // the reflectors back to doubles, this CTA's columns
        for (int c = g; c < n; c += G)
            for (int i = c + 1 + tid; i < n; i += nt)
                Ad[(size_t)c * lda + i] = ff_to_double(tri_ld(F + (size_t)c * lda + i));
    }
}

int tridiag_multi_capacity(int nmax) {
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = 3 * sizeof(double) * (size_t)nmax;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tridiag_multi_kernel<ff>, TRI_THREADS, smem);
    int per_sm64 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm64, tridiag_multi_kernel<double>, TRI_THREADS, smem);
    return nsm * std::min(per_sm, per_sm64);
}

cudaError_t launch_tridiag_multi(const TridiagDesc *descs, const int2 *items, int nitems, int nmax, int use_ff,
                                 DevStatus *st, double timeout_s, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    const size_t smem = 3 * sizeof(double) * (size_t)nmax;
    uint64_t tns = (uint64_t)(timeout_s * 1e9);
    void *args[] = {&descs, &items, &st, &tns};
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(tridiag_multi_kernel<ff>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(tridiag_multi_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    const void *fn = use_ff ? (const void *)tridiag_multi_kernel<ff> : (const void *)tridiag_multi_kernel<double>;
    return cudaLaunchCooperativeKernel(fn, dim3(nitems), dim3(TRI_THREADS), args, smem, s);
}

}  // namespace bddc
