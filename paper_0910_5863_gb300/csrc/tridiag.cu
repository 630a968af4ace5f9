// Householder tridiagonalisation of the large face-pair matrices, several CTAs per
// face (step 1 of the face kernel in eig.cu, for matrices too large for one CTA).
//
// One CTA reduces a matrix of order n in n - 2 dependent steps, each a matrix-vector
// product and a symmetric rank-2 update of the trailing block: order n^3 memory
// traffic through a single SM.  Here the G CTAs of a face share every step: CTA g
// forms the rows [i0, i1) of P = beta B x and, after a barrier of the face's CTAs,
// updates the columns [i0, i1) of B -= x W^T + W x^T (both triangles are kept, as the
// one-CTA reduction keeps them).  Each step's scalars (|x|, alpha, beta, p.x) are
// recomputed by every CTA in the same order, so all CTAs take the same decisions.
// The grid is one cooperative launch (all CTAs co-resident); the barrier of a face
// spins with a bound and records BDDC_DEV_ERR_TIMEOUT instead of hanging.
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
    T *xs = reinterpret_cast<T *>(tri_sm), *Ws = xs + n;
    double *dd = D.work, *ee = D.work + n, *bet = D.work + 2 * n;
    T *P = reinterpret_cast<T *>(D.work + 3 * n);   // shared between the face's CTAs
    unsigned *bar = D.bar;
    auto slice = [&](int len, int &a, int &b) {
        a = (int)((long long)len * g / G);
        b = (int)((long long)len * (g + 1) / G);
    };
    int c0, c1;
    if constexpr (std::is_same<T, ff>::value) {   // to double-float in place, this CTA's columns
        slice(n, c0, c1);
        for (int c = c0; c < c1; ++c)
            for (int i = tid; i < n; i += nt) F[(size_t)c * lda + i] = ff_from_double(Ad[(size_t)c * lda + i]);
    }
    if (!face_barrier(bar, G, st, timeout_ns)) return;
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        const T *x = F + (size_t)k * lda + k + 1;   // column k below the diagonal
        T acc = tri_from<T>(0.0);
        int cnt = 0;
        for (int i = tid; i < m; i += nt) {
            const T v = tri_ld(x + i);
            xs[i] = v;
            tri_fma(acc, v, v);
            if ((++cnt & 15) == 0) acc = tri_norm(acc);
        }
        const double s = tri_block_sum(tri_to(tri_norm(acc)), scratch);
        const double x0 = tri_to(xs[0]);
        const double rest = s - x0 * x0;
        if (rest <= 1e-300 * (s + 1e-300)) {   // already reduced: every CTA takes this branch
            if (g == 0 && tid == 0) {
                bet[k] = 0.0;
                ee[k] = x0;
            }
            continue;
        }
        const double nrm = sqrt(s);
        const double alpha = x0 > 0 ? -nrm : nrm;
        const double v0 = x0 - alpha;
        const double beta = 2.0 / (rest + v0 * v0);
        if (tid == 0) xs[0] = tri_from<T>(v0);
        __syncthreads();
        const T fbeta = tri_from<T>(beta);
        T *B = F + (size_t)(k + 1) * lda + k + 1;
        int i0, i1;
        slice(m, i0, i1);
        // entries [i0, i1) of P = beta B x; B is kept symmetric, so P_i is column i of B
        // against x: one warp per column, contiguous loads
        for (int i = i0 + wid; i < i1; i += nw) {
            const T *col = B + (size_t)i * lda;
            T a = tri_from<T>(0.0);
            int c = 0;
            for (int j = lane; j < m; j += 32) {
                tri_fma(a, tri_ld(col + j), xs[j]);
                if ((++c & 15) == 0) a = tri_norm(a);
            }
            a = tri_warp_sum(tri_norm(a));
            if (lane == 0) P[i] = fbeta * a;
        }
        if (!face_barrier(bar, G, st, timeout_ns)) return;
        T pa = tri_from<T>(0.0);
        cnt = 0;
        for (int i = tid; i < m; i += nt) {
            tri_fma(pa, tri_ld(P + i), xs[i]);
            if ((++cnt & 15) == 0) pa = tri_norm(pa);
        }
        const double pv = tri_block_sum(tri_to(tri_norm(pa)), scratch);
        const T K = tri_from<T>(0.5 * beta * pv);
        for (int i = tid; i < m; i += nt) Ws[i] = tri_ld(P + i) - K * xs[i];
        __syncthreads();
        // columns [i0, i1) of B -= x W^T + W x^T, one warp per column
        for (int j = i0 + wid; j < i1; j += nw) {
            const T wj = Ws[j], xj = xs[j];
            T *col = B + (size_t)j * lda;
            for (int i = lane; i < m; i += 32) col[i] = tri_ld(col + i) - (xs[i] * wj + Ws[i] * xj);
        }
        if (g == 0 && tid == 0) {
            F[(size_t)k * lda + k + 1] = tri_from<T>(v0);   // the reflector's leading entry
            bet[k] = beta;
            ee[k] = alpha;
        }
        if (!face_barrier(bar, G, st, timeout_ns)) return;
    }
    // diagonal, last off-diagonal, and (double-float) the reflectors back to doubles
    slice(n, c0, c1);
    for (int i = c0 + tid; i < c1; i += nt) dd[i] = tri_to(tri_ld(F + (size_t)i * lda + i));
    if (g == 0 && tid == 0) {
        if (n >= 2) {
            ee[n - 2] = tri_to(tri_ld(F + (size_t)(n - 2) * lda + n - 1));
            bet[n - 2] = 0.0;
        }
        bet[n - 1] = 0.0;
        ee[n - 1] = 0.0;
    }
    if constexpr (std::is_same<T, ff>::value) {
        if (!face_barrier(bar, G, st, timeout_ns)) return;   // every diagonal read before rewriting
        for (int c = c0; c < c1; ++c)
            for (int i = c + 1 + tid; i < n; i += nt)
                Ad[(size_t)c * lda + i] = ff_to_double(tri_ld(F + (size_t)c * lda + i));
    }
}

int tridiag_multi_capacity(int nmax) {
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = 2 * sizeof(double) * (size_t)nmax;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tridiag_multi_kernel<ff>, TRI_THREADS, smem);
    int per_sm64 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm64, tridiag_multi_kernel<double>, TRI_THREADS, smem);
    return nsm * std::min(per_sm, per_sm64);
}

cudaError_t launch_tridiag_multi(const TridiagDesc *descs, const int2 *items, int nitems, int nmax, int use_ff,
                                 DevStatus *st, double timeout_s, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    const size_t smem = 2 * sizeof(double) * (size_t)nmax;
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
