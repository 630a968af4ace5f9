// PCG on the reduced interface problem with the BDDC preconditioner, as one
// persistent cooperative kernel (Section 2 of the paper: PCG on the reduced
// problem, preconditioner of Lemma 2.1 / eq. (BDDC-prec); the (I-P)^T r step
// is omitted because the residual vanishes in the interiors).
//
// The preconditioner is applied in its primal (local + coarse) form, which
// the paper's Remark 5.1 states is equivalent once every constraint is a
// coarse degree of freedom:
//     r_i = R_i r,  z_i = P~_i r_i,  c_i = Phi~_i^T r_i,
//     u_c = S_C^{-1} sum_i R_ci^T c_i,
//     z   = sum_i R_i^T (z_i + Phi~_i R_ci u_c)
// with the averaging weights folded into P~ = D P D and Phi~ = D Phi.
// All reductions are deterministic: fixed per-block partial sums reduced in
// block order by every block.
#include <cooperative_groups.h>
#include "common.cuh"
#include "pcg.h"
#include <algorithm>

namespace bddc {

constexpr int PCG_THREADS = 512;
constexpr int PCG_WARPS = PCG_THREADS / 32;
constexpr int PCG_PARTIALS = 2048;   // the partials buffer holds two sets of this many blocks

// Data written by other blocks of this launch is read through L2 only
// (ld.global.cg), so no block can see a stale L1 line after a grid barrier.
__device__ __forceinline__ double ldx(const double *p) { return __ldcg(p); }

struct PcgParams {
    IfaceOps o;
    PcgBuffers b;
    int mode;
    double tol;
    int maxit;
    DevStatus *st;
    uint64_t timeout_ns;
};

// y_i = Mats_i * v_i for every (substructure, 64-row block); the blocks take
// the host's bins of items (equal cost within ~2%, the items of a bin ordered
// by substructure), v_i = R_i v is staged in shared memory once per
// substructure of a bin, then the warps split the
// columns and every lane reads two consecutive rows of a column with one
// 16-byte load (512 coalesced bytes per warp and column).  Eight columns per
// warp are loaded before they are used, so 64 KB per SM are in flight: the
// matrices are streamed from HBM once per application.  When they do not fit
// in L2 they are read with the evict-first policy, which keeps the vectors and
// the coarse data resident.
// If pold != nullptr, v[g] = z[g] + beta * pold[g] (the new search direction).
__device__ __forceinline__ double2 ld_mat2(const double *p, bool stream) {
    return stream ? __ldcs(reinterpret_cast<const double2 *>(p)) : __ldg(reinterpret_cast<const double2 *>(p));
}

// Returns this thread's share of sum_i v_i . y_i (the rows it stored), which for
// Mats = S gives p^T S p without assembling S p.
__device__ double local_gemv(const PcgParams &P, double *const *Mats, const double *vin, const double *pold,
                             double beta, double *yout, double *red, double *vs) {
    double vy = 0.0;
    const IfaceOps &o = P.o;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool stream = o.stream_mats != 0;
    int cur = -1;
    for (int bin = blockIdx.x; bin < o.nbins; bin += gridDim.x)
    for (int it = o.binptr[bin]; it < o.binptr[bin + 1]; ++it) {
        int2 w = o.rowblk[it];
        const int s = w.x, r0 = w.y;
        const int n = o.nGi[s], ld = o.ldS[s];
        if (s != cur) {
            const int *RG = o.RG + o.off[s];
            __syncthreads();
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                int g = RG[c];
                vs[c] = pold ? ldx(vin + g) + beta * ldx(pold + g) : ldx(vin + g);
            }
            __syncthreads();
            cur = s;
        }
        const double *A = Mats[s];
        const int r = r0 + 2 * lane;   // ld is even, so A + c * ld + r is 16-byte aligned
        double a0 = 0.0, a1 = 0.0;
        if (r < n) {   // rows r + 1 < ld stay inside the allocation; a row r + 1 >= n is ignored
            int c = wid;
            for (; c + 7 * PCG_WARPS < n; c += 8 * PCG_WARPS) {
                double2 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = ld_mat2(A + (size_t)(c + u * PCG_WARPS) * ld + r, stream);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const double x = vs[c + u * PCG_WARPS];
                    a0 += v[u].x * x;
                    a1 += v[u].y * x;
                }
            }
            for (; c < n; c += PCG_WARPS) {
                const double2 v = ld_mat2(A + (size_t)c * ld + r, stream);
                const double x = vs[c];
                a0 += v.x * x;
                a1 += v.y * x;
            }
        }
        red[wid * 64 + 2 * lane] = a0;
        red[wid * 64 + 2 * lane + 1] = a1;
        __syncthreads();
        if (threadIdx.x < 64) {
            double sum = 0.0;
#pragma unroll
            for (int k = 0; k < PCG_WARPS; ++k) sum += red[k * 64 + threadIdx.x];
            if (r0 + threadIdx.x < n) {
                yout[o.off[s] + r0 + threadIdx.x] = sum;
                vy += vs[r0 + threadIdx.x] * sum;
            }
        }
        __syncthreads();
    }
    return vy;
}

// c_i[m] = Phi~_i[:, m] . r_i
__device__ void coarse_dots(const PcgParams &P, const double *rin) {
    const IfaceOps &o = P.o;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int it = blockIdx.x; it < o.ncdot; it += gridDim.x) {
        int2 w = o.cdot[it];
        int s = w.x, m = w.y + wid;
        if (m < o.nci[s]) {
            int n = o.nGi[s], ld = o.ldS[s];
            const double *col = o.Phi[s] + (size_t)m * ld;
            const int *RG = o.RG + o.off[s];
            double acc = 0.0;
            int k = lane;
            for (; k + 96 < n; k += 128) {   // four independent gathers in flight
                int g[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) g[u] = RG[k + 32 * u];
                double rv[4], cv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    rv[u] = ldx(rin + g[u]);
                    cv[u] = col[k + 32 * u];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) acc += cv[u] * rv[u];
            }
            for (; k < n; k += 32) acc += col[k] * ldx(rin + RG[k]);
            acc = warp_sum(acc);
            if (lane == 0) P.b.cl[o.offc[s] + m] = acc;
        }
    }
}

// u_c = S_C^{-1} r_c; r_c is assembled redundantly in every block (shared memory)
__device__ void coarse_solve(const PcgParams &P, double *rc) {
    const IfaceOps &o = P.o;
    for (int c = threadIdx.x; c < o.nC; c += blockDim.x) {
        double s = 0.0;
        for (int e = o.cptr[c]; e < o.cptr[c + 1]; ++e) s += ldx(P.b.cl + o.cent[e]);
        rc[c] = s;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int row = blockIdx.x * PCG_WARPS + wid; row < o.nC; row += gridDim.x * PCG_WARPS) {
        const double *col = o.SCinv + (size_t)row * o.nC;
        double acc = 0.0;
        for (int c = lane; c < o.nC; c += 32) acc += col[c] * rc[c];
        acc = warp_sum(acc);
        if (lane == 0) P.b.uc[row] = acc;
    }
}

// z[x] = sum over entries (z_i[k] + Phi~_i[k, :] u_c[R_ci]); returns this thread's part of r . z
__device__ double assemble_z(const PcgParams &P, const double *rin, double *zout) {
    const IfaceOps &o = P.o;
    double part = 0.0;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < o.nG; x += gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int e = o.gptr[x]; e < o.gptr[x + 1]; ++e) {
            const ZEntry ze = o.zent[e];   // one record instead of a chain of dependent lookups
            double w = ldx(P.b.zl + ze.pe);
            const int nc = ze.nc, ld = ze.ld, k = 0;
            const double *Ph = ze.phi;
            const int *Rc = ze.rc;
            int m = 0;
            for (; m + 7 < nc; m += 8) {   // eight independent coarse gathers in flight
                int c[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) c[u] = Rc[m + u];
                double uv[8], pv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    uv[u] = ldx(P.b.uc + c[u]);
                    pv[u] = Ph[(size_t)(m + u) * ld + k];
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) w += pv[u] * uv[u];
            }
            for (; m < nc; ++m) w += Ph[(size_t)m * ld + k] * ldx(P.b.uc + Rc[m]);
            v += w;
        }
        zout[x] = v;
        part += rin[x] * v;
    }
    return part;
}

// every warp reduces the block partial sums in the same fixed order
__device__ double reduce_partials(const double *partial, int nb) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < nb; i += 32) s += ldx(partial + i);
    return warp_sum(s);
}

__global__ void __launch_bounds__(PCG_THREADS, 1) pcg_kernel(PcgParams P) {
    extern __shared__ double smem[];
    double *red = smem;                    // PCG_WARPS * 64
    double *rc = smem + PCG_WARPS * 64;    // nC (coarse phase) ...
    double *vs = rc;                       // ... or max nGi (local products)
    __shared__ double scratch[32];
    const IfaceOps &o = P.o;
    PcgBuffers &b = P.b;
    const unsigned nb = gridDim.x;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;

    if (P.mode == PCG_APPLY_M) {
        local_gemv(P, o.P, b.r, nullptr, 0.0, b.zl, red, vs);
        coarse_dots(P, b.r);
        if (!grid_barrier(P.st, nb, P.timeout_ns)) return;
        coarse_solve(P, rc);
        if (!grid_barrier(P.st, nb, P.timeout_ns)) return;
        assemble_z(P, b.r, b.z);
        return;
    }
    if (P.mode == PCG_APPLY_S) {
        local_gemv(P, o.S, b.z, nullptr, 0.0, b.yl, red, vs);
        if (!grid_barrier(P.st, nb, P.timeout_ns)) return;
        for (int x = gtid; x < o.nG; x += gstride) {
            double v = 0.0;
            for (int e = o.gptr[x]; e < o.gptr[x + 1]; ++e) v += ldx(b.yl + o.gent[e]);
            b.q[x] = v;
        }
        return;
    }

    // ---- PCG ----
    double part = 0.0;
    for (int x = gtid; x < o.nG; x += gstride) {
        b.x[x] = 0.0;
        b.p0[x] = 0.0;
        part += b.r[x] * b.r[x];
    }
    part = block_sum(part, scratch);
    if (threadIdx.x == 0) b.partial[blockIdx.x] = part;
    if (!grid_barrier(P.st, nb, P.timeout_ns)) return;
    const double r0 = sqrt(reduce_partials(b.partial, nb));
    double rz_old = 1.0, rr = r0 * r0;
    int k = 0;
    bool conv = (r0 == 0.0);
    double *pold = b.p0, *pnew = b.p1;
    while (!conv && k < P.maxit) {
        ++k;
        // z = M r
        local_gemv(P, o.P, b.r, nullptr, 0.0, b.zl, red, vs);
        coarse_dots(P, b.r);
        if (!grid_barrier(P.st, nb, P.timeout_ns)) return;
        coarse_solve(P, rc);
        if (!grid_barrier(P.st, nb, P.timeout_ns)) return;
        part = assemble_z(P, b.r, b.z);
        part = block_sum(part, scratch);
        if (threadIdx.x == 0) b.partial[blockIdx.x] = part;
        if (!grid_barrier(P.st, nb, P.timeout_ns)) return;
        // beta, p = z + beta p, y_i = S_i p_i
        const double rz = reduce_partials(b.partial, nb);
        const double beta = (k == 1) ? 0.0 : rz / rz_old;
        // p . S p = sum_i p_i . S_i p_i comes out of the local products (second partials
        // buffer: other blocks may still be reading r . z from the first)
        for (int x = gtid; x < o.nG; x += gstride) pnew[x] = b.z[x] + beta * pold[x];
        part = local_gemv(P, o.S, b.z, pold, beta, b.yl, red, vs);
        part = block_sum(part, scratch);
        if (threadIdx.x == 0) b.partial[PCG_PARTIALS + blockIdx.x] = part;
        if (!grid_barrier(P.st, nb, P.timeout_ns)) return;
        const double pq = reduce_partials(b.partial + PCG_PARTIALS, nb);
        if (!(pq > 0.0)) {
            --k;
            break;
        }
        const double alpha = rz / pq;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            b.alpha[k - 1] = alpha;
            if (k > 1) b.beta[k - 2] = beta;
        }
        // q = sum R_i^T y_i assembled on the fly; x += alpha p, r -= alpha q
        part = 0.0;
        for (int x = gtid; x < o.nG; x += gstride) {
            double q = 0.0;
            for (int e = o.gptr[x]; e < o.gptr[x + 1]; ++e) q += ldx(b.yl + o.gent[e]);
            b.x[x] += alpha * pnew[x];
            double rv = b.r[x] - alpha * q;
            b.r[x] = rv;
            part += rv * rv;
        }
        part = block_sum(part, scratch);
        if (threadIdx.x == 0) b.partial[blockIdx.x] = part;
        if (!grid_barrier(P.st, nb, P.timeout_ns)) return;
        rr = reduce_partials(b.partial, nb);
        conv = sqrt(rr) <= P.tol * r0;
        rz_old = rz;
        double *t = pold;
        pold = pnew;
        pnew = t;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *b.iters = k;
        *b.converged = conv ? 1 : 0;
        *b.relres = r0 > 0.0 ? sqrt(rr) / r0 : 0.0;
    }
}

cudaError_t launch_pcg(const IfaceOps &ops, const PcgBuffers &buf, int mode, double tol, int maxit,
                       DevStatus *st, double timeout_s, cudaStream_t s, int *nblocks_out) {
    PcgParams P;
    P.o = ops;
    P.b = buf;
    P.mode = mode;
    P.tol = tol;
    P.maxit = maxit;
    P.st = st;
    P.timeout_ns = (uint64_t)(timeout_s * 1e9);
    size_t smem = sizeof(double) * (PCG_WARPS * 64 + (size_t)std::max(std::max(ops.nC, ops.maxGi), 1));
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(pcg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_kernel, PCG_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (per_sm > 1) per_sm = 1;
    int nblocks = nsm * per_sm;
    if (nblocks > PCG_PARTIALS) nblocks = PCG_PARTIALS;   // the two partials sets of the buffer
    if (nblocks_out) *nblocks_out = nblocks;
    void *args[] = {&P};
    return cudaLaunchCooperativeKernel((void *)pcg_kernel, dim3(nblocks), dim3(PCG_THREADS), args, smem, s);
}

// Self-test of the bounded grid barrier: every block waits for `expect` arrivals.
// With expect > gridDim.x the barrier is never released, the wait runs out after
// timeout_ns, BDDC_DEV_ERR_TIMEOUT is recorded and every block returns.
__global__ void barrier_selftest_kernel(DevStatus *st, unsigned expect, uint64_t timeout_ns, int *passed) {
    if (grid_barrier(st, expect, timeout_ns) && threadIdx.x == 0) atomicAdd(passed, 1);
}

cudaError_t launch_barrier_selftest(DevStatus *st, int extra, double timeout_s, int *passed, cudaStream_t s) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    unsigned expect = (unsigned)(nsm + (extra > 0 ? extra : 0));
    uint64_t tns = (uint64_t)(timeout_s * 1e9);
    void *args[] = {&st, &expect, &tns, &passed};
    return cudaLaunchCooperativeKernel((void *)barrier_selftest_kernel, dim3(nsm), dim3(128), args, 0, s);
}

__global__ void iface_assemble_kernel(IfaceOps o, const double *packed, double *out) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < o.nG; x += gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int e = o.gptr[x]; e < o.gptr[x + 1]; ++e) v += packed[o.gent[e]];
        out[x] = v;
    }
}

__global__ void weights_kernel(IfaceOps o, const double *diag, const double *total, double *delta) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < o.nG; x += gridDim.x * blockDim.x) {
        for (int e = o.gptr[x]; e < o.gptr[x + 1]; ++e) delta[o.gent[e]] = diag[o.gent[e]] / total[x];
    }
}

__global__ void __launch_bounds__(1024) residual_norms2_kernel(const double *g, const double *q, int n, double *out) {
    __shared__ double sa[32], sb[32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double d = g[i] - q[i];
        a += d * d;
        b += g[i] * g[i];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = a;
        sb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            ta += sa[w];
            tb += sb[w];
        }
        out[0] = ta;
        out[1] = tb;
    }
}

void launch_residual_norms2(const double *g, const double *q, int n, double *out, cudaStream_t s) {
    residual_norms2_kernel<<<1, 1024, 0, s>>>(g, q, n, out);
}

void launch_iface_assemble(const IfaceOps &ops, const double *packed, double *out, cudaStream_t s) {
    int blocks = (ops.nG + 255) / 256;
    if (blocks > 0) iface_assemble_kernel<<<blocks, 256, 0, s>>>(ops, packed, out);
}

void launch_weights(const IfaceOps &ops, const double *diag_packed, double *total, double *delta_packed,
                    cudaStream_t s) {
    launch_iface_assemble(ops, diag_packed, total, s);
    int blocks = (ops.nG + 255) / 256;
    if (blocks > 0) weights_kernel<<<blocks, 256, 0, s>>>(ops, diag_packed, total, delta_packed);
}

}  // namespace bddc
