// Batched GEMM on the fifth-generation tensor cores (tcgen05, kind::tf32) with
// the three-term TF32 split ("3xTF32"):
//     x = x_hi + x_lo,  x_hi = tf32(x),  x_lo = tf32(x - x_hi),
//     a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi          (relative error ~ 2^-21),
// accumulated in FP32 in tensor memory.  It carries the FP32-class products of
// the mixed-precision interior elimination (the refinement corrections
// X += D K_s D R and the energy correction S -= X^T R of the Schur complement
// of Section 2 of the paper), where FP32 accuracy is what the FP64 refinement
// needs and TF32 alone (2^-11) would stall it.
//
// One CTA per 128 x 128 output tile of one batch item (two CTAs per SM):
//   * the operand slabs (128 rows x 32 FP32 values of A and of B, K
//     contiguous) are copied from global memory by cp.async into a raw shared
//     buffer, one slab ahead of its use; each thread copies and later reads
//     the same 16-byte chunks, so no block barrier separates the two;
//   * each thread splits its chunks into TF32 hi / lo parts and stores them
//     into the K-major 128-byte-swizzled layout (rows of 32 TF32 values = 128
//     bytes, 8-row atoms of 1024 bytes, 16-byte chunk c of row r stored at
//     chunk c ^ (r mod 8));
//   * one thread issues tcgen05.mma (M = 128, N = 128, K = 8 per instruction,
//     4 x 3 instructions per slab) into a 128-column TMEM accumulator and
//     commits them to the stage's mbarrier; the copy of slab k+1 overlaps the
//     split and the MMAs of slab k, and the other CTA on the SM covers the
//     waits of this one;
//   * the epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM
//     lanes 32 (w mod 4) .. + 31, i.e. those output rows) and adds
//     alpha * cscale[m] * acc into the FP64 (or FP32) output with coalesced
//     stores.
// Every mbarrier wait is bounded; on a timeout the CTA records
// BDDC_DEV_ERR_TIMEOUT, waits (bounded) for its issued MMAs, frees its TMEM and
// returns.
#include "common.cuh"
#include "tc_gemm.h"
#include "tcgen05.cuh"

namespace bddc {

namespace {

using namespace tc;

constexpr int TC_THREADS = 256;
constexpr int TC_KB = 32;                     // K per slab: 32 x 4 bytes = one 128-byte swizzle row
constexpr int TC_TILE_BYTES = 128 * 128;      // 128 rows x 128 bytes
constexpr int TC_STAGE_BYTES = 4 * TC_TILE_BYTES;   // A_hi, A_lo, B_hi, B_lo
constexpr int TC_STAGES = 1;                       // split (hi / lo) stage read by the MMAs
constexpr int TC_RAW_STAGES = 1;                   // raw FP32 slab in flight (cp.async)
constexpr int TC_RAW_BYTES = 2 * TC_TILE_BYTES;    // A and B slabs, 128 rows x 128 bytes each
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + TC_RAW_STAGES * TC_RAW_BYTES + 1024;   // + alignment slack
constexpr uint32_t TC_TMEM_COLS = 128;

// instruction descriptor of tcgen05.mma kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32
// (bits 7-9 = bits 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22,
// M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// round to the nearest TF32 value (10 stored mantissa bits; ties away from zero)
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// copy this thread's chunks of slab kb (rows rbase + 32 j of A and B, k values
// kb * 32 + 4 c .. + 3) into a raw stage; outside [0, rows) x [0, K) the chunk is zero
__device__ __forceinline__ void fetch_slab(const TcGemm &g, int m0, int n0, int kb, int rbase, int c, uint32_t raw) {
    const int k = kb * TC_KB + 4 * c;
    const int kv = min(max(g.K - k, 0), 4);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int r = rbase + 32 * j;
        const int ra = m0 + r, rb = n0 + r;
        const float *pa = static_cast<const float *>(g.A);
        const float *pb = static_cast<const float *>(g.B);
        const int ba = ra < g.M ? 4 * kv : 0, bb = rb < g.N ? 4 * kv : 0;
        cp_async16(raw + r * 128 + c * 16, ba ? pa + (size_t)ra * g.lda + k : pa, ba);
        cp_async16(raw + TC_TILE_BYTES + r * 128 + c * 16, bb ? pb + (size_t)rb * g.ldb + k : pb, bb);
    }
}

// split four values into TF32 hi / lo parts and store them at the swizzled chunk
__device__ __forceinline__ void store_split(uint8_t *hi_tile, uint8_t *lo_tile, int r, int c, const float (&v)[4]) {
    float4 h, l;
    float hv[4], lv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        hv[i] = tf32_round(v[i]);
        lv[i] = tf32_round(v[i] - hv[i]);
    }
    h = make_float4(hv[0], hv[1], hv[2], hv[3]);
    l = make_float4(lv[0], lv[1], lv[2], lv[3]);
    const int off = r * 128 + ((c ^ (r & 7)) << 4);
    *reinterpret_cast<float4 *>(hi_tile + off) = h;
    *reinterpret_cast<float4 *>(lo_tile + off) = l;
}

}  // namespace

__global__ void __launch_bounds__(TC_THREADS, 2)
    tc_gemm_kernel(const TcGemm *jobs, const int4 *items, int nitems, DevStatus *st, uint64_t timeout_ns) {
    extern __shared__ uint8_t tc_smem_raw[];
    __shared__ uint64_t bars[TC_STAGES];
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    const int it = blockIdx.x;
    if (it >= nitems) return;
    const int4 w = items[it];
    const TcGemm g = jobs[w.x];
    const int m0 = w.y * kTcM, n0 = w.z * kTcN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const uint32_t raw = smem_u32(tc_smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t *tiles = tc_smem_raw + (sbase - raw);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        failed = 0;
        for (int s = 0; s < TC_STAGES; ++s) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint64_t deadline = globaltimer_ns() + timeout_ns;
    const uint32_t idesc = tc_idesc(kTcM, kTcN);

    const int nkb = (g.K + TC_KB - 1) / TC_KB;
    // this thread's chunks: chunk c = tid % 8 (4 k values) of rows tid / 8 + 32 j
    const int c = tid & 7, rbase = tid >> 3;
    const uint32_t raw0 = sbase + TC_STAGES * TC_STAGE_BYTES;
    bool ok = true;
    int issued = -1;   // last slab whose MMAs were committed (uniform over the block)
    if (nkb > 0) fetch_slab(g, m0, n0, 0, rbase, c, raw0);   // prologue: slab 0 in flight
    cp_async_commit();
    const uint8_t *rawp = tc_smem_raw + (sbase - raw) + TC_STAGES * TC_STAGE_BYTES;
    for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % TC_STAGES;
        float ks[4] = {1.f, 1.f, 1.f, 1.f};
        if (g.bscale) {
            const int k = kb * TC_KB + 4 * c;
#pragma unroll
            for (int i = 0; i < 4; ++i) ks[i] = (k + i < g.K) ? __ldg(g.bscale + k + i) : 0.f;
        }
        cp_async_wait<0>();   // this thread's copies of slab kb have landed
        float4 a4[4], b4[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = rbase + 32 * j;
            a4[j] = *reinterpret_cast<const float4 *>(rawp + r * 128 + c * 16);
            b4[j] = *reinterpret_cast<const float4 *>(rawp + TC_TILE_BYTES + r * 128 + c * 16);
        }
        // slab kb + 1 is copied into the raw buffer while slab kb is split and multiplied
        // (this thread has read its own chunks of slab kb, and only it writes them)
        if (kb + 1 < nkb) fetch_slab(g, m0, n0, kb + 1, rbase, c, raw0);
        cp_async_commit();
        // the split stage is free once the MMAs of the slab that last used it have completed
        if (kb >= TC_STAGES && !mbar_wait(smem_u32(&bars[s]), (uint32_t)(((kb - TC_STAGES) / TC_STAGES) & 1),
                                          deadline)) {
            ok = false;
        }
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
        uint8_t *stage = tiles + s * TC_STAGE_BYTES;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = rbase + 32 * j;
            const float va[4] = {a4[j].x, a4[j].y, a4[j].z, a4[j].w};
            const float vb[4] = {b4[j].x * ks[0], b4[j].y * ks[1], b4[j].z * ks[2], b4[j].w * ks[3]};
            store_split(stage, stage + TC_TILE_BYTES, r, c, va);
            store_split(stage + 2 * TC_TILE_BYTES, stage + 3 * TC_TILE_BYTES, r, c, vb);
        }
        // make the generic-proxy stores visible to the tensor cores (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a_hi = smem_u32(stage), a_lo = a_hi + TC_TILE_BYTES;
            const uint32_t b_hi = a_hi + 2 * TC_TILE_BYTES, b_lo = a_hi + 3 * TC_TILE_BYTES;
#pragma unroll
            for (int kk = 0; kk < TC_KB / 8; ++kk) {
                const uint32_t koff = kk * 32;   // 8 TF32 values = 32 bytes along the swizzled row
                tc_mma(tmem, tc_sdesc(a_lo + koff), tc_sdesc(b_hi + koff), idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                tc_mma(tmem, tc_sdesc(a_hi + koff), tc_sdesc(b_lo + koff), idesc, 1u);
                tc_mma(tmem, tc_sdesc(a_hi + koff), tc_sdesc(b_hi + koff), idesc, 1u);
            }
            tc_commit(smem_u32(&bars[s]));
        }
        issued = kb;
    }
    cp_async_wait<0>();   // no copy may still target this CTA's shared memory at exit
    // the last commit covers every MMA issued before it (after a timeout: wait again, bounded)
    if (issued >= 0) {
        const uint64_t dl = ok ? deadline : globaltimer_ns() + timeout_ns;
        if (!mbar_wait(smem_u32(&bars[issued % TC_STAGES]), (uint32_t)((issued / TC_STAGES) & 1), dl)) ok = false;
    }
    if (!ok && lane == 0) atomicExch(&failed, 1);
    __syncthreads();
    tc_fence_after();
    if (!failed && nkb > 0) {
        const int q = warp & 3, half = warp >> 2;
        const int m = m0 + 32 * q + lane;
        const double csa = g.alpha * ((m < g.M && g.cscale) ? g.cscale[m] : 1.0);
        const float csa_f = (float)csa;   // the FP32 output path stays on the FP32 pipe
#pragma unroll
        for (int part = 0; part < 2; ++part) {
            const int col0 = half * 64 + part * 32;
            uint32_t v[32];
            tc_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col0, v);
            if (m < g.M) {
                if (g.c_f32) {
                    float *C = static_cast<float *>(g.C);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int n = n0 + col0 + j;
                        if (n < g.N) {
                            const float t = csa_f * __uint_as_float(v[j]);
                            C[(size_t)n * g.ldc + m] = g.store ? t : C[(size_t)n * g.ldc + m] + t;
                        }
                    }
                } else {
                    double *C = static_cast<double *>(g.C);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int n = n0 + col0 + j;
                        if (n < g.N) {
                            const double t = (double)__uint_as_float(v[j]);
                            C[(size_t)n * g.ldc + m] = g.store ? csa * t : fma(csa, t, C[(size_t)n * g.ldc + m]);
                        }
                    }
                }
            }
        }
    }
    if (failed && tid == 0) dev_fail(st, BDDC_DEV_ERR_TIMEOUT, w.x, -2);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

void launch_tc_gemm(const TcGemm *jobs, const int4 *items, int nitems, DevStatus *st, double timeout_s,
                    cudaStream_t s) {
    if (nitems <= 0) return;
    cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    const uint64_t tns = (uint64_t)(timeout_s * 1e9);
    tc_gemm_kernel<<<nitems, TC_THREADS, TC_SMEM, s>>>(jobs, items, nitems, st, tns);
}

}  // namespace bddc
