// Double-float trailing updates on the tensor cores by exact bf16 slicing (see ozaki.h).
//
// oz_split: one thread per row of the factored block column.  e_r from the largest
//   |L[r, k]| (frexp), then exactly, u = L[r, k] 2^-e_r and for p = 1..7:
//   d_p = rint(u 2^7p), u -= d_p 2^-7p, with u kept as a double-float remainder on the
//   FP32 pipe.  Digit plane p goes to the pre-swizzled layout of ozaki.h as bf16 (16-byte
//   stores of 8 digits).
//
// oz_syrk: persistent, one CTA per SM (211 KB of shared memory, all 512 TMEM columns),
//   output tiles of 128 x 32 taken round robin, three warp roles:
//   * one thread of warp 0 copies, per tile and 32-value K chunk, the 7 digit planes of rows
//     i0.. (A operand, 128 x 32 bf16 each, 8 KB) and of rows j0.. (B operand, 32 x 32, 2 KB)
//     into one of three shared-memory stages with bulk copies (cp.async.bulk; the planes are
//     stored pre-swizzled, K-major with 64-byte swizzling: row r's 16-byte chunk c at chunk
//     c ^ ((r / 2) mod 4)); the stage's mbarrier completes when all bytes have landed;
//   * one thread of warp 1 issues per K = 16 step one MMA per A plane p (tcgen05.mma
//     kind::f16, bf16 inputs, FP32 accumulate): the B planes q = 1 .. 8 - p lie back to back
//     in the stage, so A_p against all of them is one MMA of N = 32 (8 - p) whose 32-column
//     blocks land on the accumulators t = p + q (TMEM columns 224 set + 32 (t - 2) ..); it
//     commits them to the stage's "empty" mbarrier and, after the last chunk, to the set's
//     "full" mbarrier; two accumulator sets let the drain of one tile overlap the products of
//     the next;
//   * warps 2-9 (warp w reads TMEM lanes 32 (w mod 4) .., i.e. those rows, and 16 of the 32
//     columns) fetch the tile's C values while its products run, combine the seven
//     accumulators from t = 8 to t = 2, release the set, scale by 2^(e_i + e_j) and subtract
//     from C.
// Every mbarrier wait is bounded; on a timeout the CTA records BDDC_DEV_ERR_TIMEOUT,
// waits (bounded) for the MMAs it issued, frees its TMEM and returns.
#include <cuda_bf16.h>
#include "common.cuh"
#include "ozaki.h"
#include "tcgen05.cuh"

namespace bddc {

namespace {

using namespace tc;

// warp roles: 0 copies the digit planes into the stages (one thread), 1 issues the MMAs (one
// thread; the warp owns the tensor memory), 2-5 drain the accumulators (warp w reads TMEM
// lanes 32 (w mod 4) ..)
constexpr int OZ_PRODUCER_WARP = 0;
constexpr int OZ_MMA_WARP = 1;
constexpr int OZ_EPI_WARP0 = 2;
constexpr int OZ_EPI_WARPS = 8;                            // two per TMEM lane quarter, 16 columns each
constexpr int OZ_EPI_THREADS = 32 * OZ_EPI_WARPS;
constexpr int OZ_THREADS = 32 * OZ_EPI_WARP0 + OZ_EPI_THREADS;
constexpr int OZ_KC = kOzKC;                               // K per stage: 64-byte rows (64-byte swizzle)
constexpr int OZ_STAGES = 3;
constexpr int OZ_SETS = 2;                                 // accumulator sets in tensor memory
// one MMA takes all B planes of a stage (N = 7 x 32 at most: M = 128 allows N <= 256), and two
// sets of seven accumulators fill the 512 TMEM columns
static_assert(kOzTileN == 32 && kOzTileN * kOzSlices <= 256 && OZ_SETS * kOzSlices * kOzTileN <= 512,
              "tile shape: one MMA per A plane, two sets in 512 TMEM columns");
constexpr int OZ_A_BYTES = kOzTileM * OZ_KC * 2;           // one digit plane of the A operand (8 KB)
constexpr int OZ_B_BYTES = kOzTileN * OZ_KC * 2;           // (2 KB)
constexpr int OZ_STAGE_BYTES = kOzSlices * (OZ_A_BYTES + OZ_B_BYTES);

// global -> shared bulk copy (bytes a multiple of 16, both addresses 16-byte aligned), its
// completion counted in bytes on the mbarrier
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE_BYTES + 1024;
constexpr int OZ_SET_COLS = kOzSlices * kOzTileN;          // one accumulator set (7 x N columns)
constexpr uint32_t OZ_TMEM_COLS = 512;                     // two sets: the drain of a tile overlaps the next

// shared-memory matrix descriptor, K-major with 64-byte swizzling: start address >> 4,
// leading byte offset 16 (unused), stride byte offset 512 (8-row atoms of 64-byte rows),
// descriptor version 1 at bits 46-47, swizzle mode 4 (64 bytes) at bits 61-63
__device__ __forceinline__ uint64_t oz_sdesc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// tcgen05 instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9 =
// bits 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t oz_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kOzTileM >> 4) << 24);
}

// a 2^e (exact unless the result leaves the normal range, where it rounds like ldexpf)
__device__ __forceinline__ ff ff_scale2(ff a, int e) {
    if (e >= -126 && e <= 127) {
        const float p = __int_as_float((e + 127) << 23);
        return ff(a.h * p, a.l * p);
    }
    return ff(ldexpf(a.h, e), ldexpf(a.l, e));
}

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    // two-sum of a.h and b, then the low parts (b is exact; a.l carries the old tail)
    const float s = a.h + b;
    const float bb = s - a.h;
    const float e = (a.h - (s - bb)) + (b - bb);
    const float t = e + a.l;
    const float h = s + t;
    return ff(h, t - (h - s));
}

}  // namespace

__global__ void __launch_bounds__(256) oz_split_kernel(const OzSplitDesc *descs, const int2 *items, int nitems) {
    const int2 w = items[blockIdx.x];
    const OzSplitDesc d = descs[w.x];
    const int r = w.y * 256 + threadIdx.x;
    const int rows_pad = oz_rows_pad(d.rows);
    if (r >= rows_pad) return;
    float mx = 0.f;
    if (r < d.rows)
        for (int c = 0; c < d.k; ++c) mx = fmaxf(mx, fabsf(d.L[(size_t)c * d.ldl + r].h));
    int e = 0;
    if (mx > 0.f) {   // mx = f 2^e, f in [0.5, 1): 2^e > max |x_h|, so |x| 2^-e < 1
        const int be = (__float_as_int(mx) >> 23) & 0xff;
        if (be > 0) e = be - 126;   // normal: read off the exponent field
        else frexpf(mx, &e);
    }
    // 2^-e as a float when it is a normal number (then x 2^-e is exactly ldexpf(x, -e))
    const bool pow2_ok = -e >= -126 && -e <= 127;
    const float sce = pow2_ok ? __int_as_float((127 - e) << 23) : 0.f;
    if (r < d.rows) d.rexp[r] = e;
    // 16-byte chunk ch (8 digits) of row r within K chunk kc, stored at chunk ch ^ ((r / 2) mod 4)
    // of the row's 64 bytes: the shared-memory layout the tensor cores read, so that one
    // contiguous copy moves a whole (plane, chunk, row tile) block.  The digits are taken
    // from the double-float remainder (h, l) on the FP32 pipe: with d = rint(h 2^7p),
    // h - d 2^-7p is exact (Sterbenz), and a two-sum keeps the remainder normalised.
    for (int c0 = 0; c0 < kOzK; c0 += 8) {
        uint16_t dig[kOzSlices][8];
        for (int cc = 0; cc < 8; ++cc) {
            const int c = c0 + cc;
            float rh = 0.f, rl = 0.f;
            if (r < d.rows && c < d.k && mx > 0.f) {
                const ff v = d.L[(size_t)c * d.ldl + r];
                rh = pow2_ok ? v.h * sce : ldexpf(v.h, -e);
                rl = pow2_ok ? v.l * sce : ldexpf(v.l, -e);
            }
#pragma unroll
            for (int p = 0; p < kOzSlices; ++p) {
                const float sc = __int_as_float((127 + 7 * (p + 1)) << 23);    // 2^7(p+1)
                const float isc = __int_as_float((127 - 7 * (p + 1)) << 23);   // 2^-7(p+1)
                const float dp = rintf(rh * sc);
                const float a = rh - dp * isc;   // exact
                const float s2 = a + rl, bb = s2 - a;
                const float err = (a - (s2 - bb)) + (rl - bb);
                rh = s2;
                rl = err;
                dig[p][cc] = __bfloat16_as_ushort(__float2bfloat16_rn(dp));
            }
        }
        const int kc = c0 / kOzKC, ch = (c0 % kOzKC) / 8;
        const int sch = ch ^ ((r >> 1) & 3);
#pragma unroll
        for (int p = 0; p < kOzSlices; ++p) {
            uint4 pk;
            pk.x = (uint32_t)dig[p][0] | ((uint32_t)dig[p][1] << 16);
            pk.y = (uint32_t)dig[p][2] | ((uint32_t)dig[p][3] << 16);
            pk.z = (uint32_t)dig[p][4] | ((uint32_t)dig[p][5] << 16);
            pk.w = (uint32_t)dig[p][6] | ((uint32_t)dig[p][7] << 16);
            *reinterpret_cast<uint4 *>(d.slices + (((size_t)p * (kOzK / kOzKC) + kc) * rows_pad + r) * kOzKC +
                                       sch * 8) = pk;
        }
    }
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_syrk_kernel(const OzSyrkDesc *descs, const int4 *items, int nitems, DevStatus *st, uint64_t timeout_ns) {
    extern __shared__ uint8_t oz_smem_raw[];
    __shared__ uint64_t full[OZ_STAGES], empty[OZ_STAGES], accfull[OZ_SETS], accempty[OZ_SETS], done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t raw = smem_u32(oz_smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;   // swizzle atoms need aligned tiles

    if (warp == OZ_MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(OZ_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < OZ_STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int a = 0; a < OZ_SETS; ++a) {
            mbar_init(smem_u32(&accfull[a]), 1);
            mbar_init(smem_u32(&accempty[a]), OZ_EPI_THREADS);
        }
        mbar_init(smem_u32(&done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint64_t deadline = globaltimer_ns() + timeout_ns;
    auto wait = [&](uint64_t &bar, uint32_t parity) -> bool {
        unsigned spins = 0;
        while (!mbar_try_wait(smem_u32(&bar), parity)) {
            if ((++spins & 1023u) == 0 && (abort_flag || globaltimer_ns() > deadline)) {
                abort_flag = 1;
                return false;
            }
        }
        return true;
    };
    if (warp == OZ_PRODUCER_WARP) {
        // ---- one thread copies, per tile and 32-value K chunk, the 7 digit-plane blocks of rows
        // i0.. (A, 8 KB each) and of rows j0.. (B, 2 KB each) into a stage (bulk copies; the stage's
        // mbarrier completes when all their bytes have landed) ----
        if (lane == 0) {
            int g = 0;
            for (int it = blockIdx.x; it < nitems && !abort_flag; it += gridDim.x) {
                const int4 w = items[it];
                const OzSyrkDesc d = descs[w.x];
                const int i0 = w.y * kOzTileM, j0 = w.z * kOzTileN, rows_pad = oz_rows_pad(d.n),
                          rows_pad_b = oz_rows_pad(d.nb);
                for (int kc = 0; kc < kOzK / kOzKC; ++kc, ++g) {
                    const int s = g % OZ_STAGES;
                    if (g >= OZ_STAGES && !wait(empty[s], (uint32_t)(((g / OZ_STAGES) - 1) & 1))) break;
                    const uint32_t a_base = sbase + s * OZ_STAGE_BYTES, b_base = a_base + kOzSlices * OZ_A_BYTES;
                    const uint32_t fb = smem_u32(&full[s]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                 "r"((uint32_t)OZ_STAGE_BYTES)
                                 : "memory");
                    for (int p = 0; p < kOzSlices; ++p) {
                        const size_t blk = (size_t)p * (kOzK / kOzKC) + kc;
                        bulk_g2s(a_base + p * OZ_A_BYTES, d.slices + (blk * rows_pad + i0) * kOzKC, OZ_A_BYTES, fb);
                        bulk_g2s(b_base + p * OZ_B_BYTES, d.slices_b + (blk * rows_pad_b + j0) * kOzKC, OZ_B_BYTES,
                                 fb);
                    }
                }
            }
        }
    } else if (warp == OZ_MMA_WARP) {
        // ---- one thread issues the 28 digit products per K chunk into the tile's accumulator set ----
        if (lane == 0) {
            int g = 0, li = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++li) {
                const int a = li % OZ_SETS;
                if (li >= OZ_SETS && !wait(accempty[a], (uint32_t)(((li / OZ_SETS) - 1) & 1))) break;
                tc_fence_after();
                const uint32_t abase = tmem + (uint32_t)(a * OZ_SET_COLS);
                for (int kc = 0; kc < kOzK / OZ_KC && ok; ++kc, ++g) {
                    const int s = g % OZ_STAGES;
                    if (!wait(full[s], (uint32_t)((g / OZ_STAGES) & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_base = sbase + s * OZ_STAGE_BYTES, b_base = a_base + kOzSlices * OZ_A_BYTES;
                    // plane p of A against the B planes q = 1 .. 8 - p at once: they are consecutive
                    // 32-row blocks of the stage, i.e. one B operand of N = 32 (8 - p) rows, whose
                    // output block q lands on accumulator p + q (columns 32 (p + q - 2) ..) when the
                    // product starts at column 32 (p - 1).  The first product of a tile (p = 1, all
                    // seven accumulators) overwrites, every later one accumulates.
#pragma unroll
                    for (int kk = 0; kk < OZ_KC / 16; ++kk) {
                        const uint32_t koff = kk * 32;   // 16 bf16 = 32 bytes of the 64-byte row
#pragma unroll
                        for (int p = 1; p <= kOzSlices; ++p)
                            tc_mma_f16(abase + (uint32_t)(kOzTileN * (p - 1)),
                                       oz_sdesc(a_base + (p - 1) * OZ_A_BYTES + koff), oz_sdesc(b_base + koff),
                                       oz_idesc(kOzTileN * (kOzSlices + 1 - p)),
                                       (kc == 0 && kk == 0 && p == 1) ? 0u : 1u);
                    }
                    tc_commit(smem_u32(&empty[s]));   // frees the stage when these products are done
                }
                if (!ok) break;
                tc_commit(smem_u32(&accfull[a]));     // the tile's accumulators are complete
            }
            tc_commit(smem_u32(&done));               // every issued product has completed
            if (!wait(done, 0u)) {
                // bounded again: the tensor memory is freed only after the last products
                const uint64_t dl = globaltimer_ns() + timeout_ns;
                while (!mbar_try_wait(smem_u32(&done), 0u) && globaltimer_ns() < dl) {
                }
            }
        }
    } else if (warp >= OZ_EPI_WARP0) {
        // ---- epilogue: combine the seven accumulators, scale, subtract from C ----
        // Warp w reads TMEM lanes 32 (w mod 4) .. (rows of the tile) and 16 of its 32 columns.
        // The tile's C values and column exponents are fetched before its accumulators are
        // waited for (no other CTA touches this tile), so their latency overlaps the products;
        // lane l holds the exponent of column j0 + l and hands it out by shuffle.
        // Combination, in units of 2^(e_i + e_j): acc_8, acc_7, acc_6 (integers below 2^23) in
        // plain FP32, Horner in 2^-7, with a rounding error below 2^-43, under the 2^-41 of the
        // digit products p + q > 8 that the scheme drops; then acc_5 .. acc_2 one by one in
        // double-float.
        const int q4 = warp & 3, c16 = 16 * ((warp - OZ_EPI_WARP0) >> 2);
        int li = 0;
        for (int it = blockIdx.x; it < nitems && !abort_flag; it += gridDim.x, ++li) {
            const int a = li % OZ_SETS;
            const int4 w = items[it];
            const OzSyrkDesc d = descs[w.x];
            const int i = w.y * kOzTileM + 32 * q4 + lane, j0 = w.z * kOzTileN + c16;
            const bool row_ok = i < d.n, sub = d.mode == 0;
            const int ej = w.z * kOzTileN + lane < d.nb ? d.rexp_b[w.z * kOzTileN + lane] : 0;
            const int ei = row_ok ? d.rexp[i] : 0;
            ff cv[16];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
                const int j = j0 + jj;
                cv[jj] = (sub && row_ok && j <= i) ? d.C[(size_t)j * d.ldc + i] : ff(0.f, 0.f);
            }
            if (!wait(accfull[a], (uint32_t)((li / OZ_SETS) & 1))) break;
            tc_fence_after();
            const uint32_t tbase = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(a * OZ_SET_COLS + c16);
            auto col = [&](int t) { return tbase + (uint32_t)(kOzTileN * (t - 2)); };
            float tail[16];
            {
                uint32_t v8[16], v7[16], v6[16];
                tc_ld16_nowait(col(8), v8);
                tc_ld16_nowait(col(7), v7);
                tc_ld16_nowait(col(6), v6);
                tc_wait_ld();
                const float s7 = __int_as_float((127 - 7) << 23);   // 2^-7
#pragma unroll
                for (int jj = 0; jj < 16; ++jj)
                    tail[jj] = fmaf(fmaf(__uint_as_float(v8[jj]), s7, __uint_as_float(v7[jj])), s7,
                                    __uint_as_float(v6[jj])) * __int_as_float((127 - 42) << 23);   // 2^-42
            }
            ff acc[16];
            {
                uint32_t v5[16], v4[16], v3[16], v2[16];
                tc_ld16_nowait(col(5), v5);
                tc_ld16_nowait(col(4), v4);
                tc_ld16_nowait(col(3), v3);
                tc_ld16_nowait(col(2), v2);
                tc_wait_ld();
                tc_fence_before();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&accempty[a])) : "memory");
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    ff x(tail[jj], 0.f);
                    x = ff_add_f(x, __uint_as_float(v5[jj]) * __int_as_float((127 - 35) << 23));
                    x = ff_add_f(x, __uint_as_float(v4[jj]) * __int_as_float((127 - 28) << 23));
                    x = ff_add_f(x, __uint_as_float(v3[jj]) * __int_as_float((127 - 21) << 23));
                    acc[jj] = ff_add_f(x, __uint_as_float(v2[jj]) * __int_as_float((127 - 14) << 23));
                }
            }
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
                const int j = j0 + jj;
                const int sh = ei + __shfl_sync(0xffffffffu, ej, c16 + jj);
                if (row_ok && (sub ? j <= i : j < d.nb)) {   // mode 0: j <= i < n
                    const ff upd = ff_scale2(acc[jj], sh);
                    d.C[(size_t)j * d.ldc + i] = sub ? cv[jj] - upd : upd;
                }
            }
        }
    }
    __syncthreads();
    if (abort_flag && tid == 0) dev_fail(st, BDDC_DEV_ERR_TIMEOUT, blockIdx.x, -3);
    tc_fence_before();
    __syncthreads();
    if (warp == OZ_MMA_WARP) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS)
                     : "memory");
    }
}

constexpr int OZD_THREADS = 1024;
constexpr int OZD_PITCH = kOzK + 1;   // shared-memory row pitch (ff)

__global__ void __launch_bounds__(OZD_THREADS) oz_diag_kernel(const OzDiagDesc *descs, DevStatus *st) {
    extern __shared__ ff ozd_sm[];
    const OzDiagDesc d = descs[blockIdx.x];
    ff *S = ozd_sm;                        // S[r * pitch + c]: L[r][c] for r >= c, Y[r][c] at S[c * pitch + r]
    ff *yd = ozd_sm + kOzK * OZD_PITCH;     // diagonal of Y
    __shared__ ff invs[kOzK];
    __shared__ int bad;
    const int w = d.w, tid = threadIdx.x, nt = blockDim.x;
    auto at = [&](int r, int c) -> ff & { return S[r * OZD_PITCH + c]; };
    for (int e = tid; e < w * w; e += nt) {
        const int r = e % w, c = e / w;
        if (r >= c) at(r, c) = d.A[(size_t)c * d.ld + r];
        else at(r, c) = ff(0.f, 0.f);   // Y[c][r] = 0
    }
    for (int k = tid; k < w; k += nt) yd[k] = ff(1.f, 0.f);
    // Pivot k: column k of L and row k of Y scaled by 1 / sqrt(d_k), then the trailing block of L
    // and the rows of Y below k updated.  The thread that updates the next diagonal entry forms
    // its reciprocal square root at once, so every pivot costs two barriers.
    auto pivot = [&](int k) {
        ff dk = at(k, k);
        if (!(dk > ff(0.f, 0.f))) {
            bad = 1;
            dk = ff(1.f, 0.f);
            at(k, k) = dk;
        }
        invs[k] = ff_rsqrt(dk);
    };
    if (tid == 0) {
        bad = 0;
        if (w > 0) pivot(0);
    }
    __syncthreads();
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    for (int k = 0; k < w; ++k) {
        const ff inv = invs[k];
        if (tid == 0) at(k, k) = at(k, k) * inv;                              // sqrt(d_k)
        for (int r = k + 1 + tid; r < w; r += nt) at(r, k) *= inv;           // column k of L
        for (int c = tid; c <= k; c += nt) {                                 // row k of Y
            if (c < k) at(c, k) *= inv;
            else yd[k] *= inv;
        }
        __syncthreads();
        const int m = w - k - 1;
        // trailing block of L: lower triangle, a warp per column
        for (int c = k + 1 + wid; c < w; c += nw) {
            const ff lck = at(c, k);
            for (int r = c + lane; r < w; r += 32) {
                at(r, c) -= at(r, k) * lck;
                if (r == k + 1 && c == k + 1) pivot(k + 1);   // thread 0
            }
        }
        // rows below k of Y, columns <= k (flattened, rows fastest: contiguous in shared memory)
        if (m > 0) {
            const int tot = m * (k + 1), dc = nt / m, dr = nt % m;
            int c = tid / m, r = tid % m;
            for (int e = tid; e < tot; e += nt) {
                const ff yk = c < k ? at(c, k) : yd[k];
                at(c, k + 1 + r) -= at(k + 1 + r, k) * yk;
                r += dr;
                c += dc;
                if (r >= m) {
                    r -= m;
                    ++c;
                }
            }
        }
        __syncthreads();
    }
    if (bad && tid == 0) {
        if (d.fail)
            *d.fail = 1;
        else
            dev_fail(st, BDDC_DEV_ERR_NOTSPD, d.tag * 100000 + blockIdx.x, 0);
    }
    for (int e = tid; e < w * w; e += nt) {
        const int r = e % w, c = e / w;
        if (r >= c) d.A[(size_t)c * d.ld + r] = at(r, c);
    }
    for (int e = tid; e < kOzK * kOzK; e += nt) {
        const int r = e % kOzK, c = e / kOzK;
        ff v(0.f, 0.f);
        if (r < w && c < w) v = r > c ? at(c, r) : (r == c ? yd[r] : ff(0.f, 0.f));
        d.Linv[(size_t)c * kOzK + r] = v;
    }
}

void launch_oz_diag(const OzDiagDesc *d, int nd, DevStatus *st, cudaStream_t s) {
    if (nd <= 0) return;
    const int smem = (int)sizeof(ff) * (kOzK * OZD_PITCH + kOzK);
    cudaFuncSetAttribute(oz_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    oz_diag_kernel<<<nd, OZD_THREADS, smem, s>>>(d, st);
}

void launch_oz_split(const OzSplitDesc *d, const int2 *items, int nitems, cudaStream_t s) {
    if (nitems > 0) oz_split_kernel<<<nitems, 256, 0, s>>>(d, items, nitems);
}

void launch_oz_syrk(const OzSyrkDesc *d, const int4 *items, int nitems, DevStatus *st, double timeout_s,
                    cudaStream_t s) {
    if (nitems <= 0) return;
    cudaFuncSetAttribute(oz_syrk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = nitems < nsm ? nitems : nsm;   // persistent: one CTA per SM, tiles round robin
    const uint64_t tns = (uint64_t)(timeout_s * 1e9);
    oz_syrk_kernel<<<grid, OZ_THREADS, OZ_SMEM, s>>>(d, items, nitems, st, tns);
}

}  // namespace bddc
