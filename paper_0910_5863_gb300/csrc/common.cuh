// Shared device helpers of the adaptive BDDC library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define BDDC_DEV_ERR_NOTSPD 3
#define BDDC_DEV_ERR_TIMEOUT 6
#define BDDC_DEV_ERR_BOUNDS 9

// Device status block: [0] error code (first writer wins), [1] item id,
// [2] position, [3] barrier arrive counter, [4] barrier generation.
struct DevStatus {
    int code;
    int item;
    int pos;
    unsigned arrive;
    unsigned gen;
    unsigned minpiv;   // FP32 factorizations: bits of the smallest positive pivot seen
    unsigned pad[2];
};

__device__ __forceinline__ void dev_fail(DevStatus *st, int code, int item, int pos) {
    if (atomicCAS(&st->code, 0, code) == 0) {
        st->item = item;
        st->pos = pos;
    }
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  The
// wait is bounded: after timeout_ns it records BDDC_DEV_ERR_TIMEOUT and
// returns false, so every block leaves the kernel instead of hanging.
__device__ __forceinline__ bool grid_barrier(DevStatus *st, unsigned nblocks, uint64_t timeout_ns) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *vgen = &st->gen;
        unsigned g = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(&st->arrive, 1u);
        if (arrived == nblocks - 1) {
            st->arrive = 0;
            __threadfence();
            atomicAdd(&st->gen, 1u);
        } else {
            uint64_t t0 = globaltimer_ns();
            unsigned spins = 0;
            while (*vgen == g) {
                __nanosleep(64);
                if ((++spins & 255u) == 0) {
                    if (globaltimer_ns() - t0 > timeout_ns) {
                        dev_fail(st, BDDC_DEV_ERR_TIMEOUT, -1, -1);
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
        if (*(volatile int *)&st->code == BDDC_DEV_ERR_TIMEOUT) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum; every thread gets the result.  scratch: >= 32 entries.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *scratch) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    T r = 0;
    for (int w = 0; w < nw; ++w) r += scratch[w];
    __syncthreads();
    return r;
}
