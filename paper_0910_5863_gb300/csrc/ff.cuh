// Double-float ("float-float") arithmetic: a value is the unevaluated sum h + l
// of two FP32 numbers with |l| <= ulp(h) / 2, about 48 significant bits.  It runs
// on the FP32 pipe, which on this GPU is ~64x faster than the FP64 pipe, and is
// used for the FP64-class dense factorizations of the mixed precision modes.
//
// The error-free transformations are the classical ones: Knuth's two-sum,
// Dekker's fast two-sum (|a| >= |b|) and the FMA form of the exact product
// (p = a*b, e = fma(a, b, -p), a*b = p + e exactly).  The roundings that these
// rely on use the __f*_rn intrinsics, which the compiler never contracts into
// FMAs or reassociates.
#pragma once
#include <cuda_runtime.h>

namespace bddc {

struct ff {
    float h, l;
    ff() = default;
    __host__ __device__ constexpr ff(float hi, float lo) : h(hi), l(lo) {}
    __host__ __device__ constexpr ff(int v) : h((float)v), l(0.f) {}
};
static_assert(sizeof(ff) == 8, "ff must occupy the bytes of one double");

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ ff ff_from_double(double x) {
    const float h = __double2float_rn(x);
    return ff(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ ff operator+(ff a, ff b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    float h, l;
    fast_two_sum(s, e, h, l);
    return ff(h, l);
}

__device__ __forceinline__ ff operator-(ff a) { return ff(-a.h, -a.l); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }

__device__ __forceinline__ ff operator*(ff a, ff b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    float h, l;
    fast_two_sum(p, e, h, l);
    return ff(h, l);
}

__device__ __forceinline__ ff &operator+=(ff &a, ff b) { return a = a + b; }
__device__ __forceinline__ ff &operator-=(ff &a, ff b) { return a = a - b; }
__device__ __forceinline__ ff &operator*=(ff &a, ff b) { return a = a * b; }
__device__ __forceinline__ bool operator>(ff a, ff b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }

// 1 / sqrt(a) for a > 0: the FP32 estimate refined by one Newton step in ff,
// r1 = r0 + r0 (1 - a r0^2) / 2, which doubles its ~22 correct bits.
__device__ __forceinline__ ff ff_rsqrt(ff a) {
    const ff r0(rsqrtf(a.h), 0.f);
    const ff t = ff(1, 0) - a * (r0 * r0);
    const ff c = r0 * t;
    return r0 + ff(0.5f * c.h, 0.5f * c.l);
}

// acc += a * b without renormalising the low word (the fused inner step of the
// trailing update; acc.l grows by at most a few ulps of acc.h per step and is
// folded in by the caller).
__device__ __forceinline__ void ff_fma_acc(ff &acc, ff a, ff b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    float s, err;
    two_sum(acc.h, p, s, err);
    acc.h = s;
    acc.l = __fadd_rn(acc.l, __fadd_rn(err, e));
}

// acc += a * b for an FP32 b (the same steps as ff_fma_acc with a zero low word of b)
__device__ __forceinline__ void ff_fma_acc_f(ff &acc, ff a, float b) {
    const float p = __fmul_rn(a.h, b);
    float e = fmaf(a.h, b, -p);
    e = fmaf(a.l, b, e);
    float s, err;
    two_sum(acc.h, p, s, err);
    acc.h = s;
    acc.l = __fadd_rn(acc.l, __fadd_rn(err, e));
}

__device__ __forceinline__ ff ff_norm(ff a) {
    float h, l;
    fast_two_sum(a.h, a.l, h, l);
    return ff(h, l);
}

}  // namespace bddc
