// Float-float ("double-float") arithmetic on the FP32 pipes.
//
// GB300 issues FP32 at about 64 times its FP64 rate, so kernels that need more than FP32
// accuracy (refinement residuals, Krylov reductions over FP32 operators) carry a value as an
// unevaluated sum hi + lo of two floats (about 44 significant bits) using the error-free
// transformations TwoSum (Knuth) and TwoProduct via FMA (Dekker/Ogita-Rump-Oishi).
// Every step uses explicit round-to-nearest intrinsics so that the compiler never contracts
// the error-free steps into fused operations.
#pragma once

#include <cuda_runtime.h>

struct ff {
    float h, l;
};

__device__ __forceinline__ ff ff_from_double(double v) {
    const float h = __double2float_rn(v);
    return ff{h, __double2float_rn(v - (double)h)};
}

// the same split on the host (kernel arguments)
inline ff ff_from_double_host(double v) {
    const float h = (float)v;
    return ff{h, (float)(v - (double)h)};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.h + (double)a.l; }

// exact: a + b = s + e
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// renormalise so that |l| <= ulp(h)/2
__device__ __forceinline__ ff ff_norm(float h, float l) {
    const float s = __fadd_rn(h, l);
    return ff{s, __fsub_rn(l, __fsub_rn(s, h))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return ff_norm(s, e);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return ff_norm(p, e);
}

// acc += a * b (products exact to ~2^-48, sum by TwoSum; acc is left unnormalised:
// acc.l gathers the small parts and is folded in by ff_norm at the end)
__device__ __forceinline__ void ff_fma(ff& acc, ff a, ff b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    float s, t;
    two_sum(acc.h, p, s, t);
    acc.h = s;
    acc.l = __fadd_rn(acc.l, __fadd_rn(t, e));
}

// acc += a * (xh + xl) for a plain float a
__device__ __forceinline__ void ff_fma_f(ff& acc, float a, ff x) {
    const float p = __fmul_rn(a, x.h);
    float e = fmaf(a, x.h, -p);
    e = fmaf(a, x.l, e);
    float s, t;
    two_sum(acc.h, p, s, t);
    acc.h = s;
    acc.l = __fadd_rn(acc.l, __fadd_rn(t, e));
}

// warp-wide sum of (h, l) pairs; the result is valid in lane 0
__device__ __forceinline__ ff ff_warp_sum(ff a) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ff b;
        b.h = __shfl_down_sync(0xffffffffu, a.h, off);
        b.l = __shfl_down_sync(0xffffffffu, a.l, off);
        a = ff_add(a, b);
    }
    return a;
}
