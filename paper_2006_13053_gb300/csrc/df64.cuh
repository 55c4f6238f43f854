// Double-float arithmetic: a value is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2, giving about 48 significant bits on the FP32 pipes.  The operations are
// built from the error-free transformations two-sum (Knuth) and two-product via a fused
// multiply-add (Dekker's product with FMA).  Addition is Dekker's double-word sum (two-sum of
// the high words, low words added, one renormalisation): its error is bounded relative to
// |a| + |b| (not |a + b|), which is the normwise bound an FFT's error analysis uses.
// Multiplication keeps the cross terms hi*lo.
// Used for the refinement's model evaluation, where FP64 throughput is the bottleneck.
#pragma once
#include <cuda_runtime.h>

namespace sfft {

// explicitly rounded float operations: never contracted into FMAs by the compiler
#ifdef __CUDA_ARCH__
#define DF_ADD(a, b) __fadd_rn((a), (b))
#define DF_SUB(a, b) __fsub_rn((a), (b))
#define DF_MUL(a, b) __fmul_rn((a), (b))
#else
#define DF_ADD(a, b) ((a) + (b))
#define DF_SUB(a, b) ((a) - (b))
#define DF_MUL(a, b) ((a) * (b))
#endif

struct alignas(8) df64 {
    float hi, lo;
};

__host__ __device__ __forceinline__ df64 df_two_sum(float a, float b) {
    float s = DF_ADD(a, b);
    float bb = DF_SUB(s, a);
    float e = DF_ADD(DF_SUB(a, DF_SUB(s, bb)), DF_SUB(b, bb));
    return df64{s, e};
}
__host__ __device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {  // needs |a| >= |b|
    float s = DF_ADD(a, b);
    float e = DF_SUB(b, DF_SUB(s, a));
    return df64{s, e};
}
__host__ __device__ __forceinline__ df64 operator+(df64 a, df64 b) {
    df64 s = df_two_sum(a.hi, b.hi);
    s.lo = DF_ADD(s.lo, DF_ADD(a.lo, b.lo));
    return df_fast_two_sum(s.hi, s.lo);
}
__host__ __device__ __forceinline__ df64 operator-(df64 a) { return df64{-a.hi, -a.lo}; }
__host__ __device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__host__ __device__ __forceinline__ df64 operator*(df64 a, df64 b) {
    float p = DF_MUL(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
__host__ __device__ __forceinline__ df64 df_from(double v) {
    float h = (float)v;
    return df64{h, (float)(v - (double)h)};
}
__host__ __device__ __forceinline__ double df_to(df64 a) { return (double)a.hi + (double)a.lo; }

// ------------------------------------------------------------------ scalar traits
template <class T> __host__ __device__ __forceinline__ T kc(double v) { return (T)v; }
template <> __host__ __device__ __forceinline__ df64 kc<df64>(double v) { return df_from(v); }

__host__ __device__ __forceinline__ double to_d(float v) { return (double)v; }
__host__ __device__ __forceinline__ double to_d(double v) { return v; }
__host__ __device__ __forceinline__ double to_d(df64 v) { return df_to(v); }

template <class T> __host__ __device__ __forceinline__ T from_d(double v) { return (T)v; }
template <> __host__ __device__ __forceinline__ df64 from_d<df64>(double v) { return df_from(v); }

}  // namespace sfft
