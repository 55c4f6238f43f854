// Device code of the batched Bluestein transforms (Algorithm 2): a length-M DFT becomes
// a cyclic convolution of length N = 2^a 3^b 5^c >= 2M-1, computed by an in-place mixed-radix
// decimation-in-frequency FFT (natural order in, digit-reversed out), a pointwise product with
// the precomputed filter (itself stored digit-reversed) and the matching decimation-in-time
// inverse (digit-reversed in, natural order out), so no reordering pass is needed.  One CTA
// transforms one lattice; the work buffer lives in shared memory when N complex values fit, in
// the shared memory of a two-CTA cluster when half of them fit, otherwise in an L2-resident
// global scratch buffer.  Included by one translation unit per arithmetic type (fft_f64.cu,
// fft_f32.cu, fft_df64.cu).
#pragma once
#include <math.h>

#include <cooperative_groups.h>

#include <type_traits>

#include "common.cuh"

namespace sfft {

// ================================================================== device arithmetic helpers
// scalar conversion between float, double and df64 (direct for equal types)
template <class D, class S> __device__ __forceinline__ D scv(S v) {
    if constexpr (std::is_same<D, S>::value) return v;
    else if constexpr (std::is_same<D, df64>::value) {
        if constexpr (std::is_same<S, float>::value) return df64{v, 0.f};
        else return from_d<df64>((double)v);
    }
    else if constexpr (std::is_same<S, df64>::value) {
        if constexpr (std::is_same<D, float>::value) return v.hi + v.lo;
        else return (double)v.hi + (double)v.lo;
    } else return (D)v;
}
template <class D, class S> __device__ __forceinline__ cplx<D> ccv(cplx<S> a) { return {scv<D>(a.x), scv<D>(a.y)}; }

// load of a transform input in the transform precision
template <class T, class TI> __device__ __forceinline__ cplx<T> load_in(const cplx<TI>* p) { return ccv<T>(*p); }

// read-only loads of table entries in the transform precision
__device__ __forceinline__ cplx<df64> ldg(const cplx<df64>* p) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return {df64{v.x, v.y}, df64{v.z, v.w}};
}

// ================================================================== device butterflies
// R-point DFT in registers: y_p = sum_q v_q omega^{pq}, omega = exp(S * 2 pi i / R), S = -1 / +1
constexpr double kC1 = 0.309016994374947424102293417182819059;   // cos(2 pi/5)
constexpr double kC2 = -0.809016994374947424102293417182819059;  // cos(4 pi/5)
constexpr double kS1 = 0.951056516295153572116439333379382143;   // sin(2 pi/5)
constexpr double kS2 = 0.587785252292473129168705954639072769;   // sin(4 pi/5)
constexpr double kH3 = 0.866025403784438646763723170752936183;   // sqrt(3)/2

// multiply by S*i
template <int S, class T> __device__ __forceinline__ cplx<T> mul_si(cplx<T> a) {
    return S < 0 ? cplx<T>{a.y, -a.x} : cplx<T>{-a.y, a.x};
}

// Butterfly sums.  Double-float: Knuth two-sum of the high words plus the low words, without the
// final renormalisation (8 instead of 11 instructions).  The pair still represents the sum to
// ~2^-47 relative as long as |lo| stays within a few ulps of hi; every product renormalises, and
// values are renormalised when they are written to the work buffer (qnorm).
__device__ __forceinline__ df64 df_add_q(df64 a, df64 b) {
    const df64 s = df_two_sum(a.hi, b.hi);
    return df64{s.hi, DF_ADD(s.lo, DF_ADD(a.lo, b.lo))};
}
template <class T> __device__ __forceinline__ cplx<T> qadd(cplx<T> a, cplx<T> b) { return a + b; }
template <class T> __device__ __forceinline__ cplx<T> qsub(cplx<T> a, cplx<T> b) { return a - b; }
template <class T> __device__ __forceinline__ cplx<T> qnorm(cplx<T> a) { return a; }
template <> __device__ __forceinline__ cplx<df64> qadd(cplx<df64> a, cplx<df64> b) {
    return {df_add_q(a.x, b.x), df_add_q(a.y, b.y)};
}
template <> __device__ __forceinline__ cplx<df64> qsub(cplx<df64> a, cplx<df64> b) {
    return {df_add_q(a.x, -b.x), df_add_q(a.y, -b.y)};
}
template <> __device__ __forceinline__ cplx<df64> qnorm(cplx<df64> a) {
    return {df_fast_two_sum(a.x.hi, a.x.lo), df_fast_two_sum(a.y.hi, a.y.lo)};
}

template <int R, int S, class T> __device__ __forceinline__ void bfly(cplx<T>* v) {
    if constexpr (R == 2) {
        cplx<T> a = v[0], b = v[1];
        v[0] = qadd(a, b);
        v[1] = qsub(a, b);
    } else if constexpr (R == 4) {
        cplx<T> t0 = qadd(v[0], v[2]), t1 = qsub(v[0], v[2]), t2 = qadd(v[1], v[3]);
        cplx<T> t3 = mul_si<S>(qsub(v[1], v[3]));
        v[0] = qadd(t0, t2);
        v[2] = qsub(t0, t2);
        v[1] = qadd(t1, t3);
        v[3] = qsub(t1, t3);
    } else if constexpr (R == 3) {
        cplx<T> t1 = qadd(v[1], v[2]), t2 = qsub(v[1], v[2]);
        cplx<T> a = qsub(v[0], half(t1));
        cplx<T> b = mul_si<S>(t2 * kc<T>(kH3));
        v[0] = qadd(v[0], t1);
        v[1] = qadd(a, b);
        v[2] = qsub(a, b);
    } else if constexpr (R == 5) {
        cplx<T> t1 = qadd(v[1], v[4]), t2 = qadd(v[2], v[3]), t3 = qsub(v[1], v[4]), t4 = qsub(v[2], v[3]);
        cplx<T> b1 = v[0] + t1 * kc<T>(kC1) + t2 * kc<T>(kC2);
        cplx<T> b2 = v[0] + t1 * kc<T>(kC2) + t2 * kc<T>(kC1);
        cplx<T> d1 = mul_si<S>(t3 * kc<T>(kS1) + t4 * kc<T>(kS2));
        cplx<T> d2 = mul_si<S>(t3 * kc<T>(kS2) - t4 * kc<T>(kS1));
        v[0] = qadd(qadd(v[0], t1), t2);
        v[1] = qadd(b1, d1);
        v[4] = qsub(b1, d1);
        v[2] = qadd(b2, d2);
        v[3] = qsub(b2, d2);
    }
}

// cos and sin of 2 pi j / R (R = 6, 8, 9, 10, 12, 15, 16; 0 < j < R, not a quarter turn) for the
// inner twiddles of the fused radix pairs, as doubles and as double-float pairs (hi = nearest
// float, lo = the remainder); values from 50-digit evaluations
struct RootCS {
    double c, s;
    float ch, cl, sh, sl;
};
__host__ __device__ constexpr RootCS root_cs(int R, int j) {
    switch (R * 64 + j) {
        case 385: return RootCS{0.5, 0.8660254037844386, 0.5f, 0.0f, 0.8660253882408142f, 1.5543625053737742e-08f};  // 1/6
        case 386: return RootCS{-0.5, 0.8660254037844386, -0.5f, 0.0f, 0.8660253882408142f, 1.5543625053737742e-08f};  // 2/6
        case 388: return RootCS{-0.5, -0.8660254037844386, -0.5f, -0.0f, -0.8660253882408142f, -1.5543625053737742e-08f};  // 4/6
        case 389: return RootCS{0.5, -0.8660254037844386, 0.5f, 0.0f, -0.8660253882408142f, -1.5543625053737742e-08f};  // 5/6
        case 513: return RootCS{0.7071067811865476, 0.7071067811865476, 0.7071067690849304f, 1.2101617485882343e-08f, 0.7071067690849304f, 1.2101617485882343e-08f};  // 1/8
        case 515: return RootCS{-0.7071067811865476, 0.7071067811865476, -0.7071067690849304f, -1.2101617485882343e-08f, 0.7071067690849304f, 1.2101617485882343e-08f};  // 3/8
        case 517: return RootCS{-0.7071067811865476, -0.7071067811865476, -0.7071067690849304f, -1.2101617485882343e-08f, -0.7071067690849304f, -1.2101617485882343e-08f};  // 5/8
        case 519: return RootCS{0.7071067811865476, -0.7071067811865476, 0.7071067690849304f, 1.2101617485882343e-08f, -0.7071067690849304f, -1.2101617485882343e-08f};  // 7/8
        case 577: return RootCS{0.766044443118978, 0.6427876096865394, 0.7660444378852844f, 5.2336934786012534e-09f, 0.6427876353263855f, -2.5639845802061245e-08f};  // 1/9
        case 578: return RootCS{0.17364817766693036, 0.984807753012208, 0.1736481785774231f, -9.10492736760915e-10f, 0.9848077297210693f, 2.3291137907222037e-08f};  // 2/9
        case 579: return RootCS{-0.5, 0.8660254037844386, -0.5f, -0.0f, 0.8660253882408142f, 1.5543625053737742e-08f};  // 3/9
        case 580: return RootCS{-0.9396926207859084, 0.3420201433256687, -0.9396926164627075f, -4.323200908373792e-09f, 0.3420201539993286f, -1.0673660177928923e-08f};  // 4/9
        case 581: return RootCS{-0.9396926207859084, -0.3420201433256687, -0.9396926164627075f, -4.323200908373792e-09f, -0.3420201539993286f, 1.0673660177928923e-08f};  // 5/9
        case 582: return RootCS{-0.5, -0.8660254037844386, -0.5f, 0.0f, -0.8660253882408142f, -1.5543625053737742e-08f};  // 6/9
        case 583: return RootCS{0.17364817766693036, -0.984807753012208, 0.1736481785774231f, -9.10492736760915e-10f, -0.9848077297210693f, -2.3291137907222037e-08f};  // 7/9
        case 584: return RootCS{0.766044443118978, -0.6427876096865394, 0.7660444378852844f, 5.2336934786012534e-09f, -0.6427876353263855f, 2.5639845802061245e-08f};  // 8/9
        case 641: return RootCS{0.8090169943749475, 0.5877852522924731, 0.80901700258255f, -8.207602597565256e-09f, 0.5877852439880371f, 8.304436249773062e-09f};  // 1/10
        case 642: return RootCS{0.30901699437494745, 0.9510565162951535, 0.30901700258255005f, -8.207602597565256e-09f, 0.9510565400123596f, -2.3717205976936384e-08f};  // 2/10
        case 643: return RootCS{-0.30901699437494745, 0.9510565162951535, -0.30901700258255005f, 8.207602597565256e-09f, 0.9510565400123596f, -2.3717205976936384e-08f};  // 3/10
        case 644: return RootCS{-0.8090169943749475, 0.5877852522924731, -0.80901700258255f, 8.207602597565256e-09f, 0.5877852439880371f, 8.304436249773062e-09f};  // 4/10
        case 646: return RootCS{-0.8090169943749475, -0.5877852522924731, -0.80901700258255f, 8.207602597565256e-09f, -0.5877852439880371f, -8.304436249773062e-09f};  // 6/10
        case 647: return RootCS{-0.30901699437494745, -0.9510565162951535, -0.30901700258255005f, 8.207602597565256e-09f, -0.9510565400123596f, 2.3717205976936384e-08f};  // 7/10
        case 648: return RootCS{0.30901699437494745, -0.9510565162951535, 0.30901700258255005f, -8.207602597565256e-09f, -0.9510565400123596f, 2.3717205976936384e-08f};  // 8/10
        case 649: return RootCS{0.8090169943749475, -0.5877852522924731, 0.80901700258255f, -8.207602597565256e-09f, -0.5877852439880371f, -8.304436249773062e-09f};  // 9/10
        case 769: return RootCS{0.8660254037844386, 0.5, 0.8660253882408142f, 1.5543625053737742e-08f, 0.5f, 0.0f};  // 1/12
        case 770: return RootCS{0.5, 0.8660254037844386, 0.5f, 0.0f, 0.8660253882408142f, 1.5543625053737742e-08f};  // 2/12
        case 772: return RootCS{-0.5, 0.8660254037844386, -0.5f, 0.0f, 0.8660253882408142f, 1.5543625053737742e-08f};  // 4/12
        case 773: return RootCS{-0.8660254037844386, 0.5, -0.8660253882408142f, -1.5543625053737742e-08f, 0.5f, 0.0f};  // 5/12
        case 775: return RootCS{-0.8660254037844386, -0.5, -0.8660253882408142f, -1.5543625053737742e-08f, -0.5f, 0.0f};  // 7/12
        case 776: return RootCS{-0.5, -0.8660254037844386, -0.5f, -0.0f, -0.8660253882408142f, -1.5543625053737742e-08f};  // 8/12
        case 778: return RootCS{0.5, -0.8660254037844386, 0.5f, 0.0f, -0.8660253882408142f, -1.5543625053737742e-08f};  // 10/12
        case 779: return RootCS{0.8660254037844386, -0.5, 0.8660253882408142f, 1.5543625053737742e-08f, -0.5f, -0.0f};  // 11/12
        case 961: return RootCS{0.9135454576426009, 0.4067366430758002, 0.9135454297065735f, 2.7936026825159388e-08f, 0.4067366421222687f, 9.535314760000801e-10f};  // 1/15
        case 962: return RootCS{0.6691306063588582, 0.7431448254773942, 0.6691306233406067f, -1.698174934006147e-08f, 0.7431448101997375f, 1.527765647324486e-08f};  // 2/15
        case 963: return RootCS{0.30901699437494745, 0.9510565162951535, 0.30901700258255005f, -8.207602597565256e-09f, 0.9510565400123596f, -2.3717205976936384e-08f};  // 3/15
        case 964: return RootCS{-0.10452846326765347, 0.9945218953682733, -0.10452846437692642f, 1.1092728957606823e-09f, 0.9945219159126282f, -2.054435555010059e-08f};  // 4/15
        case 965: return RootCS{-0.5, 0.8660254037844386, -0.5f, 0.0f, 0.8660253882408142f, 1.5543625053737742e-08f};  // 5/15
        case 966: return RootCS{-0.8090169943749475, 0.5877852522924731, -0.80901700258255f, 8.207602597565256e-09f, 0.5877852439880371f, 8.304436249773062e-09f};  // 6/15
        case 967: return RootCS{-0.9781476007338057, 0.20791169081775934, -0.9781476259231567f, 2.5189351049448305e-08f, 0.2079116851091385f, 5.708620687272514e-09f};  // 7/15
        case 968: return RootCS{-0.9781476007338057, -0.20791169081775934, -0.9781476259231567f, 2.5189351049448305e-08f, -0.2079116851091385f, -5.708620687272514e-09f};  // 8/15
        case 969: return RootCS{-0.8090169943749475, -0.5877852522924731, -0.80901700258255f, 8.207602597565256e-09f, -0.5877852439880371f, -8.304436249773062e-09f};  // 9/15
        case 970: return RootCS{-0.5, -0.8660254037844386, -0.5f, -0.0f, -0.8660253882408142f, -1.5543625053737742e-08f};  // 10/15
        case 971: return RootCS{-0.10452846326765347, -0.9945218953682733, -0.10452846437692642f, 1.1092728957606823e-09f, -0.9945219159126282f, 2.054435555010059e-08f};  // 11/15
        case 972: return RootCS{0.30901699437494745, -0.9510565162951535, 0.30901700258255005f, -8.207602597565256e-09f, -0.9510565400123596f, 2.3717205976936384e-08f};  // 12/15
        case 973: return RootCS{0.6691306063588582, -0.7431448254773942, 0.6691306233406067f, -1.698174934006147e-08f, -0.7431448101997375f, -1.527765647324486e-08f};  // 13/15
        case 974: return RootCS{0.9135454576426009, -0.4067366430758002, 0.9135454297065735f, 2.7936026825159388e-08f, -0.4067366421222687f, -9.535314760000801e-10f};  // 14/15
        case 1025: return RootCS{0.9238795325112867, 0.3826834323650898, 0.9238795042037964f, 2.830748968563057e-08f, 0.3826834261417389f, 6.2233507236442165e-09f};  // 1/16
        case 1026: return RootCS{0.7071067811865476, 0.7071067811865476, 0.7071067690849304f, 1.2101617485882343e-08f, 0.7071067690849304f, 1.2101617485882343e-08f};  // 2/16
        case 1027: return RootCS{0.3826834323650898, 0.9238795325112867, 0.3826834261417389f, 6.2233507236442165e-09f, 0.9238795042037964f, 2.830748968563057e-08f};  // 3/16
        case 1029: return RootCS{-0.3826834323650898, 0.9238795325112867, -0.3826834261417389f, -6.2233507236442165e-09f, 0.9238795042037964f, 2.830748968563057e-08f};  // 5/16
        case 1030: return RootCS{-0.7071067811865476, 0.7071067811865476, -0.7071067690849304f, -1.2101617485882343e-08f, 0.7071067690849304f, 1.2101617485882343e-08f};  // 6/16
        case 1031: return RootCS{-0.9238795325112867, 0.3826834323650898, -0.9238795042037964f, -2.830748968563057e-08f, 0.3826834261417389f, 6.2233507236442165e-09f};  // 7/16
        case 1033: return RootCS{-0.9238795325112867, -0.3826834323650898, -0.9238795042037964f, -2.830748968563057e-08f, -0.3826834261417389f, -6.2233507236442165e-09f};  // 9/16
        case 1034: return RootCS{-0.7071067811865476, -0.7071067811865476, -0.7071067690849304f, -1.2101617485882343e-08f, -0.7071067690849304f, -1.2101617485882343e-08f};  // 10/16
        case 1035: return RootCS{-0.3826834323650898, -0.9238795325112867, -0.3826834261417389f, -6.2233507236442165e-09f, -0.9238795042037964f, -2.830748968563057e-08f};  // 11/16
        case 1037: return RootCS{0.3826834323650898, -0.9238795325112867, 0.3826834261417389f, 6.2233507236442165e-09f, -0.9238795042037964f, -2.830748968563057e-08f};  // 13/16
        case 1038: return RootCS{0.7071067811865476, -0.7071067811865476, 0.7071067690849304f, 1.2101617485882343e-08f, -0.7071067690849304f, -1.2101617485882343e-08f};  // 14/16
        case 1039: return RootCS{0.9238795325112867, -0.3826834323650898, 0.9238795042037964f, 2.830748968563057e-08f, -0.3826834261417389f, -6.2233507236442165e-09f};  // 15/16
        default: return RootCS{1.0, 0.0, 1.0f, 0.0f, 0.0f, 0.0f};
    }
}

// v * exp(S 2 pi i j / R); j is a constant once the pass loops are unrolled
template <int R, int S, class T> __device__ __forceinline__ cplx<T> rot(cplx<T> v, int j) {
    j %= R;
    if (j == 0) return v;
    if (4 * j == R) return mul_si<S>(v);
    if (2 * j == R) return cplx<T>{-v.x, -v.y};
    if (4 * j == 3 * R) return mul_si<-S>(v);
    constexpr float sf = (float)S;
    const RootCS r = root_cs(R, j);
    if constexpr (std::is_same<T, df64>::value) {
        return v * cplx<df64>{df64{r.ch, r.cl}, df64{sf * r.sh, sf * r.sl}};
    } else if constexpr (std::is_same<T, float>::value) {
        return v * c32{r.ch, sf * r.sh};
    } else {
        return v * cplx<T>{(T)r.c, (T)S * (T)r.s};
    }
}

// twiddle exp(-2 pi i k / N) for 0 <= k < N
template <class T> struct TwFull {  // full table in global memory (L2 / L1 resident)
    const cplx<T>* tw;
    __device__ __forceinline__ cplx<T> operator()(int k) const { return ldg(&tw[k]); }
};
struct TwTwo {  // FP32: product of two small shared-memory tables, k = 256 a + b
    const c32* a;
    const c32* b;
    __device__ __forceinline__ c32 operator()(int k) const { return a[k >> 8] * b[k & 255]; }
};

// The table twiddles of one group, tw(n j) for j = p1 + R1 p2.  FP32 (two-level tables in
// shared memory): one lookup w = tw(n), then products of powers, w^j = w^p1 w^(R1 p2), with the
// powers formed by repeated squaring (error a few ulps, well inside the FP32 zero test's band);
// this replaces R1 R2 - 2 table lookups by products.  Other types: full-table lookups.
template <int R1, int R2, class T, class TW>
struct TwRow {
    const TW& tw;
    int n;
    __device__ __forceinline__ TwRow(const TW& t, int n_) : tw(t), n(n_) {}
    __device__ __forceinline__ cplx<T> operator()(int p1, int p2) const { return tw(n * (p1 + R1 * p2)); }
};
template <int R1, int R2>
struct TwRow<R1, R2, float, TwTwo> {
    c32 a[R1], b[R2];  // a[p1] = w^p1, b[p2] = w^(R1 p2)
    __device__ __forceinline__ TwRow(const TwTwo& t, int n) {
        a[0] = c32{1.f, 0.f};
        a[1] = t(n);
#pragma unroll
        for (int p = 2; p < R1; ++p) a[p] = a[p / 2] * a[p - p / 2];
        b[0] = a[0];
        if constexpr (R2 > 1) {
            b[1] = R1 % 2 ? a[R1 / 2] * a[R1 - R1 / 2] : a[R1 / 2] * a[R1 / 2];
#pragma unroll
            for (int p = 2; p < R2; ++p) b[p] = b[p / 2] * b[p - p / 2];
        }
    }
    __device__ __forceinline__ c32 operator()(int p1, int p2) const {
        return p2 == 0 ? a[p1] : p1 == 0 ? b[p2] : a[p1] * b[p2];
    }
};

// ------------------------------------------------------------------ radix passes
// A pass applies one DIF stage (R2 = 1) or two consecutive DIF stages fused in registers:
// radix R1 on the sub-transforms of size Ns, then radix R2 on those of size Ns / R1.  Each
// thread transforms the R1*R2 elements b*Ns + n2 + q2*m2 + q1*m1 (m1 = Ns/R1, m2 = m1/R2), so a
// fused pass reads and writes the work buffer once for two stages.  Twiddles: a single stage
// multiplies output p by exp(-2 pi i n p / Ns) = tw(n p s1), s1 = N/Ns.  For a pair the first
// stage's twiddle of block q2 splits into tw(n2 p1 s1) omega_{R1 R2}^{q2 p1}; the first factor
// is common to the second stage's sum and merges with its twiddle tw(n2 p2 s1 R1), so a fused
// pass applies the constants omega_{R1 R2}^{q2 p1} between the stages and one table twiddle
// tw(n2 s1 (p1 + R1 p2)) per output: R1 R2 - 1 table twiddles instead of 2 R1 R2 - R1 - R2.
// The block index b = floor(i / m2) is formed with a float reciprocal: (i + 1/2) / m2 is at least
// 1/(2 m2) away from an integer, which the float product resolves exactly for i < 2^22.
// C supplies the buffer accesses (c.dif_load / c.dif_store / c.dit_load / c.dit_store: the work
// buffer's layout); the input, the filter product and the output are handled outside the generic
// passes (BlueIo's phases and mid_pass).
template <int R1, int R2, int S, class T, class TW, class C>
__device__ __forceinline__ void dif_pass(C& c, int Ns, const TW& tw) {
    const int N = c.N, m1 = Ns / R1, m2 = m1 / R2, s1 = N / Ns * c.tws, ng = N / (R1 * R2);
    const float rm = 1.0f / (float)m2;
    // a cluster of two CTAs splits the groups at a block boundary (see BlueIo)
    const int g0 = c.rank * (ng >> 1), g1 = (c.nrank == 1 || c.rank == 1) ? ng : (ng >> 1);
    for (int i = g0 + threadIdx.x; i < g1; i += blockDim.x) {
        const int b = (int)(((float)i + 0.5f) * rm), n2 = i - b * m2, base = b * Ns + n2;
        cplx<T> v[R2][R1];
#pragma unroll
        for (int q2 = 0; q2 < R2; ++q2)
#pragma unroll
            for (int q1 = 0; q1 < R1; ++q1) v[q2][q1] = c.dif_load(base + q2 * m2 + q1 * m1);
#pragma unroll
        for (int q2 = 0; q2 < R2; ++q2) bfly<R1, S>(v[q2]);
        const TwRow<R1, R2, T, TW> w(tw, n2 * s1);
        if constexpr (R2 == 1) {
#pragma unroll
            for (int p1 = 1; p1 < R1; ++p1) v[0][p1] = v[0][p1] * w(p1, 0);
#pragma unroll
            for (int p1 = 0; p1 < R1; ++p1) c.dif_store(base + p1 * m1, v[0][p1]);
        } else {
            // the two stages form an R1 R2-point DFT: inner twiddles omega_{R1 R2}^{q2 p1} between
            // them, then one outer twiddle tw(n2 s1 (p1 + R1 p2)) per output
#pragma unroll
            for (int q2 = 1; q2 < R2; ++q2)
#pragma unroll
                for (int p1 = 1; p1 < R1; ++p1) v[q2][p1] = rot<R1 * R2, S>(v[q2][p1], q2 * p1);
#pragma unroll
            for (int p1 = 0; p1 < R1; ++p1) {
                cplx<T> u[R2];
#pragma unroll
                for (int q2 = 0; q2 < R2; ++q2) u[q2] = v[q2][p1];
                bfly<R2, S>(u);
#pragma unroll
                for (int p2 = 0; p2 < R2; ++p2)
                    c.dif_store(base + p1 * m1 + p2 * m2, (p1 | p2) ? u[p2] * w(p1, p2) : u[p2]);
            }
        }
    }
}

// exact adjoint of dif_pass: conjugate twiddles and inverse butterflies in reverse order
template <int R1, int R2, class T, class TW, class C>
__device__ __forceinline__ void dit_pass(C& c, int Ns, const TW& tw) {
    const int N = c.N, m1 = Ns / R1, m2 = m1 / R2, s1 = N / Ns * c.tws, ng = N / (R1 * R2);
    const float rm = 1.0f / (float)m2;
    const int g0 = c.rank * (ng >> 1), g1 = (c.nrank == 1 || c.rank == 1) ? ng : (ng >> 1);
    for (int i = g0 + threadIdx.x; i < g1; i += blockDim.x) {
        const int b = (int)(((float)i + 0.5f) * rm), n2 = i - b * m2, base = b * Ns + n2;
        const TwRow<R1, R2, T, TW> w(tw, n2 * s1);
        cplx<T> v[R2][R1];
        if constexpr (R2 == 1) {
#pragma unroll
            for (int p1 = 0; p1 < R1; ++p1) {
                const cplx<T> x = c.dit_load(base + p1 * m1);
                v[0][p1] = p1 ? mulc(x, w(p1, 0)) : x;
            }
        } else {
#pragma unroll
            for (int p1 = 0; p1 < R1; ++p1) {
                cplx<T> u[R2];
#pragma unroll
                for (int p2 = 0; p2 < R2; ++p2) {
                    const cplx<T> x = c.dit_load(base + p1 * m1 + p2 * m2);
                    u[p2] = (p1 | p2) ? mulc(x, w(p1, p2)) : x;
                }
                bfly<R2, 1>(u);
#pragma unroll
                for (int q2 = 0; q2 < R2; ++q2) v[q2][p1] = u[q2];
            }
#pragma unroll
            for (int q2 = 1; q2 < R2; ++q2)
#pragma unroll
                for (int p1 = 1; p1 < R1; ++p1) v[q2][p1] = rot<R1 * R2, 1>(v[q2][p1], q2 * p1);
        }
#pragma unroll
        for (int q2 = 0; q2 < R2; ++q2) {
            bfly<R1, 1>(v[q2]);
#pragma unroll
            for (int q1 = 0; q1 < R1; ++q1) c.dit_store(base + q2 * m2 + q1 * m1, v[q2][q1]);
        }
    }
}

// The last DIF pass, the filter product and the first DIT pass in one: both passes work on the
// blocks of R1 R2 consecutive elements (sub-transform size Ns = R1 R2, so n2 = 0 and every outer
// twiddle is 1), so each thread takes a block through the forward R1 R2-point DFT, multiplies by
// the filter (its loads issued with the block's shared-memory loads) and back through the
// inverse DFT: one shared-memory round trip and one barrier fewer per transform.
template <int R1, int R2, class T, class C>
__device__ __forceinline__ void mid_pass(C& c) {
    constexpr int m1 = R2;  // m2 = 1
    const int ng = c.N / (R1 * R2);
    const int g0 = c.rank * (ng >> 1), g1 = (c.nrank == 1 || c.rank == 1) ? ng : (ng >> 1);
    for (int i = g0 + threadIdx.x; i < g1; i += blockDim.x) {
        const int base = i * (R1 * R2);
        cplx<T> v[R2][R1], f[R1][R2];
#pragma unroll
        for (int p1 = 0; p1 < R1; ++p1)
#pragma unroll
            for (int p2 = 0; p2 < R2; ++p2) f[p1][p2] = ldg(&c.filt[base + p1 * m1 + p2]);
#pragma unroll
        for (int q2 = 0; q2 < R2; ++q2)
#pragma unroll
            for (int q1 = 0; q1 < R1; ++q1) v[q2][q1] = c.dif_load(base + q2 + q1 * m1);
#pragma unroll
        for (int q2 = 0; q2 < R2; ++q2) bfly<R1, -1>(v[q2]);
        if constexpr (R2 > 1) {
#pragma unroll
            for (int q2 = 1; q2 < R2; ++q2)
#pragma unroll
                for (int p1 = 1; p1 < R1; ++p1) v[q2][p1] = rot<R1 * R2, -1>(v[q2][p1], q2 * p1);
#pragma unroll
            for (int p1 = 0; p1 < R1; ++p1) {
                cplx<T> u[R2];
#pragma unroll
                for (int q2 = 0; q2 < R2; ++q2) u[q2] = v[q2][p1];
                bfly<R2, -1>(u);
#pragma unroll
                for (int p2 = 0; p2 < R2; ++p2) u[p2] = u[p2] * f[p1][p2];
                bfly<R2, 1>(u);
#pragma unroll
                for (int q2 = 0; q2 < R2; ++q2) v[q2][p1] = u[q2];
            }
#pragma unroll
            for (int q2 = 1; q2 < R2; ++q2)
#pragma unroll
                for (int p1 = 1; p1 < R1; ++p1) v[q2][p1] = rot<R1 * R2, 1>(v[q2][p1], q2 * p1);
        } else {
#pragma unroll
            for (int p1 = 0; p1 < R1; ++p1) v[0][p1] = v[0][p1] * f[p1][0];
        }
#pragma unroll
        for (int q2 = 0; q2 < R2; ++q2) {
            bfly<R1, 1>(v[q2]);
#pragma unroll
            for (int q1 = 0; q1 < R1; ++q1) c.dit_store(base + q2 + q1 * m1, v[q2][q1]);
        }
    }
}

// mode 0: DIF pass, 1: DIT pass, 2: the fused middle pass
template <class T, class TW, class C>
__device__ __forceinline__ void run_pass(int mode, int r1, int r2, C& c, int Ns, const TW& tw) {
    // pairs above the type's register budget are never planned, so they are not compiled
#define SFFT_PASS(A, B)                                              \
    if constexpr (A * B <= pass_maxprod<T>()) {                      \
        if (r1 == A && r2 == B) {                                    \
            if (mode == 0) dif_pass<A, B, -1, T>(c, Ns, tw);         \
            else if (mode == 1) dit_pass<A, B, T>(c, Ns, tw);        \
            else mid_pass<A, B, T>(c);                               \
            return;                                                  \
        }                                                            \
    }
    SFFT_PASS(4, 4) SFFT_PASS(3, 3) SFFT_PASS(4, 3) SFFT_PASS(4, 2) SFFT_PASS(2, 3) SFFT_PASS(3, 5)
    SFFT_PASS(2, 5) SFFT_PASS(4, 1) SFFT_PASS(3, 1) SFFT_PASS(2, 1) SFFT_PASS(5, 1)
#undef SFFT_PASS
}

// A transform whose passes are all the same fused pair (UP = r1 | r2 << 4, e.g. N = 20736 =
// 12^4 for M = 10331) runs a kernel compiled with that pair only: no run-time dispatch and a
// fraction of the generic kernel's code (fewer instruction-fetch stalls).  UP = 0: generic.
template <int UP, class T, class TW, class C>
__device__ __forceinline__ void run_pass_u(int mode, int r1, int r2, C& c, int Ns, const TW& tw) {
    if constexpr (UP != 0) {
        constexpr int A = UP & 15, B = UP >> 4;
        if (mode == 0) dif_pass<A, B, -1, T>(c, Ns, tw);
        else if (mode == 1) dit_pass<A, B, T>(c, Ns, tw);
        else mid_pass<A, B, T>(c);
    } else {
        run_pass<T>(mode, r1, r2, c, Ns, tw);
    }
}

// CTA-wide sum of a and maximum of b in one pass (three barriers), in the statistics precision R:
// float for float and double-float transforms (FP64 instructions are scarce on this GPU and the
// statistics only place the zero test's guard band), double for double transforms.  red holds at
// least 2 x 32 values of R.
template <class R>
__device__ __forceinline__ void block_reduce_sum_max(R& a, R& b, R* red) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) { red[w] = a; red[32 + w] = b; }
    __syncthreads();
    if (w == 0) {
        R x = l < nw ? red[l] : R(0), y = l < nw ? red[32 + l] : R(0);
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y = fmax(y, __shfl_xor_sync(0xffffffffu, y, o));
        }
        if (l == 0) { red[0] = x; red[32] = y; }
    }
    __syncthreads();
    a = red[0];
    b = red[32];
}

// Largest CTA of a transform (the register budget follows from it): FP32 transforms run up to
// 576 threads (18 warps, 113 registers), so that the 1728 groups of a radix-12 pass of N = 20736
// take three rounds of every thread (measured against 512 threads at 128 registers and 864 at 72:
// the step's transforms 0.332 ms at 576, 0.346 at 864, 0.375 at 512); double and double-float
// transforms need more registers per thread and stop at 512.
#ifndef SFFT_BLUE_F32_THREADS
#define SFFT_BLUE_F32_THREADS 576
#endif
template <class T> constexpr int blue_max_threads() { return std::is_same<T, float>::value ? SFFT_BLUE_F32_THREADS : 512; }
// the same for a buffer mode: the global-scratch (0) and cluster (2) modes have longer address
// arithmetic and stay at 512 threads so that they do not spill
template <class T> constexpr int blue_max_threads(int mode) { return mode == 1 ? blue_max_threads<T>() : 512; }

// Buffer access of one Bluestein transform: the first DIF pass reads the chirp-weighted input
// (zero padded to N), the last DIF pass multiplies by the filter before its store, and the last
// DIT pass writes the chirp-weighted outputs h < M instead of the buffer.
template <class T, class TI, class TO, bool SMB, bool CL>
struct BlueIo {  // SMB: buffer in shared memory (padded layout); CL: split over a two-CTA cluster
    // statistics precision: the transform's own for float and double, float for double-float
    // (they only place the zero test's guard band and the maximum's search window)
    using R = typename std::conditional<std::is_same<T, df64>::value, float, T>::type;
    cplx<T>* buf;        // work buffer (CL: this CTA's half, elements [rank N/2, (rank+1) N/2))
    cplx<T>* rbuf;       // CL: the other CTA's half (distributed shared memory)
    int hN = 0, rank = 0, nrank = 1;
    int N, M, epi;
    int tws = 1;  // twiddle stride factor: the table is for tws N (a block of a longer transform)
    bool inv;
    const cplx<TI>* in;
    const cplx<T>* chirp;
    const cplx<T>* filt;
    cplx<TO>* out;
    const void* auxp;
    T sc;
    R ss = 0, mx2 = 0;  // EPI_ANALYZE: sum |x|^2 and max |X|^2 of this thread

    __device__ __forceinline__ cplx<T>* at(int e) {
        constexpr int P = blue_pad_shift(sizeof(cplx<T>));
        if constexpr (CL) {
            const int o = e >= hN ? 1 : 0;
            const int le = e - o * hN;
            return (o == rank ? buf : rbuf) + (P ? le + (le >> P) : le);
        } else if constexpr (SMB && P > 0) {
            return buf + e + (e >> P);
        } else {
            return buf + e;
        }
    }
    __device__ __forceinline__ cplx<T> dif_load(int e) { return *at(e); }
    __device__ __forceinline__ void dif_store(int e, cplx<T> v) { *at(e) = qnorm(v); }
    __device__ __forceinline__ cplx<T> dit_load(int e) { return *at(e); }
    __device__ __forceinline__ void dit_store(int e, cplx<T> v) { *at(e) = qnorm(v); }

    // Input and output run as phases of their own over elements [e0, e1) of this CTA, in natural
    // order (coalesced) with kIoUnroll elements per thread whose global loads are issued together:
    // the passes then only touch shared memory, and the loads' latency is paid once per batch
    // instead of once per butterfly group.
    static constexpr int kIoUnroll = 8;
    // work buffer = x_j chirp_j (conjugate chirp for the inverse) on [0, M), zero on [M, N)
    __device__ __forceinline__ void load_input(int e0, int e1) {
        for (int b = e0 + (int)threadIdx.x; b < e1; b += kIoUnroll * (int)blockDim.x) {
            cplx<TI> xv[kIoUnroll];
            cplx<T> wv[kIoUnroll];
#pragma unroll
            for (int u = 0; u < kIoUnroll; ++u) {
                const int e = b + u * (int)blockDim.x;
                if (e < e1 && e < M) {
                    xv[u] = in[e];
                    wv[u] = ldg(&chirp[e]);
                }
            }
#pragma unroll
            for (int u = 0; u < kIoUnroll; ++u) {
                const int e = b + u * (int)blockDim.x;
                if (e >= e1) break;
                cplx<T> v = {kc<T>(0.0), kc<T>(0.0)};
                if (e < M) {
                    const cplx<T> x = ccv<T>(xv[u]);
                    if (epi == EPI_ANALYZE) ss += scv<R>(abs2(x));
                    v = inv ? mulc(x, wv[u]) : x * wv[u];
                }
                *at(e) = v;
            }
        }
    }
    // Input of the sparse-polynomial sampler (eq. 2.3) built in place: the bucket sums
    // sum_{q : k_q.z_l = h mod M} c_q of lattice l (terms of instance I, coefficients rounded to the
    // transform precision, summed by shared-memory atomics), zero on [M, N), then the chirp product
    // on [0, M).  Only for a buffer in this CTA's shared memory.
    __device__ __forceinline__ void scatter_terms(const InstDesc& I, int l) {
        for (int e = threadIdx.x; e < N; e += blockDim.x) *at(e) = cplx<T>{kc<T>(0.0), kc<T>(0.0)};
        __syncthreads();
        const int d = I.d;
        const int32_t* __restrict__ kv = I.samp_kvec;
        const int32_t* __restrict__ zl = I.z + (int64_t)l * d;
        // h = k.z mod M term by term in 32-bit arithmetic: |k_t| mod M by a Barrett reduction
        // (mu = floor((2^32 - 1) / M) leaves a remainder below 2M for any operand below 2^32: one
        // conditional subtraction), its sign applied, then the product with z_t < M, below M^2 <
        // 2^32 while M < 2^16 (always so for a buffer in one CTA's shared memory), reduced the same
        // way; larger M take the int64 sum and remainder
        const uint32_t uM = (uint32_t)M, mu = 0xffffffffu / uM;
        auto red = [&](uint32_t x) -> uint32_t {
            const uint32_t r = x - __umulhi(x, mu) * uM;
            return min(r, r - uM);
        };
        for (int64_t q = threadIdx.x; q < I.samp_nterms; q += blockDim.x) {
            uint32_t h = 0;
            if (uM < 65536u) {
                for (int t = 0; t < d; ++t) {
                    const int32_t k = kv[q * d + t];
                    uint32_t rk = red(k < 0 ? 0u - (uint32_t)k : (uint32_t)k);
                    if (k < 0 && rk) rk = uM - rk;
                    h += red(rk * (uint32_t)zl[t]);
                    h = min(h, h - uM);
                }
            } else {
                int64_t x = 0;
                for (int t = 0; t < d; ++t) x += (int64_t)kv[q * d + t] * zl[t];
                int64_t r = x % (int64_t)M;
                if (r < 0) r += M;
                h = (uint32_t)r;
            }
            const cplx<T> v = ccv<T>(I.samp_coef[q]);
            cplx<T>* p = at((int)h);
            atomicAdd(&p->x, v.x);
            atomicAdd(&p->y, v.y);
        }
        __syncthreads();
        for (int b = threadIdx.x; b < M; b += kIoUnroll * (int)blockDim.x) {
            cplx<T> xv[kIoUnroll], wv[kIoUnroll];
#pragma unroll
            for (int u = 0; u < kIoUnroll; ++u) {
                const int e = b + u * (int)blockDim.x;
                if (e < M) {
                    xv[u] = *at(e);
                    wv[u] = ldg(&chirp[e]);
                }
            }
#pragma unroll
            for (int u = 0; u < kIoUnroll; ++u) {
                const int e = b + u * (int)blockDim.x;
                if (e >= M) break;
                *at(e) = inv ? mulc(xv[u], wv[u]) : xv[u] * wv[u];
            }
        }
    }
    // outputs j in [e0, e1), e1 <= M: chirp product, scale and the epilogue (the noise of
    // EPI_ADDNOISE is complex float for float transforms, complex double otherwise)
    using NZ = typename std::conditional<std::is_same<T, float>::value, c32, c64>::type;
    __device__ __forceinline__ void store_output(int e0, int e1) {
        const NZ* noise = epi == EPI_ADDNOISE ? reinterpret_cast<const NZ*>(auxp) : nullptr;
        for (int b = e0 + (int)threadIdx.x; b < e1; b += kIoUnroll * (int)blockDim.x) {
            cplx<T> vv[kIoUnroll], wv[kIoUnroll];
            NZ zv[kIoUnroll];
#pragma unroll
            for (int u = 0; u < kIoUnroll; ++u) {
                const int e = b + u * (int)blockDim.x;
                if (e < e1) {
                    vv[u] = *at(e);
                    wv[u] = ldg(&chirp[e]);
                    if (noise) zv[u] = noise[e];
                }
            }
#pragma unroll
            for (int u = 0; u < kIoUnroll; ++u) {
                const int e = b + u * (int)blockDim.x;
                if (e >= e1) break;
                emit(e, vv[u], wv[u], noise ? &zv[u] : nullptr);
            }
        }
    }
    __device__ __forceinline__ void emit(int e, cplx<T> v, cplx<T> w, const NZ* zp) {
        cplx<T> X = inv ? mulc(v, w) : v * w;
        X = X * sc;
        if (epi == EPI_PLAIN || epi == EPI_ANALYZE) {
            if constexpr (std::is_same<T, df64>::value && std::is_same<TO, float>::value) {
                // float output of a double-float value: high words out, low words to aux
                out[e] = cplx<TO>{X.x.hi, X.y.hi};
                if (auxp) reinterpret_cast<c32*>(const_cast<void*>(auxp))[e] = c32{X.x.lo, X.y.lo};
            } else {
                out[e] = ccv<TO>(X);
            }
            if (epi == EPI_ANALYZE) mx2 = fmax(mx2, scv<R>(abs2(X)));
        } else {  // EPI_ADDNOISE (noise added in the transform precision)
            if constexpr (std::is_same<T, float>::value) {
                if (zp) X = X + *zp;
                out[e] = ccv<TO>(X);
            } else {
                c64 r = ccv<double>(X);
                if (zp) r = r + *zp;
                out[e] = ccv<TO>(r);
            }
        }
    }
};

// EPI_ANALYZE: the CTA's (cluster's) sum |x|^2 and max |X|^2 to the lattice's statistics
template <class T, class TI, class TO, bool SMB, bool CL>
__device__ __forceinline__ void analyze_epilogue(const BlueJob& J, BlueIo<T, TI, TO, SMB, CL>& c, int epi, int rank,
                                                 double* red, double* xchg) {
    if (epi == EPI_ANALYZE) {
        using R = typename BlueIo<T, TI, TO, SMB, CL>::R;
        R ssr = c.ss, mxr = c.mx2;
        block_reduce_sum_max(ssr, mxr, reinterpret_cast<R*>(red));
        double ssd = (double)ssr, mx2 = (double)mxr;
        if constexpr (CL) {  // partials of both CTAs to rank 0
            auto cl = cooperative_groups::this_cluster();
            double* x0 = cl.map_shared_rank(xchg, 0);
            if (threadIdx.x == 0) { x0[2 * rank] = ssd; x0[2 * rank + 1] = mx2; }
            cl.sync();
            if (rank != 0) return;
            ssd = xchg[0] + xchg[2];
            mx2 = fmax(xchg[1], xchg[3]);
        }
        if (threadIdx.x == 0) {
            const double mx = sqrt(mx2);
            LatStats& S = *J.stat;
            S.max32 = (float)mx;
            S.max_abs = mx;
            S.rms = sqrt(ssd / (double)J.M);
        }
    }
}

// Copy of a block of n elements between the global-scratch buffer g and the padded shared-memory
// buffer of cb (to shared memory if IN), kIoUnroll elements per thread in flight.
template <bool IN, class C, class T>
__device__ __forceinline__ void stage_block(C& cb, cplx<T>* g, int n) {
    constexpr int U = 8;
    for (int e0 = threadIdx.x; e0 < n; e0 += U * blockDim.x) {
        cplx<T> v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            if (e < n) v[u] = IN ? g[e] : *cb.at(e);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            if (e < n) {
                if (IN) *cb.at(e) = v[u];
                else g[e] = v[u];
            }
        }
    }
}

// CL: the transform of one lattice is split over a cluster of two CTAs, each holding half of the
// work buffer in its shared memory.  Only the first DIF pass and the last DIT pass (sub-transform
// size N) touch the other half; every later pass works on blocks of size N / (first pass radix
// product), which lie inside one half when that product is even, so a CTA takes the groups of
// its own blocks.  The input and output phases touch only the CTA's own half.  Cluster barriers
// follow the input phase (both halves filled, both CTAs running before any remote access), follow
// the first pass, and come before and after the last one; after that no CTA reads the other's
// half, so either may leave.
template <class T, class TI, class TO, bool SMB, bool CL, int UP, class TW>
__device__ __forceinline__ void bluestein_body(const BlueJob& J, cplx<T>* buf, cplx<T>* rbuf, int rank, const TW& tw,
                                               int sign, int epi, const void* inp, const void* auxp, void* outp,
                                               double* red, double* xchg, cplx<T>* smem, const InstDesc* insts) {
    BlueIo<T, TI, TO, SMB, CL> c;
    c.buf = buf;
    c.rbuf = rbuf;
    if constexpr (CL) {
        c.hN = J.N >> 1;
        c.rank = rank;
        c.nrank = 2;
    }
    c.N = J.N;
    c.M = J.M;
    c.epi = epi;
    c.inv = sign > 0;
    c.in = reinterpret_cast<const cplx<TI>*>(inp);
    c.chirp = reinterpret_cast<const cplx<T>*>(J.chirp);
    c.filt = reinterpret_cast<const cplx<T>*>(J.filt);
    c.out = reinterpret_cast<cplx<TO>*>(outp);
    c.auxp = auxp;
    c.sc = kc<T>(J.scale);
    auto sync = [&](bool cluster_wide) {
        if constexpr (CL) {
            if (cluster_wide) {
                cooperative_groups::this_cluster().sync();
                return;
            }
        }
        __syncthreads();
    };
    // ---- input phase (this CTA's half of the buffer when split over a cluster)
    const int h0 = CL ? rank * (J.N >> 1) : 0, h1 = CL ? h0 + (J.N >> 1) : J.N;
    bool built = false;
    if constexpr (SMB && !CL && (std::is_same<T, float>::value || std::is_same<T, double>::value)) {
        if (J.io_flags & 64) {
            c.scatter_terms(insts[J.inst], J.lat);
            built = true;
        }
    }
    if (!built) c.load_input(h0, h1);
    // the first pass reads both halves: both CTAs' inputs must be in place
    sync(true);
    const int np = J.npass;
    if constexpr (!SMB && !CL) {
        // global-scratch buffer: only the first DIF pass and the last DIT pass need the whole
        // buffer; every pass between them works inside the blocks of N / R0 elements that the first
        // pass leaves (R0 = its radix product), so each block is staged in shared memory for them
        const int R0 = (J.pass_r[0] & 15) * (J.pass_r[0] >> 4), Nb = J.N / R0;
        unsigned dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        constexpr int PS = blue_pad_shift(sizeof(cplx<T>));
        const size_t need = (size_t)(Nb + (PS ? (Nb >> PS) + 1 : 0)) * sizeof(cplx<T>);
        if (np >= 2 && smem && need <= dyn) {
            run_pass_u<UP, T>(0, J.pass_r[0] & 15, J.pass_r[0] >> 4, c, J.N, tw);
            __syncthreads();
            BlueIo<T, TI, TO, true, false> cb;
            cb.buf = smem;
            cb.N = Nb;
            cb.M = J.M;
            cb.tws = R0;
            for (int b = 0; b < R0; ++b) {
                cb.filt = c.filt + (size_t)b * Nb;
                cplx<T>* gb = c.buf + (size_t)b * Nb;
                stage_block<true>(cb, gb, Nb);
                __syncthreads();
                int Ns = Nb;
                for (int p = 1; p < np - 1; ++p) {
                    const int r1 = J.pass_r[p] & 15, r2 = J.pass_r[p] >> 4;
                    run_pass_u<UP, T>(0, r1, r2, cb, Ns, tw);
                    Ns /= r1 * r2;
                    __syncthreads();
                }
                run_pass_u<UP, T>(2, J.pass_r[np - 1] & 15, J.pass_r[np - 1] >> 4, cb, Ns, tw);
                __syncthreads();
                for (int p = np - 2; p >= 1; --p) {
                    const int r1 = J.pass_r[p] & 15, r2 = J.pass_r[p] >> 4;
                    Ns *= r1 * r2;
                    run_pass_u<UP, T>(1, r1, r2, cb, Ns, tw);
                    __syncthreads();
                }
                stage_block<false>(cb, gb, Nb);
                __syncthreads();
            }
            run_pass_u<UP, T>(1, J.pass_r[0] & 15, J.pass_r[0] >> 4, c, J.N, tw);
            __syncthreads();
            c.store_output(h0, min(h1, J.M));
            analyze_epilogue<T, TI, TO, SMB, CL>(J, c, epi, rank, red, xchg);
            return;
        }
    }
    // ---- DIF passes, the fused middle pass (last DIF pass, filter, first DIT pass), DIT passes
    // in reverse order (the last writes into both halves)
    for (int p = 0, Ns = J.N; p < np - 1; ++p) {
        const int r1 = J.pass_r[p] & 15, r2 = J.pass_r[p] >> 4;
        run_pass_u<UP, T>(0, r1, r2, c, Ns, tw);
        Ns /= r1 * r2;
        sync(p == 0);
    }
    int Ns = (J.pass_r[np - 1] & 15) * (J.pass_r[np - 1] >> 4);
    run_pass_u<UP, T>(2, J.pass_r[np - 1] & 15, J.pass_r[np - 1] >> 4, c, Ns, tw);
    // cluster-wide when this pass was also the first (np = 1) or the last DIT pass comes next
    sync(np <= 2);
    for (int p = np - 2; p >= 0; --p) {
        const int r1 = J.pass_r[p] & 15, r2 = J.pass_r[p] >> 4;
        Ns *= r1 * r2;
        run_pass_u<UP, T>(1, r1, r2, c, Ns, tw);
        sync(p <= 1);
    }
    // ---- output phase over this CTA's elements below M
    c.store_output(h0, min(h1, J.M));
    analyze_epilogue<T, TI, TO, SMB, CL>(J, c, epi, rank, red, xchg);
}

// One CTA (MODE 0, 1) or a cluster of two CTAs (MODE 2) = one Bluestein transform.  T:
// arithmetic (float, double or df64); TI/TO: element type of input/output.  MODE 0: work buffer
// in J.scratch (global, L2-resident); 1: in dynamic shared memory; 2: split over the two CTAs'
// shared memory.
template <class T, class TI, class TO, int MODE, int UP>
__device__ __forceinline__ void bluestein_cta(const BlueJob* __restrict__ jobs, int job, int rank, int sign, int epi,
                                              const InstDesc* __restrict__ insts, void* out_base,
                                              const void* aux_base) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[64];
    __shared__ double xchg[4];
    const BlueJob& J = jobs[job];
    cplx<T>* buf = MODE ? reinterpret_cast<cplx<T>*>(smem_raw) : reinterpret_cast<cplx<T>*>(J.scratch);
    cplx<T>* rbuf = nullptr;
    if constexpr (MODE == 2) rbuf = cooperative_groups::this_cluster().map_shared_rank(buf, rank ^ 1);
    // MODE 0: the dynamic shared memory stages the blocks between the first and the last pass
    cplx<T>* stage = MODE == 0 ? reinterpret_cast<cplx<T>*>(smem_raw) : nullptr;
    const void* inp = J.in;
    const void* auxp = J.aux;
    void* outp = J.out;
    if (J.io_flags & 3) {
        const InstDesc& I = insts[J.inst];
        const size_t esz = I.prec ? sizeof(c32) : sizeof(c64);
        if (J.io_flags & 1) inp = (const char*)I.samples + J.io_off * esz;
        if (J.io_flags & 2) auxp = (const char*)I.samples + J.io_off * esz;
    }
    if (J.io_flags & 48) {
        const InstDesc& I = insts[J.inst];
        if (J.io_flags & 16) outp = (char*)I.samp_out + J.io_off * sizeof(cplx<TO>);
        if (J.io_flags & 32)
            auxp = I.samp_noise ? (const void*)((const char*)I.samp_noise + J.io_off * (I.prec ? sizeof(c32) : sizeof(c64)))
                                : nullptr;
    }
    if (J.io_flags & 4) outp = (char*)out_base + J.io_off * sizeof(cplx<TO>);
    if (J.io_flags & 8) auxp = aux_base ? (const void*)((const c64*)aux_base + J.io_off) : nullptr;
    if constexpr (std::is_same<T, float>::value) {
        __shared__ c32 s_twa[1024], s_twb[256];
        const c32* ga = reinterpret_cast<const c32*>(J.twa);
        const c32* gb = reinterpret_cast<const c32*>(J.twb);
        for (int i = threadIdx.x; i < J.tw_na; i += blockDim.x) s_twa[i] = ga[i];
        for (int i = threadIdx.x; i < 256; i += blockDim.x) s_twb[i] = gb[i];
        __syncthreads();
        bluestein_body<T, TI, TO, MODE != 0, MODE == 2, UP>(J, buf, rbuf, rank, TwTwo{s_twa, s_twb}, sign, epi, inp, auxp, outp,
                                             red, xchg, stage, insts);
    } else {
        bluestein_body<T, TI, TO, MODE != 0, MODE == 2, UP>(J, buf, rbuf, rank, TwFull<T>{reinterpret_cast<const cplx<T>*>(J.tw)},
                                             sign, epi, inp, auxp, outp, red, xchg, stage, insts);
    }
}

template <class T, class TI, class TO, int MODE, int UP = 0>
__global__ void __launch_bounds__(blue_max_threads<T>(MODE), 1) k_bluestein(const BlueJob* __restrict__ jobs, int sign, int epi,
                                                            const InstDesc* __restrict__ insts, void* out_base,
                                                            const void* aux_base) {
    bluestein_cta<T, TI, TO, MODE, UP>(jobs, blockIdx.x, 0, sign, epi, insts, out_base, aux_base);
}

template <class T, class TI, class TO>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(blue_max_threads<T>(2), 1)
    k_bluestein_pair(const BlueJob* __restrict__ jobs, int sign, int epi, const InstDesc* __restrict__ insts,
                     void* out_base, const void* aux_base) {
    const int rank = (int)cooperative_groups::this_cluster().block_rank();
    bluestein_cta<T, TI, TO, 2, 0>(jobs, blockIdx.x >> 1, rank, sign, epi, insts, out_base, aux_base);
}

// ================================================================== launch of one instantiation

// upair: the pass pair shared by every pass of every job (r1 | r2 << 4), or 0; FP32 transforms in
// shared memory whose passes are all (4, 3) run the kernel specialised for that pair
constexpr int kUniformPair43 = 4 | (3 << 4);
template <class T, class TI, class TO>
int launch_t(const BlueJob* djobs, int njobs, int maxN, int mode, int sign, int epi, const InstDesc* insts,
             cudaStream_t st, void* ob, const void* ab, int threads, int upair) {
    // 0 (or any size the kernel cannot take): the largest CTA
    const int tmax = blue_max_threads<T>(mode);
    if (threads < 64 || threads > tmax || threads % 32) threads = tmax;
    if (njobs == 0) return SFFT_OK;
    if (mode == 1 || mode == 2) {
        const size_t bytes = blue_smem_bytes(mode == 2 ? maxN / 2 : maxN, sizeof(cplx<T>));
        if (bytes > blue_smem_limit() || (mode == 2 && maxN % 2)) {
            set_error("Bluestein length %d does not fit the shared-memory mode %d", maxN, mode);
            return SFFT_EINVAL;
        }
        if constexpr (std::is_same<T, float>::value) {
            if (mode == 1 && upair == kUniformPair43) {
                SFFT_TRY(allow_smem((const void*)k_bluestein<T, TI, TO, 1, kUniformPair43>, (int)blue_smem_limit()));
                k_bluestein<T, TI, TO, 1, kUniformPair43><<<njobs, threads, bytes, st>>>(djobs, sign, epi, insts, ob, ab);
                return launch_check("k_bluestein");
            }
        }
        if (mode == 1) SFFT_TRY(allow_smem((const void*)k_bluestein<T, TI, TO, 1>, (int)blue_smem_limit()));
        else SFFT_TRY(allow_smem((const void*)k_bluestein_pair<T, TI, TO>, (int)blue_smem_limit()));
        if (mode == 1) k_bluestein<T, TI, TO, 1><<<njobs, threads, bytes, st>>>(djobs, sign, epi, insts, ob, ab);
        else k_bluestein_pair<T, TI, TO><<<2 * njobs, threads, bytes, st>>>(djobs, sign, epi, insts, ob, ab);
    } else {
        // the global-scratch mode stages the blocks of its middle passes in shared memory (the
        // kernel falls back to global passes when a block does not fit)
        const size_t bytes = blue_smem_limit();
        SFFT_TRY(allow_smem((const void*)k_bluestein<T, TI, TO, 0>, (int)bytes));
        k_bluestein<T, TI, TO, 0><<<njobs, threads, bytes, st>>>(djobs, sign, epi, insts, ob, ab);
    }
    return launch_check("k_bluestein");
}

}  // namespace sfft
