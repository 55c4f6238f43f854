// Shared definitions of the sm_103a sparse-FFT library: complex arithmetic, error
// plumbing and the descriptors that the kernels of every stage consume.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sfft.h"
#include "df64.cuh"

namespace sfft {

// ------------------------------------------------------------------ complex numbers
template <class T>
struct alignas(2 * sizeof(T)) cplx {
    T x, y;
};
using c32 = cplx<float>;
using c64 = cplx<double>;

template <class T> __host__ __device__ __forceinline__ cplx<T> mk(T a, T b) { return cplx<T>{a, b}; }
template <class T> __host__ __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <class T> __host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <class T> __host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class T> __host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, T s) { return {a.x * s, a.y * s}; }
template <class T> __host__ __device__ __forceinline__ cplx<T> conj(cplx<T> a) { return {a.x, -a.y}; }
// a * conj(b)
template <class T> __host__ __device__ __forceinline__ cplx<T> mulc(cplx<T> a, cplx<T> b) {
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <class T> __host__ __device__ __forceinline__ T abs2(cplx<T> a) { return a.x * a.x + a.y * a.y; }

// double-float complex products: each component a*b + c*d with error-free FMA products and one
// renormalisation (19 FP32 instructions instead of two products and a sum, 25); the error is
// bounded relative to |a b| + |c d|, the normwise bound an FFT needs
__host__ __device__ __forceinline__ df64 df_dot2(df64 a, df64 b, df64 c, df64 d) {
    const float p1 = DF_MUL(a.hi, b.hi), e1 = fmaf(a.hi, b.hi, -p1);
    const float p2 = DF_MUL(c.hi, d.hi), e2 = fmaf(c.hi, d.hi, -p2);
    const df64 s = df_two_sum(p1, p2);
    float t = DF_ADD(e1, e2);
    t = fmaf(a.hi, b.lo, t);
    t = fmaf(a.lo, b.hi, t);
    t = fmaf(c.hi, d.lo, t);
    t = fmaf(c.lo, d.hi, t);
    return df_fast_two_sum(s.hi, DF_ADD(s.lo, t));
}
__host__ __device__ __forceinline__ cplx<df64> operator*(cplx<df64> a, cplx<df64> b) {
    return {df_dot2(a.x, b.x, -a.y, b.y), df_dot2(a.x, b.y, a.y, b.x)};
}
__host__ __device__ __forceinline__ cplx<df64> mulc(cplx<df64> a, cplx<df64> b) {
    return {df_dot2(a.x, b.x, a.y, b.y), df_dot2(a.y, b.x, -a.x, b.y)};
}
// exact halving
template <class T> __host__ __device__ __forceinline__ cplx<T> half(cplx<T> a) { return {a.x * (T)0.5, a.y * (T)0.5}; }
__host__ __device__ __forceinline__ cplx<df64> half(cplx<df64> a) {
    return {df64{DF_MUL(a.x.hi, 0.5f), DF_MUL(a.x.lo, 0.5f)}, df64{DF_MUL(a.y.hi, 0.5f), DF_MUL(a.y.lo, 0.5f)}};
}

template <class T, class U> __host__ __device__ __forceinline__ cplx<T> cvt(cplx<U> a) { return {(T)a.x, (T)a.y}; }

#ifdef __CUDACC__
// read-only cached loads of complex values
__device__ __forceinline__ c32 ldg(const c32* p) {
    float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ c64 ldg(const c64* p) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
}
#endif

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
const char* get_error();

#define SFFT_CU(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            ::sfft::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return SFFT_ECUDA;                                                                 \
        }                                                                                      \
    } while (0)

#define SFFT_TRY(expr)            \
    do {                          \
        int rc_ = (expr);         \
        if (rc_ != SFFT_OK) return rc_; \
    } while (0)

#define SFFT_CHECK(cond, code, ...)           \
    do {                                      \
        if (!(cond)) {                        \
            ::sfft::set_error(__VA_ARGS__);   \
            return (code);                    \
        }                                     \
    } while (0)

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current device; the attribute is
// set once per (kernel, device) and the record is guarded by a mutex (thread-safe, multi-GPU).
int allow_smem(const void* kernel, int bytes);

inline int launch_check(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("launch of %s failed: %s", what, cudaGetErrorString(e));
        return SFFT_ECUDA;
    }
    return SFFT_OK;
}

// ------------------------------------------------------------------ constants
constexpr int kMaxD = 32;      // candidate dimension limit
constexpr int kMaxL = 64;      // lattices per reconstruction
constexpr int kMaxStages = 24; // mixed-radix stages of one Bluestein length

// ------------------------------------------------------------------ FFT tables
// Everything needed to run a length-M DFT by Bluestein's algorithm through a length-N
// cyclic convolution, N = 2^a 3^b 5^c >= 2M-1, computed once per distinct M.
struct FftTables {
    int64_t M = 0, N = 0;
    int nstages = 0;
    int radix[kMaxStages];
    // device tables; the *32 copies are the double tables rounded to float
    c64* tw64 = nullptr;   // [N] exp(-2 pi i n / N)
    c32* tw32 = nullptr;
    c64* chirp64 = nullptr; // [M] exp(-pi i (j^2 mod 2M) / M)
    c32* chirp32 = nullptr;
    c64* filt64[2] = {nullptr, nullptr}; // [N] DIF(b)/N, digit-reversed; [0] forward, [1] inverse
    c32* filt32[2] = {nullptr, nullptr};
    c64* dft64 = nullptr;  // [M] exp(-2 pi i m / M) for single-bucket FP64 DFTs
    // FP32 twiddles as two small tables: exp(-2 pi i k/N) = twa[k >> 8] * twb[k & 255]
    c32* twa32 = nullptr;  // [tw_na] exp(-2 pi i 256 a / N)
    c32* twb32 = nullptr;  // [256]   exp(-2 pi i b / N)
    int tw_na = 0;
    // double-float copies (hi, lo words of each double entry)
    void* twdf = nullptr;     // [N]
    void* chirpdf = nullptr;  // [M]
    void* dftdf = nullptr;    // [M] exp(-2 pi i m / M), single-bucket re-tests of FP32 samples
    void* filtdf[2] = {nullptr, nullptr};
    int refs = 0;
    int device = -1;
};

int tables_acquire(int64_t M, FftTables** out);
void tables_release(FftTables* t);
int64_t bluestein_size(int64_t M);

// ------------------------------------------------------------------ per-lattice job
// One Bluestein transform (a length-M DFT of one lattice).
struct BlueJob {
    const void* in;      // input complex (element type by launch), M entries
    void* out;           // output complex, M entries
    const void* aux;     // epilogue side buffer: noise input (EPI_ADDNOISE) or low-word output
                         // (EPI_ANALYZE of a double-float transform with float output), M entries
    void* scratch;       // global work buffer of N complex (used when the buffer is not in smem)
    const void* tw;      // twiddles of the transform precision (full table)
    const void* twa;     // FP32 two-level twiddle tables
    const void* twb;
    const void* chirp;
    const void* filt;    // filter of the requested direction
    const double* dft64; // single-bucket root table (guard re-tests of FP64 samples)
    struct LatStats* stat; // side outputs of EPI_ANALYZE
    double scale;        // output scale (1/M for the normalised forward DFT)
    int M, N, nstages, tw_na;
    // io_flags: bit 0 in = samples of instance `inst` + io_off; bit 1 aux = those samples;
    //           bit 2 out = out_base (launch argument) + io_off; bit 3 aux = aux_base + io_off;
    //           bit 4 out = samp_out of instance `inst` + io_off; bit 5 aux = its samp_noise + io_off;
    //           bit 6 input = the sparse-polynomial terms of instance `inst` (samp_kvec, samp_coef),
    //           summed into the buckets of lattice `lat` in the CTA's shared-memory buffer (buffer
    //           mode 1 only; `in` is then unused)
    int inst, io_flags, lat;
    int64_t io_off;
    uint8_t radix[kMaxStages];  // stage radices in DIF order
    // passes over the work buffer: one stage or two consecutive stages fused in registers;
    // pass_r[p] = r1 | r2 << 4 (r2 = 1 for a single stage)
    uint8_t npass;
    uint8_t pass_r[kMaxStages];
};

// epilogue modes of the Bluestein kernel
enum BlueEpi : int {
    EPI_PLAIN = 0,    // out = scale * y
    EPI_ANALYZE = 1,  // out = y / M; per-lattice max|y| and sum |x|^2 recorded; a double-float
                      // transform with float output also writes the low words of y / M to aux
    EPI_ADDNOISE = 2, // out = y + aux (aux complex double)
};

struct LatStats {
    double max_abs;   // max_h |ghat_h| (FP64 after the guard re-test of the maximum)
    double rms;       // sqrt(sum_j |x_j|^2 / M)
    double tau;       // zero-test threshold
    double band;      // guard half-width around tau
    float max32;      // max_h |ghat_h| of the working-precision transform
    int pad;
};

// One launch of Bluestein transforms over a device job array.  prec: 0 double, 1 float,
// 2 double-float; in_prec/out_prec: 0 double, 1 float.  mode: work buffer in global scratch (0),
// in shared memory (1: N <= maxN complex values fit one CTA), or split over a two-CTA cluster
// (2: every N even, N/2 values fit one CTA).
struct InstDesc;
// upair: r1 | r2 << 4 when every pass of every job is the fused pair (r1, r2) (uniform_pair), else 0.
int launch_bluestein(const BlueJob* djobs, int njobs, int maxN, int mode, int prec, int in_prec, int out_prec, int sign,
                     int epi, const InstDesc* insts, cudaStream_t st, void* out_base = nullptr,
                     const void* aux_base = nullptr, int threads = 0, int upair = 0);
// the pass pair shared by every pass of the jobs (r1 | r2 << 4), or 0
int uniform_pair(const BlueJob* jobs, size_t n);
size_t blue_smem_limit();
// Shared-memory work buffers of 8-byte complex values are padded against bank conflicts of the
// strided passes: element e lives at e + (e >> 5).  (16-byte values: measured slower padded, the
// index arithmetic costs more than the conflicts.)
constexpr int blue_pad_shift(size_t esz) { return esz == 8 ? 5 : 0; }
inline size_t blue_smem_bytes(int64_t n, size_t esz) {
    const int p = blue_pad_shift(esz);
    return (size_t)(n + (p ? (n >> p) + 1 : 0)) * esz;
}
// per-type launchers behind launch_bluestein (one translation unit each)
int launch_bluestein_f64(const BlueJob* djobs, int njobs, int maxN, int mode, int sign, int epi, const InstDesc* insts,
                         cudaStream_t st, void* ob, const void* ab, int threads, int upair);
int launch_bluestein_f32(bool in_double, const BlueJob* djobs, int njobs, int maxN, int mode, int sign, int epi,
                         const InstDesc* insts, cudaStream_t st, void* ob, const void* ab, int threads, int upair);
int launch_bluestein_df64(const BlueJob* djobs, int njobs, int maxN, int mode, int sign, int epi, const InstDesc* insts,
                          cudaStream_t st, void* ob, const void* ab, int threads, int upair);
// stage pairs that the transform kernels implement as one fused pass (run_pass lists the same)
constexpr bool pass_fusable(int r1, int r2) {
    return (r1 == 4 && (r2 == 4 || r2 == 3 || r2 == 2)) || (r1 == 3 && (r2 == 3 || r2 == 5)) ||
           (r1 == 2 && (r2 == 3 || r2 == 5));
}
// register budget of a fused pass: elements per thread (16 complex floats, 12 complex doubles
// or double-floats, so that 512-thread CTAs stay within 128 registers per thread)
template <class T> constexpr int pass_maxprod() { return sizeof(T) == 4 ? 16 : 12; }
// greedy left-to-right fusion of consecutive stages whose radix product is at most maxprod
int plan_passes(const int* radix, int ns, int maxprod, uint8_t* pass_r);

// ------------------------------------------------------------------ instance / lattice descriptors
// Everything the per-candidate kernels need about one reconstruction problem.  Lives in
// device memory; the per-call IO pointers are refreshed before each run.
struct InstDesc {
    int d, L, need, prec;      // need = ceil(nu L) (Algorithm 1 count threshold)
    int combine, nwords;
    int cand_i8, cand_ld;      // candidate rows: int8 (1) or int32 (0); row stride in elements
    int rank_bits, spare;      // Algorithm 4 rank-key precision (sfft_params.rank_bits)
    int64_t n;                 // |Gamma|
    int64_t cap;               // capacity of the detected list
    int64_t s_tilde;
    double tau_abs, tau_rel, theta_abs, theta_rel;
    const void* cand;          // [n, cand_ld] int32 or int8
    const int32_t* z;          // [L, d]
    const int32_t* Ml;         // [L]
    const uint32_t* mu;        // [L] floor(2^32 / M_l)
    const uint32_t* offk;      // [L] multiple of M_l added before the Barrett reduction
    const int64_t* soff;       // [L+1] sample offsets
    const int32_t* boff;       // [L] bitmap word offsets
    uint32_t* nzbits;          // [nwords]
    void* ghat;                // [sum M] complex (prec)
    LatStats* stats;           // [L]
    uint32_t* detbits;         // [ceil(n/32)]
    uint8_t* cnt8;             // [n] partial counts between lattice groups (plans with several groups)
    int64_t* det;              // [cap] detected indices (ascending)
    int64_t* cnt;              // [kCntWords] counters: 0 |Itilde|, 1 n_out, 2 n_guard, 3 error flags
    c64* coef;                 // [cap]
    int32_t* H;                // [cap, L]
    uint8_t* sel;              // [cap, 2] lattice of the Re / Im median
    uint8_t* rsel;             // [cap, 2] lattice of the refinement's Re / Im median (refine plans)
    c64* adj_w;                // [cap] adjoint: cotangents of the detected set
    int32_t* coll;             // [sum M] collision counts
    c64* C;                    // [sum M] bucket scatter buffer
    c32* ghat_lo;              // [sum M] low words of a double-float forward transform, or NULL
    int32_t* outpos;           // [cap] detected position of output q
    c64* lsq_work;             // [3 cap] conjugate-gradient vectors (least-squares combine) or NULL
    int32_t* lsq_next;         // [cap, L] bucket lists of the detected entries (least squares)
    void* lsq_pairs;           // [lsq_pair_cap] colliding pairs (q, q', M_l) of the normal matrix
    int64_t lsq_pair_cap;
    // ---- per call
    const void* samples;       // [sum M] complex (prec)
    int64_t* supp_out;
    uint64_t* key_out;         // optional: the rank key of each output (sharded merges)
    c64* coef_out;
    int64_t out_cap;
    uint8_t* dcounts;          // diag
    int32_t* dhashes;          // diag
    // ---- per call of the sparse-polynomial sampler
    const int32_t* samp_kvec;  // [samp_nterms, d]
    const c64* samp_coef;      // [samp_nterms]
    int64_t samp_nterms;
    void* samp_out;            // [sum M] complex (prec)
    const void* samp_noise;    // [sum M] complex in the plan precision, or NULL
};

static_assert(sizeof(InstDesc) % 8 == 0, "descriptors are uploaded as 8-byte words");

// One lattice of one instance (for per-lattice kernels).
struct LatDesc {
    int inst, l, M, N;
    int64_t soff;
    int32_t boff;
    int pad;
    const double* dft64;       // [M] exp(-2 pi i m / M)
    const void* dftdf;         // [M] the same roots as double-float pairs (cplx<df64>)
};

// The detection bits of an instance are compacted in kCompactChunks chunks of whole words; the
// hash kernels count the detections of chunk c in cnt[8 + c] so that each chunk's compaction
// starts from the sum of the counts before it.
constexpr int kCompactChunks = 32;
constexpr int kCntWords = 8 + kCompactChunks;
__device__ __forceinline__ void mark_detected(const InstDesc& I, int64_t idx) {
    atomicOr(&I.detbits[idx >> 5], 1u << (idx & 31));
    const int64_t W = (I.n + 31) >> 5, cw = (W + kCompactChunks - 1) / kCompactChunks;
    atomicAdd(reinterpret_cast<unsigned long long*>(&I.cnt[8 + (idx >> 5) / cw]), 1ull);
}

#ifdef __CUDACC__
// Order-preserving key of a non-negative double rounded to `bits` significant bits (0: all 52):
// the bit pattern of a non-negative double orders like its value, and rounding the pattern to a
// multiple of 2^(52 - bits) (half up; a carry moves into the exponent) keeps that order.  Moduli
// whose keys agree rank by position (Algorithm 4's near-tie rule, sfft_params.rank_bits).
__device__ __forceinline__ unsigned long long rank_key(double v, int bits) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    if (bits > 0 && bits < 52) {
        const int drop = 52 - bits;
        b = ((b + (1ull << (drop - 1))) >> drop) << drop;
    }
    return b;
}

// Copy of n 32-bit words from global to shared memory by the whole CTA with kCopyBatch loads of
// every thread in flight (16-byte loads when both addresses are 16-byte aligned), so that a
// CTA's prologue pays the global-memory latency a few times instead of once per word.
template <int kCopyBatch = 4>
__device__ __forceinline__ void copy_words_to_smem(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src, int n) {
    int done = 0;
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
        const int n4 = n >> 2;
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        uint4* d4 = reinterpret_cast<uint4*>(dst);
        for (int i0 = threadIdx.x; i0 < n4; i0 += kCopyBatch * blockDim.x) {
            uint4 v[kCopyBatch];
#pragma unroll
            for (int u = 0; u < kCopyBatch; ++u) {
                const int i = i0 + u * blockDim.x;
                if (i < n4) v[u] = __ldg(s4 + i);
            }
#pragma unroll
            for (int u = 0; u < kCopyBatch; ++u) {
                const int i = i0 + u * blockDim.x;
                if (i < n4) d4[i] = v[u];
            }
        }
        done = n4 << 2;
    }
    for (int i0 = done + threadIdx.x; i0 < n; i0 += kCopyBatch * blockDim.x) {
        uint32_t v[kCopyBatch];
#pragma unroll
        for (int u = 0; u < kCopyBatch; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < n) v[u] = __ldg(src + i);
        }
#pragma unroll
        for (int u = 0; u < kCopyBatch; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < n) dst[i] = v[u];
        }
    }
}
#endif

// error flag bits (InstDesc::cnt[3])
enum : int64_t { ERR_DET_CAP = 1, ERR_GUARD_CAP = 2, ERR_OUT_CAP = 4, ERR_TC_TIMEOUT = 8 };
// counters InstDesc::cnt[4]: least-squares CG iterations; cnt[5]: colliding pairs found

}  // namespace sfft
