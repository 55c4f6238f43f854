// Per-lattice and per-candidate kernels of the reconstruction (Algorithms 1, 2 and 4):
//   zero test of the lattice DFT buckets with direct re-tests near the threshold (Remark 2.3),
//   candidate hashing k.z_l mod M_l and the majority count (Algorithm 1/2, count rule),
//   ascending compaction of the detected set, the per-candidate gather and component-wise
//   median (eq. 2.6), bucket collision counts and the Remark 2.8 combine, the refinement
//   scatter/update, and Algorithm 4's theta filter plus radix top-s_tilde selection.
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace sfft {

// ================================================================== zero test (per lattice)
// One CTA per lattice.  The working-precision |ghat| decides every bucket except those within
// `band` of tau (and the maximum, which sets tau when tau_rel > 0): those are recomputed by a
// direct DFT sum of the samples with exact integer phase (j h mod M).
//
// The phase of thread t's terms j = t, t + B, t + 2B, ... steps by B h mod M.  FP64 samples sum in
// FP64.  FP32 samples sum in double-float on the FP32 pipes (on this GPU FP64 runs at a small
// fraction of the FP32 rate): each term x_j w, w = w_hi + w_lo the root as a float pair, enters as
// float products split exactly (x w_hi = p + e by one FMA) plus x w_lo, accumulated by two-sums
// into a (hi, lo) pair; relative error ~2^-46 of sum |x_j|, the accuracy class of the FP64 sum.
__device__ __forceinline__ void df_acc(float& h, float& l, float a, df64 w) {
    const float p = a * w.hi;
    float e = fmaf(a, w.hi, -p);
    e = fmaf(a, w.lo, e);
    const float s = h + p, bb = s - h;
    l += ((h - (s - bb)) + (p - bb)) + e;
    h = s;
}

// A thread's terms are taken kBdUnroll at a time with their loads issued together (the root-table
// lookups are gathers), then accumulated in the order j = t, t + B, ... as one at a time would.
constexpr int kBdUnroll = 4;
template <class TS>
__device__ c64 bucket_dft(const cplx<TS>* __restrict__ x, int M, int h, const c64* __restrict__ tab,
                          const cplx<df64>* __restrict__ tabdf, double* red) {
    const unsigned B = blockDim.x, uM = (unsigned)M;
    unsigned ph = (unsigned)(((int64_t)threadIdx.x * h) % M);
    const unsigned inc = (unsigned)(((int64_t)B * h) % M);
    double re = 0, im = 0;
    if constexpr (sizeof(TS) == 4) {
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
        for (int j0 = threadIdx.x; j0 < M; j0 += kBdUnroll * (int)B) {
            cplx<df64> w[kBdUnroll];
            c32 v[kBdUnroll];
#pragma unroll
            for (int u = 0; u < kBdUnroll; ++u) {
                const int j = j0 + u * (int)B;
                if (j < M) {
                    w[u] = tabdf[ph];
                    v[u] = x[j];
                }
                ph += inc;
                ph = min(ph, ph - uM);  // ph + inc < 2M: one conditional subtraction
            }
#pragma unroll
            for (int u = 0; u < kBdUnroll; ++u) {
                if (j0 + u * (int)B >= M) break;
                df_acc(rh, rl, v[u].x, w[u].x);
                df_acc(rh, rl, -v[u].y, w[u].y);
                df_acc(ih, il, v[u].x, w[u].y);
                df_acc(ih, il, v[u].y, w[u].x);
            }
        }
        re = (double)rh + (double)rl;
        im = (double)ih + (double)il;
    } else {
        for (int j0 = threadIdx.x; j0 < M; j0 += kBdUnroll * (int)B) {
            c64 w[kBdUnroll], v[kBdUnroll];
#pragma unroll
            for (int u = 0; u < kBdUnroll; ++u) {
                const int j = j0 + u * (int)B;
                if (j < M) {
                    w[u] = tab[ph];
                    v[u] = cvt<double>(x[j]);
                }
                ph += inc;
                ph = min(ph, ph - uM);
            }
#pragma unroll
            for (int u = 0; u < kBdUnroll; ++u) {
                if (j0 + u * (int)B >= M) break;
                re += v[u].x * w[u].x - v[u].y * w[u].y;
                im += v[u].x * w[u].y + v[u].y * w[u].x;
            }
        }
    }
    // block sums of re, im
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) { red[2 * w] = re; red[2 * w + 1] = im; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += red[2 * i]; b += red[2 * i + 1]; }
        red[64] = a / M;
        red[65] = b / M;
    }
    __syncthreads();
    c64 r = {red[64], red[65]};
    __syncthreads();
    return r;
}

// block-wide maximum of a double (all threads get the result)
__device__ __forceinline__ double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, red[i]);
        red[64] = m;
    }
    __syncthreads();
    const double r = red[64];
    __syncthreads();
    return r;
}

constexpr int kZtThreads = 512;
constexpr int kGuardCap = 1024;

template <class TS>
__global__ void __launch_bounds__(kZtThreads, 2) k_zero_test(const LatDesc* __restrict__ lats, InstDesc* __restrict__ insts,
                                                          double kappa_u_log) {
    __shared__ double red[72];
    __shared__ int glist[kGuardCap];
    __shared__ int gcount;
    __shared__ double s_max64;
    const LatDesc& D = lats[blockIdx.x];
    InstDesc& I = insts[D.inst];
    LatStats& S = I.stats[D.l];
    const int M = D.M;
    cplx<TS>* g = reinterpret_cast<cplx<TS>*>(I.ghat) + D.soff;
    // low words of a double-float transform: ghat = g + glo to ~2^-44 relative accuracy
    c32* glo = I.ghat_lo ? I.ghat_lo + D.soff : nullptr;
    const cplx<TS>* x = reinterpret_cast<const cplx<TS>*>(I.samples) + D.soff;
    const c64* tab = reinterpret_cast<const c64*>(D.dft64);
    const cplx<df64>* tabdf = reinterpret_cast<const cplx<df64>*>(D.dftdf);
    // FP64 scalars are formed by one thread and shared: on this GPU a warp-wide FP64 instruction
    // costs as much as dozens of FP32 ones
    __shared__ double s_band, s_tlo, s_thi;
    __shared__ TS s_lo2, s_hi2;
    if (threadIdx.x == 0) s_band = kappa_u_log * log2((double)D.N) * S.rms;
    __syncthreads();
    const double band = s_band;
    auto full = [&](int h) -> c64 {  // the bucket in the transform's full precision
        cplx<TS> v = g[h];
        c64 r = {(double)v.x, (double)v.y};
        if (glo) { c32 w = glo[h]; r.x += (double)w.x; r.y += (double)w.y; }
        return r;
    };
    auto store = [&](int h, c64 v) {  // replace a bucket by its directly summed value
        cplx<TS> hi = cvt<TS>(v);
        g[h] = hi;
        if (glo) glo[h] = c32{(float)(v.x - (double)hi.x), (float)(v.y - (double)hi.y)};
    };
    if (threadIdx.x == 0) { gcount = 0; s_max64 = 0; }
    __syncthreads();
    // Squared magnitudes are formed in the working precision and compared with bounds widened
    // by a relative slack that covers their rounding; only buckets between the bounds need the
    // direct re-test.
    const double slack = sizeof(TS) == 4 ? 1e-6 : 1e-15;
    const double big = sizeof(TS) == 4 ? 3.0e38 : 1.0e300;
    // ---- exact maximum: direct re-test of every bucket that could be the maximum
    double tau = I.tau_abs;
    if (I.tau_rel > 0) {
        if (threadIdx.x == 0) {
            const double lo = fmax(S.max_abs * (1.0 - 1.0 / 1048576.0) - 2.0 * band, 0.0);
            s_lo2 = (TS)fmin(lo * lo * (1.0 - slack), big);
        }
        __syncthreads();
        const TS lo2 = s_lo2;
        for (int h = threadIdx.x; h < M; h += blockDim.x) {
            cplx<TS> v = g[h];
            if (v.x * v.x + v.y * v.y >= lo2) {
                int p = atomicAdd(&gcount, 1);
                if (p < kGuardCap) glist[p] = h;
            }
        }
        __syncthreads();
        int nc = min(gcount, kGuardCap);
        if (gcount > kGuardCap && threadIdx.x == 0) atomicOr((unsigned long long*)&I.cnt[3], (unsigned long long)ERR_GUARD_CAP);
        if (glo) {  // the double-float value is the maximum's FP64-class value
            double m = 0;
            for (int i = threadIdx.x; i < nc; i += blockDim.x) m = fmax(m, sqrt(abs2(full(glist[i]))));
            m = block_max(m, red);
            if (threadIdx.x == 0) s_max64 = m;
        } else {
            for (int i = 0; i < nc; ++i) {
                c64 v = bucket_dft(x, M, glist[i], tab, tabdf, red);
                if (threadIdx.x == 0) {
                    s_max64 = fmax(s_max64, sqrt(abs2(v)));
                    store(glist[i], v);
                }
            }
        }
        __syncthreads();
        tau = fmax(tau, I.tau_rel * s_max64);
        if (threadIdx.x == 0) { S.max_abs = s_max64; gcount = 0; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        S.tau = tau;
        S.band = band;
        s_tlo = fmax(tau - band, 0.0);
        s_thi = tau + band;
        s_lo2 = (TS)fmin(s_tlo * s_tlo * (1.0 - slack), big);  // below: certainly zero
        s_hi2 = (TS)fmin(s_thi * s_thi * (1.0 + slack), big);  // above: certainly non-zero
    }
    __syncthreads();
    // ---- threshold: one warp writes 32 consecutive buckets per ballot
    const double tlo = s_tlo, thi = s_thi;
    const TS lo2 = s_lo2, hi2 = s_hi2;
    uint32_t* words = I.nzbits + D.boff;
    const int nw = (M + 31) >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    // kZtUnroll words per warp and iteration, their loads issued together
    constexpr int kZtUnroll = 4;
    for (int w0 = warp * kZtUnroll; w0 < nw; w0 += nwarp * kZtUnroll) {
        cplx<TS> v[kZtUnroll];
#pragma unroll
        for (int u = 0; u < kZtUnroll; ++u) {
            const int h = (w0 + u) * 32 + lane;
            v[u] = h < M ? g[h] : cplx<TS>{(TS)0, (TS)0};
        }
#pragma unroll
        for (int u = 0; u < kZtUnroll; ++u) {
            const int wi = w0 + u, h = wi * 32 + lane;
            if (wi >= nw) break;
            bool nz = false;
            if (h < M) {
                TS a2 = v[u].x * v[u].x + v[u].y * v[u].y;
                nz = a2 > hi2;
                if (!nz && a2 >= lo2) {
                    // uncertain in the working precision: the double-float value decides outside
                    // the transform's error band, the direct re-test below inside it
                    bool open = true;
                    if (glo) {
                        const double a = sqrt(abs2(full(h)));
                        if (a > thi) { nz = true; open = false; }
                        else if (a < tlo) open = false;
                    }
                    if (open) {
                        int p = atomicAdd(&gcount, 1);
                        if (p < kGuardCap) glist[p] = h;
                    }
                }
            }
            uint32_t b = __ballot_sync(0xffffffffu, nz);
            if (lane == 0) words[wi] = b;
        }
    }
    __syncthreads();
    int nc = min(gcount, kGuardCap);
    if (gcount > kGuardCap && threadIdx.x == 0) atomicOr((unsigned long long*)&I.cnt[3], (unsigned long long)ERR_GUARD_CAP);
    for (int i = 0; i < nc; ++i) {
        int h = glist[i];
        c64 v = bucket_dft(x, M, h, tab, tabdf, red);
        if (threadIdx.x == 0) {
            double a = sqrt(abs2(v));
            uint32_t bit = 1u << (h & 31);
            if (a > tau) atomicOr(&words[h >> 5], bit);
            else atomicAnd(&words[h >> 5], ~bit);
            store(h, v);  // the stored bucket is the FP64 value that decided the test
        }
    }
    if (threadIdx.x == 0 && nc) atomicAdd((unsigned long long*)&I.cnt[2], (unsigned long long)nc);
}

// ================================================================== hash + count (Algorithm 1/2)
// Candidates are streamed once from HBM; the non-zero bitmap of all lattices of the instance
// and the generating vectors sit in shared memory.  h = k.z_l mod M_l is exact: the int32
// inner product is offset by a multiple of M_l to be non-negative and reduced by a Barrett
// step (q = umulhi(x, floor(2^32/M)), one conditional subtraction).
// 384 threads: the bitmap of all lattices (48 KB at L = 37, M = 10331) lets 4 CTAs share an SM, so
// 384-thread CTAs keep 48 warps resident where 256-thread ones keep 32 (measured 0.398 -> 0.363 ms
// for 16 instances of 2^20 candidates; 512 threads: 0.367 ms, limited by registers to 3 CTAs)
constexpr int kHashThreads = 384;
constexpr int kHashThreadsBig = 768;  // CTAs whose bitmap leaves room for at most two per SM
constexpr int kCPT = 2;  // candidates per thread

// Row r of int8 candidate rows of stride ld bytes as KW int8x4 words: directly when ld is a multiple
// of 4, else from the aligned words around the row by funnel shifts.  Rows below r_safe have those
// KW + 1 words inside the array; the last rows are read with bounds checks (no read past nbytes).
// Bytes past d belong to the next row (or are zero at the array's end).
template <int KW>
__device__ __forceinline__ void load_row8(const uint32_t* __restrict__ w8, const uint8_t* __restrict__ b8, int64_t r,
                                          int ld, int64_t nbytes, int64_t r_safe, uint32_t* kw) {
    if ((ld & 3) == 0) {
        const int ldw = ld >> 2;
#pragma unroll
        for (int w = 0; w < KW; ++w) kw[w] = __ldg(w8 + r * ldw + w);
        return;
    }
    const int64_t b0 = r * ld, w0 = b0 >> 2;
    const uint32_t sh = (uint32_t)(b0 & 3) * 8u;
    uint32_t wv[KW + 1];
    if (r < r_safe) {
#pragma unroll
        for (int j = 0; j <= KW; ++j) wv[j] = __ldg(w8 + w0 + j);
    } else {
#pragma unroll
        for (int j = 0; j <= KW; ++j) {
            const int64_t wj = w0 + j;
            if ((wj + 1) * 4 <= nbytes) {
                wv[j] = __ldg(w8 + wj);
            } else {  // the array's last bytes
                uint32_t v = 0;
                for (int q = 0; q < 4; ++q)
                    if (wj * 4 + q < nbytes) v |= (uint32_t)b8[wj * 4 + q] << (8 * q);
                wv[j] = v;
            }
        }
    }
#pragma unroll
    for (int w = 0; w < KW; ++w) kw[w] = __funnelshift_r(wv[w], wv[w + 1], sh);
}

template <int D, int NT = kHashThreads>
__global__ void __launch_bounds__(NT) k_hash_count(const InstDesc* __restrict__ insts, int l0, int l1in,
                                                              int mode) {
    extern __shared__ __align__(16) uint32_t hsm[];
    const InstDesc& I = insts[blockIdx.y];
    // lattice group [l0, l1): its bitmap words [w0, w1) go to shared memory
    const int L = I.L, l1 = l1in < 0 ? L : l1in, Lg = l1 - l0;
    const int w0 = I.boff[l0], w1 = l1 < L ? I.boff[l1] : I.nwords, nwords = w1 - w0;
    uint32_t* bits = hsm;
    int* sz = reinterpret_cast<int*>(hsm + nwords);     // [Lg][D]
    uint32_t* sM = reinterpret_cast<uint32_t*>(sz + Lg * D);
    uint32_t* smu = sM + Lg;
    uint32_t* soffk = smu + Lg;
    uint32_t* sbo = soffk + Lg;
    copy_words_to_smem(bits, I.nzbits + w0, nwords);
    for (int i = threadIdx.x; i < Lg * D; i += blockDim.x) sz[i] = I.z[l0 * D + i];
    for (int i = threadIdx.x; i < Lg; i += blockDim.x) {
        sM[i] = (uint32_t)I.Ml[l0 + i];
        smu[i] = I.mu[l0 + i];
        soffk[i] = I.offk[l0 + i];
        sbo[i] = (uint32_t)(I.boff[l0 + i] - w0) * 32u;
    }
    __syncthreads();
    const int64_t n = I.n;
    const int need = I.need;
    const int32_t* __restrict__ cand = reinterpret_cast<const int32_t*>(I.cand);
    const int8_t* __restrict__ cand8 = reinterpret_cast<const int8_t*>(I.cand);
    const int ld = I.cand_ld;
    uint8_t* dcounts = I.dcounts;
    int32_t* dhashes = I.dhashes;
    const uint32_t* __restrict__ cand8w = reinterpret_cast<const uint32_t*>(I.cand);
    const int64_t nbytes = n * ld;
    constexpr int KW = (D + 3) / 4;
    const int64_t r_safe = n - (4 * KW + 3) / (ld > 0 ? ld : 1) - 1;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * kCPT;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x * kCPT; base < n; base += step) {
        int k[kCPT][D];
        int64_t idx[kCPT];
        int cnt[kCPT];
#pragma unroll
        for (int c = 0; c < kCPT; ++c) {
            idx[c] = base + threadIdx.x + (int64_t)c * blockDim.x;
            cnt[c] = (mode & 1) || idx[c] >= n ? 0 : I.cnt8[idx[c]];
        }
        if (!(mode & 1) && !dhashes && !dcounts) {
            // a later lattice group: a warp none of whose candidates can still reach the count
            // threshold with this and the following groups' lattices is decided (counts unchanged)
            bool alive = false;
#pragma unroll
            for (int c = 0; c < kCPT; ++c) alive |= idx[c] < n && cnt[c] + (L - l0) >= need;
            if (!__any_sync(0xffffffffu, alive)) continue;
        }
#pragma unroll
        for (int c = 0; c < kCPT; ++c) {
            const int64_t r = idx[c] < n ? idx[c] : 0;
            const int32_t* row = cand + r * D;
            if (I.cand_i8) {  // int8 rows of stride ld bytes, read as words, sign-extended per byte
                uint32_t kw[KW];
                load_row8<KW>(cand8w, reinterpret_cast<const uint8_t*>(cand8), r, ld, nbytes, r_safe, kw);
#pragma unroll
                for (int t = 0; t < D; ++t) k[c][t] = (int)(int32_t)(kw[t >> 2] << (24 - 8 * (t & 3))) >> 24;
            } else if constexpr (D % 4 == 0) {
#pragma unroll
                for (int t = 0; t < D; t += 4) {
                    int4 v = __ldg(reinterpret_cast<const int4*>(row + t));
                    k[c][t] = v.x; k[c][t + 1] = v.y; k[c][t + 2] = v.z; k[c][t + 3] = v.w;
                }
            } else if constexpr (D % 2 == 0) {
#pragma unroll
                for (int t = 0; t < D; t += 2) {
                    int2 v = __ldg(reinterpret_cast<const int2*>(row + t));
                    k[c][t] = v.x; k[c][t + 1] = v.y;
                }
            } else {
#pragma unroll
                for (int t = 0; t < D; ++t) k[c][t] = __ldg(row + t);
            }
        }
        for (int l = 0; l < Lg; ++l) {
            int zl[D];
#pragma unroll
            for (int t = 0; t < D; ++t) zl[t] = sz[l * D + t];
            const uint32_t M = sM[l], mu = smu[l], off = soffk[l], bo = sbo[l];
#pragma unroll
            for (int c = 0; c < kCPT; ++c) {
                uint32_t xp = off;  // unsigned: the offset sum wraps modulo 2^32 by definition
#pragma unroll
                for (int t = 0; t < D; ++t) xp += (uint32_t)(k[c][t] * zl[t]);
                const uint32_t q = __umulhi(xp, mu);
                uint32_t r = xp - q * M;
                r = min(r, r - M);
                uint32_t bit = bo + r;
                cnt[c] += (bits[bit >> 5] >> (bit & 31)) & 1u;
                if (dhashes && idx[c] < n) dhashes[idx[c] * L + l0 + l] = (int32_t)r;
            }
            // count rule decided for the whole warp: every candidate has reached `need` or cannot
            // reach it (tested every fourth lattice once fewer than `need` remain: before that
            // nobody can have missed more than L - need)
            const int rem = L - 1 - (l0 + l);
            if (!dhashes && !dcounts && rem < need && (rem & 3) == 0) {
                bool alive = false;
#pragma unroll
                for (int c = 0; c < kCPT; ++c) alive |= cnt[c] < need && cnt[c] + rem >= need;
                if (!__any_sync(0xffffffffu, alive)) break;
            }
        }
#pragma unroll
        for (int c = 0; c < kCPT; ++c) {
            if (idx[c] < n) {
                if (mode & 2) {
                    if (cnt[c] >= need) mark_detected(I, idx[c]);
                    if (dcounts) dcounts[idx[c]] = (uint8_t)cnt[c];
                } else {
                    I.cnt8[idx[c]] = (uint8_t)cnt[c];
                }
            }
        }
    }
}

// Packed variant: |k_t| <= 127 and M_l < 65536, so k is stored as int8x4 words and z_l (in its
// symmetric residue range) as int16x2 words; each dp2a instruction adds two products k_t z_t
// exactly into the int32 sum.
// Per lattice a 16-byte aligned record in shared memory holds {M, mu, off, bit offset} and the
// packed z words (broadcast loads shared by all threads).  DIAG additionally writes the
// per-candidate hashes and counts.
#ifndef SFFT_HASH_CPT
#define SFFT_HASH_CPT 4
#endif
constexpr int kCPT2 = SFFT_HASH_CPT;  // candidates per thread of the packed kernel
#ifndef SFFT_HASH_CHECK_EVERY
#define SFFT_HASH_CHECK_EVERY 1
#endif
constexpr int kHashCheckEvery = SFFT_HASH_CHECK_EVERY;  // lattices between the warp's count-rule tests

template <int D> struct Pack {
    static constexpr int KW = (D + 3) / 4;             // int8x4 words of k
    static constexpr int ZW = (D + 1) / 2;             // int16x2 words of z
    static constexpr int REC = 4 + ((ZW + 3) / 4) * 4; // words per lattice record (multiple of 4)
};

// Shared-memory prologue of the packed kernels for the lattice group [l0, l1): the group's bitmap
// words and one record per lattice.  Record words: {M, mu, off, bit offset}, then the packed z
// words, z_t in the symmetric range |z_t| <= (M - 1) / 2 (k.z = k.(z - M) mod M: signed int16 for
// every prime M < 65536), one record word per thread.
template <int D>
__device__ __forceinline__ void packed_prologue(const InstDesc& I, int l0, int l1, uint32_t* rec, uint32_t* bits) {
    using PK = Pack<D>;
    const int L = I.L, Lg = l1 - l0;
    const int w0 = I.boff[l0], w1 = l1 < L ? I.boff[l1] : I.nwords;
    copy_words_to_smem(bits, I.nzbits + w0, w1 - w0);
    for (int j = threadIdx.x; j < Lg * PK::REC; j += blockDim.x) {
        const int g = j / PK::REC, w = j - g * PK::REC, l = l0 + g;
        const int Ml = I.Ml[l];
        uint32_t v;
        if (w == 0) {
            v = (uint32_t)Ml;
        } else if (w == 1) {
            v = I.mu[l];
        } else if (w == 2) {
            v = I.offk[l];
        } else if (w == 3) {
            v = (uint32_t)(I.boff[l] - w0) * 32u;
        } else {
            const int t = 2 * (w - 4), Mh = Ml / 2;
            auto zsym = [&](int tt) -> uint32_t {
                const int zv = I.z[l * D + tt];
                return (uint32_t)(zv > Mh ? zv - Ml : zv) & 0xffffu;
            };
            v = (t < D ? zsym(t) : 0u) | ((t + 1 < D ? zsym(t + 1) : 0u) << 16);
        }
        rec[j] = v;
    }
}

// One lattice's contribution to a candidate's count: bit (off + k.z mod M) of the lattice's bitmap.
// The offset seeds the dot product (32-bit wrap-around equals the unsigned sum); bytes of k at
// positions >= d meet zero z halves.
template <int D>
__device__ __forceinline__ uint32_t packed_hash(const uint32_t* kw, const uint32_t* zw, uint32_t M, uint32_t mu,
                                                uint32_t off) {
    using PK = Pack<D>;
    int x = (int)off;
#pragma unroll
    for (int w = 0; w < PK::ZW; ++w) {
        if (w & 1) x = __dp2a_hi((int)zw[w], (int)kw[w >> 1], x);
        else x = __dp2a_lo((int)zw[w], (int)kw[w >> 1], x);
    }
    const uint32_t xp = (uint32_t)x;
    const uint32_t q = __umulhi(xp, mu);
    uint32_t rr = xp - q * M;
    return min(rr, rr - M);  // one conditional subtraction: rr - M wraps above rr when rr < M
}

template <int D, bool DIAG, int NT = kHashThreads>
__global__ void __launch_bounds__(NT, NT == kHashThreads ? 4 : 2) k_hash_count_packed(const InstDesc* __restrict__ insts,
                                                                                      int l0, int l1in, int mode) {
    extern __shared__ __align__(16) uint32_t hsm[];
    using PK = Pack<D>;
    const InstDesc& I = insts[blockIdx.y];
    // lattice group [l0, l1): its bitmap words go to shared memory
    const int L = I.L, l1 = l1in < 0 ? L : l1in, Lg = l1 - l0;
    uint32_t* rec = hsm;                       // [Lg][REC]
    uint32_t* bits = hsm + Lg * PK::REC;       // [nwords]
    packed_prologue<D>(I, l0, l1, rec, bits);
    __syncthreads();
    const int64_t n = I.n;
    const int need = I.need;
    const int32_t* __restrict__ cand = reinterpret_cast<const int32_t*>(I.cand);
    const uint32_t* __restrict__ cand8w = reinterpret_cast<const uint32_t*>(I.cand);  // int8 rows as words
    const int ld = I.cand_ld, ldw = ld >> 2;
    const bool i8 = I.cand_i8 != 0, ld4 = (ld & 3) == 0;
    const int64_t nbytes = n * ld;  // int8 rows: bytes of the candidate array
    // rows below r_safe have their KW + 1 aligned words inside the array (last byte read
    // r ld + 4 KW + 3 < n ld); the last few rows are read with bounds checks
    const int64_t r_safe = n - (4 * PK::KW + 3) / (ld > 0 ? ld : 1) - 1;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * kCPT2;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x * kCPT2; base < n; base += step) {
        uint32_t kw[kCPT2][PK::KW];
        int64_t idx[kCPT2];
        int cnt[kCPT2];
#pragma unroll
        for (int c = 0; c < kCPT2; ++c) {
            idx[c] = base + threadIdx.x + (int64_t)c * blockDim.x;
            cnt[c] = (mode & 1) || idx[c] >= n ? 0 : I.cnt8[idx[c]];
        }
        if constexpr (!DIAG) {
            if (!(mode & 1)) {
                // a later lattice group: a warp none of whose candidates can still reach the count
                // threshold with this and the following groups' lattices is decided (counts unchanged)
                bool alive = false;
#pragma unroll
                for (int c = 0; c < kCPT2; ++c) alive |= idx[c] < n && cnt[c] + (L - l0) >= need;
                if (!__any_sync(0xffffffffu, alive)) continue;
            }
        }
#pragma unroll
        for (int c = 0; c < kCPT2; ++c) {
            const int64_t r = idx[c] < n ? idx[c] : 0;
            if (i8) {  // the int8 row already holds the packed words (bytes past d meet zero z entries)
                if (ld4) {
#pragma unroll
                    for (int w = 0; w < PK::KW; ++w) kw[c][w] = __ldg(cand8w + r * ldw + w);
                } else {  // rows at any byte offset: the aligned words around the row, funnel-shifted
                    const int64_t b0 = r * ld, w0 = b0 >> 2;
                    const uint32_t sh = (uint32_t)(b0 & 3) * 8u;
                    uint32_t wv[PK::KW + 1];
                    if (r < r_safe) {
#pragma unroll
                        for (int j = 0; j <= PK::KW; ++j) wv[j] = __ldg(cand8w + w0 + j);
                    } else {
#pragma unroll
                        for (int j = 0; j <= PK::KW; ++j) {
                            const int64_t wj = w0 + j;
                            if ((wj + 1) * 4 <= nbytes) {
                                wv[j] = __ldg(cand8w + wj);
                            } else {  // the array's last bytes (no read past its end)
                                const uint8_t* b8 = reinterpret_cast<const uint8_t*>(I.cand);
                                uint32_t v = 0;
                                for (int q = 0; q < 4; ++q)
                                    if (wj * 4 + q < nbytes) v |= (uint32_t)b8[wj * 4 + q] << (8 * q);
                                wv[j] = v;
                            }
                        }
                    }
#pragma unroll
                    for (int w = 0; w < PK::KW; ++w) kw[c][w] = __funnelshift_r(wv[w], wv[w + 1], sh);
                }
                continue;
            }
            const int32_t* row = cand + r * D;
            int k[PK::KW * 4];
#pragma unroll
            for (int t = 0; t < PK::KW * 4; ++t) k[t] = 0;
            if constexpr (D % 4 == 0) {
#pragma unroll
                for (int t = 0; t < D; t += 4) {
                    int4 v = __ldg(reinterpret_cast<const int4*>(row + t));
                    k[t] = v.x; k[t + 1] = v.y; k[t + 2] = v.z; k[t + 3] = v.w;
                }
            } else if constexpr (D % 2 == 0) {
#pragma unroll
                for (int t = 0; t < D; t += 2) {
                    int2 v = __ldg(reinterpret_cast<const int2*>(row + t));
                    k[t] = v.x; k[t + 1] = v.y;
                }
            } else {
#pragma unroll
                for (int t = 0; t < D; ++t) k[t] = __ldg(row + t);
            }
#pragma unroll
            for (int w = 0; w < PK::KW; ++w)
                kw[c][w] = (uint32_t)(k[4 * w] & 0xff) | ((uint32_t)(k[4 * w + 1] & 0xff) << 8) |
                           ((uint32_t)(k[4 * w + 2] & 0xff) << 16) | ((uint32_t)(k[4 * w + 3] & 0xff) << 24);
        }
        auto lattice = [&](int l) {
            const uint4* r4 = reinterpret_cast<const uint4*>(rec + l * PK::REC);
            const uint4 cst = r4[0];
            uint32_t zw[PK::REC - 4];
#pragma unroll
            for (int w = 0; w < (PK::REC - 4) / 4; ++w) {
                uint4 v = r4[1 + w];
                zw[4 * w] = v.x; zw[4 * w + 1] = v.y; zw[4 * w + 2] = v.z; zw[4 * w + 3] = v.w;
            }
            const uint32_t M = cst.x, mu = cst.y, off = cst.z;
            const uint32_t* lbits = bits + (cst.w >> 5);  // the lattice's bitmap (segments start on words)
#pragma unroll
            for (int c = 0; c < kCPT2; ++c) {
                const uint32_t rr = packed_hash<D>(kw[c], zw, M, mu, off);
                cnt[c] += __funnelshift_r(lbits[rr >> 5], 0u, rr) & 1u;  // bit rr & 31 of word rr >> 5
                if constexpr (DIAG) {
                    if (idx[c] < n && I.dhashes) I.dhashes[idx[c] * L + l0 + l] = (int32_t)rr;
                }
            }
        };
        // count rule (Algorithm 1): once every candidate of the warp is decided -- it has reached
        // `need`, or cannot reach it with the lattices left -- the rest cannot change a decision
        // (exact counts are only reported by the DIAG variant).  While rem >= need lattices
        // remain, no candidate can have missed more than L - need of them, so the warp test starts
        // below that and then runs every kHashCheckEvery lattices (every lattice measured 1.7 %
        // faster than every second, every third 0.2 % slower).
        for (int l = 0; l < Lg; ++l) {
            lattice(l);
            if constexpr (!DIAG) {
                const int rem = L - 1 - (l0 + l);
                if (rem < need && rem % kHashCheckEvery == 0) {
                    bool alive = false;
#pragma unroll
                    for (int c = 0; c < kCPT2; ++c) alive |= cnt[c] < need && cnt[c] + rem >= need;
                    if (!__any_sync(0xffffffffu, alive)) break;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < kCPT2; ++c) {
            if (idx[c] < n) {
                if (mode & 2) {
                    if (cnt[c] >= need) mark_detected(I, idx[c]);
                    if constexpr (DIAG) {
                        if (I.dcounts) I.dcounts[idx[c]] = (uint8_t)cnt[c];
                    }
                } else {
                    I.cnt8[idx[c]] = (uint8_t)cnt[c];
                }
            }
        }
    }
}

// ================================================================== compaction (ascending Itilde)
// Ascending Itilde from the detection bits.  Each instance's ceil(n/32) bit words are split into
// kCompactChunks contiguous chunks, one CTA each.  A CTA starts at the sum of the detection counts
// of the chunks before its own (kept by the hash kernels in cnt[8 + c]), scans its own chunk and
// writes its indices; the last chunk's CTA records |Itilde|.  One launch, no inter-CTA waits.
constexpr int kCompactThreads = 256;

__global__ void __launch_bounds__(kCompactThreads) k_compact(InstDesc* __restrict__ insts) {
    __shared__ int64_t wsum[32];
    InstDesc& I = insts[blockIdx.y];
    const int64_t W = (I.n + 31) >> 5;
    const int64_t chunk = (W + gridDim.x - 1) / gridDim.x;
    const int64_t c0 = min(W, (int64_t)blockIdx.x * chunk), c1 = min(W, c0 + chunk);
    const uint32_t* bits = I.detbits;
    // set bits before this chunk: the hash kernels' per-chunk detection counts
    int64_t base = 0;
    for (int b = 0; b < (int)blockIdx.x; ++b) base += I.cnt[8 + b];
    // this chunk: contiguous words per thread, block exclusive scan of their counts
    const int64_t per = (c1 - c0 + blockDim.x - 1) / blockDim.x;
    const int64_t w0 = min(c1, c0 + threadIdx.x * per), w1 = min(c1, w0 + per);
    int64_t c = 0;
    for (int64_t w = w0; w < w1; ++w) c += __popc(bits[w]);
    int64_t v = c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int64_t t = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    int64_t pos = base + v - c + (warp > 0 ? wsum[warp - 1] : 0);
    const int64_t total = base + wsum[(blockDim.x >> 5) - 1];
    for (int64_t w = w0; w < w1; ++w) {
        uint32_t b = bits[w];
        while (b) {
            int t = __ffs(b) - 1;
            b &= b - 1;
            if (pos < I.cap) I.det[pos] = w * 32 + t;
            ++pos;
        }
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        I.cnt[0] = total;
        if (total > I.cap) atomicOr((unsigned long long*)&I.cnt[3], (unsigned long long)ERR_DET_CAP);
    }
}

// ================================================================== hashes of the detected set
// One warp per detected candidate; lane l (and l+32) owns lattice l.
// h = k.z_l mod M_l of detected candidate q.  The plan bounds |k.z| so that the offset sum fits
// 32 bits: the hash kernel's exact Barrett reduction (q = umulhi(x, floor(2^32/M)) is at most one
// short, so one conditional subtraction).
__device__ __forceinline__ int32_t det_hash(const InstDesc& I, int64_t q, int l) {
    const int d = I.d;
    const int64_t row = I.det[q] * I.cand_ld;
    const int32_t* k32 = reinterpret_cast<const int32_t*>(I.cand) + row;
    const int8_t* k8 = reinterpret_cast<const int8_t*>(I.cand) + row;
    const int32_t* zl = I.z + l * d;
    uint32_t xp = I.offk[l];  // unsigned wrap-around: the sum mod 2^32, in [0, 2^32)
    for (int t = 0; t < d; ++t) xp += (uint32_t)((I.cand_i8 ? (int)__ldg(k8 + t) : __ldg(k32 + t)) * zl[t]);
    const uint32_t M = (uint32_t)I.Ml[l];
    uint32_t r = xp - __umulhi(xp, I.mu[l]) * M;
    return (int32_t)min(r, r - M);
}

__global__ void k_det_hashes(const InstDesc* __restrict__ insts) {
    const InstDesc& I = insts[blockIdx.y];
    const int64_t nd = min(I.cnt[0], I.cap);
    const int warps = blockDim.x >> 5;
    for (int64_t q = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); q < nd; q += (int64_t)gridDim.x * warps) {
        const int lane = threadIdx.x & 31, L = I.L;
        for (int l = lane; l < L; l += 32) I.H[q * L + l] = det_hash(I, q, l);
    }
}

__global__ void k_collisions(const InstDesc* __restrict__ insts) {
    const InstDesc& I = insts[blockIdx.y];
    const int64_t nd = min(I.cnt[0], I.cap);
    const int L = I.L;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nd * L; e += (int64_t)gridDim.x * blockDim.x) {
        int l = (int)(e % L);
        atomicAdd(&I.coll[I.soff[l] + I.H[e]], 1);
    }
}

// Order-preserving integer key of a double (-0 mapped to +0, NaN never occurs): the warp
// median ranks keys with integer compares instead of the low-rate FP64 pipe.
__device__ __forceinline__ long long ord_key(double v) {
    long long b = __double_as_longlong(v);
    if (b == (long long)0x8000000000000000ull) b = 0;
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}

// Median of L <= 64 packed keys spread over a warp (lane l holds the keys of lattices l and l+32)
// by a bitonic sort: element e = 2 lane + j (j = 0: lattice `lane`, j = 1: lattice `lane + 32`),
// missing lattices padded with +inf.  A packed key holds an order-preserving value key in its
// high 58 bits and the lattice in its low 6, so equal values order by lattice (lower first); the
// (L-1)/2-th smallest is the median of eq. (2.6) for odd L.  Values that differ only below the
// key's resolution (2^-46 relative for doubles, 2^-50 for double-float pairs) count as equal.
__device__ __forceinline__ long long warp_median_packed(long long ka, long long kb, int L, int lane) {
    long long k0 = lane < L ? ka : LLONG_MAX, k1 = lane + 32 < L ? kb : LLONG_MAX;
#pragma unroll
    for (int size = 2; size <= 64; size <<= 1) {
#pragma unroll
        for (int d = size >> 1; d > 0; d >>= 1) {
            if (d == 1) {  // both elements in this lane
                const bool up = ((2 * lane) & size) == 0;
                if (up == (k1 < k0)) {
                    const long long t = k0; k0 = k1; k1 = t;
                }
            } else {
                const int m = d >> 1;  // partner lane = lane ^ m, same j
                const long long p0 = __shfl_xor_sync(0xffffffffu, k0, m), p1 = __shfl_xor_sync(0xffffffffu, k1, m);
                const bool up = ((2 * lane) & size) == 0, low = ((2 * lane) & d) == 0;
                const bool want_min = up == low;
                if (want_min == (p0 < k0)) k0 = p0;
                if (want_min == (p1 < k1)) k1 = p1;
            }
        }
    }
    const int mid = (L - 1) >> 1;
    return __shfl_sync(0xffffffffu, (mid & 1) ? k1 : k0, mid >> 1);
}
__device__ __forceinline__ long long pack_key(long long value_key, int lattice) {
    return (value_key & ~63ll) | lattice;
}

// Order-preserving keys.  A normalised double-float pair (hi = fl(hi + lo)) orders like its value
// lexicographically in (hi, lo), because rounding to nearest is monotone; -0 counts as +0.
__device__ __forceinline__ int ord32(float f) {
    int b = __float_as_int(f);
    if (b == (int)0x80000000) b = 0;
    return b ^ ((b >> 31) & 0x7fffffff);
}
__device__ __forceinline__ long long df_key(float hi, float lo) {
    return (long long)(((unsigned long long)(long long)ord32(hi) << 32) | (unsigned)(ord32(lo) ^ (int)0x80000000));
}
template <class TS> __device__ __forceinline__ long long val_key(TS hi, float lo) {
    if constexpr (sizeof(TS) == 8) return ord_key((double)hi);
    else return df_key((float)hi, lo);
}
// value of lane (l & 31)'s a (l < 32) or b (l >= 32)
template <class T> __device__ __forceinline__ T pick(T a, T b, int l) {
    const T x = __shfl_sync(0xffffffffu, a, l & 31), y = __shfl_sync(0xffffffffu, b, l & 31);
    return l < 32 ? x : y;
}

__device__ __forceinline__ void zero_bucket(const InstDesc& I, int64_t b, int zc) {
    if (zc == 1) I.C[b] = c64{0.0, 0.0};
    else if (zc == 2) reinterpret_cast<c32*>(I.C)[b] = c32{0.f, 0.f};
}

// The same median for float values: a bitonic sort of 32-bit order keys (half the shuffles and
// compares of the packed 64-bit keys), then the lattice among the keys equal to the median value
// at rank mid - #(smaller keys) in lattice order, which is the element the packed (value,
// lattice) order puts at position mid.
__device__ __forceinline__ int warp_median32(int ka, int kb, int L, int lane) {
    const bool va = lane < L, vb = lane + 32 < L;
    int k0 = va ? ka : INT_MAX, k1 = vb ? kb : INT_MAX;
#pragma unroll
    for (int size = 2; size <= 64; size <<= 1) {
#pragma unroll
        for (int d = size >> 1; d > 0; d >>= 1) {
            if (d == 1) {
                const bool up = ((2 * lane) & size) == 0;
                if (up == (k1 < k0)) {
                    const int t = k0; k0 = k1; k1 = t;
                }
            } else {
                const int m = d >> 1;
                const int p0 = __shfl_xor_sync(0xffffffffu, k0, m), p1 = __shfl_xor_sync(0xffffffffu, k1, m);
                const bool up = ((2 * lane) & size) == 0, low = ((2 * lane) & d) == 0;
                const bool want_min = up == low;
                if (want_min == (p0 < k0)) k0 = p0;
                if (want_min == (p1 < k1)) k1 = p1;
            }
        }
    }
    const int mid = (L - 1) >> 1;
    const int vm = __shfl_sync(0xffffffffu, (mid & 1) ? k1 : k0, mid >> 1);
    const int less = __popc(__ballot_sync(0xffffffffu, va && ka < vm)) + __popc(__ballot_sync(0xffffffffu, vb && kb < vm));
    unsigned ea = __ballot_sync(0xffffffffu, va && ka == vm), eb = __ballot_sync(0xffffffffu, vb && kb == vm);
    int r = mid - less;  // rank among the ties, lattice order
    const int na = __popc(ea);
    if (r < na) {
        for (; r > 0; --r) ea &= ea - 1;
        return __ffs(ea) - 1;
    }
    for (r -= na; r > 0; --r) eb &= eb - 1;
    return 32 + __ffs(eb) - 1;
}

// Median combine (eq. 2.6) or the Remark 2.8 hybrid combine on the detected set: coef = combine(ghat).
// The ranking uses integer keys of the buckets (float, double-float pair or double); only the
// selected median is converted to double.
// HASH: the hashes of Itilde are formed here (and stored for the later stages) instead of by a
// separate k_det_hashes launch (every combine but the hybrid one, which needs the collision counts
// of all hashes first).
// zc: the refinement's bucket sums C are zeroed at every bucket of Itilde (1: FP64 buckets, 2: the
// FP32 buckets of the first half), the only entries its scatter and update touch, instead of
// clearing all sum M_l entries.
template <class TS, bool HASH>
__global__ void k_combine(const InstDesc* __restrict__ insts, int zc) {
    const InstDesc& I = insts[blockIdx.y];
    const int64_t nd = min(I.cnt[0], I.cap);
    const int warps = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, L = I.L;
    const cplx<TS>* g = reinterpret_cast<const cplx<TS>*>(I.ghat);
    const c32* glo = I.ghat_lo;  // low words of a double-float transform (or NULL)
    const bool hybrid = I.combine == SFFT_COMBINE_HYBRID;
    for (int64_t q = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); q < nd; q += (int64_t)gridDim.x * warps) {
        cplx<TS> ha = {0, 0}, hb = {0, 0};
        c32 la = {0.f, 0.f}, lb = {0.f, 0.f};
        int fa = 0, fb = 0;  // collision-free flags (hybrid)
        if (lane < L) {
            int32_t h;
            if constexpr (HASH) {
                h = det_hash(I, q, lane);
                I.H[q * L + lane] = h;
            } else {
                h = I.H[q * L + lane];
            }
            const int64_t b = I.soff[lane] + h;
            ha = g[b];
            if (glo) la = glo[b];
            if (hybrid) fa = I.coll[b] == 1;
            zero_bucket(I, b, zc);
        }
        if (lane + 32 < L) {
            int32_t h;
            if constexpr (HASH) {
                h = det_hash(I, q, lane + 32);
                I.H[q * L + lane + 32] = h;
            } else {
                h = I.H[q * L + lane + 32];
            }
            const int64_t b = I.soff[lane + 32] + h;
            hb = g[b];
            if (glo) lb = glo[b];
            if (hybrid) fb = I.coll[b] == 1;
            zero_bucket(I, b, zc);
        }
        int lre, lim;
        if (sizeof(TS) == 4 && !glo) {  // plain float buckets: 32-bit keys
            lre = warp_median32(ord32((float)ha.x), ord32((float)hb.x), L, lane);
            lim = warp_median32(ord32((float)ha.y), ord32((float)hb.y), L, lane);
        } else {
            lre = (int)(warp_median_packed(pack_key(val_key<TS>(ha.x, la.x), lane),
                                           pack_key(val_key<TS>(hb.x, lb.x), lane + 32), L, lane) & 63);
            lim = (int)(warp_median_packed(pack_key(val_key<TS>(ha.y, la.y), lane),
                                           pack_key(val_key<TS>(hb.y, lb.y), lane + 32), L, lane) & 63);
        }
        c64 out = {(double)pick(ha.x, hb.x, lre), (double)pick(ha.y, hb.y, lim)};
        if (glo) {
            out.x += (double)pick(la.x, lb.x, lre);
            out.y += (double)pick(la.y, lb.y, lim);
        }
        if (hybrid) {
            double sr = (fa ? (double)ha.x + (double)la.x : 0.0) + (fb ? (double)hb.x + (double)lb.x : 0.0);
            double si = (fa ? (double)ha.y + (double)la.y : 0.0) + (fb ? (double)hb.y + (double)lb.y : 0.0);
            int nf = fa + fb;
            for (int o = 16; o > 0; o >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                si += __shfl_xor_sync(0xffffffffu, si, o);
                nf += __shfl_xor_sync(0xffffffffu, nf, o);
            }
            if (nf > 0) out = c64{sr / nf, si / nf};
        }
        if (lane == 0) {
            I.coef[q] = out;
            I.sel[2 * q] = (uint8_t)lre;
            I.sel[2 * q + 1] = (uint8_t)lim;
        }
    }
}

// Refinement update: the residual f - sum_{k in Itilde} c_k e^{2 pi i k.x} has the lattice DFT
// r_hat_h = ghat_h - C_h (aliasing formula, eq. 2.3), C_h = sum of c_k over the detected k with
// h_kl = h.  c_k += median_l Re r_hat + i median_l Im r_hat at h_kl, in FP64; ghat is the forward
// transform (FP64, or a double-float pair hi + lo for FP32 plans with refinement).
// FP32 buckets (F32: FP32 transforms, C accumulated in float): r_hat in float, whose rounding is
// far below the transform's own error, and 32-bit median keys; the update itself stays FP64.
template <class TS, bool F32>
__global__ void k_refine_update(const InstDesc* __restrict__ insts) {
    const InstDesc& I = insts[blockIdx.y];
    const int64_t nd = min(I.cnt[0], I.cap);
    const int warps = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, L = I.L;
    const cplx<TS>* g = reinterpret_cast<const cplx<TS>*>(I.ghat);
    const c32* glo = I.ghat_lo;
    if constexpr (F32) {
        const c32* g32 = reinterpret_cast<const c32*>(I.ghat);
        const c32* C32 = reinterpret_cast<const c32*>(I.C);
        for (int64_t q = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); q < nd; q += (int64_t)gridDim.x * warps) {
            auto rhat = [&](int l) -> c32 {
                const int64_t b = I.soff[l] + I.H[q * L + l];
                const c32 v = g32[b], c = C32[b];
                return c32{v.x - c.x, v.y - c.y};
            };
            c32 va = {0.f, 0.f}, vb = {0.f, 0.f};
            if (lane < L) va = rhat(lane);
            if (lane + 32 < L) vb = rhat(lane + 32);
            const int lre = warp_median32(ord32(va.x), ord32(vb.x), L, lane);
            const int lim = warp_median32(ord32(va.y), ord32(vb.y), L, lane);
            const float dre = pick(va.x, vb.x, lre), dim = pick(va.y, vb.y, lim);
            if (lane == 0) {
                const c64 c = I.coef[q];
                I.coef[q] = c64{c.x + (double)dre, c.y + (double)dim};
                if (I.rsel) {
                    I.rsel[2 * q] = (uint8_t)lre;
                    I.rsel[2 * q + 1] = (uint8_t)lim;
                }
            }
        }
        return;
    }
    for (int64_t q = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); q < nd; q += (int64_t)gridDim.x * warps) {
        auto rhat = [&](int l) -> c64 {
            const int64_t b = I.soff[l] + I.H[q * L + l];
            const cplx<TS> v = g[b];
            c64 r = {(double)v.x, (double)v.y};
            if (glo) {
                const c32 w = glo[b];
                r.x += (double)w.x;
                r.y += (double)w.y;
            }
            const c64 c = I.C[b];
            return c64{r.x - c.x, r.y - c.y};
        };
        c64 va = {0, 0}, vb = {0, 0};
        if (lane < L) va = rhat(lane);
        if (lane + 32 < L) vb = rhat(lane + 32);
        const int lre = (int)(warp_median_packed(pack_key(ord_key(va.x), lane), pack_key(ord_key(vb.x), lane + 32), L,
                                                 lane) & 63);
        const int lim = (int)(warp_median_packed(pack_key(ord_key(va.y), lane), pack_key(ord_key(vb.y), lane + 32), L,
                                                 lane) & 63);
        const double dre = pick(va.x, vb.x, lre), dim = pick(va.y, vb.y, lim);
        if (lane == 0) {
            const c64 c = I.coef[q];
            I.coef[q] = c64{c.x + dre, c.y + dim};
            if (I.rsel) {
                I.rsel[2 * q] = (uint8_t)lre;
                I.rsel[2 * q + 1] = (uint8_t)lim;
            }
        }
    }
}

// Least-squares post-processing (Remark 2.8).  With A the sampling matrix of the detected set at
// all lattice nodes, the aliasing formula (eq. 2.3) gives A^H A = G = sum_l M_l P_l^T P_l (P_l maps
// k to its bucket h_kl) and A^H f = b, b_k = sum_l M_l ghat^(l)_{h_kl}.  G = D + E with the
// diagonal D_k = sum_l M_l and E_kk' = sum of M_l over the lattices where k and k' collide: with
// M ~ 10 s, E has a few entries per row.  Three grid-wide kernels build the bucket lists of the
// detected entries (the collision-count buffer holds the list heads), the right-hand side, and the
// list of colliding pairs; one CTA per instance then runs conjugate gradients on G c = b from the
// median estimates with G v = D v + E v over the pairs.  When the pairs exceed their capacity
// (many-way collisions) G v falls back to a scatter of v into the buckets and a weighted gather.
constexpr int kLsqThreads = 1024;
struct LsqPair {
    int32_t q, q2;
    double w;
};

// mode 0: heads of the touched buckets := -1, r := 0, pair count := 0
// mode 1: push every entry e = q L + l on its bucket's list; r_q += M_l ghat^(l)_{h_ql} (= b)
template <class TS>
__global__ void k_lsq_prep(InstDesc* __restrict__ insts, int mode) {
    InstDesc& I = insts[blockIdx.y];
    if (I.combine != SFFT_COMBINE_LSQ || I.lsq_work == nullptr) return;
    const int64_t nd = min(I.cnt[0], I.cap);
    const int L = I.L;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (mode == 0) {
        for (int64_t e = t0; e < nd * L; e += stride) I.coll[I.soff[e % L] + I.H[e]] = -1;
        for (int64_t q = t0; q < nd; q += stride) I.lsq_work[q] = c64{0, 0};
        if (t0 == 0) I.cnt[5] = 0;
        return;
    }
    const cplx<TS>* g = reinterpret_cast<const cplx<TS>*>(I.ghat);
    for (int64_t e = t0; e < nd * L; e += stride) {
        const int l = (int)(e % L);
        const int64_t b = I.soff[l] + I.H[e];
        I.lsq_next[e] = atomicExch(&I.coll[b], (int32_t)e);
        const cplx<TS> v = g[b];
        double vx = (double)v.x, vy = (double)v.y;
        if (I.ghat_lo) { vx += (double)I.ghat_lo[b].x; vy += (double)I.ghat_lo[b].y; }
        const double m = (double)I.Ml[l];
        atomicAdd(&I.lsq_work[e / L].x, m * vx);
        atomicAdd(&I.lsq_work[e / L].y, m * vy);
    }
}

// every ordered colliding pair (q, q') of a lattice, with weight M_l
__global__ void k_lsq_pairs(InstDesc* __restrict__ insts) {
    InstDesc& I = insts[blockIdx.y];
    if (I.combine != SFFT_COMBINE_LSQ || I.lsq_work == nullptr) return;
    const int64_t nd = min(I.cnt[0], I.cap);
    const int L = I.L;
    LsqPair* pairs = reinterpret_cast<LsqPair*>(I.lsq_pairs);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nd * L; e += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(e % L);
        const int64_t b = I.soff[l] + I.H[e];
        for (int32_t f = I.coll[b]; f >= 0; f = I.lsq_next[f]) {
            if (f == (int32_t)e) continue;
            const unsigned long long k = atomicAdd((unsigned long long*)&I.cnt[5], 1ull);
            if ((int64_t)k < I.lsq_pair_cap) pairs[k] = LsqPair{(int32_t)(e / L), (int32_t)(f / L), (double)I.Ml[l]};
        }
    }
}

// block sum of a double: warp sums, then warp 0 sums the partials and broadcasts (FP64 work is
// costly on this GPU, so no thread repeats the final sum)
__device__ double block_sum_f64(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double r = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if (threadIdx.x == 0) sh[32] = r;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

constexpr int kLsqSmemVec = 2048;  // detected sets up to this size keep the CG vectors in shared memory

__global__ void __launch_bounds__(kLsqThreads) k_lsq_cg(InstDesc* __restrict__ insts, int max_iter, double tol) {
    extern __shared__ __align__(16) unsigned char lsq_smem[];
    __shared__ double red[33];
    InstDesc& I = insts[blockIdx.x];
    if (I.combine != SFFT_COMBINE_LSQ || I.lsq_work == nullptr) return;
    const int64_t nd = min(I.cnt[0], I.cap);
    if (nd == 0) return;
    const int L = I.L;
    const int64_t ne = nd * L;
    const bool in_smem = nd <= kLsqSmemVec;
    c64* x = in_smem ? reinterpret_cast<c64*>(lsq_smem) : I.coef;
    c64* r = in_smem ? x + kLsqSmemVec : I.lsq_work;  // holds b on entry
    c64* p = in_smem ? r + kLsqSmemVec : I.lsq_work + I.cap;
    c64* Ap = in_smem ? p + kLsqSmemVec : p + I.cap;
    if (in_smem) {
        for (int64_t q = threadIdx.x; q < nd; q += blockDim.x) {
            x[q] = I.coef[q];
            r[q] = I.lsq_work[q];
        }
        __syncthreads();
    }
    const int64_t npair = I.cnt[5];
    const bool sparse = npair <= I.lsq_pair_cap;
    const LsqPair* pairs = reinterpret_cast<const LsqPair*>(I.lsq_pairs);
    double dg = 0;  // D_k = sum_l M_l
    for (int l = 0; l < L; ++l) dg += (double)I.Ml[l];
    auto matvec = [&](const c64* v, c64* out) {
        if (sparse) {
            for (int64_t q = threadIdx.x; q < nd; q += blockDim.x) out[q] = c64{dg * v[q].x, dg * v[q].y};
            __syncthreads();
            for (int64_t j = threadIdx.x; j < npair; j += blockDim.x) {
                const LsqPair pr = pairs[j];
                atomicAdd(&out[pr.q].x, pr.w * v[pr.q2].x);
                atomicAdd(&out[pr.q].y, pr.w * v[pr.q2].y);
            }
            __syncthreads();
            return;
        }
        for (int64_t e = threadIdx.x; e < ne; e += blockDim.x) I.C[I.soff[e % L] + I.H[e]] = c64{0, 0};
        __syncthreads();
        for (int64_t e = threadIdx.x; e < ne; e += blockDim.x) {
            c64* c = &I.C[I.soff[e % L] + I.H[e]];
            atomicAdd(&c->x, v[e / L].x);
            atomicAdd(&c->y, v[e / L].y);
        }
        __syncthreads();
        for (int64_t q = threadIdx.x; q < nd; q += blockDim.x) {
            double sx = 0, sy = 0;
            for (int l = 0; l < L; ++l) {
                const c64 c = I.C[I.soff[l] + I.H[q * L + l]];
                sx += (double)I.Ml[l] * c.x;
                sy += (double)I.Ml[l] * c.y;
            }
            out[q] = c64{sx, sy};
        }
        __syncthreads();
    };
    // r = b - G x,  p = r
    matvec(x, Ap);
    double rr = 0, bb = 0;
    for (int64_t q = threadIdx.x; q < nd; q += blockDim.x) {
        const c64 bq = r[q];
        const c64 rq = {bq.x - Ap[q].x, bq.y - Ap[q].y};
        r[q] = rq;
        p[q] = rq;
        rr += rq.x * rq.x + rq.y * rq.y;
        bb += bq.x * bq.x + bq.y * bq.y;
    }
    rr = block_sum_f64(rr, red);
    bb = block_sum_f64(bb, red);
    int it = 0;
    for (; it < max_iter && rr > tol * tol * bb; ++it) {
        matvec(p, Ap);
        double pAp = 0;
        for (int64_t q = threadIdx.x; q < nd; q += blockDim.x) pAp += p[q].x * Ap[q].x + p[q].y * Ap[q].y;
        pAp = block_sum_f64(pAp, red);
        if (!(pAp > 0)) break;
        const double alpha = rr / pAp;
        double rn = 0;
        for (int64_t q = threadIdx.x; q < nd; q += blockDim.x) {
            x[q] = c64{x[q].x + alpha * p[q].x, x[q].y + alpha * p[q].y};
            const c64 rq = {r[q].x - alpha * Ap[q].x, r[q].y - alpha * Ap[q].y};
            r[q] = rq;
            rn += rq.x * rq.x + rq.y * rq.y;
        }
        rn = block_sum_f64(rn, red);
        const double beta = rn / rr;
        for (int64_t q = threadIdx.x; q < nd; q += blockDim.x) p[q] = c64{r[q].x + beta * p[q].x, r[q].y + beta * p[q].y};
        __syncthreads();
        rr = rn;
    }
    if (in_smem)
        for (int64_t q = threadIdx.x; q < nd; q += blockDim.x) I.coef[q] = x[q];
    if (threadIdx.x == 0) I.cnt[4] = it;  // iterations taken (diagnostics)
}

// scatter the detected coefficients into their buckets: C_l[h_kl] += c_k (FP64, or float buckets
// in the first half of the buffer for FP32 transforms)
template <bool F32>
__global__ void k_scatter_coef(const InstDesc* __restrict__ insts) {
    const InstDesc& I = insts[blockIdx.y];
    const int64_t nd = min(I.cnt[0], I.cap);
    const int L = I.L;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nd * L; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t q = e / L;
        int l = (int)(e - q * L);
        c64 c = I.coef[q];
        const int64_t b = I.soff[l] + I.H[e];
        if constexpr (F32) {
            c32* C32 = reinterpret_cast<c32*>(I.C);
            atomicAdd(&C32[b].x, (float)c.x);
            atomicAdd(&C32[b].y, (float)c.y);
        } else {
            atomicAdd(&I.C[b].x, c.x);
            atomicAdd(&I.C[b].y, c.y);
        }
    }
}

// ================================================================== Algorithm 4 selection
constexpr int kSelThreads = 1024;


__device__ int64_t block_sum64(int64_t v, int64_t* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    int64_t r = 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
        sh[32] = r;
    }
    __syncthreads();
    r = sh[32];
    __syncthreads();
    return r;
}

// exclusive block scan of int flags processed in chunks of blockDim (returns prefix, sets total)
__device__ int block_excl_scan(int f, int* sh, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int v = f;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    __syncthreads();
    if (lane == 31) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        sh[lane] = t;
    }
    __syncthreads();
    int pre = v - f + (warp > 0 ? sh[warp - 1] : 0);
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return pre;
}

// |c| of the first kSelCache coefficients is computed once (FP64 hypot is costly here) and kept
// in shared memory; beyond that it is recomputed in each pass.
constexpr int kSelCache = 4096;

__global__ void __launch_bounds__(kSelThreads) k_select(InstDesc* __restrict__ insts) {
    __shared__ int64_t sh64[33];
    __shared__ int shi[33];
    __shared__ unsigned int hist[256];
    __shared__ double smax[32];
    __shared__ double mag[kSelCache];
    InstDesc& I = insts[blockIdx.x];
    const int64_t nd = min(I.cnt[0], I.cap);
    auto absc = [&](int64_t q) -> double {
        if (q < kSelCache) return mag[q];
        const c64 c = I.coef[q];
        return hypot(c.x, c.y);
    };
    for (int64_t q = threadIdx.x; q < min(nd, (int64_t)kSelCache); q += blockDim.x) {
        const c64 c = I.coef[q];
        mag[q] = hypot(c.x, c.y);
    }
    __syncthreads();
    // theta = max(theta_abs, theta_rel * max |c|)
    double mx = 0;
    for (int64_t q = threadIdx.x; q < nd; q += blockDim.x) mx = fmax(mx, absc(q));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, smax[i]);
        smax[0] = m;
    }
    __syncthreads();
    const double theta = fmax(I.theta_abs, I.theta_rel * smax[0]);
    __syncthreads();
    // kept set and its size
    int64_t kept = 0;
    for (int64_t q = threadIdx.x; q < nd; q += blockDim.x) kept += absc(q) >= theta;
    kept = block_sum64(kept, sh64);
    int64_t want = (I.s_tilde > 0 && I.s_tilde < kept) ? I.s_tilde : kept;
    // radix select of the want-th largest key among kept items (only if truncating)
    uint64_t prefix = 0, mask = 0;
    int64_t need = want;
    const bool trunc = want < kept;
    if (trunc) {
        for (int p = 7; p >= 0; --p) {
            for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
            __syncthreads();
            for (int64_t q = threadIdx.x; q < nd; q += blockDim.x) {
                const double a = absc(q);
                const uint64_t key = rank_key(a, I.rank_bits);
                if (a >= theta && (key & mask) == prefix) atomicAdd(&hist[(key >> (8 * p)) & 255u], 1u);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int64_t acc = 0;
                int b = 255;
                for (; b > 0; --b) {
                    if (acc + hist[b] >= need) break;
                    acc += hist[b];
                }
                sh64[0] = acc;
                shi[0] = b;
            }
            __syncthreads();
            need -= sh64[0];
            prefix |= (uint64_t)shi[0] << (8 * p);
            mask |= (uint64_t)255 << (8 * p);
            __syncthreads();
        }
    }
    // prefix = key of the want-th largest; 'need' = how many items equal to it are taken
    // (lowest indices first, i.e. first in detected order)
    int64_t eq_taken = 0, outn = 0;
    for (int64_t q0 = 0; q0 < nd; q0 += blockDim.x) {
        int64_t q = q0 + threadIdx.x;
        int sel = 0, eq = 0;
        c64 c = {0, 0};
        uint64_t key = 0;
        if (q < nd) {
            c = I.coef[q];
            const double a = absc(q);
            key = rank_key(a, I.rank_bits);
            if (a >= theta) {
                if (!trunc || key > prefix) sel = 1;
                else if (key == prefix) eq = 1;
            }
        }
        int tot_eq;
        int pre_eq = block_excl_scan(eq, shi, &tot_eq);
        if (eq && eq_taken + pre_eq < need) sel = 1;
        eq_taken += tot_eq;
        int tot_sel;
        int pre_sel = block_excl_scan(sel, shi, &tot_sel);
        if (sel) {
            int64_t pos = outn + pre_sel;
            if (pos < I.out_cap) {
                I.supp_out[pos] = I.det[q];
                I.coef_out[pos] = c;
                if (I.key_out) I.key_out[pos] = key;
            }
            if (pos < I.cap) I.outpos[pos] = (int32_t)q;
        }
        outn += tot_sel;
    }
    if (threadIdx.x == 0) {
        I.cnt[1] = outn;
        if (outn > I.out_cap) atomicOr((unsigned long long*)&I.cnt[3], (unsigned long long)ERR_OUT_CAP);
    }
}

// ================================================================== samplers and adjoint scatter
// scatter coefficients of a sparse polynomial into the lattice buckets (eq. 2.3)
__global__ void k_scatter_terms(const InstDesc* __restrict__ insts) {
    const InstDesc& I = insts[blockIdx.y];
    const int L = I.L, d = I.d;
    const int32_t* __restrict__ kvec = I.samp_kvec;
    const c64* __restrict__ coef = I.samp_coef;
    const int64_t nterms = I.samp_nterms;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nterms * L; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t q = e / L;
        int l = (int)(e - q * L);
        int64_t x = 0;
        for (int t = 0; t < d; ++t) x += (int64_t)kvec[q * d + t] * I.z[l * d + t];
        int64_t M = I.Ml[l];
        int64_t r = x % M;
        if (r < 0) r += M;
        if (I.prec) {  // FP32 plans: FP32 buckets (the samples are FP32)
            c32* dst = reinterpret_cast<c32*>(I.C) + I.soff[l] + r;
            atomicAdd(&dst->x, (float)coef[q].x);
            atomicAdd(&dst->y, (float)coef[q].y);
        } else {
            c64* dst = I.C + I.soff[l] + r;
            atomicAdd(&dst->x, coef[q].x);
            atomicAdd(&dst->y, coef[q].y);
        }
    }
}

// ---- adjoint (vector-Jacobian product) with the support and every median's selected lattices held
// fixed.  The median coefficient is p_q = Re ghat^(lre)_h + i Im ghat^(lim)_h; with one refinement
// step c_q = p_q + Re rhat^(mre)_h + i Im rhat^(mim)_h, rhat = ghat - C, C_l[h] = sum of p over the
// detected frequencies in bucket h.  Both are linear in ghat, so the cotangent of ghat is G1 + G2:
// G1 puts the output cotangents W into the refinement's selected buckets, the median coefficients
// receive V = W - sum_l G1_l[h_ql] (their path through C), and G2 puts V into the median's buckets.
// Without refinement G1 = 0 and V = W.  The sample cotangent is the adjoint of the 1/M-normalised
// DFT applied to G (an inverse transform).

// W: dense cotangents of the detected set (adj_w cleared before; 0 for frequencies not selected)
__global__ void k_adj_dense(const InstDesc* __restrict__ insts, const c64* __restrict__ dcoef) {
    const InstDesc& I = insts[blockIdx.y];
    const int64_t nout = min(I.cnt[1], min(I.out_cap, I.cap));
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nout; p += (int64_t)gridDim.x * blockDim.x)
        I.adj_w[I.outpos[p]] = dcoef[p];
}

// G1: W into the buckets the refinement's median selected (C holds the cotangent of ghat)
__global__ void k_adj_refine_scatter(const InstDesc* __restrict__ insts) {
    const InstDesc& I = insts[blockIdx.y];
    const int64_t nd = min(I.cnt[0], I.cap);
    const int L = I.L;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nd; q += (int64_t)gridDim.x * blockDim.x) {
        const c64 w = I.adj_w[q];
        const int mre = I.rsel[2 * q], mim = I.rsel[2 * q + 1];
        if (w.x != 0.0) atomicAdd(&I.C[I.soff[mre] + I.H[q * L + mre]].x, w.x);
        if (w.y != 0.0) atomicAdd(&I.C[I.soff[mim] + I.H[q * L + mim]].y, w.y);
    }
}

// V = W - sum_l G1_l[h_ql], in place (G1 is only read here)
__global__ void k_adj_refine_gather(const InstDesc* __restrict__ insts) {
    const InstDesc& I = insts[blockIdx.y];
    const int64_t nd = min(I.cnt[0], I.cap);
    const int L = I.L;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nd; q += (int64_t)gridDim.x * blockDim.x) {
        double sx = 0.0, sy = 0.0;
        for (int l = 0; l < L; ++l) {
            const c64 g = I.C[I.soff[l] + I.H[q * L + l]];
            sx += g.x;
            sy += g.y;
        }
        const c64 w = I.adj_w[q];
        I.adj_w[q] = c64{w.x - sx, w.y - sy};
    }
}

// G2: V into the buckets the combine's median selected (added to G1)
__global__ void k_adj_median_scatter(const InstDesc* __restrict__ insts) {
    const InstDesc& I = insts[blockIdx.y];
    const int64_t nd = min(I.cnt[0], I.cap);
    const int L = I.L;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nd; q += (int64_t)gridDim.x * blockDim.x) {
        const c64 v = I.adj_w[q];
        const int lre = I.sel[2 * q], lim = I.sel[2 * q + 1];
        if (v.x != 0.0) atomicAdd(&I.C[I.soff[lre] + I.H[q * L + lre]].x, v.x);
        if (v.y != 0.0) atomicAdd(&I.C[I.soff[lim] + I.H[q * L + lim]].y, v.y);
    }
}

// lattice nodes: numer = j z mod M (exact), x = numer / M
__global__ void k_points(const InstDesc* __restrict__ insts, int32_t* numer, double* xout) {
    const InstDesc& I = insts[0];
    const int L = I.L, d = I.d;
    const int64_t tot = I.soff[L] * d;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t node = e / d;
        int t = (int)(e - node * d);
        int l = 0;
        while (I.soff[l + 1] <= node) ++l;
        int64_t j = node - I.soff[l];
        int64_t M = I.Ml[l];
        int64_t v = (j * (int64_t)I.z[l * d + t]) % M;
        if (numer) numer[e] = (int32_t)v;
        if (xout) xout[e] = (double)v / (double)M;
    }
}

// per-dimension min / max of the candidates (plan validation: N_Gamma, |k| bound)
__global__ void k_cand_stats(const void* __restrict__ cand, int i8, int ld, int64_t n, int d, int* mn, int* mx) {
    __shared__ int smn[kMaxD], smx[kMaxD];
    if (threadIdx.x < d) { smn[threadIdx.x] = INT_MAX; smx[threadIdx.x] = INT_MIN; }
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * d; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / d;
        const int t = (int)(e - r * d);
        const int v = i8 ? (int)reinterpret_cast<const int8_t*>(cand)[r * ld + t]
                         : reinterpret_cast<const int32_t*>(cand)[r * ld + t];
        atomicMin(&smn[t], v);
        atomicMax(&smx[t], v);
    }
    __syncthreads();
    if (threadIdx.x < d) {
        atomicMin(&mn[threadIdx.x], smn[threadIdx.x]);
        atomicMax(&mx[threadIdx.x], smx[threadIdx.x]);
    }
}

__global__ void k_to_c64(const void* src, int prec, c64* dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = prec ? cvt<double>(reinterpret_cast<const c32*>(src)[i]) : reinterpret_cast<const c64*>(src)[i];
}

__global__ void k_clear_inst(InstDesc* __restrict__ insts, int clear_det, int clear_coll, int clear_C) {
    InstDesc& I = insts[blockIdx.y];
    const int64_t W = (I.n + 31) >> 5;
    const int64_t SM = I.soff[I.L];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (clear_det)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < W; i += stride) I.detbits[i] = 0;
    if (clear_coll)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < SM; i += stride) I.coll[i] = 0;
    if (clear_C == 1)  // FP64 buckets
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < SM; i += stride) I.C[i] = c64{0, 0};
    if (clear_C == 2)  // FP32 buckets of the sampler of FP32 plans (first half of the buffer)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < SM; i += stride)
            reinterpret_cast<c32*>(I.C)[i] = c32{0.f, 0.f};
    if (clear_det && blockIdx.x == 0 && threadIdx.x < kCntWords) I.cnt[threadIdx.x] = 0;
}

// Copy from pinned host memory (device-accessible through unified addressing) by a kernel on the
// caller's stream: descriptor uploads do not queue behind bulk transfers on the copy engines.
__global__ void k_upload(uint64_t* __restrict__ dst, const uint64_t* __restrict__ src, int64_t words) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// ================================================================== launch wrappers
int launch_upload(void* dst, const void* pinned_src, size_t bytes, cudaStream_t st) {
    if (bytes % 8 || ((uintptr_t)dst | (uintptr_t)pinned_src) % 8) {
        set_error("upload of %zu bytes needs 8-byte sizes and alignment", bytes);
        return SFFT_EINVAL;
    }
    const int64_t words = (int64_t)(bytes / 8);
    const int gx = (int)std::min<int64_t>(64, (words + 255) / 256 + 1);
    k_upload<<<gx, 256, 0, st>>>(reinterpret_cast<uint64_t*>(dst), reinterpret_cast<const uint64_t*>(pinned_src), words);
    return launch_check("k_upload");
}

int launch_cand_stats(const void* cand, int i8, int ld, int64_t n, int d, int* mn, int* mx, cudaStream_t st) {
    int gx = (int)std::min<int64_t>(4 * 152, (n * d + 255) / 256 + 1);
    k_cand_stats<<<gx, 256, 0, st>>>(cand, i8, ld, n, d, mn, mx);
    return launch_check("k_cand_stats");
}

int launch_to_c64(const void* src, int prec, c64* dst, int64_t n, cudaStream_t st) {
    int gx = (int)std::min<int64_t>(4 * 152, (n + 255) / 256 + 1);
    k_to_c64<<<gx, 256, 0, st>>>(src, prec, dst, n);
    return launch_check("k_to_c64");
}

int launch_clear(InstDesc* di, int ninst, int clear_det, int clear_coll, int clear_C, cudaStream_t st) {
    k_clear_inst<<<dim3(64, ninst), 256, 0, st>>>(di, clear_det, clear_coll, clear_C);
    return launch_check("k_clear_inst");
}

template <int D>
static int launch_hash_d(const InstDesc* di, int ninst, int gx, size_t smem, int variant, int l0, int l1, int mode,
                         cudaStream_t st) {
    // variant: 0 int32 kernel, 1 packed kernel, 2 packed kernel with diagnostics (3: hash_tc.cu);
    // the CTA size follows the bitmap's shared memory (hash_threads)
    const int nt = variant == 2 ? kHashThreads : hash_threads(variant == 1, smem);
    if (variant == 0) {
        if (nt == kHashThreadsBig) {
            SFFT_TRY(allow_smem((const void*)k_hash_count<D, kHashThreadsBig>, 220 * 1024));
            k_hash_count<D, kHashThreadsBig><<<dim3(gx, ninst), nt, smem, st>>>(di, l0, l1, mode);
        } else {
            SFFT_TRY(allow_smem((const void*)k_hash_count<D>, 220 * 1024));
            k_hash_count<D><<<dim3(gx, ninst), kHashThreads, smem, st>>>(di, l0, l1, mode);
        }
    } else if (variant == 1) {
        if (nt == kHashThreadsBig) {
            SFFT_TRY(allow_smem((const void*)k_hash_count_packed<D, false, kHashThreadsBig>, 220 * 1024));
            k_hash_count_packed<D, false, kHashThreadsBig><<<dim3(gx, ninst), nt, smem, st>>>(di, l0, l1, mode);
        } else {
            SFFT_TRY(allow_smem((const void*)k_hash_count_packed<D, false>, 220 * 1024));
            k_hash_count_packed<D, false><<<dim3(gx, ninst), kHashThreads, smem, st>>>(di, l0, l1, mode);
        }
    } else {
        SFFT_TRY(allow_smem((const void*)k_hash_count_packed<D, true>, 220 * 1024));
        k_hash_count_packed<D, true><<<dim3(gx, ninst), kHashThreads, smem, st>>>(di, l0, l1, mode);
    }
    return launch_check("k_hash_count");
}

int hash_ctas_per_sm(size_t smem) { return std::max<int>(1, std::min<int>(8, (int)((228 * 1024) / (smem + 1024)))); }

// CTA size of the hash kernels for a bitmap segment of smem bytes: 384 threads while 3 or more CTAs
// share an SM; 768 when the bitmap leaves room for one CTA (both kernels) or two (the packed
// kernel, 40 registers), so that an SM keeps 24 or 48 warps instead of 12 or 24
int hash_threads(bool packed, size_t smem) {
    const int per_sm = hash_ctas_per_sm(smem);
    return per_sm == 1 || (packed && per_sm == 2) ? kHashThreadsBig : kHashThreads;
}

int64_t hash_tile(bool packed, size_t smem) { return (int64_t)hash_threads(packed, smem) * (packed ? kCPT2 : kCPT); }

size_t hash_smem_bytes(int d, int L, int64_t nwords, bool packed) {
    if (!packed) return sizeof(uint32_t) * (size_t)nwords + sizeof(int32_t) * (size_t)L * (d + 4);
    const int ZW = (d + 1) / 2, REC = 4 + ((ZW + 3) / 4) * 4;
    return sizeof(uint32_t) * ((size_t)nwords + (size_t)L * REC);
}

int launch_hash_count(const InstDesc* di, int ninst, int d, int gx, size_t smem, int variant, int l0, int l1, int mode,
                      cudaStream_t st) {
    if (variant == 3) return launch_hash_count_tc(di, ninst, gx, smem, st);  // tensor-core products
    switch (d) {
#define SFFT_HD(D) case D: return launch_hash_d<D>(di, ninst, gx, smem, variant, l0, l1, mode, st);
        SFFT_HD(1) SFFT_HD(2) SFFT_HD(3) SFFT_HD(4) SFFT_HD(5) SFFT_HD(6) SFFT_HD(7) SFFT_HD(8)
        SFFT_HD(9) SFFT_HD(10) SFFT_HD(11) SFFT_HD(12) SFFT_HD(13) SFFT_HD(14) SFFT_HD(15) SFFT_HD(16)
        SFFT_HD(17) SFFT_HD(18) SFFT_HD(19) SFFT_HD(20) SFFT_HD(21) SFFT_HD(22) SFFT_HD(23) SFFT_HD(24)
        SFFT_HD(25) SFFT_HD(26) SFFT_HD(27) SFFT_HD(28) SFFT_HD(29) SFFT_HD(30) SFFT_HD(31) SFFT_HD(32)
#undef SFFT_HD
        default: set_error("dimension %d not supported", d); return SFFT_EINVAL;
    }
}

int launch_zero_test(const LatDesc* dl, int nlat, InstDesc* di, int prec, double kappa_u, cudaStream_t st) {
    if (prec) k_zero_test<float><<<nlat, kZtThreads, 0, st>>>(dl, di, kappa_u);
    else k_zero_test<double><<<nlat, kZtThreads, 0, st>>>(dl, di, kappa_u);
    return launch_check("k_zero_test");
}

int launch_compact(InstDesc* di, int ninst, cudaStream_t st) {
    k_compact<<<dim3(kCompactChunks, ninst), kCompactThreads, 0, st>>>(di);
    return launch_check("k_compact");
}

// per-detected-candidate kernels: one warp per candidate in a grid-stride loop over a grid of
// about 8 resident CTAs per SM for the whole batch (|Itilde| is only known on the device)
static int det_grid(int64_t maxdet, int ninst) {
    const int64_t need = (maxdet + 7) / 8, cap = (152 * 8 + ninst - 1) / ninst;
    return (int)std::max<int64_t>(1, std::min(need, cap));
}

int launch_det_hashes(const InstDesc* di, int ninst, int64_t maxdet, cudaStream_t st) {
    const int gx = det_grid(maxdet, ninst);
    k_det_hashes<<<dim3(gx, ninst), 256, 0, st>>>(di);
    return launch_check("k_det_hashes");
}

int launch_collisions(const InstDesc* di, int ninst, cudaStream_t st) {
    k_collisions<<<dim3(152, ninst), 256, 0, st>>>(di);
    return launch_check("k_collisions");
}

int launch_combine(const InstDesc* di, int ninst, int64_t maxdet, int prec, int mode, cudaStream_t st, int zc) {
    const int gx = det_grid(maxdet, ninst);
    if (mode == 1 || mode == 2) {  // 2: FP32 buckets
        if (mode == 2) k_refine_update<float, true><<<dim3(gx, ninst), 256, 0, st>>>(di);
        else if (prec) k_refine_update<float, false><<<dim3(gx, ninst), 256, 0, st>>>(di);
        else k_refine_update<double, false><<<dim3(gx, ninst), 256, 0, st>>>(di);
        return launch_check("k_refine_update");
    }
    if (mode == 3) {  // combine that forms the hashes of Itilde itself
        if (prec) k_combine<float, true><<<dim3(gx, ninst), 256, 0, st>>>(di, zc);
        else k_combine<double, true><<<dim3(gx, ninst), 256, 0, st>>>(di, zc);
    } else {
        if (prec) k_combine<float, false><<<dim3(gx, ninst), 256, 0, st>>>(di, zc);
        else k_combine<double, false><<<dim3(gx, ninst), 256, 0, st>>>(di, zc);
    }
    return launch_check("k_combine");
}

int launch_lsq(InstDesc* di, int ninst, int prec, cudaStream_t st) {
    const dim3 grid(152, ninst);
    for (int mode = 0; mode < 2; ++mode) {
        if (prec) k_lsq_prep<float><<<grid, 256, 0, st>>>(di, mode);
        else k_lsq_prep<double><<<grid, 256, 0, st>>>(di, mode);
        SFFT_TRY(launch_check("k_lsq_prep"));
    }
    k_lsq_pairs<<<grid, 256, 0, st>>>(di);
    SFFT_TRY(launch_check("k_lsq_pairs"));
    const int smem = 4 * kLsqSmemVec * (int)sizeof(c64);
    SFFT_TRY(allow_smem((const void*)k_lsq_cg, smem));
    k_lsq_cg<<<ninst, kLsqThreads, smem, st>>>(di, 64, 1e-12);
    return launch_check("k_lsq_cg");
}

int launch_scatter_coef(const InstDesc* di, int ninst, bool f32, cudaStream_t st) {
    if (f32) k_scatter_coef<true><<<dim3(152, ninst), 256, 0, st>>>(di);
    else k_scatter_coef<false><<<dim3(152, ninst), 256, 0, st>>>(di);
    return launch_check("k_scatter_coef");
}

int launch_select(InstDesc* di, int ninst, cudaStream_t st) {
    k_select<<<ninst, kSelThreads, 0, st>>>(di);
    return launch_check("k_select");
}

int launch_scatter_terms(const InstDesc* di, int ninst, int64_t max_terms_x_L, cudaStream_t st) {
    int gx = (int)std::min<int64_t>(1024, (max_terms_x_L + 255) / 256 + 1);
    k_scatter_terms<<<dim3(gx, ninst), 256, 0, st>>>(di);
    return launch_check("k_scatter_terms");
}

int launch_adjoint_buckets(const InstDesc* di, const c64* dcoef, bool refine, int64_t maxdet, cudaStream_t st) {
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(4 * 152, (maxdet + 255) / 256));
    if (dcoef) {
        k_adj_dense<<<dim3(gx, 1), 256, 0, st>>>(di, dcoef);
        SFFT_TRY(launch_check("k_adj_dense"));
    }
    if (refine) {
        k_adj_refine_scatter<<<dim3(gx, 1), 256, 0, st>>>(di);
        SFFT_TRY(launch_check("k_adj_refine_scatter"));
        k_adj_refine_gather<<<dim3(gx, 1), 256, 0, st>>>(di);
        SFFT_TRY(launch_check("k_adj_refine_gather"));
    }
    k_adj_median_scatter<<<dim3(gx, 1), 256, 0, st>>>(di);
    return launch_check("k_adj_median_scatter");
}

int launch_points(const InstDesc* di, int32_t* numer, double* x, int64_t tot, cudaStream_t st) {
    int gx = (int)std::min<int64_t>(4096, (tot + 255) / 256 + 1);
    k_points<<<gx, 256, 0, st>>>(di, numer, x);
    return launch_check("k_points");
}

}  // namespace sfft
