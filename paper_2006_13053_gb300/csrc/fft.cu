// Batched prime-length DFTs of the lattice samples (Algorithm 2, line 2) by Bluestein's
// algorithm: a length-M DFT becomes a cyclic convolution of length N = 2^a 3^b 5^c >= 2M-1.
// The convolution is computed by an in-place mixed-radix decimation-in-frequency FFT
// (natural order in, digit-reversed out), a pointwise product with the precomputed filter
// (itself stored digit-reversed) and the matching decimation-in-time inverse (digit-reversed
// in, natural order out), so no reordering pass is needed.  One CTA transforms one lattice;
// the work buffer lives in shared memory when N complex values fit (FP32 up to N = 28672),
// otherwise in an L2-resident global scratch buffer.  Chirp phases j^2 mod 2M and all
// twiddle indices are exact integers; the tables are computed once per distinct M in double.
#include <math.h>

#include <map>
#include <mutex>
#include <type_traits>

#include "common.cuh"

namespace sfft {

// ================================================================== host tables
int64_t bluestein_size(int64_t M) {
    int64_t need = 2 * M - 1, best = -1;
    for (int64_t p5 = 1; p5 < 4 * need; p5 *= 5)
        for (int64_t p3 = p5; p3 < 4 * need; p3 *= 3)
            for (int64_t p2 = p3; p2 < 4 * need; p2 *= 2)
                if (p2 >= need && (best < 0 || p2 < best)) best = p2;
    return best;
}

static int factor_radices(int64_t N, int* rad) {
    int n = 0;
    int64_t v = N;
    while (v % 4 == 0) { rad[n++] = 4; v /= 4; }
    while (v % 2 == 0) { rad[n++] = 2; v /= 2; }
    while (v % 3 == 0) { rad[n++] = 3; v /= 3; }
    while (v % 5 == 0) { rad[n++] = 5; v /= 5; }
    return v == 1 ? n : -1;
}

// host DIF (same stage order and indexing as the device kernel), double precision
static void host_dif(std::vector<c64>& a, int64_t N, const int* rad, int ns, const std::vector<c64>& tw) {
    int64_t Ns = N;
    for (int s = 0; s < ns; ++s) {
        int R = rad[s];
        int64_t m = Ns / R, stride = N / Ns;
        for (int64_t b = 0; b < N / Ns; ++b)
            for (int64_t n = 0; n < m; ++n) {
                c64 v[5], y[5];
                for (int q = 0; q < R; ++q) v[q] = a[b * Ns + n + q * m];
                for (int p = 0; p < R; ++p) {
                    double re = 0, im = 0;
                    for (int q = 0; q < R; ++q) {
                        int64_t e = ((int64_t)p * q) % R;  // omega_R^{pq} = tw[e * N / R]
                        c64 w = tw[e * (N / R)];
                        re += v[q].x * w.x - v[q].y * w.y;
                        im += v[q].x * w.y + v[q].y * w.x;
                    }
                    y[p] = c64{re, im};
                }
                for (int p = 0; p < R; ++p) {
                    c64 w = tw[(n * p * stride) % N];
                    a[b * Ns + n + p * m] = y[p] * w;
                }
            }
        Ns = m;
    }
}

static std::mutex g_tab_mu;
static std::map<std::pair<int, int64_t>, FftTables*> g_tabs;

static int upload64(c64** dst, const std::vector<c64>& src) {
    SFFT_CU(cudaMalloc((void**)dst, sizeof(c64) * src.size()));
    SFFT_CU(cudaMemcpy(*dst, src.data(), sizeof(c64) * src.size(), cudaMemcpyHostToDevice));
    return SFFT_OK;
}
static int upload32(c32** dst, const std::vector<c64>& src) {
    std::vector<c32> tmp(src.size());
    for (size_t i = 0; i < src.size(); ++i) tmp[i] = c32{(float)src[i].x, (float)src[i].y};
    SFFT_CU(cudaMalloc((void**)dst, sizeof(c32) * tmp.size()));
    SFFT_CU(cudaMemcpy(*dst, tmp.data(), sizeof(c32) * tmp.size(), cudaMemcpyHostToDevice));
    return SFFT_OK;
}

static int upload_df(void** dst, const std::vector<c64>& src) {
    std::vector<cplx<df64>> tmp(src.size());
    for (size_t i = 0; i < src.size(); ++i) tmp[i] = cplx<df64>{df_from(src[i].x), df_from(src[i].y)};
    SFFT_CU(cudaMalloc(dst, sizeof(cplx<df64>) * tmp.size()));
    SFFT_CU(cudaMemcpy(*dst, tmp.data(), sizeof(cplx<df64>) * tmp.size(), cudaMemcpyHostToDevice));
    return SFFT_OK;
}

int tables_acquire(int64_t M, FftTables** out) {
    int dev = 0;
    SFFT_CU(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tab_mu);
    auto key = std::make_pair(dev, M);
    auto it = g_tabs.find(key);
    if (it != g_tabs.end()) {
        it->second->refs++;
        *out = it->second;
        return SFFT_OK;
    }
    FftTables* t = new FftTables();
    t->M = M;
    t->N = bluestein_size(M);
    t->device = dev;
    t->nstages = factor_radices(t->N, t->radix);
    if (t->nstages <= 0 || t->nstages > kMaxStages || t->N > 262144) {
        delete t;
        set_error("no mixed-radix plan for Bluestein length of M=%lld", (long long)M);
        return SFFT_EINVAL;
    }
    const int64_t N = t->N;
    std::vector<c64> tw(N), chirp(M), dft(M), b(N, c64{0, 0});
    for (int64_t i = 0; i < N; ++i) {
        double a = -2.0 * M_PI * (double)i / (double)N;
        tw[i] = c64{cos(a), sin(a)};
    }
    for (int64_t j = 0; j < M; ++j) {
        int64_t ph = (int64_t)((__int128)j * j % (2 * M));  // exact j^2 mod 2M
        double a = -M_PI * (double)ph / (double)M;
        chirp[j] = c64{cos(a), sin(a)};
        double a2 = -2.0 * M_PI * (double)j / (double)M;
        dft[j] = c64{cos(a2), sin(a2)};
    }
    int rc = SFFT_OK;
    t->tw_na = (int)((N + 255) / 256);
    std::vector<c64> twa(t->tw_na), twb(256);
    for (int a = 0; a < t->tw_na; ++a) {
        double ang = -2.0 * M_PI * (double)((int64_t)a * 256) / (double)N;
        twa[a] = c64{cos(ang), sin(ang)};
    }
    for (int b2 = 0; b2 < 256; ++b2) {
        double ang = -2.0 * M_PI * (double)b2 / (double)N;
        twb[b2] = c64{cos(ang), sin(ang)};
    }
    if (rc == SFFT_OK) rc = upload32(&t->twa32, twa);
    if (rc == SFFT_OK) rc = upload32(&t->twb32, twb);
    // filters: forward b_n = conj(chirp_|n|), inverse b_n = chirp_|n| (circular), then DIF / N
    for (int dir = 0; dir < 2 && rc == SFFT_OK; ++dir) {
        std::fill(b.begin(), b.end(), c64{0, 0});
        for (int64_t n = 0; n < M; ++n) {
            c64 v = dir == 0 ? conj(chirp[n]) : chirp[n];
            b[n] = v;
            if (n > 0) b[N - n] = v;
        }
        host_dif(b, N, t->radix, t->nstages, tw);
        for (auto& v : b) v = v * (1.0 / (double)N);
        if ((rc = upload64(&t->filt64[dir], b)) == SFFT_OK) rc = upload32(&t->filt32[dir], b);
        if (rc == SFFT_OK) rc = upload_df(&t->filtdf[dir], b);
    }
    if (rc == SFFT_OK) rc = upload64(&t->tw64, tw);
    if (rc == SFFT_OK) rc = upload32(&t->tw32, tw);
    if (rc == SFFT_OK) rc = upload64(&t->chirp64, chirp);
    if (rc == SFFT_OK) rc = upload32(&t->chirp32, chirp);
    if (rc == SFFT_OK) rc = upload64(&t->dft64, dft);
    if (rc == SFFT_OK) rc = upload_df(&t->twdf, tw);
    if (rc == SFFT_OK) rc = upload_df(&t->chirpdf, chirp);
    if (rc != SFFT_OK) {
        t->refs = 1;
        tables_release(t);
        return rc;
    }
    t->refs = 1;
    g_tabs[key] = t;
    *out = t;
    return SFFT_OK;
}

void tables_release(FftTables* t) {
    if (!t) return;
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if (--t->refs > 0) return;
    g_tabs.erase(std::make_pair(t->device, t->M));
    cudaFree(t->tw64); cudaFree(t->tw32); cudaFree(t->chirp64); cudaFree(t->chirp32); cudaFree(t->dft64);
    for (int d = 0; d < 2; ++d) { cudaFree(t->filt64[d]); cudaFree(t->filt32[d]); cudaFree(t->filtdf[d]); }
    cudaFree(t->twa32); cudaFree(t->twb32); cudaFree(t->twdf); cudaFree(t->chirpdf);
    delete t;
}

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

template <int R, int S, class T> __device__ __forceinline__ void bfly(cplx<T>* v) {
    if constexpr (R == 2) {
        cplx<T> a = v[0], b = v[1];
        v[0] = a + b;
        v[1] = a - b;
    } else if constexpr (R == 4) {
        cplx<T> t0 = v[0] + v[2], t1 = v[0] - v[2], t2 = v[1] + v[3], t3 = mul_si<S>(v[1] - v[3]);
        v[0] = t0 + t2;
        v[2] = t0 - t2;
        v[1] = t1 + t3;
        v[3] = t1 - t3;
    } else if constexpr (R == 3) {
        cplx<T> t1 = v[1] + v[2], t2 = v[1] - v[2];
        cplx<T> a = v[0] - t1 * kc<T>(0.5);
        cplx<T> b = mul_si<S>(t2 * kc<T>(kH3));
        v[0] = v[0] + t1;
        v[1] = a + b;
        v[2] = a - b;
    } else if constexpr (R == 5) {
        cplx<T> t1 = v[1] + v[4], t2 = v[2] + v[3], t3 = v[1] - v[4], t4 = v[2] - v[3];
        cplx<T> b1 = v[0] + t1 * kc<T>(kC1) + t2 * kc<T>(kC2);
        cplx<T> b2 = v[0] + t1 * kc<T>(kC2) + t2 * kc<T>(kC1);
        cplx<T> d1 = mul_si<S>(t3 * kc<T>(kS1) + t4 * kc<T>(kS2));
        cplx<T> d2 = mul_si<S>(t3 * kc<T>(kS2) - t4 * kc<T>(kS1));
        v[0] = v[0] + t1 + t2;
        v[1] = b1 + d1;
        v[4] = b1 - d1;
        v[2] = b2 + d2;
        v[3] = b2 - d2;
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

// DIF stage: sub-transform size Ns, radix R, m = Ns / R; twiddle exp(-2 pi i n p / Ns).
// The block index b = floor(i / m) is formed with a float reciprocal: (i + 1/2) / m is at least
// 1/(2m) away from an integer, which the float product resolves exactly for i < 2^22.
template <int R, class T, class TW>
__device__ __forceinline__ void dif_stage(cplx<T>* __restrict__ buf, int N, int Ns, const TW& tw) {
    const int m = Ns / R, stride = N / Ns, nb = N / R;
    const float rm = 1.0f / (float)m;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        int b = (int)(((float)i + 0.5f) * rm), n = i - b * m;
        cplx<T>* base = buf + (size_t)b * Ns + n;
        cplx<T> v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = base[q * m];
        bfly<R, -1>(v);
        base[0] = v[0];
#pragma unroll
        for (int p = 1; p < R; ++p) base[p * m] = v[p] * tw(n * p * stride);
    }
}

// DIT stage (exact adjoint of dif_stage): conj twiddles, then inverse R-point DFT
template <int R, class T, class TW>
__device__ __forceinline__ void dit_stage(cplx<T>* __restrict__ buf, int N, int Ns, const TW& tw) {
    const int m = Ns / R, stride = N / Ns, nb = N / R;
    const float rm = 1.0f / (float)m;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        int b = (int)(((float)i + 0.5f) * rm), n = i - b * m;
        cplx<T>* base = buf + (size_t)b * Ns + n;
        cplx<T> v[R];
        v[0] = base[0];
#pragma unroll
        for (int p = 1; p < R; ++p) v[p] = mulc(base[p * m], tw(n * p * stride));
        bfly<R, 1>(v);
#pragma unroll
        for (int q = 0; q < R; ++q) base[q * m] = v[q];
    }
}

template <class T, class TW>
__device__ __forceinline__ void run_stage(bool dif, int R, cplx<T>* buf, int N, int Ns, const TW& tw) {
    if (dif) {
        switch (R) {
            case 4: dif_stage<4>(buf, N, Ns, tw); break;
            case 2: dif_stage<2>(buf, N, Ns, tw); break;
            case 3: dif_stage<3>(buf, N, Ns, tw); break;
            default: dif_stage<5>(buf, N, Ns, tw); break;
        }
    } else {
        switch (R) {
            case 4: dit_stage<4>(buf, N, Ns, tw); break;
            case 2: dit_stage<2>(buf, N, Ns, tw); break;
            case 3: dit_stage<3>(buf, N, Ns, tw); break;
            default: dit_stage<5>(buf, N, Ns, tw); break;
        }
    }
}

__device__ __forceinline__ double block_reduce_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (threadIdx.x == 0) red[0] = r;
    __syncthreads();
    double out = red[0];
    __syncthreads();
    return out;
}

__device__ __forceinline__ double block_reduce_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (threadIdx.x == 0) red[0] = r;
    __syncthreads();
    double out = red[0];
    __syncthreads();
    return out;
}

constexpr int kBlueThreads = 512;

template <class T, class TI, class TO, class TW>
__device__ __forceinline__ void bluestein_body(const BlueJob& J, cplx<T>* buf, const TW& tw, int sign, int epi,
                                               const void* inp, const void* auxp, void* outp, double* red) {
    // max of |x|^2 in the transform precision (double for df64, whose analysis is never requested)
    using R = typename std::conditional<std::is_same<T, df64>::value, double, T>::type;
    const int M = J.M, N = J.N, ns = J.nstages;
    const cplx<T>* __restrict__ chirp = reinterpret_cast<const cplx<T>*>(J.chirp);
    const cplx<T>* __restrict__ filt = reinterpret_cast<const cplx<T>*>(J.filt);
    const cplx<TI>* __restrict__ in = reinterpret_cast<const cplx<TI>*>(inp);
    const bool inv = sign > 0;
    // ---- load x_j * w_j (w = chirp for the forward DFT, conj(chirp) for the inverse), zero pad
    R ss = 0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        cplx<T> v = {kc<T>(0.0), kc<T>(0.0)};
        if (i < M) {
            cplx<T> x = load_in<T, TI>(in + i);
            if (epi == EPI_ANALYZE) ss += scv<R>(abs2(x));
            cplx<T> w = ldg(&chirp[i]);
            v = inv ? mulc(x, w) : x * w;
        }
        buf[i] = v;
    }
    double ssd = 0;
    if (epi == EPI_ANALYZE) ssd = block_reduce_sum((double)ss, red);
    __syncthreads();
    // ---- DIF stages
    int Ns = N;
    for (int s = 0; s < ns; ++s) {
        int Rr = J.radix[s];
        run_stage<T>(true, Rr, buf, N, Ns, tw);
        Ns /= Rr;
        __syncthreads();
    }
    // ---- pointwise product with the (digit-reversed) filter
    for (int i = threadIdx.x; i < N; i += blockDim.x) buf[i] = buf[i] * ldg(&filt[i]);
    __syncthreads();
    // ---- DIT stages, reverse order
    Ns = 1;
    for (int s = ns - 1; s >= 0; --s) {
        int Rr = J.radix[s];
        Ns *= Rr;
        run_stage<T>(false, Rr, buf, N, Ns, tw);
        __syncthreads();
    }
    // ---- epilogue: X_h = w_h conv_h
    cplx<TO>* __restrict__ out = reinterpret_cast<cplx<TO>*>(outp);
    R mx2 = 0;
    const T sc = kc<T>(J.scale);
    for (int h = threadIdx.x; h < M; h += blockDim.x) {
        cplx<T> w = ldg(&chirp[h]);
        cplx<T> X = inv ? mulc(buf[h], w) : buf[h] * w;
        X = X * sc;
        if (epi == EPI_PLAIN || epi == EPI_ANALYZE) {
            if constexpr (std::is_same<T, df64>::value && std::is_same<TO, float>::value) {
                // float output of a double-float value: high words out, low words to aux
                out[h] = cplx<TO>{X.x.hi, X.y.hi};
                if (auxp) reinterpret_cast<c32*>(const_cast<void*>(auxp))[h] = c32{X.x.lo, X.y.lo};
            } else {
                out[h] = ccv<TO>(X);
            }
            if (epi == EPI_ANALYZE) mx2 = fmax(mx2, scv<R>(abs2(X)));
        } else {  // EPI_ADDNOISE
            const c64* aux = reinterpret_cast<const c64*>(auxp);
            c64 r = ccv<double>(X);
            if (aux) r = r + aux[h];
            out[h] = ccv<TO>(r);
        }
    }
    if (epi == EPI_ANALYZE) {
        double mx = sqrt(block_reduce_max((double)mx2, red));
        if (threadIdx.x == 0) {
            LatStats& S = *J.stat;
            S.max32 = (float)mx;
            S.max_abs = mx;
            S.rms = sqrt(ssd / (double)M);
        }
    }
}

// One CTA = one Bluestein transform.  T: arithmetic (float, double or df64); TI/TO: element
// type of input/output.  SM: work buffer in dynamic shared memory, else in J.scratch.
template <class T, class TI, class TO, bool SM>
__global__ void __launch_bounds__(kBlueThreads, 1) k_bluestein(const BlueJob* __restrict__ jobs, int sign, int epi,
                                                            const InstDesc* __restrict__ insts, void* out_base,
                                                            const void* aux_base) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    const BlueJob& J = jobs[blockIdx.x];
    cplx<T>* buf = SM ? reinterpret_cast<cplx<T>*>(smem_raw) : reinterpret_cast<cplx<T>*>(J.scratch);
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
        if (J.io_flags & 32) auxp = I.samp_noise ? (const void*)(I.samp_noise + J.io_off) : nullptr;
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
        bluestein_body<T, TI, TO>(J, buf, TwTwo{s_twa, s_twb}, sign, epi, inp, auxp, outp, red);
    } else {
        bluestein_body<T, TI, TO>(J, buf, TwFull<T>{reinterpret_cast<const cplx<T>*>(J.tw)}, sign, epi, inp, auxp,
                                  outp, red);
    }
}

// ================================================================== host launcher
size_t blue_smem_limit() { return 207 * 1024; }

template <class T, class TI, class TO>
static int launch_t(const BlueJob* djobs, int njobs, int maxN, bool sm, int sign, int epi, const InstDesc* insts,
                    cudaStream_t st, void* ob, const void* ab, int threads) {
    if (threads < 64 || threads > kBlueThreads || threads % 32) threads = kBlueThreads;
    if (njobs == 0) return SFFT_OK;
    if (sm) {
        size_t bytes = (size_t)maxN * sizeof(cplx<T>);
        if (bytes > blue_smem_limit()) {
            set_error("Bluestein length %d does not fit shared memory", maxN);
            return SFFT_EINVAL;
        }
        static bool attr_done = false;  // one attribute call per instantiation
        if (!attr_done) {
            SFFT_CU(cudaFuncSetAttribute(k_bluestein<T, TI, TO, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)blue_smem_limit()));
            attr_done = true;
        }
        k_bluestein<T, TI, TO, true><<<njobs, threads, bytes, st>>>(djobs, sign, epi, insts, ob, ab);
    } else {
        k_bluestein<T, TI, TO, false><<<njobs, threads, 0, st>>>(djobs, sign, epi, insts, ob, ab);
    }
    return launch_check("k_bluestein");
}

int launch_bluestein(const BlueJob* djobs, int njobs, int maxN, bool sm, int prec, int in_prec, int out_prec, int sign,
                     int epi, const InstDesc* insts, cudaStream_t st, void* ob, const void* ab, int threads) {
    // prec: 0 double, 1 float, 2 double-float; in/out: 0 double, 1 float
    if (prec == 2) {  // double-float: float samples in, float high words out (low words to aux)
        if (in_prec != 1 || out_prec != 1) { set_error("double-float transforms take and give float"); return SFFT_EINVAL; }
        return launch_t<df64, float, float>(djobs, njobs, maxN, sm, sign, epi, insts, st, ob, ab, threads);
    }
    int key = prec * 4 + in_prec * 2 + out_prec;
    switch (key) {
        case 0: return launch_t<double, double, double>(djobs, njobs, maxN, sm, sign, epi, insts, st, ob, ab, threads);
        case 1: return launch_t<double, double, float>(djobs, njobs, maxN, sm, sign, epi, insts, st, ob, ab, threads);
        case 2: return launch_t<double, float, double>(djobs, njobs, maxN, sm, sign, epi, insts, st, ob, ab, threads);
        case 3: return launch_t<double, float, float>(djobs, njobs, maxN, sm, sign, epi, insts, st, ob, ab, threads);
        case 4: return launch_t<float, double, double>(djobs, njobs, maxN, sm, sign, epi, insts, st, ob, ab, threads);
        case 5: return launch_t<float, double, float>(djobs, njobs, maxN, sm, sign, epi, insts, st, ob, ab, threads);
        case 6: return launch_t<float, float, double>(djobs, njobs, maxN, sm, sign, epi, insts, st, ob, ab, threads);
        default: return launch_t<float, float, float>(djobs, njobs, maxN, sm, sign, epi, insts, st, ob, ab, threads);
    }
}

}  // namespace sfft
