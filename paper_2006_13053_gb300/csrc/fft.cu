// Host side of the batched prime-length DFTs (Algorithm 2) by Bluestein's algorithm:
// per distinct M the Bluestein length N = 2^a 3^b 5^c >= 2M-1, its radix order and pass plan,
// and the chirp, filter and twiddle tables (computed once in double: chirp phases j^2 mod 2M
// and all twiddle indices are exact integers), plus the launch dispatcher over the arithmetic
// types.  The kernels are in bluestein.cuh.
#include <math.h>

#include <map>
#include <mutex>

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

// Stage order of N = 4^f 2^t 3^b 5^c (t <= 1): radix-4 and radix-3 stages alternate while both
// remain, so that the kernels can fuse them pairwise (4 x 3 = 12 elements per thread), then the
// remaining 4s, the 2, the remaining 3s and the 5s.
static int factor_radices(int64_t N, int* rad) {
    int64_t v = N;
    int f = 0, t = 0, b = 0, c = 0;
    while (v % 4 == 0) { ++f; v /= 4; }
    while (v % 2 == 0) { ++t; v /= 2; }
    while (v % 3 == 0) { ++b; v /= 3; }
    while (v % 5 == 0) { ++c; v /= 5; }
    if (v != 1 || f + t + b + c > kMaxStages) return -1;
    int n = 0;
    while (f > 0 && b > 0) { rad[n++] = 4; rad[n++] = 3; --f; --b; }
    while (f-- > 0) rad[n++] = 4;
    while (t-- > 0) rad[n++] = 2;
    while (b-- > 0) rad[n++] = 3;
    while (c-- > 0) rad[n++] = 5;
    return n;
}

int plan_passes(const int* radix, int ns, int maxprod, uint8_t* pass_r) {
    int np = 0;
    for (int s = 0; s < ns;) {
        const int r1 = radix[s];
        if (s + 1 < ns && r1 * radix[s + 1] <= maxprod && pass_fusable(r1, radix[s + 1])) {
            pass_r[np++] = (uint8_t)(r1 | (radix[s + 1] << 4));
            s += 2;
        } else {
            pass_r[np++] = (uint8_t)(r1 | (1 << 4));
            s += 1;
        }
    }
    return np;
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
    if (rc == SFFT_OK) rc = upload_df(&t->dftdf, dft);
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
    cudaFree(t->twa32); cudaFree(t->twb32); cudaFree(t->twdf); cudaFree(t->chirpdf); cudaFree(t->dftdf);
    delete t;
}

size_t blue_smem_limit() { return 207 * 1024; }

int uniform_pair(const BlueJob* jobs, size_t n) {
    int up = -1;
    for (size_t j = 0; j < n; ++j)
        for (int p = 0; p < jobs[j].npass; ++p) {
            if (up < 0) up = jobs[j].pass_r[p];
            else if (up != jobs[j].pass_r[p]) return 0;
        }
    return up < 0 ? 0 : up;
}

int launch_bluestein(const BlueJob* djobs, int njobs, int maxN, int mode, int prec, int in_prec, int out_prec, int sign,
                     int epi, const InstDesc* insts, cudaStream_t st, void* ob, const void* ab, int threads, int upair) {
    // prec: 0 double, 1 float, 2 double-float; in/out: 0 double, 1 float
    if (prec == 2) {  // double-float: float samples in, float high words out (low words to aux)
        if (in_prec != 1 || out_prec != 1) { set_error("double-float transforms take and give float"); return SFFT_EINVAL; }
        return launch_bluestein_df64(djobs, njobs, maxN, mode, sign, epi, insts, st, ob, ab, threads, upair);
    }
    // the element-type combinations the library uses: FP64 everything; FP32 with FP32 or FP64 input
    if (prec == 0 && in_prec == 0 && out_prec == 0)
        return launch_bluestein_f64(djobs, njobs, maxN, mode, sign, epi, insts, st, ob, ab, threads, upair);
    if (prec == 1 && out_prec == 1)
        return launch_bluestein_f32(in_prec == 0, djobs, njobs, maxN, mode, sign, epi, insts, st, ob, ab, threads, upair);
    set_error("unsupported transform precision combination (%d, %d, %d)", prec, in_prec, out_prec);
    return SFFT_EINVAL;
}

}  // namespace sfft
