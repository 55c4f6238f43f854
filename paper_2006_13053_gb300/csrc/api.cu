// C ABI of the library: plans (Corollary 2.6 / eq. 4.2 parameter rules, lattice generation),
// workspace layout, and the stage sequence of one reconstruction (Algorithm 2 -> optional
// Remark 2.8 combine -> optional FP64 refinement -> Algorithm 4 selection), the synthetic
// samplers and the adjoint.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "philox.cuh"
#include "plan.cuh"

namespace sfft {

// ================================================================== errors
static thread_local std::string g_err;
void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}
const char* get_error() { return g_err.c_str(); }

int allow_smem(const void* kernel, int bytes) {
    int dev = 0;
    SFFT_CU(cudaGetDevice(&dev));
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> done;  // (kernel, device) -> limit set
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(kernel, dev);
    const auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return SFFT_OK;
    SFFT_CU(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done[key] = bytes;
    return SFFT_OK;
}

// ================================================================== Philox4x64-10 (philox.cuh)
uint64_t philox_word0(uint64_t key0, uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3) {
    return philox4x64_w0(key0, c0, c1, c2, c3);
}

double philox_u01(uint64_t key, uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3) {
    return philox4x64_u01(key, c0, c1, c2, c3);
}

// ================================================================== number theory / rules
static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((unsigned __int128)a * b % m); }
static uint64_t powmod(uint64_t a, uint64_t e, uint64_t m) {
    uint64_t r = 1;
    a %= m;
    while (e) {
        if (e & 1) r = mulmod(r, a, m);
        a = mulmod(a, a, m);
        e >>= 1;
    }
    return r;
}
bool is_prime(int64_t n) {
    if (n < 2) return false;
    for (int64_t p : {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37}) {
        if (n % p == 0) return n == p;
    }
    uint64_t d = (uint64_t)n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (uint64_t a : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 17ull, 19ull, 23ull, 29ull, 31ull, 37ull}) {
        uint64_t x = powmod(a, d, (uint64_t)n);
        if (x == 1 || x == (uint64_t)n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; ++r) {
            x = mulmod(x, x, (uint64_t)n);
            if (x == (uint64_t)n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}
int64_t next_prime_above(double x) {
    int64_t p = (int64_t)floor(x) + 1;
    if (p < 2) p = 2;
    while (!is_prime(p)) ++p;
    return p;
}
static int odd_ceil(double v) {
    int n = (int)ceil(v - 1e-12);
    if (n < 1) n = 1;
    return (n % 2) ? n : n + 1;
}
int L_rule(int rule, int64_t n, double delta, double c) {
    const double base = 4.0 * c / ((c - 2.0) * log(c - 1.0)) * (log((double)n) - log(delta));
    switch (rule) {
        case SFFT_L_COR26: return odd_ceil(base);
        case SFFT_L_EQ42: return odd_ceil(0.25 * base);
        default: {
            int v = (int)ceil(2.0 * log((double)n)) + 1;
            return (v % 2) ? v : v + 1;
        }
    }
}

// ================================================================== plan lifecycle
static int dmalloc(void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        return SFFT_ENOMEM;
    }
    return SFFT_OK;
}
#define DMALLOC(ptr, bytes) SFFT_TRY(dmalloc((void**)&(ptr), (bytes)))

int Plan::io_begin() {
    if (io_ev) SFFT_CU(cudaEventSynchronize(io_ev));
    return SFFT_OK;
}
int Plan::io_upload() {
    SFFT_TRY(launch_upload(d_inst, h_inst, sizeof(InstDesc), st));
    SFFT_CU(cudaEventRecord(io_ev, st));
    return SFFT_OK;
}

void Plan::release() {
    if (io_ev) { cudaEventSynchronize(io_ev); cudaEventDestroy(io_ev); io_ev = nullptr; }
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    for (auto* t : tabs) tables_release(t);
    tabs.clear();
    if (h_inst) cudaFreeHost(h_inst);
    if (h_cnt) cudaFreeHost(h_cnt);
    h_inst = nullptr;
    h_cnt = nullptr;
}

int Plan::alloc(void** p, size_t bytes) {
    SFFT_TRY(dmalloc(p, bytes));
    allocs.push_back(*p);
    return SFFT_OK;
}

size_t Plan::esz() const { return prec ? sizeof(c32) : sizeof(c64); }

// prec: 0 double, 1 float, 2 double-float arithmetic
BlueJob make_blue_job(const FftTables* t, int prec, int dir, double scale) {
    BlueJob J;
    memset(&J, 0, sizeof J);
    J.M = (int)t->M;
    J.N = (int)t->N;
    J.nstages = t->nstages;
    for (int s = 0; s < t->nstages; ++s) J.radix[s] = (uint8_t)t->radix[s];
    J.npass = (uint8_t)plan_passes(t->radix, t->nstages, prec == 1 ? pass_maxprod<float>() : pass_maxprod<double>(),
                                   J.pass_r);
    if (prec == 1) {
        J.tw = t->tw32; J.chirp = t->chirp32; J.filt = t->filt32[dir];
    } else if (prec == 0) {
        J.tw = t->tw64; J.chirp = t->chirp64; J.filt = t->filt64[dir];
    } else {
        J.tw = t->twdf; J.chirp = t->chirpdf; J.filt = t->filtdf[dir];
    }
    J.twa = t->twa32;
    J.twb = t->twb32;
    J.tw_na = t->tw_na;
    J.dft64 = (const double*)t->dft64;
    J.scale = scale;
    return J;
}

bool Plan::fits_smem(int tprec) const {
    size_t e = tprec == 1 ? sizeof(c32) : sizeof(c64);  // double and double-float: 16 bytes
    return blue_smem_bytes(maxN, e) <= blue_smem_limit();
}

int Plan::buf_mode(int tprec) const {
    if (fits_smem(tprec)) return 1;
    const size_t e = tprec == 1 ? sizeof(c32) : sizeof(c64);
    bool even = true;
    for (const FftTables* t : tabs) even &= t->N % 2 == 0;
    return even && blue_smem_bytes(maxN / 2, e) <= blue_smem_limit() ? 2 : 0;
}

// FP32 plans with refinement run the forward transform in double-float unless the caller asks
// for FP32: the refinement's residual spectrum is r_hat = ghat - C (eq. 2.3), as accurate as
// ghat, without further transforms.
int Plan::fwd_prec() const {
    if (prec == SFFT_FP32 && (p.refine || p.combine == SFFT_COMBINE_LSQ)) return p.dft == SFFT_DFT_FP32 ? 1 : 2;
    return prec;
}

int Plan::build_jobs() {
    const size_t e = esz();
    char* ghat_b = (char*)ghat;
    const int fp = fwd_prec();
    jobs_fwd.clear(); jobs_samp.clear();
    for (int l = 0; l < L; ++l) {
        const FftTables* t = tabs[l];
        const int64_t o = soff[l];
        // forward analyse: ghat = DFT(samples)/M (double-float: low words to ghat_lo)
        BlueJob a = make_blue_job(t, fp, 0, 1.0 / (double)M[l]);
        a.io_flags = 1; a.io_off = o; a.inst = 0;
        a.out = ghat_b + o * e;
        a.aux = ghat_lo ? (const void*)(ghat_lo + o) : nullptr;
        a.stat = stats + l;
        a.scratch = buf_mode(fp) ? nullptr : (char*)scratch + (size_t)l * maxN * sizeof(c64);
        jobs_fwd.push_back(a);
        // sampler: out (launch argument) = IDFT(C) + noise (launch argument), plan precision
        BlueJob sj = make_blue_job(t, prec, 1, 1.0);
        // FP32 plans scatter FP32 buckets into the first half of C (see k_scatter_terms)
        sj.in = prec ? (const void*)(reinterpret_cast<c32*>(C) + o) : (const void*)(C + o);
        sj.io_flags = 16 | 32; sj.io_off = o; sj.inst = 0; sj.lat = l;
        // a transform in one CTA's shared memory sums its buckets there (no global bucket pass)
        if (buf_mode(prec) == 1) sj.io_flags |= 64;
        sj.scratch = buf_mode(prec) ? nullptr : (char*)scratch + (size_t)l * maxN * sizeof(c64);
        jobs_samp.push_back(sj);
    }
    return SFFT_OK;
}

// The adjoint's inverse lattice transforms run in FP64 for every plan precision (their output, the
// sample cotangent, is rounded to the plan precision only at the end).  Built on the first backward
// call: the job list, a global work buffer when a length fits neither one CTA nor a two-CTA cluster
// in FP64, and for FP32 plans an FP64 output buffer.
int Plan::prepare_adjoint() {
    if (d_jobs_adj) return SFFT_OK;
    const int mode = buf_mode(0);
    void* scr = nullptr;
    if (mode == 0) SFFT_TRY(alloc(&scr, sizeof(c64) * (size_t)maxN * L));
    if (prec != SFFT_FP64) SFFT_TRY(alloc((void**)&adj_out, sizeof(c64) * (size_t)sumM));
    jobs_adj.clear();
    for (int l = 0; l < L; ++l) {
        // out (launch argument) = (1/M) IDFT(C) in FP64
        BlueJob aj = make_blue_job(tabs[l], 0, 1, 1.0 / (double)M[l]);
        aj.in = C + soff[l]; aj.io_flags = 4; aj.io_off = soff[l];
        aj.scratch = mode ? nullptr : (char*)scr + (size_t)l * maxN * sizeof(c64);
        jobs_adj.push_back(aj);
    }
    return upload_jobs(jobs_adj, &d_jobs_adj, &allocs);
}

// upload a job list into a device array (static lists: once at plan creation)
int upload_jobs(const std::vector<BlueJob>& v, BlueJob** dst, std::vector<void*>* owner) {
    SFFT_TRY(dmalloc((void**)dst, sizeof(BlueJob) * std::max<size_t>(1, v.size())));
    owner->push_back(*dst);
    SFFT_CU(cudaMemcpy(*dst, v.data(), sizeof(BlueJob) * v.size(), cudaMemcpyHostToDevice));
    return SFFT_OK;
}

// N_Gamma = max_t (max k_t - min k_t) (eq. 2.4) and max |k_t| of n candidate rows in the plan's layout
static int candidate_bounds(Plan* P, const void* cand, int64_t n, int64_t* NG_out, int64_t* kmax_out) {
    const int d = P->d;
    cudaStream_t st = P->st;
    if (!P->d_minmax) SFFT_TRY(P->alloc((void**)&P->d_minmax, sizeof(int) * 2 * kMaxD));
    int* dmn = P->d_minmax;
    int* dmx = P->d_minmax + kMaxD;
    std::vector<int> mn(d, INT32_MAX), mx(d, INT32_MIN);
    SFFT_CU(cudaMemcpyAsync(dmn, mn.data(), sizeof(int) * d, cudaMemcpyHostToDevice, st));
    SFFT_CU(cudaMemcpyAsync(dmx, mx.data(), sizeof(int) * d, cudaMemcpyHostToDevice, st));
    SFFT_TRY(launch_cand_stats(cand, P->p.cand_type == SFFT_CAND_I8, P->p.cand_ld, n, d, dmn, dmx, st));
    SFFT_CU(cudaMemcpyAsync(mn.data(), dmn, sizeof(int) * d, cudaMemcpyDeviceToHost, st));
    SFFT_CU(cudaMemcpyAsync(mx.data(), dmx, sizeof(int) * d, cudaMemcpyDeviceToHost, st));
    SFFT_CU(cudaStreamSynchronize(st));
    int64_t NG = 0, kmax = 0;
    for (int t = 0; t < d; ++t) {
        NG = std::max<int64_t>(NG, (int64_t)mx[t] - mn[t]);
        kmax = std::max<int64_t>(kmax, std::max<int64_t>(std::llabs(mn[t]), std::llabs(mx[t])));
    }
    *NG_out = NG;
    *kmax_out = kmax;
    return SFFT_OK;
}

int plan_create(Plan* P, int d, const void* cand, int64_t n, int64_t s, int Lin, const int64_t* Min,
                const int64_t* zin, const sfft_params* pin, cudaStream_t st) {
    sfft_params p;
    if (pin) p = *pin; else sfft_params_default(&p);
    SFFT_CHECK(d >= 1 && d <= kMaxD, SFFT_EINVAL, "d=%d must be in [1, %d]", d, kMaxD);
    SFFT_CHECK(cand != nullptr && n >= 1, SFFT_EINVAL, "empty candidate set");
    SFFT_CHECK(n < ((int64_t)1 << 31), SFFT_EINVAL, "|Gamma| must be < 2^31");
    SFFT_CHECK(s >= 1, SFFT_EINVAL, "s must be >= 1");
    SFFT_CHECK(p.nu > 0 && p.nu <= 0.5, SFFT_EINVAL, "nu must be in (0, 1/2]");
    SFFT_CHECK(p.c > 1.0 / p.nu && p.c > 2.0, SFFT_EINVAL, "c must exceed max(2, 1/nu)");
    SFFT_CHECK(p.delta > 0 && p.delta < 1, SFFT_EINVAL, "delta must be in (0, 1)");
    SFFT_CHECK(p.precision == SFFT_FP64 || p.precision == SFFT_FP32, SFFT_EINVAL, "bad precision");
    SFFT_CHECK(p.refine == 0 || p.refine == 1, SFFT_EINVAL, "refine must be 0 or 1");
    SFFT_CHECK(p.combine == SFFT_COMBINE_MEDIAN || p.combine == SFFT_COMBINE_HYBRID || p.combine == SFFT_COMBINE_LSQ,
               SFFT_EINVAL, "bad combine mode");
    SFFT_CHECK(p.cand_type == SFFT_CAND_I32 || p.cand_type == SFFT_CAND_I8, SFFT_EINVAL, "bad cand_type");
    SFFT_CHECK(p.dft == SFFT_DFT_DF64 || p.dft == SFFT_DFT_FP32, SFFT_EINVAL, "bad dft arithmetic %d", p.dft);
    SFFT_CHECK(p.rank_bits >= 0 && p.rank_bits <= 52, SFFT_EINVAL, "rank_bits must be in [0, 52]");
    if (p.cand_type == SFFT_CAND_I32) {
        SFFT_CHECK(p.cand_ld == 0 || p.cand_ld == d, SFFT_EINVAL, "int32 candidate rows are dense (cand_ld 0 or d)");
        // the hash kernels read a row as int4 words (d % 4 == 0) or int2 words (d % 2 == 0)
        const uintptr_t al = d % 4 == 0 ? 16 : d % 2 == 0 ? 8 : 4;
        SFFT_CHECK((uintptr_t)cand % al == 0, SFFT_EINVAL,
                   "int32 candidate rows of d = %d must start %d-byte aligned", d, (int)al);
        p.cand_ld = d;
    } else {
        SFFT_CHECK(p.cand_ld >= d, SFFT_EINVAL, "int8 candidate rows need a stride cand_ld >= d (got %d)", p.cand_ld);
        SFFT_CHECK(((uintptr_t)cand & 3) == 0, SFFT_EINVAL, "int8 candidate rows must start 4-byte aligned");
    }
    P->d = d; P->cand = cand; P->n = n; P->s = s; P->p = p; P->prec = p.precision; P->st = st;
    // ---- L and M (Corollary 2.6 / eq. 4.2 / fallback)
    int L = Lin > 0 ? Lin : L_rule(p.L_rule, n, p.delta, p.c);
    SFFT_CHECK(L >= 1 && L <= kMaxL, SFFT_EINVAL, "L=%d must be in [1, %d]", L, kMaxL);
    SFFT_CHECK(L % 2 == 1, SFFT_EINVAL, "L=%d must be odd (component-wise median, Algorithm 2)", L);
    P->L = L;
    P->M.resize(L);
    if (Min) {
        for (int l = 0; l < L; ++l) P->M[l] = Min[l];
    } else if (p.L_rule == SFFT_L_FALLBACK) {
        int64_t q = next_prime_above((double)(4 * s - 1));
        for (int l = 0; l < L; ++l) { P->M[l] = q; q = next_prime_above((double)q); }
    } else {
        int64_t q = next_prime_above(p.c * (double)s);
        for (int l = 0; l < L; ++l) P->M[l] = q;
    }
    for (int l = 0; l < L; ++l) {
        SFFT_CHECK(P->M[l] >= 2 && P->M[l] < (1 << 27), SFFT_EINVAL, "M_%d=%lld out of range", l, (long long)P->M[l]);
        SFFT_CHECK(is_prime(P->M[l]), SFFT_ENOTPRIME, "M_%d=%lld is not prime", l, (long long)P->M[l]);
    }
    // ---- candidate bounds: N_Gamma (eq. 2.4) and max |k_t|
    SFFT_TRY(candidate_bounds(P, cand, n, &P->N_gamma, &P->kmax));
    for (int l = 0; l < L; ++l) {
        SFFT_CHECK(P->M[l] > P->N_gamma, SFFT_EALIAS,
                   "M_%d=%lld <= N_Gamma=%lld: |Gamma mod M| = |Gamma| is not guaranteed (pass an admissible M)", l,
                   (long long)P->M[l], (long long)P->N_gamma);
        const double bound = (double)d * (double)P->kmax * (double)(P->M[l] - 1);
        SFFT_CHECK(bound + (double)P->M[l] < 2147483647.0, SFFT_EOVERFLOW,
                   "d*max|k|*(M-1) = %.0f does not fit the exact 32-bit hash", bound);
    }
    // ---- generating vectors
    P->z.resize((size_t)L * d);
    for (int l = 0; l < L; ++l)
        for (int t = 0; t < d; ++t) {
            int64_t v;
            if (zin) v = zin[(size_t)l * d + t];
            else v = (int64_t)(philox_word0(p.seed, (uint64_t)t, (uint64_t)l, 0, 0) % (uint64_t)P->M[l]);
            SFFT_CHECK(v >= 0 && v < P->M[l], SFFT_EINVAL, "z[%d][%d]=%lld outside [0, M)", l, t, (long long)v);
            P->z[(size_t)l * d + t] = v;
        }
    // ---- offsets and tables
    P->soff.assign(L + 1, 0);
    P->boff.assign(L, 0);
    int64_t words = 0;
    for (int l = 0; l < L; ++l) {
        P->soff[l + 1] = P->soff[l] + P->M[l];
        P->boff[l] = (int32_t)words;
        words += (P->M[l] + 31) / 32;
    }
    P->nwords = (int)words;
    P->sumM = P->soff[L];
    P->maxN = 0;
    for (int l = 0; l < L; ++l) {
        FftTables* t = nullptr;
        SFFT_TRY(tables_acquire(P->M[l], &t));
        P->tabs.push_back(t);
        P->maxN = std::max<int>(P->maxN, (int)t->N);
    }
    // ---- workspace
    const int64_t cap = std::min<int64_t>(n, p.detect_cap > 0 ? p.detect_cap : std::max<int64_t>(4 * s + 4096, 16384));
    P->cap = cap;
    P->cap_alloc = cap;
    P->n_alloc = n;
    const size_t e = P->esz();
    std::vector<int32_t> z32(P->z.begin(), P->z.end()), M32(P->M.begin(), P->M.end());
    std::vector<uint32_t> mu(L), offk(L);
    for (int l = 0; l < L; ++l) {
        mu[l] = (uint32_t)((1ull << 32) / (uint64_t)P->M[l]);
        const double bound = (double)d * (double)P->kmax * (double)(P->M[l] - 1);
        offk[l] = (uint32_t)(P->M[l] * ((int64_t)ceil(bound / (double)P->M[l]) + 1));
    }
    int32_t *dz, *dM, *dboff;
    uint32_t *dmu, *doffk;
    int64_t* dsoff;
    SFFT_TRY(P->alloc((void**)&dz, sizeof(int32_t) * z32.size()));
    P->d_z = dz;
    SFFT_TRY(P->alloc((void**)&dM, sizeof(int32_t) * L));
    SFFT_TRY(P->alloc((void**)&dmu, sizeof(uint32_t) * L));
    SFFT_TRY(P->alloc((void**)&doffk, sizeof(uint32_t) * L));
    SFFT_TRY(P->alloc((void**)&dsoff, sizeof(int64_t) * (L + 1)));
    SFFT_TRY(P->alloc((void**)&dboff, sizeof(int32_t) * L));
    SFFT_CU(cudaMemcpy(dz, z32.data(), sizeof(int32_t) * z32.size(), cudaMemcpyHostToDevice));
    SFFT_CU(cudaMemcpy(dM, M32.data(), sizeof(int32_t) * L, cudaMemcpyHostToDevice));
    SFFT_CU(cudaMemcpy(dmu, mu.data(), sizeof(uint32_t) * L, cudaMemcpyHostToDevice));
    SFFT_CU(cudaMemcpy(doffk, offk.data(), sizeof(uint32_t) * L, cudaMemcpyHostToDevice));
    SFFT_CU(cudaMemcpy(dsoff, P->soff.data(), sizeof(int64_t) * (L + 1), cudaMemcpyHostToDevice));
    SFFT_CU(cudaMemcpy(dboff, P->boff.data(), sizeof(int32_t) * L, cudaMemcpyHostToDevice));
    SFFT_TRY(P->alloc((void**)&P->nzbits, sizeof(uint32_t) * words));
    SFFT_TRY(P->alloc(&P->ghat, e * P->sumM));
    SFFT_TRY(P->alloc((void**)&P->stats, sizeof(LatStats) * L));
    SFFT_TRY(P->alloc((void**)&P->detbits, sizeof(uint32_t) * ((n + 31) / 32)));
    SFFT_TRY(P->alloc((void**)&P->det, sizeof(int64_t) * cap));
    SFFT_TRY(P->alloc((void**)&P->cnt, sizeof(int64_t) * kCntWords));
    SFFT_TRY(P->alloc((void**)&P->coef, sizeof(c64) * cap));
    SFFT_TRY(P->alloc((void**)&P->H, sizeof(int32_t) * cap * L));
    SFFT_TRY(P->alloc((void**)&P->sel, 2 * cap));
    if (p.refine) SFFT_TRY(P->alloc((void**)&P->rsel, 2 * cap));
    SFFT_TRY(P->alloc((void**)&P->adj_w, sizeof(c64) * cap));
    SFFT_TRY(P->alloc((void**)&P->outpos, sizeof(int32_t) * cap));
    SFFT_TRY(P->alloc((void**)&P->coll, sizeof(int32_t) * P->sumM));
    SFFT_TRY(P->alloc((void**)&P->C, sizeof(c64) * P->sumM));
    if (P->fwd_prec() == 2) SFFT_TRY(P->alloc((void**)&P->ghat_lo, sizeof(c32) * P->sumM));
    if (p.combine == SFFT_COMBINE_LSQ) {
        SFFT_TRY(P->alloc((void**)&P->lsq_work, sizeof(c64) * 3 * cap));
        SFFT_TRY(P->alloc((void**)&P->lsq_next, sizeof(int32_t) * cap * L));
        P->lsq_pair_cap = 16 * cap;  // off-diagonal entries; more (many-way collisions): bucket matvec
        SFFT_TRY(P->alloc(&P->lsq_pairs, 16 * (size_t)P->lsq_pair_cap));
    }
    if (!P->buf_mode(P->fwd_prec()) || !P->buf_mode(P->prec))
        SFFT_TRY(P->alloc(&P->scratch, sizeof(c64) * (size_t)P->maxN * L));
    SFFT_TRY(P->alloc((void**)&P->sop_a, sizeof(double) * 2 * 16 * 129));
    SFFT_TRY(P->alloc((void**)&P->sop_tri, sizeof(int32_t) * 3 * 16));
    // ---- instance descriptor
    SFFT_CU(cudaMallocHost((void**)&P->h_inst, sizeof(InstDesc)));
    SFFT_CU(cudaMallocHost((void**)&P->h_cnt, sizeof(int64_t) * 8));
    InstDesc& I = *P->h_inst;
    memset(&I, 0, sizeof I);
    I.d = d; I.L = L; I.prec = P->prec; I.combine = p.combine; I.nwords = (int)words;
    I.need = (int)ceil(p.nu * L - 1e-9);
    I.n = n; I.cap = cap; I.s_tilde = p.s_tilde;
    I.tau_abs = p.tau_abs; I.tau_rel = p.tau_rel; I.theta_abs = p.theta_abs; I.theta_rel = p.theta_rel;
    I.rank_bits = p.rank_bits;
    I.cand = cand; I.cand_i8 = p.cand_type == SFFT_CAND_I8; I.cand_ld = p.cand_ld; I.z = dz; I.Ml = dM; I.mu = dmu; I.offk = doffk; I.soff = dsoff; I.boff = dboff;
    I.nzbits = P->nzbits; I.ghat = P->ghat; I.stats = P->stats; I.detbits = P->detbits; I.det = P->det;
    I.cnt = P->cnt; I.coef = P->coef; I.H = P->H; I.sel = P->sel; I.coll = P->coll; I.C = P->C;
    I.rsel = P->rsel; I.adj_w = P->adj_w;
    I.ghat_lo = P->ghat_lo; I.lsq_work = P->lsq_work; I.outpos = P->outpos;
    I.lsq_next = P->lsq_next; I.lsq_pairs = P->lsq_pairs; I.lsq_pair_cap = P->lsq_pair_cap;
    SFFT_CU(cudaEventCreateWithFlags(&P->io_ev, cudaEventDisableTiming));
    SFFT_TRY(P->alloc((void**)&P->d_inst, sizeof(InstDesc)));
    SFFT_CU(cudaMemcpy(P->d_inst, &I, sizeof(InstDesc), cudaMemcpyHostToDevice));
    // ---- lattice descriptors and static transform jobs
    std::vector<LatDesc> lats(L);
    for (int l = 0; l < L; ++l) {
        lats[l] = LatDesc{0, l, (int)P->M[l], (int)P->tabs[l]->N, P->soff[l], P->boff[l], 0,
                          (const double*)P->tabs[l]->dft64, P->tabs[l]->dftdf};
    }
    SFFT_TRY(P->alloc((void**)&P->d_lats, sizeof(LatDesc) * L));
    SFFT_CU(cudaMemcpy(P->d_lats, lats.data(), sizeof(LatDesc) * L, cudaMemcpyHostToDevice));
    SFFT_TRY(P->build_jobs());
    SFFT_TRY(upload_jobs(P->jobs_fwd, &P->d_jobs_fwd, &P->allocs));
    SFFT_TRY(upload_jobs(P->jobs_samp, &P->d_jobs_samp, &P->allocs));
    // hash-count kernel choice; lattices split into groups whose bitmaps fit shared memory
    int64_t maxM = *std::max_element(P->M.begin(), P->M.end());
    P->packed = P->kmax <= 127 && maxM < 65536;  // int8 k, int16 z in the symmetric range
    const size_t kHashSmem = 200 * 1024;
    for (int l0 = 0; l0 < L;) {
        int l1 = l0 + 1;
        while (l1 < L) {
            int64_t wds = (l1 + 1 < L ? P->boff[l1 + 1] : words) - P->boff[l0];
            if (hash_smem_bytes(d, l1 + 1 - l0, wds, P->packed) > kHashSmem) break;
            ++l1;
        }
        int64_t wds = (l1 < L ? P->boff[l1] : words) - P->boff[l0];
        size_t sm = hash_smem_bytes(d, l1 - l0, wds, P->packed);
        SFFT_CHECK(sm <= 220 * 1024, SFFT_EINVAL, "the bitmap of lattice %d alone does not fit shared memory", l0);
        P->hgroups.push_back({l0, l1});
        P->hsmem.push_back(sm);
        l0 = l1;
    }
    P->hash_smem = *std::max_element(P->hsmem.begin(), P->hsmem.end());
    // tensor-core inner products: exact while every |k.z| (and partial sum) is below 2^24, the
    // bucket bit indices below 2^22, d <= 16 (2d <= 32) and L <= 64 (tensor-memory columns)
    // (int8 rows are read as whole words there: strides of a multiple of 4 bytes)
    if (P->packed && d <= 16 && L <= 64 && P->hgroups.size() == 1 && P->p.cand_ld % 4 == 0 &&
        maxM <= 32768 && (double)d * (double)P->kmax * (double)(maxM - 1) < 16777216.0 && words * 32 < (1 << 22)) {
        P->tc_smem = hash_tc_smem_bytes(L, words);
        P->hash_tc = P->tc_smem <= 220 * 1024;
    }
    if (P->hgroups.size() > 1) {
        SFFT_TRY(P->alloc((void**)&P->cnt8, (size_t)n));
        P->h_inst->cnt8 = P->cnt8;
        SFFT_CU(cudaMemcpy(P->d_inst, P->h_inst, sizeof(InstDesc), cudaMemcpyHostToDevice));
    }
    return SFFT_OK;
}

// ================================================================== the reconstruction stage sequence
// Runs every stage for `ninst` instances described by d_inst (all of precision prec).
static int mark(const PipeArgs& a, int stage, cudaStream_t st) {
    if (!a.timer) return SFFT_OK;
    SFFT_CU(cudaEventRecord(a.timer->ev[stage], st));
    a.timer->recorded[stage] = true;
    return SFFT_OK;
}

int run_pipeline(const PipeArgs& a, cudaStream_t st) {
    const int ni = a.ninst;
    // FP32 transforms: float buckets C for the refinement (their rounding is far below the
    // transform's error); the second half of a sharded reconstruction gets FP64 buckets
    const bool f32 = a.prec == 1 && a.fwd_prec == 1 && a.phase == 0;
    // a whole reconstruction with refinement zeroes C at the buckets of Itilde in the combine (the
    // least-squares combine uses C as scratch in between, so it keeps the full clear)
    const int zc = a.refine && a.phase == 0 && !a.lsq ? (f32 ? 2 : 1) : 0;
    if (a.timer)
        for (int i = 0; i <= ST_COUNT; ++i) a.timer->recorded[i] = false;
    if (a.phase != 2) {
        SFFT_TRY(mark(a, ST_CLEAR, st));
        SFFT_TRY(launch_clear(a.d_inst, ni, 1, a.hybrid, 0, st));
        // Algorithm 2: lattice DFTs (normalised by 1/M) + per-lattice statistics
        SFFT_TRY(mark(a, ST_FFT_FWD, st));
        for (const auto& f : a.fwd)
            SFFT_TRY(launch_bluestein(f.jobs, f.njobs, f.maxN, f.mode, a.fwd_prec, a.prec, a.prec, -1, EPI_ANALYZE,
                                      a.d_inst, st, nullptr, nullptr, f.threads, f.upair));
        // zero test with direct re-tests inside the guard band (Remark 2.3); unit roundoff of the
        // transform arithmetic (double-float: 2^-44, a bound with margin for its ~48-bit operations)
        SFFT_TRY(mark(a, ST_ZERO_TEST, st));
        const double u = a.fwd_prec == 1 ? 5.9604644775390625e-08 : a.fwd_prec == 2 ? 5.684341886080802e-14
                                                                                     : 1.1102230246251565e-16;
        SFFT_TRY(launch_zero_test(a.d_lats, a.nlat, a.d_inst, a.prec, 32.0 * u, st));
        // count rule over all candidates, ascending compaction of Itilde
        SFFT_TRY(mark(a, ST_HASH, st));
        for (const auto& h : a.hash)
            SFFT_TRY(launch_hash_count(a.d_inst + h.off, h.count, h.d, h.gx, h.smem, h.variant, h.l0, h.l1, h.mode, st));
        SFFT_TRY(mark(a, ST_COMPACT, st));
        SFFT_TRY(launch_compact(a.d_inst, ni, st));
        // hashes of Itilde, collision counts, median / hybrid combine
        // (the median combine forms the hashes itself; the hybrid one needs all collision counts first)
        SFFT_TRY(mark(a, ST_DET_HASH, st));
        if (a.hybrid) SFFT_TRY(launch_det_hashes(a.d_inst, ni, a.maxcap, st));
        SFFT_TRY(mark(a, ST_COMBINE, st));
        if (a.hybrid) SFFT_TRY(launch_collisions(a.d_inst, ni, st));
        SFFT_TRY(launch_combine(a.d_inst, ni, a.maxcap, a.prec, a.hybrid ? 0 : 3, st, zc));
        if (a.lsq) {  // Remark 2.8 least squares on the detected set, from the medians
            SFFT_TRY(mark(a, ST_LSQ, st));
            SFFT_TRY(launch_lsq(a.d_inst, ni, a.prec, st));
        }
        if (a.phase == 1) {  // a shard's part of C (FP64 buckets), summed over the shards by the caller
            SFFT_TRY(launch_clear(a.d_inst, ni, 0, 0, 1, st));
            SFFT_TRY(launch_scatter_coef(a.d_inst, ni, false, st));
            SFFT_TRY(mark(a, ST_COUNT, st));
            return SFFT_OK;
        }
    }
    if (a.refine) {
        if (a.phase == 0) {
            SFFT_TRY(mark(a, ST_SCATTER, st));
            if (!zc) SFFT_TRY(launch_clear(a.d_inst, ni, 0, 0, f32 ? 2 : 1, st));
            SFFT_TRY(launch_scatter_coef(a.d_inst, ni, f32, st));
        }
        // residual spectrum r_hat = ghat - C at the buckets of Itilde (eq. 2.3), median update
        SFFT_TRY(mark(a, ST_DELTA, st));
        SFFT_TRY(launch_combine(a.d_inst, ni, a.maxcap, a.prec, f32 ? 2 : 1, st));
    }
    // Algorithm 4: theta filter and top-s_tilde, ascending output
    SFFT_TRY(mark(a, ST_SELECT, st));
    SFFT_TRY(launch_select(a.d_inst, ni, st));
    SFFT_TRY(mark(a, ST_COUNT, st));
    return SFFT_OK;
}

// grid of the tensor-core hash kernel: resident CTAs per SM from shared memory, tiles of 128
int tc_grid(size_t smem, int64_t tiles, int count) {
    const int per_sm = std::max<int>(1, std::min<int>(4, (int)((228 * 1024) / (smem + 1024))));
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, ((int64_t)152 * per_sm + count - 1) / count));
}

int Plan::hash_grid() const {
    const int per_sm = hash_ctas_per_sm(hash_smem);
    const int64_t tile = hash_tile(packed, hash_smem), tiles = (n + tile - 1) / tile;
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)152 * per_sm));
}

PipeArgs Plan::pipe_args() {
    PipeArgs a;
    a.ninst = 1; a.d_inst = d_inst; a.d_lats = d_lats; a.nlat = L;
    a.prec = prec; a.fwd_prec = fwd_prec(); a.maxcap = cap;
    a.hybrid = p.combine == SFFT_COMBINE_HYBRID; a.refine = p.refine; a.lsq = p.combine == SFFT_COMBINE_LSQ;
    a.fwd.push_back(FftLaunch{d_jobs_fwd, L, maxN, buf_mode(fwd_prec())});
    a.fwd.back().upair = uniform_pair(jobs_fwd.data(), jobs_fwd.size());
    const int ng = (int)hgroups.size();
    for (int g = 0; g < ng; ++g) {
        HashGroup h;
        h.off = 0; h.count = 1; h.d = d; h.gx = h.gx0 = hash_grid(); h.smem = hsmem[g];
        h.variant = packed ? (diag_run ? 2 : 1) : 0;
        if (hash_tc && !diag_run) {  // per-candidate diagnostics come from the packed kernel
            h.tc_ok = true;
            h.tc_smem = tc_smem;
            h.tc_tiles = (n + 127) / 128;
            h.tc_gx0 = tc_grid(tc_smem, h.tc_tiles, 1);
        }
        h.l0 = hgroups[g].first;
        h.l1 = g + 1 < ng ? hgroups[g].second : -1;
        h.mode = (g == 0 ? 1 : 0) | (g + 1 == ng ? 2 : 0);
        a.hash.push_back(h);
    }
    return a;
}

}  // namespace sfft

using namespace sfft;

// ================================================================== C ABI
extern "C" {

void sfft_params_default(sfft_params* p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->c = 10.33;
    p->delta = 0.1;
    p->nu = 0.5;
    p->tau_abs = 0.0;
    p->tau_rel = 1e-10;
    p->theta_abs = 0.0;
    p->theta_rel = 0.0;
    p->s_tilde = 0;
    p->precision = SFFT_FP64;
    p->refine = 0;
    p->L_rule = SFFT_L_COR26;
    p->combine = SFFT_COMBINE_MEDIAN;
    p->seed = 0;
    p->detect_cap = 0;
}

const char* sfft_last_error(void) { return get_error(); }

uint64_t sfft_philox4x64_word0(uint64_t key0, uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3) {
    return philox_word0(key0, c0, c1, c2, c3);
}

int64_t sfft_next_prime_above(double x) { return next_prime_above(x); }

int sfft_L_rule(int rule, int64_t n_cand, double delta, double c) {
    if (n_cand < 1 || !(delta > 0 && delta < 1) || !(c > 2)) return -1;
    return L_rule(rule, n_cand, delta, c);
}

int sfft_plan_create(sfft_plan** out, int d, const void* cand, int64_t n_cand, int64_t s, int L, const int64_t* M,
                     const int64_t* z, const sfft_params* p, void* stream) {
    if (!out) { set_error("out is NULL"); return SFFT_EINVAL; }
    *out = nullptr;
    Plan* P = new Plan();
    int rc = plan_create(P, d, cand, n_cand, s, L, M, z, p, (cudaStream_t)stream);
    if (rc != SFFT_OK) {
        P->release();
        delete P;
        return rc;
    }
    *out = reinterpret_cast<sfft_plan*>(P);
    return SFFT_OK;
}

void sfft_plan_destroy(sfft_plan* plan) {
    if (!plan) return;
    Plan* P = reinterpret_cast<Plan*>(plan);
    cudaStreamSynchronize(P->st);
    P->release();
    delete P;
}

int sfft_plan_set_candidates(sfft_plan* plan, const void* cand, int64_t n_cand) {
    if (!plan || !cand) { set_error("null argument"); return SFFT_EINVAL; }
    Plan* P = reinterpret_cast<Plan*>(plan);
    SFFT_CHECK(n_cand >= 1 && n_cand <= P->n_alloc, SFFT_EINVAL,
               "n_cand = %lld must be in [1, %lld] (the plan's workspace size)", (long long)n_cand,
               (long long)P->n_alloc);
    const int d = P->d;
    if (P->p.cand_type == SFFT_CAND_I32) {
        const uintptr_t al = d % 4 == 0 ? 16 : d % 2 == 0 ? 8 : 4;
        SFFT_CHECK((uintptr_t)cand % al == 0, SFFT_EINVAL,
                   "int32 candidate rows of d = %d must start %d-byte aligned", d, (int)al);
    } else {
        SFFT_CHECK(((uintptr_t)cand & 3) == 0, SFFT_EINVAL, "int8 candidate rows must start 4-byte aligned");
    }
    SFFT_TRY(P->io_begin());
    int64_t NG = 0, kmax = 0;
    SFFT_TRY(candidate_bounds(P, cand, n_cand, &NG, &kmax));
    // the hash offsets, the kernel choice and the overflow check were derived from the plan's bound
    // on |k_t|: a set within that bound keeps them valid
    SFFT_CHECK(kmax <= P->kmax, SFFT_EINVAL,
               "max |k_t| = %lld exceeds the plan's %lld (create a new plan for this candidate set)",
               (long long)kmax, (long long)P->kmax);
    for (int l = 0; l < P->L; ++l)
        SFFT_CHECK(P->M[l] > NG, SFFT_EALIAS, "M_%d=%lld <= N_Gamma=%lld of the new candidate set", l,
                   (long long)P->M[l], (long long)NG);
    P->cand = cand;
    P->n = n_cand;
    P->N_gamma = NG;
    P->cap = std::min<int64_t>(n_cand, P->cap_alloc);
    InstDesc& I = *P->h_inst;
    I.cand = cand;
    I.n = n_cand;
    I.cap = P->cap;
    SFFT_TRY(P->io_upload());
    P->have_forward = false;
    return SFFT_OK;
}

int sfft_plan_set_generators(sfft_plan* plan, const int64_t* z) {
    if (!plan || !z) { set_error("null argument"); return SFFT_EINVAL; }
    Plan* P = reinterpret_cast<Plan*>(plan);
    const int L = P->L, d = P->d;
    std::vector<int32_t> z32((size_t)L * d);
    for (int l = 0; l < L; ++l)
        for (int t = 0; t < d; ++t) {
            const int64_t v = z[(size_t)l * d + t];
            SFFT_CHECK(v >= 0 && v < P->M[l], SFFT_EINVAL, "z[%d][%d]=%lld outside [0, M)", l, t, (long long)v);
            z32[(size_t)l * d + t] = (int32_t)v;
        }
    // the hash offsets depend on M and the bound on |k_t| only, the FFT tables on M only
    SFFT_CU(cudaStreamSynchronize(P->st));  // no launch of this plan may still read the old vectors
    SFFT_CU(cudaMemcpy(P->d_z, z32.data(), sizeof(int32_t) * z32.size(), cudaMemcpyHostToDevice));
    for (size_t i = 0; i < z32.size(); ++i) P->z[i] = z[i];
    P->have_forward = false;
    return SFFT_OK;
}

int sfft_plan_info(const sfft_plan* plan, int* L, int64_t* M, int64_t* z, int64_t* n_samples) {
    if (!plan) { set_error("plan is NULL"); return SFFT_EINVAL; }
    const Plan* P = reinterpret_cast<const Plan*>(plan);
    if (L) *L = P->L;
    if (M) for (int l = 0; l < P->L; ++l) M[l] = P->M[l];
    if (z) for (size_t i = 0; i < P->z.size(); ++i) z[i] = P->z[i];
    if (n_samples) *n_samples = P->sumM;
    return SFFT_OK;
}

int sfft_sample_points(const sfft_plan* plan, int32_t* numer_out, double* x_out, int64_t* offsets) {
    if (!plan) { set_error("plan is NULL"); return SFFT_EINVAL; }
    const Plan* P = reinterpret_cast<const Plan*>(plan);
    if (offsets) for (int l = 0; l <= P->L; ++l) offsets[l] = P->soff[l];
    if (numer_out || x_out) {
        SFFT_TRY(launch_points(P->d_inst, numer_out, x_out, P->sumM * P->d, P->st));
        SFFT_CU(cudaStreamSynchronize(P->st));
    }
    return SFFT_OK;
}

int sfft_reconstruct(sfft_plan* plan, const void* samples, int64_t* supp_out, double* coef_out, int64_t cap,
                     int64_t* n_out, sfft_diag* diag) {
    if (!plan || !samples || (cap > 0 && (!supp_out || !coef_out))) {
        set_error("sfft_reconstruct: null argument");
        return SFFT_EINVAL;
    }
    Plan* P = reinterpret_cast<Plan*>(plan);
    SFFT_TRY(P->io_begin());
    InstDesc& I = *P->h_inst;
    I.samples = samples;
    I.supp_out = supp_out;
    I.coef_out = reinterpret_cast<c64*>(coef_out);
    I.out_cap = cap;
    I.dcounts = diag ? diag->counts : nullptr;
    I.dhashes = diag ? diag->hashes : nullptr;
    I.key_out = nullptr;
    cudaStream_t st = P->st;
    SFFT_TRY(P->io_upload());
    P->shard_open = false;
    P->diag_run = diag && (diag->counts || diag->hashes);
    SFFT_TRY(run_pipeline(P->pipe_args(), st));
    SFFT_CU(cudaMemcpyAsync(P->h_cnt, P->cnt, sizeof(int64_t) * 8, cudaMemcpyDeviceToHost, st));
    if (diag) {
        const int64_t nd_cap = P->cap;
        if (diag->detected) SFFT_CU(cudaMemcpyAsync(diag->detected, P->det, sizeof(int64_t) * nd_cap, cudaMemcpyDeviceToDevice, st));
        if (diag->pcheck) SFFT_CU(cudaMemcpyAsync(diag->pcheck, P->coef, sizeof(c64) * nd_cap, cudaMemcpyDeviceToDevice, st));
        if (diag->ghat) SFFT_TRY(launch_to_c64(P->ghat, P->prec, reinterpret_cast<c64*>(diag->ghat), P->sumM, st));
        if (diag->collisions) {
            if (I.combine != SFFT_COMBINE_HYBRID) {  // the combine did not need them: count over Itilde now
                SFFT_CU(cudaMemsetAsync(P->coll, 0, sizeof(int32_t) * P->sumM, st));
                SFFT_TRY(launch_collisions(P->d_inst, 1, st));
            }
            SFFT_CU(cudaMemcpyAsync(diag->collisions, P->coll, sizeof(int32_t) * P->sumM, cudaMemcpyDeviceToDevice, st));
        }
        if (diag->tau) {
            std::vector<LatStats> S(P->L);
            SFFT_CU(cudaMemcpyAsync(S.data(), P->stats, sizeof(LatStats) * P->L, cudaMemcpyDeviceToHost, st));
            SFFT_CU(cudaStreamSynchronize(st));
            std::vector<double> tau(P->L);
            for (int l = 0; l < P->L; ++l) tau[l] = S[l].tau;
            SFFT_CU(cudaMemcpy(diag->tau, tau.data(), sizeof(double) * P->L, cudaMemcpyHostToDevice));
        }
    }
    SFFT_CU(cudaStreamSynchronize(st));
    const int64_t* c = P->h_cnt;
    if (diag) {
        diag->n_detected = c[0];
        diag->n_guard = c[2];
        diag->lsq_iters = c[4];
    }
    if (n_out) *n_out = c[1];
    P->have_forward = true;
    P->last_nout = c[1];
    if (c[3] & ERR_GUARD_CAP) {
        set_error("more than 1024 buckets of one lattice lie inside the FP64 guard band around tau: the zero-test "
                  "threshold is below what the working precision resolves (raise tau or use an FP64 plan)");
        return SFFT_ECAPACITY;
    }
    if (c[3] & ERR_DET_CAP) { set_error("|Itilde| = %lld exceeds detect_cap = %lld", (long long)c[0], (long long)P->cap); return SFFT_ECAPACITY; }
    if (c[3] & ERR_OUT_CAP) { set_error("%lld selected frequencies exceed cap = %lld", (long long)c[1], (long long)cap); return SFFT_ECAPACITY; }
    return SFFT_OK;
}

static int read_counts(Plan* P) {
    SFFT_CU(cudaMemcpyAsync(P->h_cnt, P->cnt, sizeof(int64_t) * 8, cudaMemcpyDeviceToHost, P->st));
    SFFT_CU(cudaStreamSynchronize(P->st));
    const int64_t* c = P->h_cnt;
    if (c[3] & ERR_GUARD_CAP) {
        set_error("more than 1024 buckets of one lattice lie inside the FP64 guard band around tau");
        return SFFT_ECAPACITY;
    }
    if (c[3] & ERR_DET_CAP) { set_error("|Itilde| = %lld exceeds detect_cap = %lld", (long long)c[0], (long long)P->cap); return SFFT_ECAPACITY; }
    return SFFT_OK;
}

int sfft_reconstruct_shard_begin(sfft_plan* plan, const void* samples, double* C_out, int64_t* n_detected) {
    if (!plan || !samples || !C_out) { set_error("null argument"); return SFFT_EINVAL; }
    Plan* P = reinterpret_cast<Plan*>(plan);
    SFFT_CHECK(P->p.combine == SFFT_COMBINE_MEDIAN, SFFT_EINVAL, "sharded reconstructions use the median combine");
    SFFT_CHECK(P->p.theta_rel == 0.0, SFFT_EINVAL,
               "sharded reconstructions need an absolute theta (theta_rel = 0: the largest modulus is global)");
    SFFT_TRY(P->io_begin());
    InstDesc& I = *P->h_inst;
    I.samples = samples;
    I.supp_out = nullptr;
    I.coef_out = nullptr;
    I.key_out = nullptr;
    I.out_cap = 0;
    I.dcounts = nullptr;
    I.dhashes = nullptr;
    SFFT_TRY(P->io_upload());
    P->diag_run = false;
    PipeArgs a = P->pipe_args();
    a.phase = 1;
    SFFT_TRY(run_pipeline(a, P->st));
    SFFT_CU(cudaMemcpyAsync(C_out, P->C, sizeof(c64) * P->sumM, cudaMemcpyDeviceToDevice, P->st));
    SFFT_TRY(read_counts(P));
    if (n_detected) *n_detected = P->h_cnt[0];
    P->have_forward = false;
    P->shard_open = true;
    return SFFT_OK;
}

int sfft_reconstruct_shard_end(sfft_plan* plan, const double* C_sum, int64_t* supp_out, double* coef_out,
                               uint64_t* keys_out, int64_t cap, int64_t* n_out) {
    if (!plan || !C_sum || (cap > 0 && (!supp_out || !coef_out))) { set_error("null argument"); return SFFT_EINVAL; }
    Plan* P = reinterpret_cast<Plan*>(plan);
    SFFT_CHECK(P->shard_open, SFFT_ESTATE, "sfft_reconstruct_shard_end without sfft_reconstruct_shard_begin");
    P->shard_open = false;
    SFFT_TRY(P->io_begin());
    InstDesc& I = *P->h_inst;
    I.supp_out = supp_out;
    I.coef_out = reinterpret_cast<c64*>(coef_out);
    I.key_out = keys_out;
    I.out_cap = cap;
    SFFT_TRY(P->io_upload());
    SFFT_CU(cudaMemcpyAsync(P->C, C_sum, sizeof(c64) * P->sumM, cudaMemcpyDeviceToDevice, P->st));
    PipeArgs a = P->pipe_args();
    a.phase = 2;
    SFFT_TRY(run_pipeline(a, P->st));
    SFFT_TRY(read_counts(P));
    if (n_out) *n_out = P->h_cnt[1];
    if (P->h_cnt[3] & ERR_OUT_CAP) {
        set_error("%lld selected frequencies exceed cap = %lld", (long long)P->h_cnt[1], (long long)cap);
        return SFFT_ECAPACITY;
    }
    return SFFT_OK;
}

int sfft_reconstruct_backward(sfft_plan* plan, const double* dcoef, void* dsamples) {
    if (!plan || !dsamples) { set_error("null argument"); return SFFT_EINVAL; }
    Plan* P = reinterpret_cast<Plan*>(plan);
    SFFT_CHECK(P->have_forward, SFFT_ESTATE, "sfft_reconstruct_backward before sfft_reconstruct");
    SFFT_CHECK(P->p.combine == SFFT_COMBINE_MEDIAN, SFFT_ESTATE, "the adjoint is defined for the median combine");
    SFFT_TRY(P->prepare_adjoint());
    cudaStream_t st = P->st;
    SFFT_CU(cudaMemsetAsync(P->C, 0, sizeof(c64) * P->sumM, st));
    SFFT_CU(cudaMemsetAsync(P->adj_w, 0, sizeof(c64) * P->cap, st));
    SFFT_TRY(launch_adjoint_buckets(P->d_inst, P->last_nout > 0 ? reinterpret_cast<const c64*>(dcoef) : nullptr,
                                    P->p.refine != 0, P->cap, st));
    // dsamples = A^H gbar with (A^H g)_j = (1/M) sum_h g_h exp(+2 pi i j h / M), in FP64
    void* out = P->prec == SFFT_FP64 ? dsamples : (void*)P->adj_out;
    SFFT_TRY(launch_bluestein(P->d_jobs_adj, P->L, P->maxN, P->buf_mode(0), 0, 0, 0, +1, EPI_PLAIN, P->d_inst, st, out,
                              nullptr));
    if (P->prec != SFFT_FP64)
        SFFT_TRY(launch_c64_to_c32(P->adj_out, reinterpret_cast<c32*>(dsamples), P->sumM, st));
    SFFT_CU(cudaStreamSynchronize(st));
    return SFFT_OK;
}

int sfft_sample_sparse_poly(const sfft_plan* plan, const int32_t* kvec, const double* coef, int64_t n_terms,
                            const void* noise, void* samples_out) {
    if (!plan || !samples_out || n_terms < 0 || (n_terms > 0 && (!kvec || !coef))) {
        set_error("null argument");
        return SFFT_EINVAL;
    }
    Plan* P = const_cast<Plan*>(reinterpret_cast<const Plan*>(plan));
    cudaStream_t st = P->st;
    SFFT_TRY(P->io_begin());
    InstDesc& I = *P->h_inst;
    I.samp_kvec = kvec;
    I.samp_coef = reinterpret_cast<const c64*>(coef);
    I.samp_nterms = n_terms;
    I.samp_out = samples_out;
    I.samp_noise = noise;
    SFFT_TRY(P->io_upload());
    // buckets in the plan precision (eq. 2.3), inverse lattice DFTs, noise; transforms in shared
    // memory sum their own buckets
    if (P->buf_mode(P->prec) != 1) {
        SFFT_TRY(launch_clear(P->d_inst, 1, 0, 0, P->prec ? 2 : 1, st));
        if (n_terms > 0) SFFT_TRY(launch_scatter_terms(P->d_inst, 1, n_terms * P->L, st));
    }
    SFFT_TRY(launch_bluestein(P->d_jobs_samp, P->L, P->maxN, P->buf_mode(P->prec), P->prec, P->prec, P->prec, +1,
                              EPI_ADDNOISE, P->d_inst, st, nullptr, nullptr, 0,
                              uniform_pair(P->jobs_samp.data(), P->jobs_samp.size())));
    return SFFT_OK;
}

static int sop_prepare(Plan* P, const int32_t* triples, const double* theta, int n_terms, int K, double width) {
    SFFT_CHECK(triples && theta && n_terms >= 1 && n_terms <= 16 && K >= 0 && K <= 128 && width > 0, SFFT_EINVAL,
               "sum-of-products: need 1 <= n_terms <= 16, 0 <= K <= 128, width > 0");
    for (int i = 0; i < 3 * n_terms; ++i)
        SFFT_CHECK(triples[i] >= 0 && triples[i] < P->d, SFFT_EINVAL, "triple entry %d outside [0, d)", triples[i]);
    SFFT_CU(cudaMemcpyAsync(P->sop_tri, triples, sizeof(int32_t) * 3 * n_terms, cudaMemcpyHostToDevice, P->st));
    return launch_sop_coefs(theta, n_terms, K, width, P->sop_a, P->sop_a + 16 * 129, P->st);
}

int sfft_sample_sop(const sfft_plan* plan, const int32_t* triples, const double* theta, int n_terms, int K, double width,
                    void* samples_out) {
    if (!plan || !samples_out) { set_error("null argument"); return SFFT_EINVAL; }
    Plan* P = const_cast<Plan*>(reinterpret_cast<const Plan*>(plan));
    SFFT_TRY(sop_prepare(P, triples, theta, n_terms, K, width));
    SFFT_TRY(launch_sop_sample(P->d_inst, P->sop_tri, n_terms, K, P->sop_a, samples_out, P->prec, P->st));
    return SFFT_OK;
}

int sfft_sample_sop_backward(const sfft_plan* plan, const int32_t* triples, const double* theta, int n_terms, int K,
                             double width, const void* dsamples, double* dtheta) {
    if (!plan || !dsamples || !dtheta) { set_error("null argument"); return SFFT_EINVAL; }
    Plan* P = const_cast<Plan*>(reinterpret_cast<const Plan*>(plan));
    SFFT_TRY(sop_prepare(P, triples, theta, n_terms, K, width));
    SFFT_CU(cudaMemsetAsync(dtheta, 0, sizeof(double) * n_terms, P->st));
    SFFT_TRY(launch_sop_backward(P->d_inst, P->sop_tri, n_terms, K, P->sop_a, P->sop_a + 16 * 129, dsamples, P->prec,
                                 dtheta, P->st));
    SFFT_CU(cudaStreamSynchronize(P->st));
    return SFFT_OK;
}

}  // extern "C"
