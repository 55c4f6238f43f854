// Dimension-incremental sparse FFT (Algorithm 3) with Algorithm 4 (plus one refinement step)
// in the role of Algorithm A, on a box candidate set Gamma = prod_t [lo_t, hi_t].
//   Step 1: for every coordinate t, r random node tails; K_t-point DFTs along coordinate t
//           (Bluestein kernel, FP64); keep the s_local largest projections of modulus >= theta.
//   Step 2: for t = 2..d: J_t = I^(1..t-1) x I^(t) (device pairing), t-dimensional lattices of
//           size M = nextprime(c s) and L by eq. (4.2), the black box sampled at the lattice
//           nodes followed by a random tail, Algorithm 4; the union over the r calls.
//   Step 3: the coefficients of the final (t = d) call, top-s.
// Random draws (Philox4x64-10, key = (seed, 0), word 0 of the output block):
//   Step 1 node components  x'_u = U01(c0=u, c1=i, c2=t, c3=1)
//   Step 2 tail             x'_u = U01(c0=u, c1=i, c2=t, c3=2)
//   Step 2 generators       z_{l,u} = u64(c0=u, c1=l, c2=t*2^20 + i, c3=3) mod M
// with 0-based t (number of the coordinate being added), i (repetition), l, u.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <numeric>
#include <set>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "plan.cuh"

namespace sfft {
namespace {

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    int ensure(size_t bytes) {
        if (bytes <= cap) return SFFT_OK;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 256));
        if (e != cudaSuccess) {
            set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
            return SFFT_ENOMEM;
        }
        cap = std::max<size_t>(bytes, 256);
        return SFFT_OK;
    }
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

// out = (1/K) DFT(in) of length K (any K >= 2) in FP64 through the Bluestein kernel
int small_dft(int K, const c64* in, c64* out, DevBuf& jobbuf, cudaStream_t st) {
    FftTables* t = nullptr;
    SFFT_TRY(tables_acquire(K, &t));
    BlueJob J = make_blue_job(t, 0, 0, 1.0 / (double)K);
    J.in = in;
    J.out = out;
    int rc = jobbuf.ensure(sizeof(BlueJob));
    if (rc == SFFT_OK) {
        cudaError_t e = cudaMemcpyAsync(jobbuf.p, &J, sizeof J, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { set_error("job upload: %s", cudaGetErrorString(e)); rc = SFFT_ECUDA; }
    }
    const bool sm = blue_smem_bytes(t->N, sizeof(c64)) <= blue_smem_limit();
    if (rc == SFFT_OK && !sm) { set_error("Step 1 length K=%d too large", K); rc = SFFT_EINVAL; }
    if (rc == SFFT_OK) rc = launch_bluestein(jobbuf.as<BlueJob>(), 1, (int)t->N, 1, 0, 0, 0, -1, EPI_PLAIN, nullptr, st);
    if (rc == SFFT_OK) {
        cudaError_t e = cudaStreamSynchronize(st);  // the tables may be released below
        if (e != cudaSuccess) { set_error("small DFT: %s", cudaGetErrorString(e)); rc = SFFT_ECUDA; }
    }
    tables_release(t);
    return rc;
}

// positions of the s_keep largest |v| with |v| >= theta (ties: lower position), ascending
std::vector<int64_t> top_positions(const std::vector<c64>& v, int64_t s_keep, double theta) {
    std::vector<int64_t> keep;
    std::vector<double> a(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        a[i] = hypot(v[i].x, v[i].y);
        if (a[i] >= theta) keep.push_back((int64_t)i);
    }
    if (s_keep >= 0 && (int64_t)keep.size() > s_keep) {
        std::stable_sort(keep.begin(), keep.end(), [&](int64_t x, int64_t y) { return a[x] > a[y]; });
        keep.resize(s_keep);
        std::sort(keep.begin(), keep.end());
    }
    return keep;
}

struct Driver {
    int d = 0;
    const sfft_dimincr_params* p = nullptr;
    sfft_sample_fn f = nullptr;
    void* ctx = nullptr;
    cudaStream_t st = nullptr;
    int64_t nsamp = 0;
    DevBuf X, y, y32, tail, jobbuf, dft, prev, cur, J, supp, coef, rows;

    int eval(const double* Xd, int64_t n, double* yd) {
        int rc = f(ctx, Xd, n, yd, (void*)st);
        if (rc != 0) {
            set_error("black-box function returned %d", rc);
            return SFFT_EINVAL;
        }
        nsamp += n;
        SFFT_CHECK(p->max_samples <= 0 || nsamp <= p->max_samples, SFFT_ECAPACITY, "sample budget %lld exceeded",
                   (long long)p->max_samples);
        return SFFT_OK;
    }
    int upload_tail(uint64_t i, uint64_t t, uint64_t tag) {
        std::vector<double> tl(d);
        for (int u = 0; u < d; ++u) tl[u] = philox_u01(p->seed, (uint64_t)u, i, t, tag);
        SFFT_TRY(tail.ensure(sizeof(double) * d));
        SFFT_CU(cudaMemcpyAsync(tail.p, tl.data(), sizeof(double) * d, cudaMemcpyHostToDevice, st));
        SFFT_CU(cudaStreamSynchronize(st));  // tl is released on return
        return SFFT_OK;
    }

    // Step 1: single frequency component identification for coordinate t
    int step1(int t, int lo, int hi, std::vector<int32_t>* It) {
        const int K = hi - lo + 1;
        std::set<int32_t> sel;
        for (int i = 0; i < p->r; ++i) {
            SFFT_TRY(upload_tail((uint64_t)i, (uint64_t)t, 1));
            SFFT_TRY(X.ensure(sizeof(double) * (size_t)K * d));
            SFFT_TRY(y.ensure(sizeof(c64) * K));
            SFFT_TRY(dft.ensure(sizeof(c64) * K));
            SFFT_TRY(launch_step1_nodes(tail.as<double>(), d, t, K, X.as<double>(), st));
            SFFT_TRY(eval(X.as<double>(), K, y.as<double>()));
            std::vector<c64> ph(K);
            if (K >= 2) {
                SFFT_TRY(small_dft(K, y.as<c64>(), dft.as<c64>(), jobbuf, st));
                SFFT_CU(cudaMemcpy(ph.data(), dft.p, sizeof(c64) * K, cudaMemcpyDeviceToHost));
            } else {
                SFFT_CU(cudaMemcpy(ph.data(), y.p, sizeof(c64) * K, cudaMemcpyDeviceToHost));
            }
            // vals[q] = ph[k_q mod K] for k_q = lo + q
            std::vector<c64> vals(K);
            double mx = 0;
            for (int q = 0; q < K; ++q) {
                int k = lo + q;
                vals[q] = ph[((k % K) + K) % K];
                mx = std::max(mx, hypot(vals[q].x, vals[q].y));
            }
            const double th = std::max(p->theta_abs, p->theta_rel * mx);
            for (int64_t q : top_positions(vals, p->s_local, th)) sel.insert(lo + (int32_t)q);
        }
        It->assign(sel.begin(), sel.end());
        return SFFT_OK;
    }

    // one Algorithm 4 call of Step 2 on J (device [nJ, tc]); adds the selected rows to acc
    int step2_call(int t, int i, int64_t nJ, int64_t NJ, int64_t st_, std::map<std::vector<int32_t>, c64>* acc) {
        const int tc = t + 1;
        const int64_t M = next_prime_above(p->c * (double)p->s);
        SFFT_CHECK(M > NJ, SFFT_EALIAS, "lattice size %lld <= expansion %lld of J_t", (long long)M, (long long)NJ);
        const int L = L_rule(SFFT_L_EQ42, nJ, p->delta, p->c);
        std::vector<int64_t> Mv(L, M), z((size_t)L * tc);
        for (int l = 0; l < L; ++l)
            for (int u = 0; u < tc; ++u)
                z[(size_t)l * tc + u] = (int64_t)(philox_word0(p->seed, (uint64_t)u, (uint64_t)l,
                                                               (uint64_t)t * (1ull << 20) + (uint64_t)i, 3) % (uint64_t)M);
        sfft_params q;
        sfft_params_default(&q);
        q.c = p->c;
        q.delta = p->delta;
        q.tau_abs = p->tau_abs;
        q.tau_rel = p->tau_rel;
        q.theta_abs = p->theta_abs;
        q.theta_rel = p->theta_rel;
        q.s_tilde = st_;
        q.precision = p->precision;
        q.refine = p->refine;
        q.seed = p->seed;
        q.detect_cap = nJ;  // every candidate of J_t may be detected (compressible functions)
        Plan P;
        int rc = plan_create(&P, tc, J.as<int32_t>(), nJ, p->s, L, Mv.data(), z.data(), &q, st);
        if (rc == SFFT_OK) rc = run_call(P, t, i, tc, st_, acc);
        cudaStreamSynchronize(st);
        P.release();
        return rc;
    }

    int run_call(Plan& P, int t, int i, int tc, int64_t st_, std::map<std::vector<int32_t>, c64>* acc) {
        const int64_t n = P.sumM;
        SFFT_TRY(X.ensure(sizeof(double) * (size_t)n * d));
        SFFT_TRY(y.ensure(sizeof(c64) * n));
        SFFT_TRY(rows.ensure(sizeof(double) * (size_t)n * tc));  // lattice coordinates
        SFFT_TRY(launch_points(P.d_inst, nullptr, rows.as<double>(), n * tc, st));
        SFFT_TRY(upload_tail((uint64_t)i, (uint64_t)t, 2));
        SFFT_TRY(launch_assemble_nodes(rows.as<double>(), n, tc, tail.as<double>(), d, X.as<double>(), st));
        SFFT_TRY(eval(X.as<double>(), n, y.as<double>()));
        const void* samples = y.p;
        if (P.prec == SFFT_FP32) {
            SFFT_TRY(y32.ensure(sizeof(c32) * n));
            SFFT_TRY(launch_c64_to_c32(y.as<c64>(), y32.as<c32>(), n, st));
            samples = y32.p;
        }
        const int64_t cap = std::max<int64_t>(st_, 1);
        SFFT_TRY(supp.ensure(sizeof(int64_t) * cap));
        SFFT_TRY(coef.ensure(sizeof(c64) * cap));
        int64_t nout = 0;
        SFFT_TRY(sfft_reconstruct(reinterpret_cast<sfft_plan*>(&P), samples, supp.as<int64_t>(), coef.as<double>(), cap,
                                  &nout, nullptr));
        if (nout == 0) return SFFT_OK;
        SFFT_TRY(rows.ensure(sizeof(int32_t) * (size_t)nout * tc));
        SFFT_TRY(launch_gather_rows(J.as<int32_t>(), tc, supp.as<int64_t>(), nout, rows.as<int32_t>(), st));
        std::vector<int32_t> hr((size_t)nout * tc);
        std::vector<c64> hc(nout);
        SFFT_CU(cudaMemcpyAsync(hr.data(), rows.p, sizeof(int32_t) * hr.size(), cudaMemcpyDeviceToHost, st));
        SFFT_CU(cudaMemcpyAsync(hc.data(), coef.p, sizeof(c64) * nout, cudaMemcpyDeviceToHost, st));
        SFFT_CU(cudaStreamSynchronize(st));
        for (int64_t q = 0; q < nout; ++q) {
            std::vector<int32_t> key(hr.begin() + q * tc, hr.begin() + (q + 1) * tc);
            (*acc)[key] = hc[q];  // a later call overwrites an earlier coefficient of the same row
        }
        return SFFT_OK;
    }
};

}  // namespace
}  // namespace sfft

using namespace sfft;

extern "C" {

void sfft_dimincr_params_default(sfft_dimincr_params* p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->s = 1;
    p->s_local = 0;
    p->r = 1;
    p->theta_abs = 1e-12;
    p->theta_rel = 0.0;
    p->delta = 0.9;
    p->c = 10.33;
    p->tau_abs = 0.0;
    p->tau_rel = 1e-10;
    p->precision = SFFT_FP64;
    p->refine = 1;
    p->seed = 0;
    p->max_samples = 0;
}

int sfft_dim_incremental(int d, const int32_t* box_lo, const int32_t* box_hi, const sfft_dimincr_params* pin,
                         sfft_sample_fn f, void* ctx, int32_t* supp_out, double* coef_out, int64_t cap, int64_t* n_out,
                         int64_t* n_samples, void* stream) {
    SFFT_CHECK(d >= 1 && d <= kMaxD && box_lo && box_hi && pin && f && n_out && (cap == 0 || (supp_out && coef_out)),
               SFFT_EINVAL, "sfft_dim_incremental: bad argument");
    sfft_dimincr_params p = *pin;
    if (p.s_local <= 0) p.s_local = 2 * p.s;
    SFFT_CHECK(p.s >= 1 && p.r >= 1 && p.s_local >= p.s && p.delta > 0 && p.delta < 1 && p.c > 2, SFFT_EINVAL,
               "sfft_dim_incremental: bad parameters");
    for (int t = 0; t < d; ++t) SFFT_CHECK(box_hi[t] >= box_lo[t], SFFT_EINVAL, "empty box in dimension %d", t);
    Driver D;
    D.d = d;
    D.p = &p;
    D.f = f;
    D.ctx = ctx;
    D.st = (cudaStream_t)stream;
    // ---- Step 1
    std::vector<std::vector<int32_t>> I1(d);
    for (int t = 0; t < d; ++t) SFFT_TRY(D.step1(t, box_lo[t], box_hi[t], &I1[t]));
    // ---- Step 2
    std::vector<int32_t> Icur(I1[0].begin(), I1[0].end());  // rows of width t
    std::vector<c64> coef;
    int width = 1;
    if (d == 1) {
        // a single coordinate: Step 1 alone identifies the frequencies; coefficients by one call on Gamma = I^(1)
        coef.assign(Icur.size(), c64{0, 0});
    }
    for (int t = 1; t < d; ++t) {
        const bool last = t == d - 1;
        const int rt = last ? 1 : p.r;
        const int64_t st_ = last ? p.s : p.s_local;
        std::map<std::vector<int32_t>, c64> acc;
        const int64_t np = (int64_t)Icur.size() / width, nt = (int64_t)I1[t].size();
        const int64_t nJ = np * nt;
        // expansion of J_t: the column ranges of I^(1..t-1) and of I^(t)
        int64_t NJ = 0;
        if (nJ > 0) {
            for (int u = 0; u < width; ++u) {
                int32_t mn = INT32_MAX, mx = INT32_MIN;
                for (int64_t a = 0; a < np; ++a) { mn = std::min(mn, Icur[a * width + u]); mx = std::max(mx, Icur[a * width + u]); }
                NJ = std::max<int64_t>(NJ, (int64_t)mx - mn);
            }
            NJ = std::max<int64_t>(NJ, (int64_t)I1[t].back() - I1[t].front());
        }
        for (int i = 0; i < rt && nJ > 0; ++i) {
            SFFT_TRY(D.prev.ensure(sizeof(int32_t) * Icur.size()));
            SFFT_TRY(D.cur.ensure(sizeof(int32_t) * nt));
            SFFT_TRY(D.J.ensure(sizeof(int32_t) * (size_t)nJ * (t + 1)));
            SFFT_CU(cudaMemcpyAsync(D.prev.p, Icur.data(), sizeof(int32_t) * Icur.size(), cudaMemcpyHostToDevice, D.st));
            SFFT_CU(cudaMemcpyAsync(D.cur.p, I1[t].data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice, D.st));
            SFFT_TRY(launch_pairing(D.prev.as<int32_t>(), np, width, D.cur.as<int32_t>(), (int)nt, D.J.as<int32_t>(), D.st));
            SFFT_TRY(D.step2_call(t, i, nJ, NJ, st_, &acc));
        }
        Icur.clear();
        coef.clear();
        for (const auto& kv : acc) {
            Icur.insert(Icur.end(), kv.first.begin(), kv.first.end());
            coef.push_back(kv.second);
        }
        width = t + 1;
    }
    // ---- Step 3: coefficients of the final call, top-s by modulus
    const int64_t nrow = width > 0 ? (int64_t)Icur.size() / width : 0;
    std::vector<int64_t> pos = top_positions(coef, p.s, 0.0);
    *n_out = (int64_t)pos.size();
    if (n_samples) *n_samples = D.nsamp;
    (void)nrow;
    const int64_t nw = std::min<int64_t>(cap, (int64_t)pos.size());
    for (int64_t q = 0; q < nw; ++q) {
        for (int u = 0; u < d; ++u) supp_out[q * d + u] = Icur[pos[q] * width + u];
        coef_out[2 * q] = coef[pos[q]].x;
        coef_out[2 * q + 1] = coef[pos[q]].y;
    }
    if ((int64_t)pos.size() > cap) {
        set_error("%lld frequencies exceed cap = %lld", (long long)pos.size(), (long long)cap);
        return SFFT_ECAPACITY;
    }
    return SFFT_OK;
}

int sfft_fn_sparse_poly(void* ctx, const double* x, int64_t n, double* y, void* stream) {
    auto* c = reinterpret_cast<sfft_fn_sparse_poly_ctx*>(ctx);
    if (!c || !x || !y) return SFFT_EINVAL;
    return launch_sparse_eval_points(x, n, c->d, c->kvec, c->coef, c->n_terms, y, (cudaStream_t)stream);
}

int sfft_fn_sop(void* ctx, const double* x, int64_t n, double* y, void* stream) {
    auto* c = reinterpret_cast<sfft_fn_sop_ctx*>(ctx);
    if (!c || !x || !y || !c->work || !c->triples || !c->theta) return SFFT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    double* a = reinterpret_cast<double*>(c->work);
    double* da = a + (size_t)c->n_terms * (c->K + 1);
    int32_t* tri = reinterpret_cast<int32_t*>(da + (size_t)c->n_terms * (c->K + 1));
    for (int i = 0; i < 3 * c->n_terms; ++i)
        if (c->triples[i] < 0 || c->triples[i] >= c->d) return SFFT_EINVAL;
    SFFT_CU(cudaMemcpyAsync(tri, c->triples, sizeof(int32_t) * 3 * c->n_terms, cudaMemcpyHostToDevice, st));
    SFFT_TRY(launch_sop_coefs(c->theta, c->n_terms, c->K, c->width, a, da, st));
    return launch_sop_eval_points(x, n, c->d, tri, c->n_terms, c->K, a, y, st);
}

}  // extern "C"
