// Dimension-incremental sparse FFT (Algorithm 3) with Algorithm 4 (plus one refinement step)
// in the role of Algorithm A, on a box candidate set Gamma = prod_t [lo_t, hi_t].
//   Step 1: for every coordinate t, r random node tails; K_t-point DFTs along coordinate t
//           (Bluestein kernel, FP64); keep the s_local largest projections of modulus >= theta
//           (one-CTA radix select on the device) and unite them over the r tails.
//   Step 2: for t = 2..d: J_t = I^(1..t-1) x I^(t) (device pairing), t-dimensional lattices of
//           size M = nextprime(c s) and L by eq. (4.2), the black box sampled at the lattice
//           nodes followed by a random tail, Algorithm 4; the union over the r calls (scatter
//           by row of J_t, ordered compaction).
//   Step 3: the coefficients of the final (t = d) call, whose Algorithm 4 keeps the s largest.
// Every index set stays in device memory; the host reads only set sizes (to size the next
// launches) and, at the end, the output.
// Random draws (Philox4x64-10, key = (seed, 0), word 0 of the output block):
//   Step 1 node components  x'_u = U01(c0=u, c1=i, c2=t, c3=1)
//   Step 2 tail             x'_u = U01(c0=u, c1=i, c2=t, c3=2)
//   Step 2 generators       z_{l,u} = u64(c0=u, c1=l, c2=t*2^20 + i, c3=3) mod M
// with 0-based t (number of the coordinate being added), i (repetition), l, u.
#include <math.h>
#include <string.h>

#include <algorithm>
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

// FFT tables held by the driver for its whole run (one acquisition per distinct length), so that
// the per-call plans and the Step-1 transforms neither rebuild them nor wait for their release
struct TableCache {
    std::vector<FftTables*> held;
    int get(int64_t M, FftTables** out) {
        for (FftTables* t : held)
            if (t->M == M) { *out = t; return SFFT_OK; }
        SFFT_TRY(tables_acquire(M, out));
        held.push_back(*out);
        return SFFT_OK;
    }
    ~TableCache() {
        for (FftTables* t : held) tables_release(t);
    }
};

struct Driver {
    int d = 0;
    const sfft_dimincr_params* p = nullptr;
    sfft_sample_fn f = nullptr;
    void* ctx = nullptr;
    cudaStream_t st = nullptr;
    int64_t nsamp = 0;
    TableCache tabs;
    DevBuf X, y, y32, tail, jobbuf, dft, mag, mask, pos, cnts, J, supp, coef, rows, flags, acc, Icur, Icoef, Inext;
    std::vector<DevBuf> I1;      // Step 1 sets I^(t): device int32, ascending
    std::vector<int64_t> n1;     // their sizes
    int64_t* h_cnt = nullptr;    // pinned: device counts read by the host

    ~Driver() {
        if (h_cnt) cudaFreeHost(h_cnt);
    }
    int init() {
        SFFT_CU(cudaMallocHost((void**)&h_cnt, 64));
        return SFFT_OK;
    }
    // a device int64 count -> host (the sizes of the next sets)
    int read_count(const int64_t* dev, int64_t* out) {
        SFFT_CU(cudaMemcpyAsync(h_cnt, dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        SFFT_CU(cudaStreamSynchronize(st));
        *out = h_cnt[0];
        return SFFT_OK;
    }
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
    // random node components U01(c0 = u, c1 = i, c2 = t, c3 = tag), u < d, drawn on the device
    int draw_tail(uint64_t i, uint64_t t, uint64_t tag) {
        SFFT_TRY(tail.ensure(sizeof(double) * d));
        return launch_philox_tail(p->seed, i, t, tag, d, tail.as<double>(), st);
    }
    // out = (1/K) DFT(in) of length K >= 2 in FP64 through the Bluestein kernel
    int small_dft(int K, const c64* in, c64* out) {
        FftTables* t = nullptr;
        SFFT_TRY(tabs.get(K, &t));
        SFFT_CHECK(blue_smem_bytes(t->N, sizeof(c64)) <= blue_smem_limit(), SFFT_EINVAL, "Step 1 length K=%d too large",
                   K);
        BlueJob Jb = make_blue_job(t, 0, 0, 1.0 / (double)K);
        Jb.in = in;
        Jb.out = out;
        SFFT_TRY(jobbuf.ensure(sizeof(BlueJob)));
        // pageable source: the copy is staged before the call returns, so Jb may go out of scope
        SFFT_CU(cudaMemcpyAsync(jobbuf.p, &Jb, sizeof Jb, cudaMemcpyHostToDevice, st));
        return launch_bluestein(jobbuf.as<BlueJob>(), 1, (int)t->N, 1, 0, 0, 0, -1, EPI_PLAIN, nullptr, st);
    }

    // Step 1: single frequency component identification for coordinate t (r node tails, the
    // s_local largest projections of each, their union) -> I^(t) on the device
    int step1(int t, int lo, int hi) {
        const int K = hi - lo + 1;
        SFFT_TRY(mask.ensure(K));
        SFFT_CU(cudaMemsetAsync(mask.p, 0, K, st));
        SFFT_TRY(mag.ensure(sizeof(double) * K));
        for (int i = 0; i < p->r; ++i) {
            SFFT_TRY(draw_tail((uint64_t)i, (uint64_t)t, 1));
            SFFT_TRY(X.ensure(sizeof(double) * (size_t)K * d));
            SFFT_TRY(y.ensure(sizeof(c64) * K));
            SFFT_TRY(dft.ensure(sizeof(c64) * K));
            SFFT_TRY(launch_step1_nodes(tail.as<double>(), d, t, K, X.as<double>(), st));
            SFFT_TRY(eval(X.as<double>(), K, y.as<double>()));
            const c64* ph = y.as<c64>();
            if (K >= 2) {
                SFFT_TRY(small_dft(K, y.as<c64>(), dft.as<c64>()));
                ph = dft.as<c64>();
            }
            SFFT_TRY(launch_step1_select(ph, K, lo, p->s_local, p->theta_abs, p->theta_rel, p->rank_bits,
                                         mag.as<double>(), mask.as<uint8_t>(), st));
        }
        SFFT_TRY(pos.ensure(sizeof(int64_t) * K));
        SFFT_TRY(cnts.ensure(sizeof(int64_t) * (flag_compact_blocks(K) + 1)));
        int64_t* total = cnts.as<int64_t>() + flag_compact_blocks(K);
        SFFT_TRY(launch_flag_compact(mask.as<uint8_t>(), K, cnts.as<int64_t>(), pos.as<int64_t>(), total, st));
        int64_t n = 0;
        SFFT_TRY(read_count(total, &n));
        SFFT_TRY(I1[t].ensure(sizeof(int32_t) * std::max<int64_t>(n, 1)));
        SFFT_TRY(launch_positions_to_values(pos.as<int64_t>(), n, lo, I1[t].as<int32_t>(), st));
        n1[t] = n;
        return SFFT_OK;
    }

    // one Algorithm 4 call of Step 2 on J (device [nJ, tc]); its selection goes into the union
    // (flags / acc over the rows of J)
    int step2_call(int t, int i, int64_t nJ, int64_t st_) {
        const int tc = t + 1;
        const int64_t M = next_prime_above(p->c * (double)p->s);
        // eq. (4.2) with delta (the paper's numerics), or Corollary 2.6 with the theory's failure
        // probability gamma_A = delta / (3 d r) of one Algorithm 4 call (Section 3.3)
        const int L = p->L_rule == SFFT_L_COR26 ? L_rule(SFFT_L_COR26, nJ, p->delta / (3.0 * d * p->r), p->c)
                                                : L_rule(SFFT_L_EQ42, nJ, p->delta, p->c);
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
        q.rank_bits = p->rank_bits;
        q.detect_cap = nJ;  // every candidate of J_t may be detected (compressible functions)
        FftTables* hold = nullptr;
        SFFT_TRY(tabs.get(M, &hold));  // keeps the tables alive between the per-call plans
        Plan P;
        int rc = plan_create(&P, tc, J.as<int32_t>(), nJ, p->s, L, Mv.data(), z.data(), &q, st);
        if (rc == SFFT_OK) rc = run_call(P, t, i, tc, st_, nJ);
        cudaStreamSynchronize(st);
        P.release();
        return rc;
    }

    int run_call(Plan& P, int t, int i, int tc, int64_t st_, int64_t nJ) {
        const int64_t n = P.sumM;
        SFFT_TRY(X.ensure(sizeof(double) * (size_t)n * d));
        SFFT_TRY(y.ensure(sizeof(c64) * n));
        SFFT_TRY(rows.ensure(sizeof(double) * (size_t)n * tc));  // lattice coordinates
        SFFT_TRY(launch_points(P.d_inst, nullptr, rows.as<double>(), n * tc, st));
        SFFT_TRY(draw_tail((uint64_t)i, (uint64_t)t, 2));
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
        (void)nJ;
        return launch_union_scatter(supp.as<int64_t>(), coef.as<c64>(), nout, flags.as<uint8_t>(), acc.as<c64>(), st);
    }

    // Step 2 for coordinate t: J_t = I^(1..t-1) x I^(t) (rows in lexicographic order, because
    // I^(1..t-1) is and I^(t) is ascending), r (or 1) calls, the union in row order -> I^(1..t)
    int step2(int t, int64_t* np_io) {
        const bool last = t == d - 1;
        const int rt = last ? 1 : p->r;
        const int64_t st_ = last ? p->s : p->s_local;
        const int64_t np = *np_io, nt = n1[t];
        const int64_t nJ = np * nt;
        const int w = t;  // columns of I^(1..t-1)
        if (nJ == 0) {
            *np_io = 0;
            return SFFT_OK;
        }
        SFFT_TRY(J.ensure(sizeof(int32_t) * (size_t)nJ * (t + 1)));
        SFFT_TRY(launch_pairing(Icur.as<int32_t>(), np, w, I1[t].as<int32_t>(), (int)nt, J.as<int32_t>(), st));
        SFFT_TRY(flags.ensure(nJ));
        SFFT_CU(cudaMemsetAsync(flags.p, 0, nJ, st));
        SFFT_TRY(acc.ensure(sizeof(c64) * nJ));
        for (int i = 0; i < rt; ++i) SFFT_TRY(step2_call(t, i, nJ, st_));
        SFFT_TRY(pos.ensure(sizeof(int64_t) * nJ));
        SFFT_TRY(cnts.ensure(sizeof(int64_t) * (flag_compact_blocks(nJ) + 1)));
        int64_t* total = cnts.as<int64_t>() + flag_compact_blocks(nJ);
        SFFT_TRY(launch_flag_compact(flags.as<uint8_t>(), nJ, cnts.as<int64_t>(), pos.as<int64_t>(), total, st));
        int64_t nu = 0;
        SFFT_TRY(read_count(total, &nu));
        SFFT_TRY(Inext.ensure(sizeof(int32_t) * (size_t)std::max<int64_t>(nu, 1) * (t + 1)));
        SFFT_TRY(launch_gather_rows(J.as<int32_t>(), t + 1, pos.as<int64_t>(), nu, Inext.as<int32_t>(), st));
        SFFT_TRY(Icoef.ensure(sizeof(c64) * std::max<int64_t>(nu, 1)));
        SFFT_TRY(launch_gather_c64(acc.as<c64>(), pos.as<int64_t>(), nu, Icoef.as<c64>(), st));
        std::swap(Icur.p, Inext.p);
        std::swap(Icur.cap, Inext.cap);
        *np_io = nu;
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
    p->rank_bits = 0;
    p->L_rule = SFFT_L_EQ42;
}

int sfft_dim_incremental(int d, const int32_t* box_lo, const int32_t* box_hi, const sfft_dimincr_params* pin,
                         sfft_sample_fn f, void* ctx, int32_t* supp_out, double* coef_out, int64_t cap, int64_t* n_out,
                         int64_t* n_samples, void* stream) {
    SFFT_CHECK(d >= 2 && d <= kMaxD && box_lo && box_hi && pin && f && n_out && (cap == 0 || (supp_out && coef_out)),
               SFFT_EINVAL, "sfft_dim_incremental: bad argument (2 <= d <= %d)", kMaxD);
    sfft_dimincr_params p = *pin;
    if (p.s_local <= 0) p.s_local = 2 * p.s;
    SFFT_CHECK(p.s >= 1 && p.r >= 0 && p.s_local >= p.s && p.delta > 0 && p.delta < 1 && p.c > 2 && p.rank_bits >= 0 &&
                   p.rank_bits <= 52 && (p.L_rule == SFFT_L_EQ42 || p.L_rule == SFFT_L_COR26),
               SFFT_EINVAL, "sfft_dim_incremental: bad parameters");
    if (p.r == 0) {  // Section 3.3: r = ceil(2 s ln(3 d s / delta)) detection iterations
        const double r = ceil(2.0 * (double)p.s * log(3.0 * d * (double)p.s / p.delta));
        SFFT_CHECK(r < 1e9, SFFT_EINVAL, "the theory's r = %.0f is too large", r);
        p.r = (int)r;
    }
    for (int t = 0; t < d; ++t) SFFT_CHECK(box_hi[t] >= box_lo[t], SFFT_EINVAL, "empty box in dimension %d", t);
    Driver D;
    D.d = d;
    D.p = &p;
    D.f = f;
    D.ctx = ctx;
    D.st = (cudaStream_t)stream;
    SFFT_TRY(D.init());
    D.I1.resize(d);
    D.n1.assign(d, 0);
    // ---- Step 1: I^(t) for every coordinate
    for (int t = 0; t < d; ++t) SFFT_TRY(D.step1(t, box_lo[t], box_hi[t]));
    // ---- Step 2: I^(1..t) = union of Algorithm 4 outputs on J_t, t = 2..d (0-based t = 1..d-1)
    int64_t np = D.n1[0];
    SFFT_TRY(D.Icur.ensure(sizeof(int32_t) * std::max<int64_t>(np, 1)));
    SFFT_CU(cudaMemcpyAsync(D.Icur.p, D.I1[0].p, sizeof(int32_t) * np, cudaMemcpyDeviceToDevice, D.st));
    for (int t = 1; t < d; ++t) SFFT_TRY(D.step2(t, &np));
    // ---- Step 3: the coefficients of the final call (its Algorithm 4 already kept the s largest)
    *n_out = np;
    if (n_samples) *n_samples = D.nsamp;
    const int64_t nw = std::min<int64_t>(cap, np);
    if (nw > 0) {
        SFFT_CU(cudaMemcpyAsync(supp_out, D.Icur.p, sizeof(int32_t) * (size_t)nw * d, cudaMemcpyDeviceToHost, D.st));
        SFFT_CU(cudaMemcpyAsync(coef_out, D.Icoef.p, sizeof(c64) * nw, cudaMemcpyDeviceToHost, D.st));
    }
    SFFT_CU(cudaStreamSynchronize(D.st));
    if (np > cap) {
        set_error("%lld frequencies exceed cap = %lld", (long long)np, (long long)cap);
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
