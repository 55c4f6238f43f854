// Section 4.3's approximately sparse test function (eq. 4.3) at the lattice nodes: a sum of
// products of periodic B-splines, f(x) = sum_q prod_{t in dims_q} N_{m_q}(x_t), with
//   N_m(x) = C_m sum_k sinc(pi k/m)^m (-1)^k exp(2 pi i k x),   ||N_m||_{L2(T)} = 1.
// Its Fourier series is the periodisation of the cardinal B-spline M_m (knots 0, 1, ..., m,
// Fourier transform ((1 - e^{-i w}) / (i w))^m) scaled to one period: N_m(x) = C_m m M_m(m x)
// for x in [0, 1) (the (-1)^k is the half-period shift from the centred to the cardinal
// spline).  M_m is evaluated by the Cox-de Boor recurrence on uniform knots,
//   M_k(v) = (v M_{k-1}(v) + (k - v) M_{k-1}(v - 1)) / (k - 1),
// for the k values M_k(f + r), r = 0..k-1 (f the fractional part of v) at once: O(m^2) FP64
// operations, no truncated series.  C_m = (m M_2m(m))^(-1/2): the L2 norm of m M_m(m .) over a
// period is m times the autocorrelation of M_m at 0, which is M_2m at its centre.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "plan.cuh"

namespace sfft {

constexpr int kBsMaxTerms = 8;
constexpr int kBsMaxDims = 4;
constexpr int kBsMaxOrder = 12;

struct BsTerms {
    int n;
    int ndim[kBsMaxTerms];
    int dims[kBsMaxTerms][kBsMaxDims];
    int m[kBsMaxTerms];
    double scale[kBsMaxTerms];  // C_m m
};

// M_m(v) for v in [0, m) (cardinal B-spline of order m <= MAXO); 0 outside
template <int MAXO>
__host__ __device__ inline double cardinal_bspline(int m, double v) {
    if (!(v >= 0.0) || v >= (double)m || m > MAXO) return 0.0;
    const int i = (int)floor(v);
    const double f = v - (double)i;
    double b[MAXO];
    b[0] = 1.0;  // order 1: M_1(f) = 1
    for (int k = 2; k <= m; ++k) {
        // b[r] = M_{k-1}(f + r), r < k - 1; new b[r] = M_k(f + r), r < k
        double prev = 0.0;  // M_{k-1}(f + r - 1)
        for (int r = 0; r < k; ++r) {
            const double cur = r < k - 1 ? b[r] : 0.0;
            const double x = f + (double)r;
            b[r] = (x * cur + ((double)k - x) * prev) / (double)(k - 1);
            prev = cur;
        }
    }
    return b[i];
}

template <class T>
__global__ void k_bspline_sample(const InstDesc* __restrict__ insts, BsTerms terms, void* out) {
    const InstDesc& I = insts[0];
    const int L = I.L, d = I.d;
    const int64_t tot = I.soff[L];
    cplx<T>* y = reinterpret_cast<cplx<T>*>(out);
    for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < tot; node += (int64_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (I.soff[l + 1] <= node) ++l;
        const int64_t j = node - I.soff[l], M = I.Ml[l];
        double f = 0.0;
        for (int q = 0; q < terms.n; ++q) {
            const int m = terms.m[q];
            double p = 1.0;
            for (int u = 0; u < terms.ndim[q]; ++u) {
                const int t = terms.dims[q][u];
                const int64_t num = (j * (int64_t)I.z[l * d + t]) % M;  // exact node numerator
                p *= terms.scale[q] * cardinal_bspline<kBsMaxOrder>(m, (double)(m * num) / (double)M);
            }
            f += p;
        }
        y[node] = cplx<T>{(T)f, (T)0};
    }
}

// f at arbitrary nodes x [n, d] (FP64), output complex double (imaginary part 0): the black box of
// Algorithm 3 for this test function
__global__ void k_bspline_eval_points(const double* __restrict__ x, int64_t n, int d, BsTerms terms, double* y) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double f = 0.0;
        for (int q = 0; q < terms.n; ++q) {
            const int m = terms.m[q];
            double p = 1.0;
            for (int u = 0; u < terms.ndim[q]; ++u) {
                const double xv = x[j * d + terms.dims[q][u]];
                p *= terms.scale[q] * cardinal_bspline<kBsMaxOrder>(m, (double)m * (xv - floor(xv)));
            }
            f += p;
        }
        y[2 * j] = f;
        y[2 * j + 1] = 0.0;
    }
}

// the terms from the host arrays of the C ABI (dims [n_terms, 4], -1 ends a term; orders [n_terms])
static int make_terms(const int32_t* dims, const int32_t* orders, int n_terms, int d, BsTerms* T) {
    SFFT_CHECK(dims && orders, SFFT_EINVAL, "null argument");
    SFFT_CHECK(n_terms >= 1 && n_terms <= kBsMaxTerms, SFFT_EINVAL, "B-spline sums take 1 to %d terms", kBsMaxTerms);
    *T = BsTerms{};
    T->n = n_terms;
    for (int q = 0; q < n_terms; ++q) {
        const int m = orders[q];
        SFFT_CHECK(m >= 1 && m <= kBsMaxOrder, SFFT_EINVAL, "B-spline order %d must be in [1, %d]", m, kBsMaxOrder);
        T->m[q] = m;
        int nd = 0;
        for (int u = 0; u < kBsMaxDims; ++u) {
            const int t = dims[q * kBsMaxDims + u];
            if (t < 0) break;
            SFFT_CHECK(t < d, SFFT_EINVAL, "term %d: dimension %d is not below d = %d", q, t, d);
            for (int w = 0; w < nd; ++w)
                SFFT_CHECK(T->dims[q][w] != t, SFFT_EINVAL, "term %d repeats dimension %d", q, t);
            T->dims[q][nd++] = t;
        }
        SFFT_CHECK(nd >= 1, SFFT_EINVAL, "term %d has no dimension", q);
        T->ndim[q] = nd;
        // C_m = (m M_2m(m))^(-1/2)
        T->scale[q] = (double)m / sqrt((double)m * cardinal_bspline<2 * kBsMaxOrder>(2 * m, (double)m));
    }
    return SFFT_OK;
}

}  // namespace sfft

using namespace sfft;

extern "C" int sfft_fn_bspline(void* ctx, const double* x, int64_t n, double* y, void* stream) {
    auto* c = reinterpret_cast<sfft_fn_bspline_ctx*>(ctx);
    if (!c || !x || !y) return SFFT_EINVAL;
    BsTerms T;
    SFFT_TRY(make_terms(c->dims, c->orders, c->n_terms, c->d, &T));
    if (n <= 0) return SFFT_OK;
    const int gx = (int)std::min<int64_t>(4 * 152, (n + 255) / 256 + 1);
    k_bspline_eval_points<<<gx, 256, 0, (cudaStream_t)stream>>>(x, n, c->d, T, y);
    return launch_check("k_bspline_eval_points");
}

extern "C" int sfft_sample_bspline(const sfft_plan* plan, const int32_t* dims, const int32_t* orders, int n_terms,
                                   void* samples_out) {
    if (!plan || !dims || !orders || !samples_out) { set_error("null argument"); return SFFT_EINVAL; }
    const Plan* P = reinterpret_cast<const Plan*>(plan);
    BsTerms T;
    SFFT_TRY(make_terms(dims, orders, n_terms, P->d, &T));
    if (P->prec) k_bspline_sample<float><<<4 * 152, 256, 0, P->st>>>(P->d_inst, T, samples_out);
    else k_bspline_sample<double><<<4 * 152, 256, 0, P->st>>>(P->d_inst, T, samples_out);
    return launch_check("k_bspline_sample");
}
