// Synthetic black-box functions sampled at lattice nodes or arbitrary points:
//   * the sum-of-products function f(x) = sum_m prod_{t in T_m} g_{theta_m}(x_t) with the
//     periodic kernel g_theta(x) = sum_{|k|<=K} a_k(theta) e^{2 pi i k x},
//     a_k = sinc(pi k / (width theta))^4 (a smooth variant of the tensor-product test function
//     of the paper's Section 4.2.2), its adjoint with respect to theta, recomputing the
//     factors at every node instead of storing them;
//   * direct evaluation of a sparse trigonometric polynomial (eq. 2.2) at arbitrary nodes.
// g_theta is real and even: g(x) = a_0 + 2 sum_k a_k cos(2 pi k x), evaluated by Clenshaw's
// recurrence on cos(2 pi x).
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace sfft {

constexpr int kMaxTerms = 16;
constexpr int kMaxK = 128;

__global__ void k_sop_coefs(const double* __restrict__ theta, int n_terms, int K, double width, double* a, double* da) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_terms * (K + 1)) return;
    int m = e / (K + 1), k = e - m * (K + 1);
    double th = theta[m];
    double u = M_PI * k / (width * th);
    double sn = k == 0 ? 1.0 : sin(u) / u;
    double dsn = k == 0 ? 0.0 : (u * cos(u) - sin(u)) / (u * u);
    a[e] = sn * sn * sn * sn;
    da[e] = 4.0 * sn * sn * sn * dsn * (-u / th);
}

// g(c) = a_0 + 2 sum_{k>=1} a_k T_k(c), c = cos(2 pi x)   (Clenshaw)
template <class T> __device__ __forceinline__ T clenshaw(const T* a, int K, T c) {
    T b1 = 0, b2 = 0;
    for (int k = K; k >= 1; --k) {
        T b0 = (T)2 * a[k] + (T)2 * c * b1 - b2;
        b2 = b1;
        b1 = b0;
    }
    return a[0] + c * b1 - b2;
}

template <class T> __device__ __forceinline__ T cos2pi_frac(int64_t num, int64_t M) {
    if constexpr (sizeof(T) == 4) return cospif(2.0f * ((float)num / (float)M));
    else return cospi(2.0 * ((double)num / (double)M));
}

// f at the plan's lattice nodes.  The kernels are evaluated in FP64 for either plan precision and
// only the stored sample is rounded to T: an FP32 plan receives the correctly rounded FP32 value of
// f at each node (not an FP32 Clenshaw sum, whose error grows with K).
template <class T>
__global__ void k_sop_sample(const InstDesc* __restrict__ insts, const int32_t* __restrict__ triples, int n_terms, int K,
                             const double* __restrict__ a64, void* out) {
    __shared__ double sa[kMaxTerms * (kMaxK + 1)];
    __shared__ int str[kMaxTerms * 3];
    const InstDesc& I = insts[0];
    for (int i = threadIdx.x; i < n_terms * (K + 1); i += blockDim.x) sa[i] = a64[i];
    for (int i = threadIdx.x; i < n_terms * 3; i += blockDim.x) str[i] = triples[i];
    __syncthreads();
    const int L = I.L, d = I.d;
    const int64_t tot = I.soff[L];
    cplx<T>* y = reinterpret_cast<cplx<T>*>(out);
    for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < tot; node += (int64_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (I.soff[l + 1] <= node) ++l;
        const int64_t j = node - I.soff[l], M = I.Ml[l];
        double f = 0;
        for (int m = 0; m < n_terms; ++m) {
            double p = 1;
            for (int u = 0; u < 3; ++u) {
                int t = str[3 * m + u];
                int64_t num = (j * (int64_t)I.z[l * d + t]) % M;
                p *= clenshaw<double>(sa + m * (K + 1), K, cos2pi_frac<double>(num, M));
            }
            f += p;
        }
        y[node] = cplx<T>{(T)f, (T)0};
    }
}

// theta-adjoint of k_sop_sample: the factors and their theta-derivatives are recomputed at every
// node in FP64 (nothing is stored), the sample cotangent is read in the plan precision
template <class T>
__global__ void k_sop_backward(const InstDesc* __restrict__ insts, const int32_t* __restrict__ triples, int n_terms, int K,
                               const double* __restrict__ a64, const double* __restrict__ da64, const void* dsamples,
                               double* dtheta) {
    __shared__ double sa[kMaxTerms * (kMaxK + 1)];
    __shared__ double sda[kMaxTerms * (kMaxK + 1)];
    __shared__ int str[kMaxTerms * 3];
    __shared__ double red[32];
    const InstDesc& I = insts[0];
    for (int i = threadIdx.x; i < n_terms * (K + 1); i += blockDim.x) {
        sa[i] = a64[i];
        sda[i] = da64[i];
    }
    for (int i = threadIdx.x; i < n_terms * 3; i += blockDim.x) str[i] = triples[i];
    __syncthreads();
    const int L = I.L, d = I.d;
    const int64_t tot = I.soff[L];
    const cplx<T>* w = reinterpret_cast<const cplx<T>*>(dsamples);
    double acc[kMaxTerms];
    for (int m = 0; m < kMaxTerms; ++m) acc[m] = 0;
    for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < tot; node += (int64_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (I.soff[l + 1] <= node) ++l;
        const int64_t j = node - I.soff[l], M = I.Ml[l];
        const double wr = (double)w[node].x;
        for (int m = 0; m < n_terms; ++m) {
            double g[3], dg[3];
            for (int u = 0; u < 3; ++u) {
                int t = str[3 * m + u];
                int64_t num = (j * (int64_t)I.z[l * d + t]) % M;
                double c = cos2pi_frac<double>(num, M);
                g[u] = clenshaw<double>(sa + m * (K + 1), K, c);
                dg[u] = clenshaw<double>(sda + m * (K + 1), K, c);
            }
            acc[m] += wr * (dg[0] * g[1] * g[2] + g[0] * dg[1] * g[2] + g[0] * g[1] * dg[2]);
        }
    }
    for (int m = 0; m < n_terms; ++m) {
        double v = acc[m];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
            atomicAdd(&dtheta[m], s);
        }
    }
}

// f at arbitrary nodes x [n, d] (double), output complex double (imaginary part 0); FP64
__global__ void k_sop_eval_points(const double* __restrict__ x, int64_t n, int d, const int32_t* __restrict__ triples,
                                  int n_terms, int K, const double* __restrict__ a64, double* y) {
    __shared__ double sa[kMaxTerms * (kMaxK + 1)];
    __shared__ int str[kMaxTerms * 3];
    for (int i = threadIdx.x; i < n_terms * (K + 1); i += blockDim.x) sa[i] = a64[i];
    for (int i = threadIdx.x; i < n_terms * 3; i += blockDim.x) str[i] = triples[i];
    __syncthreads();
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double f = 0;
        for (int m = 0; m < n_terms; ++m) {
            double p = 1;
            for (int u = 0; u < 3; ++u) {
                double xv = x[j * d + str[3 * m + u]];
                double c = cospi(2.0 * (xv - floor(xv)));
                p *= clenshaw<double>(sa + m * (K + 1), K, c);
            }
            f += p;
        }
        y[2 * j] = f;
        y[2 * j + 1] = 0;
    }
}

// p(x) = sum_q c_q exp(2 pi i k_q . x) at arbitrary nodes (direct, FP64)
__global__ void k_sparse_eval_points(const double* __restrict__ x, int64_t n, int d, const int32_t* __restrict__ kvec,
                                     const double* __restrict__ coef, int64_t nterms, double* y) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double re = 0, im = 0;
        for (int64_t q = 0; q < nterms; ++q) {
            double ph = 0;
            for (int t = 0; t < d; ++t) {
                double v = (double)kvec[q * d + t] * x[j * d + t];
                ph += v - floor(v);
            }
            ph -= floor(ph);
            double s, c;
            sincospi(2.0 * ph, &s, &c);
            re += coef[2 * q] * c - coef[2 * q + 1] * s;
            im += coef[2 * q] * s + coef[2 * q + 1] * c;
        }
        y[2 * j] = re;
        y[2 * j + 1] = im;
    }
}

int launch_sop_coefs(const double* theta, int n_terms, int K, double width, double* a, double* da, cudaStream_t st) {
    SFFT_CHECK(n_terms >= 1 && n_terms <= kMaxTerms && K >= 0 && K <= kMaxK, SFFT_EINVAL,
               "sum-of-products: need 1 <= n_terms <= %d and 0 <= K <= %d", kMaxTerms, kMaxK);
    int tot = n_terms * (K + 1);
    k_sop_coefs<<<(tot + 255) / 256, 256, 0, st>>>(theta, n_terms, K, width, a, da);
    return launch_check("k_sop_coefs");
}

int launch_sop_sample(const InstDesc* di, const int32_t* triples_dev, int n_terms, int K, const double* a, void* out,
                      int prec, cudaStream_t st) {
    if (prec) k_sop_sample<float><<<4 * 152, 256, 0, st>>>(di, triples_dev, n_terms, K, a, out);
    else k_sop_sample<double><<<4 * 152, 256, 0, st>>>(di, triples_dev, n_terms, K, a, out);
    return launch_check("k_sop_sample");
}

int launch_sop_backward(const InstDesc* di, const int32_t* triples_dev, int n_terms, int K, const double* a,
                        const double* da, const void* dsamples, int prec, double* dtheta, cudaStream_t st) {
    if (prec) k_sop_backward<float><<<2 * 152, 256, 0, st>>>(di, triples_dev, n_terms, K, a, da, dsamples, dtheta);
    else k_sop_backward<double><<<2 * 152, 256, 0, st>>>(di, triples_dev, n_terms, K, a, da, dsamples, dtheta);
    return launch_check("k_sop_backward");
}

int launch_sop_eval_points(const double* x, int64_t n, int d, const int32_t* triples_dev, int n_terms, int K,
                           const double* a, double* y, cudaStream_t st) {
    int gx = (int)std::min<int64_t>(4 * 152, (n + 255) / 256 + 1);
    k_sop_eval_points<<<gx, 256, 0, st>>>(x, n, d, triples_dev, n_terms, K, a, y);
    return launch_check("k_sop_eval_points");
}

int launch_sparse_eval_points(const double* x, int64_t n, int d, const int32_t* kvec, const double* coef,
                              int64_t nterms, double* y, cudaStream_t st) {
    int gx = (int)std::min<int64_t>(8 * 152, (n + 127) / 128 + 1);
    k_sparse_eval_points<<<gx, 128, 0, st>>>(x, n, d, kvec, coef, nterms, y);
    return launch_check("k_sparse_eval_points");
}

}  // namespace sfft
