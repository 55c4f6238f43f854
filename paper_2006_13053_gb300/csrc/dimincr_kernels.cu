// Device kernels of the dimension-incremental driver (Algorithm 3): the pairing of the
// already identified index sets into the candidate set J_t, the assembly of the full
// d-dimensional sampling nodes (lattice coordinates followed by the random tail), precision
// conversion of black-box samples and the gather of selected candidate rows.
#include "common.cuh"
#include "kernels.cuh"

namespace sfft {

// J_t = I^(1..t-1) x I^(t): row a*nt + b = (prev[a, 0..t-1], cur[b])  (t = columns of prev)
__global__ void k_pairing(const int32_t* __restrict__ prev, int64_t np, int t, const int32_t* __restrict__ cur, int nt,
                          int32_t* __restrict__ out) {
    const int64_t tot = np * nt;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < tot; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = r / nt;
        const int b = (int)(r - a * nt);
        int32_t* o = out + r * (t + 1);
        for (int u = 0; u < t; ++u) o[u] = prev[a * t + u];
        o[t] = cur[b];
    }
}

// X[j, 0..tc-1] = lattice node coordinates, X[j, tc..d-1] = tail[tc..d-1]
__global__ void k_assemble_nodes(const double* __restrict__ xl, int64_t n, int tc, const double* __restrict__ tail, int d,
                                 double* __restrict__ X) {
    const int64_t tot = n * d;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / d;
        const int u = (int)(e - j * d);
        X[e] = u < tc ? xl[j * tc + u] : tail[u];
    }
}

// Step 1 nodes: X[l, u] = tail[u] for u != t, X[l, t] = l / K
__global__ void k_step1_nodes(const double* __restrict__ tail, int d, int t, int K, double* __restrict__ X) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * d; e += gridDim.x * blockDim.x) {
        const int l = e / d, u = e - l * d;
        X[e] = u == t ? (double)l / (double)K : tail[u];
    }
}

__global__ void k_c64_to_c32(const c64* __restrict__ a, c32* __restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = c32{(float)a[i].x, (float)a[i].y};
}

// rows[q, :] = J[idx[q], :]
__global__ void k_gather_rows(const int32_t* __restrict__ J, int w, const int64_t* __restrict__ idx, int64_t n,
                              int32_t* __restrict__ rows) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * w; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e / w;
        rows[e] = J[idx[q] * w + (e - q * w)];
    }
}

static int grid_for(int64_t n) { return (int)std::min<int64_t>(4 * 152, (n + 255) / 256 + 1); }

int launch_pairing(const int32_t* prev, int64_t np, int t, const int32_t* cur, int nt, int32_t* out, cudaStream_t st) {
    k_pairing<<<grid_for(np * nt), 256, 0, st>>>(prev, np, t, cur, nt, out);
    return launch_check("k_pairing");
}
int launch_assemble_nodes(const double* xl, int64_t n, int tc, const double* tail, int d, double* X, cudaStream_t st) {
    k_assemble_nodes<<<grid_for(n * d), 256, 0, st>>>(xl, n, tc, tail, d, X);
    return launch_check("k_assemble_nodes");
}
int launch_step1_nodes(const double* tail, int d, int t, int K, double* X, cudaStream_t st) {
    k_step1_nodes<<<grid_for((int64_t)K * d), 256, 0, st>>>(tail, d, t, K, X);
    return launch_check("k_step1_nodes");
}
int launch_c64_to_c32(const c64* a, c32* b, int64_t n, cudaStream_t st) {
    k_c64_to_c32<<<grid_for(n), 256, 0, st>>>(a, b, n);
    return launch_check("k_c64_to_c32");
}
int launch_gather_rows(const int32_t* J, int w, const int64_t* idx, int64_t n, int32_t* rows, cudaStream_t st) {
    if (n <= 0) return SFFT_OK;
    k_gather_rows<<<grid_for(n * w), 256, 0, st>>>(J, w, idx, n, rows);
    return launch_check("k_gather_rows");
}

}  // namespace sfft
