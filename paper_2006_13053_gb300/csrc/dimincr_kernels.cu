// Device kernels of the dimension-incremental driver (Algorithm 3): the pairing of the
// already identified index sets into the candidate set J_t, the assembly of the full
// d-dimensional sampling nodes (lattice coordinates followed by the random tail), the random
// node components, Step 1's selection of the s_local largest projections, the union of the
// r Step-2 calls (scatter by candidate index + ordered compaction), precision conversion of
// black-box samples and the gathers of selected candidate rows and coefficients.  The index sets
// I^(t), I^(1..t) and J_t never leave the device.
#include <limits.h>

#include "common.cuh"
#include "kernels.cuh"
#include "philox.cuh"

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

// out[u] = U01(c0 = u, c1, c2, c3) for u < d: the random node components of Algorithm 3
__global__ void k_philox_tail(uint64_t key, uint64_t c1, uint64_t c2, uint64_t c3, int d, double* __restrict__ out) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < d) out[u] = philox4x64_u01(key, (uint64_t)u, c1, c2, c3);
}

constexpr int kSel1Threads = 1024;

// exclusive block scan of 0/1 flags (all threads of the block call it); returns the prefix and
// the block total
__device__ int block_scan01(int f, int* sh, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned b = __ballot_sync(0xffffffffu, f);
    const int pre_w = __popc(b & ((1u << lane) - 1u));
    __syncthreads();
    if (lane == 0) sh[warp] = __popc(b);
    __syncthreads();
    if (warp == 0) {
        int v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        sh[32 + lane] = v;  // inclusive
    }
    __syncthreads();
    *total = sh[32 + (blockDim.x >> 5) - 1];
    const int r = pre_w + (warp > 0 ? sh[32 + warp - 1] : 0);
    __syncthreads();
    return r;
}

// Step 1 selection (Algorithm 3, Step 1c): the projections v_q = ph[(lo + q) mod K], q < K, of the
// coordinate's K-point DFT; keep the s_keep largest moduli among those >= theta = max(theta_abs,
// theta_rel max |v|) (ties and equal rank keys: lower q first) and OR them into mask[q].  One CTA:
// a radix select over the rank keys of the moduli (8 passes of 8 bits), then an ordered scan for
// the moduli equal to the s_keep-th key.  mag: global scratch of K doubles.
__global__ void __launch_bounds__(kSel1Threads) k_step1_select(const c64* __restrict__ ph, int K, int lo,
                                                               int64_t s_keep, double theta_abs, double theta_rel,
                                                               int rank_bits, double* __restrict__ mag,
                                                               uint8_t* __restrict__ mask) {
    __shared__ unsigned int hist[256];
    __shared__ int shi[72];
    __shared__ double smax[32];
    __shared__ long long sl[2];
    double mx = 0;
    for (int q = threadIdx.x; q < K; q += blockDim.x) {
        int h = (lo + q) % K;
        if (h < 0) h += K;
        const c64 v = ph[h];
        const double a = hypot(v.x, v.y);
        mag[q] = a;
        mx = fmax(mx, a);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
    __syncthreads();  // also orders the mag[] writes before the reads below (same block)
    if (threadIdx.x == 0) {
        double m = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, smax[i]);
        smax[0] = m;
    }
    __syncthreads();
    const double theta = fmax(theta_abs, theta_rel * smax[0]);
    int kept = 0;
    for (int q = threadIdx.x; q < K; q += blockDim.x) kept += mag[q] >= theta;
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) shi[threadIdx.x >> 5] = kept;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += shi[i];
        shi[0] = t;
    }
    __syncthreads();
    kept = shi[0];
    __syncthreads();
    if (s_keep < 0 || kept <= s_keep) {
        for (int q = threadIdx.x; q < K; q += blockDim.x)
            if (mag[q] >= theta) mask[q] = 1;
        return;
    }
    unsigned long long prefix = 0, msk = 0;
    long long need = s_keep;
    for (int p = 7; p >= 0; --p) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int q = threadIdx.x; q < K; q += blockDim.x) {
            const unsigned long long key = rank_key(mag[q], rank_bits);
            if (mag[q] >= theta && (key & msk) == prefix) atomicAdd(&hist[(key >> (8 * p)) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long acc = 0;
            int b = 255;
            for (; b > 0; --b) {
                if (acc + hist[b] >= need) break;
                acc += hist[b];
            }
            sl[0] = acc;
            sl[1] = b;
        }
        __syncthreads();
        need -= sl[0];
        prefix |= (unsigned long long)sl[1] << (8 * p);
        msk |= 255ull << (8 * p);
        __syncthreads();
    }
    // keys above the s_keep-th key, plus the first `need` equal keys in position order
    long long eq_taken = 0;
    for (int q0 = 0; q0 < K; q0 += blockDim.x) {
        const int q = q0 + threadIdx.x;
        int eq = 0, sel = 0;
        if (q < K && mag[q] >= theta) {
            const unsigned long long key = rank_key(mag[q], rank_bits);
            if (key > prefix) sel = 1;
            else if (key == prefix) eq = 1;
        }
        int tot;
        const int pre = block_scan01(eq, shi, &tot);
        if (eq && eq_taken + pre < need) sel = 1;
        eq_taken += tot;
        if (sel) mask[q] = 1;
    }
}

// union of the r Step-2 calls: flag[supp[q]] = 1 and acc[supp[q]] = coef[q] (a later call, run
// after this one on the same stream, overwrites an earlier coefficient of the same candidate)
__global__ void k_union_scatter(const int64_t* __restrict__ supp, const c64* __restrict__ coef, int64_t n,
                                uint8_t* __restrict__ flag, c64* __restrict__ acc) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = supp[q];
        flag[i] = 1;
        acc[i] = coef[q];
    }
}

// ordered compaction of 0/1 flags: block b owns the chunk [b ch, (b + 1) ch); pass 0 counts, pass 1
// starts at the sum of the counts of the chunks before its own and writes the positions in order
constexpr int kFlagThreads = 256;

__global__ void __launch_bounds__(kFlagThreads) k_flag_compact(const uint8_t* __restrict__ flag, int64_t n, int64_t ch,
                                                               int pass, int64_t* __restrict__ counts,
                                                               int64_t* __restrict__ out, int64_t* __restrict__ total) {
    __shared__ int shi[72];
    __shared__ long long sbase;
    const int64_t c0 = min(n, (int64_t)blockIdx.x * ch), c1 = min(n, c0 + ch);
    if (pass == 0) {
        int cnt = 0;
        for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) cnt += flag[i] != 0;
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if ((threadIdx.x & 31) == 0) shi[threadIdx.x >> 5] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += shi[i];
            counts[blockIdx.x] = t;
        }
        return;
    }
    if (threadIdx.x == 0) {
        long long b = 0;
        for (int i = 0; i < (int)blockIdx.x; ++i) b += counts[i];
        sbase = b;
        if (blockIdx.x == gridDim.x - 1) *total = b + counts[blockIdx.x];
    }
    __syncthreads();
    long long pos = sbase;
    for (int64_t i0 = c0; i0 < c1; i0 += blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        const int f = i < c1 && flag[i] != 0;
        int tot;
        const int pre = block_scan01(f, shi, &tot);
        if (f) out[pos + pre] = i;
        pos += tot;
    }
}

// out[q] = v[idx[q]]
__global__ void k_gather_c64(const c64* __restrict__ v, const int64_t* __restrict__ idx, int64_t n, c64* __restrict__ out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = v[idx[q]];
}

// I^(t) values from Step 1's positions: out[q] = lo + pos[q]
__global__ void k_positions_to_values(const int64_t* __restrict__ pos, int64_t n, int lo, int32_t* __restrict__ out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = lo + (int32_t)pos[q];
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
int launch_philox_tail(uint64_t key, uint64_t c1, uint64_t c2, uint64_t c3, int d, double* out, cudaStream_t st) {
    k_philox_tail<<<(d + 63) / 64, 64, 0, st>>>(key, c1, c2, c3, d, out);
    return launch_check("k_philox_tail");
}
int launch_step1_select(const c64* ph, int K, int lo, int64_t s_keep, double theta_abs, double theta_rel, int rank_bits,
                        double* mag, uint8_t* mask, cudaStream_t st) {
    k_step1_select<<<1, kSel1Threads, 0, st>>>(ph, K, lo, s_keep, theta_abs, theta_rel, rank_bits, mag, mask);
    return launch_check("k_step1_select");
}
int launch_union_scatter(const int64_t* supp, const c64* coef, int64_t n, uint8_t* flag, c64* acc, cudaStream_t st) {
    if (n <= 0) return SFFT_OK;
    k_union_scatter<<<grid_for(n), 256, 0, st>>>(supp, coef, n, flag, acc);
    return launch_check("k_union_scatter");
}
int64_t flag_compact_blocks(int64_t n) { return std::max<int64_t>(1, std::min<int64_t>(1024, (n + 4095) / 4096)); }
int launch_flag_compact(const uint8_t* flag, int64_t n, int64_t* counts, int64_t* out, int64_t* total, cudaStream_t st) {
    const int64_t B = flag_compact_blocks(n), ch = (n + B - 1) / B;
    for (int pass = 0; pass < 2; ++pass) {
        k_flag_compact<<<(int)B, kFlagThreads, 0, st>>>(flag, n, ch, pass, counts, out, total);
        SFFT_TRY(launch_check("k_flag_compact"));
    }
    return SFFT_OK;
}
int launch_gather_c64(const c64* v, const int64_t* idx, int64_t n, c64* out, cudaStream_t st) {
    if (n <= 0) return SFFT_OK;
    k_gather_c64<<<grid_for(n), 256, 0, st>>>(v, idx, n, out);
    return launch_check("k_gather_c64");
}
int launch_positions_to_values(const int64_t* pos, int64_t n, int lo, int32_t* out, cudaStream_t st) {
    if (n <= 0) return SFFT_OK;
    k_positions_to_values<<<grid_for(n), 256, 0, st>>>(pos, n, lo, out);
    return launch_check("k_positions_to_values");
}

}  // namespace sfft
