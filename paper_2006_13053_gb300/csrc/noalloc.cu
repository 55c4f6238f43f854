// Detection step (zero test, candidate hashing with the majority count, ascending compaction)
// for callers that must not allocate device memory, e.g. code running inside a host callback,
// a custom allocator or a memory-capped service process where cudaMalloc is forbidden or could
// fail mid-run.  All scratch (the non-zero bitmap, the per-candidate detection bits, the lattice
// constants, the counters and the instance descriptor) lives in one file-scope device array of
// fixed size that every GPU loading this library holds until the process exits.  The caller
// passes only inputs and outputs.  Every call shares this array and leaves its contents behind;
// calls whose work overlaps on the GPU (different streams, or threads of one process) race on it.
#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace sfft {
namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;  // 8 MiB per device
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// device address of the scratch array on the current device.  Looked up at every call (cheap), so
// that a device reset or a re-created primary context between calls cannot leave a stale address.
int scratch_address(void** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
        set_error("cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
        return SFFT_ECUDA;
    }
    *out = p;
    return SFFT_OK;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// non-zero bitmap from given FP64 lattice DFTs: bit h of lattice l is |ghat^(l)_h| > tau_l
__global__ void k_nz_from_ghat(const c64* __restrict__ ghat, const InstDesc* __restrict__ inst,
                               const double* __restrict__ tau) {
    const InstDesc& I = *inst;
    const int l = blockIdx.x;
    const int M = I.Ml[l];
    const c64* g = ghat + I.soff[l];
    uint32_t* words = I.nzbits + I.boff[l];
    const int nw = (M + 31) >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const double t = tau[l];
    for (int wi = warp; wi < nw; wi += nwarp) {
        int h = wi * 32 + lane;
        bool nz = false;
        if (h < M) nz = sqrt(abs2(g[h])) > t;
        uint32_t b = __ballot_sync(0xffffffffu, nz);
        if (lane == 0) words[wi] = b;
    }
}

}  // namespace
}  // namespace sfft

using namespace sfft;

extern "C" int sfft_detect_noalloc(int d, const int32_t* cand, int64_t n_cand, int L, const int64_t* M,
                                   const int64_t* z, const double* ghat, const double* tau, double nu,
                                   int64_t* detected_out, int64_t cap, int64_t* n_detected, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    SFFT_CHECK(d >= 1 && d <= kMaxD && L >= 1 && L <= kMaxL, SFFT_EINVAL, "need 1 <= d <= %d and 1 <= L <= %d", kMaxD,
               kMaxL);
    SFFT_CHECK(cand && n_cand >= 1 && M && z && ghat && tau && n_detected && (cap == 0 || detected_out), SFFT_EINVAL,
               "null argument");
    SFFT_CHECK(nu > 0 && nu <= 0.5, SFFT_EINVAL, "nu must be in (0, 1/2]");
    // the hash kernels read an int32 row as int4 words (d % 4 == 0) or int2 words (d % 2 == 0)
    const uintptr_t al = d % 4 == 0 ? 16 : d % 2 == 0 ? 8 : 4;
    SFFT_CHECK((uintptr_t)cand % al == 0, SFFT_EINVAL, "candidate rows of d = %d must start %d-byte aligned", d,
               (int)al);
    // ---- scratch layout (bytes, 256-aligned pieces)
    int64_t words = 0, sumM = 0, maxM = 0;
    for (int l = 0; l < L; ++l) {
        SFFT_CHECK(M[l] >= 2 && M[l] < (1 << 27), SFFT_EINVAL, "M_%d out of range", l);
        words += (M[l] + 31) / 32;
        sumM += M[l];
        maxM = std::max<int64_t>(maxM, M[l]);
    }
    size_t off = 0;
    const size_t o_inst = off; off = align256(off + sizeof(InstDesc));
    const size_t o_z = off;    off = align256(off + sizeof(int32_t) * L * d);
    const size_t o_M = off;    off = align256(off + sizeof(int32_t) * L);
    const size_t o_mu = off;   off = align256(off + sizeof(uint32_t) * L);
    const size_t o_offk = off; off = align256(off + sizeof(uint32_t) * L);
    const size_t o_boff = off; off = align256(off + sizeof(int32_t) * L);
    const size_t o_soff = off; off = align256(off + sizeof(int64_t) * (L + 1));
    const size_t o_tau = off;  off = align256(off + sizeof(double) * L);
    const size_t o_cnt = off;  off = align256(off + sizeof(int64_t) * kCntWords);
    const size_t o_mnx = off;  off = align256(off + sizeof(int) * 2 * kMaxD);
    const size_t o_nz = off;   off = align256(off + sizeof(uint32_t) * words);
    const size_t o_det = off;  off = align256(off + sizeof(uint32_t) * ((n_cand + 31) / 32));
    SFFT_CHECK(off <= kScratchBytes, SFFT_ECAPACITY,
               "the allocation-free detection holds at most %zu bytes of scratch (needs %zu: |Gamma| = %lld, "
               "sum M = %lld); use sfft_reconstruct for larger problems",
               kScratchBytes, off, (long long)n_cand, (long long)sumM);
    void* base = nullptr;
    SFFT_TRY(scratch_address(&base));
    char* S = reinterpret_cast<char*>(base);
    // ---- candidate bounds (|k| for the overflow check and the packed kernel)
    int mnx[2 * kMaxD];
    for (int t = 0; t < kMaxD; ++t) { mnx[t] = INT32_MAX; mnx[kMaxD + t] = INT32_MIN; }
    int* dmn = reinterpret_cast<int*>(S + o_mnx);
    SFFT_CU(cudaMemcpyAsync(dmn, mnx, sizeof mnx, cudaMemcpyHostToDevice, st));
    SFFT_TRY(launch_cand_stats(cand, 0, d, n_cand, d, dmn, dmn + kMaxD, st));
    SFFT_CU(cudaMemcpyAsync(mnx, dmn, sizeof mnx, cudaMemcpyDeviceToHost, st));
    SFFT_CU(cudaStreamSynchronize(st));
    int64_t kmax = 0;
    for (int t = 0; t < d; ++t)
        kmax = std::max<int64_t>(kmax, std::max<int64_t>(std::llabs(mnx[t]), std::llabs(mnx[kMaxD + t])));
    // ---- lattice constants (host stack arrays, copied into the scratch array)
    int32_t zz[kMaxL * kMaxD], Mm[kMaxL], bo[kMaxL];
    uint32_t mu[kMaxL], offk[kMaxL];
    int64_t so[kMaxL + 1];
    so[0] = 0;
    int64_t w = 0;
    for (int l = 0; l < L; ++l) {
        const double bound = (double)d * (double)kmax * (double)(M[l] - 1);
        SFFT_CHECK(bound + (double)M[l] < 2147483647.0, SFFT_EOVERFLOW,
                   "d*max|k|*(M-1) = %.0f does not fit the exact 32-bit hash", bound);
        for (int t = 0; t < d; ++t) {
            SFFT_CHECK(z[l * d + t] >= 0 && z[l * d + t] < M[l], SFFT_EINVAL, "z[%d][%d] outside [0, M)", l, t);
            zz[l * d + t] = (int32_t)z[l * d + t];
        }
        Mm[l] = (int32_t)M[l];
        mu[l] = (uint32_t)((1ull << 32) / (uint64_t)M[l]);
        offk[l] = (uint32_t)(M[l] * ((int64_t)ceil(bound / (double)M[l]) + 1));
        bo[l] = (int32_t)w;
        w += (M[l] + 31) / 32;
        so[l + 1] = so[l] + M[l];
    }
    const bool packed = kmax <= 127 && maxM < 65536;
    const size_t smem = hash_smem_bytes(d, L, (int)words, packed);
    SFFT_CHECK(smem <= 220 * 1024, SFFT_ECAPACITY, "non-zero bitmap of %lld words does not fit shared memory",
               (long long)words);
    InstDesc I;
    memset(&I, 0, sizeof I);
    I.d = d; I.L = L; I.need = (int)ceil(nu * L - 1e-9); I.nwords = (int)words;
    I.n = n_cand; I.cap = cap;
    I.cand = cand;
    I.cand_ld = d;  // dense int32 rows
    I.z = reinterpret_cast<int32_t*>(S + o_z);
    I.Ml = reinterpret_cast<int32_t*>(S + o_M);
    I.mu = reinterpret_cast<uint32_t*>(S + o_mu);
    I.offk = reinterpret_cast<uint32_t*>(S + o_offk);
    I.boff = reinterpret_cast<int32_t*>(S + o_boff);
    I.soff = reinterpret_cast<int64_t*>(S + o_soff);
    I.cnt = reinterpret_cast<int64_t*>(S + o_cnt);
    I.nzbits = reinterpret_cast<uint32_t*>(S + o_nz);
    I.detbits = reinterpret_cast<uint32_t*>(S + o_det);
    I.det = detected_out;
    InstDesc* dI = reinterpret_cast<InstDesc*>(S + o_inst);
    SFFT_CU(cudaMemcpyAsync(dI, &I, sizeof I, cudaMemcpyHostToDevice, st));
    SFFT_CU(cudaMemcpyAsync(S + o_z, zz, sizeof(int32_t) * L * d, cudaMemcpyHostToDevice, st));
    SFFT_CU(cudaMemcpyAsync(S + o_M, Mm, sizeof(int32_t) * L, cudaMemcpyHostToDevice, st));
    SFFT_CU(cudaMemcpyAsync(S + o_mu, mu, sizeof(uint32_t) * L, cudaMemcpyHostToDevice, st));
    SFFT_CU(cudaMemcpyAsync(S + o_offk, offk, sizeof(uint32_t) * L, cudaMemcpyHostToDevice, st));
    SFFT_CU(cudaMemcpyAsync(S + o_boff, bo, sizeof(int32_t) * L, cudaMemcpyHostToDevice, st));
    SFFT_CU(cudaMemcpyAsync(S + o_soff, so, sizeof(int64_t) * (L + 1), cudaMemcpyHostToDevice, st));
    SFFT_CU(cudaMemcpyAsync(S + o_tau, tau, sizeof(double) * L, cudaMemcpyHostToDevice, st));
    // the array keeps the previous call's contents: clear what must start at zero
    SFFT_CU(cudaMemsetAsync(S + o_cnt, 0, sizeof(int64_t) * kCntWords, st));
    SFFT_CU(cudaMemsetAsync(S + o_det, 0, sizeof(uint32_t) * ((n_cand + 31) / 32), st));
    // ---- zero test, count rule, compaction
    k_nz_from_ghat<<<L, 256, 0, st>>>(reinterpret_cast<const c64*>(ghat), dI, reinterpret_cast<const double*>(S + o_tau));
    SFFT_TRY(launch_check("k_nz_from_ghat"));
    int per_sm = std::max<int>(1, std::min<int>(8, (int)((228 * 1024) / (smem + 1024))));
    int gx = (int)std::max<int64_t>(1, std::min<int64_t>((n_cand + 511) / 512, (int64_t)152 * per_sm));
    SFFT_TRY(launch_hash_count(dI, 1, d, gx, smem, packed ? 1 : 0, 0, -1, 3, st));
    SFFT_TRY(launch_compact(dI, 1, st));
    int64_t cnt0 = 0;
    SFFT_CU(cudaMemcpyAsync(&cnt0, S + o_cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SFFT_CU(cudaStreamSynchronize(st));
    *n_detected = cnt0;
    if (cnt0 > cap) {
        set_error("%lld detected candidates exceed cap = %lld", (long long)cnt0, (long long)cap);
        return SFFT_ECAPACITY;
    }
    return SFFT_OK;
}
