// Hash + count (Algorithm 2, lines 4-6) with the inner products k.z_l on the tensor cores.
//
// For a tile of 128 candidates the products k.z_l of all L lattices form one small GEMM
// D = A B^T: A [128 x 2d] holds each candidate's k twice, B [L x 2d] holds z_l split as
// (z mod 128, 128 floor(z / 128)), so every entry of both is an integer that bf16 represents
// exactly and D[i, l] = k_i.z_l.  One tcgen05.mma (kind::f16, bf16 inputs, FP32 accumulator in
// tensor memory) per 16 of 2d computes D; while |k.z| < 2^24 every partial sum is an integer
// that FP32 holds exactly.  The epilogue reads a thread's row of D with tcgen05.ld and reduces
// each entry modulo M_l in FP32 (round-to-nearest quotient through the 1.5 * 2^23 shift, exact
// FMA remainder, one correction), then tests the lattice's bit of the non-zero bitmap.
// Operands live in shared memory in the K-major layout without swizzle: core matrices of 8 rows
// x 16 bytes, 128 bytes apart along K, 8-row groups (2d padded to 32: 512 bytes) apart along M/N.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace sfft {

constexpr int kTcThreads = 128;  // one candidate per thread and tile, TMEM lane = thread
constexpr int kTcK = 32;         // 2d padded to 32 (d <= 16)
constexpr int kTcCols = 64;      // TMEM columns: L <= 64
constexpr float kTcMagic = 12582912.0f;  // 1.5 * 2^23: x + magic rounds x to an integer

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ int kmaj_off(int r, int k) {  // byte offset of element (r, k)
    return (r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {  // LBO 128 B (K), SBO 512 B (M/N)
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
           (1ull << 46);
}

size_t hash_tc_smem_bytes(int L, int64_t nwords) {
    return (size_t)128 * kTcK * 2 + (size_t)kTcCols * kTcK * 2 + sizeof(float4) * (size_t)L +
           sizeof(uint32_t) * (size_t)nwords + 64;
}

// mode bit 0: first lattice group (counts start at 0), bit 1: last group (threshold); the host
// uses this kernel only for plans with one lattice group (mode 3)
__global__ void __launch_bounds__(kTcThreads) k_hash_count_tc(const InstDesc* __restrict__ insts) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const InstDesc& I = insts[blockIdx.y];
    const int L = I.L, d = I.d, tid = threadIdx.x, warp = tid >> 5;
    const int nwords = I.nwords;
    unsigned char* sa = tsm;                                   // A tile [128 x 32] bf16
    unsigned char* sb = sa + 128 * kTcK * 2;                   // B [64 x 32] bf16
    float4* cst = reinterpret_cast<float4*>(sb + kTcCols * kTcK * 2);  // {M, 1/M, bit offset + magic, -}
    uint32_t* bits = reinterpret_cast<uint32_t*>(cst + L);
    for (int i = tid; i < nwords; i += blockDim.x) bits[i] = I.nzbits[i];
    for (int e = tid; e < 128 * kTcK / 2; e += blockDim.x) reinterpret_cast<uint32_t*>(sa)[e] = 0u;
    for (int e = tid; e < kTcCols * kTcK; e += blockDim.x) {
        const int n = e / kTcK, k = e % kTcK;
        float v = 0.f;
        if (n < L && k < 2 * d) {
            const int z = I.z[n * d + (k < d ? k : k - d)];
            v = k < d ? (float)(z & 127) : (float)(z & ~127);  // z = (z mod 128) + 128 floor(z / 128)
        }
        *reinterpret_cast<__nv_bfloat16*>(sb + kmaj_off(n, k)) = __float2bfloat16(v);
    }
    for (int l = tid; l < L; l += blockDim.x) {
        const float M = (float)I.Ml[l];
        cst[l] = make_float4(M, 1.0f / M, (float)(I.boff[l] * 32) + kTcMagic, 0.f);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                     "n"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = tslot;
    const int ks = (2 * d + 15) / 16;  // K = 16 steps
    const int npad = (L + 15) & ~15;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(npad >> 3) << 17) | (8u << 24);
    // base of the bitmap words addressed by (float bits of bit + magic) >> 5: magic's bits are a
    // multiple of 32, so word = bits_base[float_bits >> 5] and the bit is float_bits & 31
    const uint32_t* bits_base = bits - (0x4B400000u >> 5);
    const int64_t n = I.n;
    const int need = I.need;
    const uint32_t* cand8w = reinterpret_cast<const uint32_t*>(I.cand);
    const int32_t* cand32 = reinterpret_cast<const int32_t*>(I.cand);
    const int ld = I.cand_ld;
    const int64_t ntiles = (n + 127) / 128;
    uint32_t phase = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t idx = tile * 128 + tid;
        // ---- A row of this thread's candidate: (k, k) in bf16 (zeros past the end of Gamma)
        if (idx >= n) {
            for (int t = 0; t < 2 * d; ++t) *reinterpret_cast<__nv_bfloat16*>(sa + kmaj_off(tid, t)) = __float2bfloat16(0.f);
        } else {
            if (I.cand_i8) {
                const uint32_t* row = cand8w + idx * (ld >> 2);
                for (int w = 0; w < (d + 3) / 4; ++w) {
                    const uint32_t word = __ldg(row + w);
                    for (int b = 0; b < 4 && 4 * w + b < d; ++b) {
                        const int t = 4 * w + b;
                        const __nv_bfloat16 v = __float2bfloat16((float)(int8_t)(word >> (8 * b)));
                        *reinterpret_cast<__nv_bfloat16*>(sa + kmaj_off(tid, t)) = v;
                        *reinterpret_cast<__nv_bfloat16*>(sa + kmaj_off(tid, d + t)) = v;
                    }
                }
            } else {
                for (int t = 0; t < d; ++t) {
                    const __nv_bfloat16 v = __float2bfloat16((float)__ldg(cand32 + idx * ld + t));
                    *reinterpret_cast<__nv_bfloat16*>(sa + kmaj_off(tid, t)) = v;
                    *reinterpret_cast<__nv_bfloat16*>(sa + kmaj_off(tid, d + t)) = v;
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---- D = A B^T in tensor memory
        if (tid == 0) {
            for (int s = 0; s < ks; ++s) {
                const uint64_t ad = smem_desc(smem_u32(sa) + s * 256), bd = smem_desc(smem_u32(sb) + s * 256);
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
                             "l"(ad), "l"(bd), "r"(idesc), "r"(s));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar)));
        }
        uint32_t done = 0;
        for (int spin = 0; spin < (1 << 24) && !done; ++spin) {
            asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                         "selp.b32 %0, 1, 0, q;\n\t}"
                         : "=r"(done)
                         : "r"(smem_u32(&mbar)), "r"(phase));
        }
        phase ^= 1u;
        if (__syncthreads_or(!done)) {  // the MMA never completed: report and stop (no hang)
            if (tid == 0) atomicOr((unsigned long long*)&I.cnt[3], (unsigned long long)ERR_TC_TIMEOUT);
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---- epilogue: count the lattices whose bucket of k is non-zero
        int cnt = 0;
        for (int c0 = 0; c0 < L; c0 += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int l = c0 + j;
                if (l < L) {
                    const float4 c = cst[l];
                    const float x = __uint_as_float(v[j]);
                    const float q = __fadd_rn(__fmaf_rn(x, c.y, kTcMagic), -kTcMagic);  // round(x / M)
                    float r = __fmaf_rn(-q, c.x, x);                                      // exact, |r| < M
                    r = r < 0.f ? __fadd_rn(r, c.x) : r;
                    const uint32_t fb = __float_as_uint(__fadd_rn(r, c.z));  // bits of (bit + magic)
                    cnt += (bits_base[fb >> 5] >> (fb & 31)) & 1u;
                }
            }
            // count rule (Algorithm 1): stop once no candidate of the warp can still reach need
            const int rem = L - min(L, c0 + 16);
            if (!__any_sync(0xffffffffu, idx < n && cnt + rem >= need)) break;
        }
        if (idx < n && cnt >= need) atomicOr(&I.detbits[idx >> 5], 1u << (idx & 31));
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();  // tensor memory read and A free before the next tile's MMA
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(kTcCols));
}

int launch_hash_count_tc(const InstDesc* di, int ninst, int gx, size_t smem, cudaStream_t st) {
    static bool attr_done = false;
    if (!attr_done) {
        SFFT_CU(cudaFuncSetAttribute(k_hash_count_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
        attr_done = true;
    }
    k_hash_count_tc<<<dim3(gx, ninst), kTcThreads, smem, st>>>(di);
    return launch_check("k_hash_count_tc");
}

}  // namespace sfft
