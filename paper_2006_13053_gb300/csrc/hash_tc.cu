// Hash + count (Algorithm 2) with the inner products k.z_l on the tensor cores.
//
// For a tile of 128 candidates the products k.z_l of all L lattices form one small GEMM
// D = A B^T: A [128 x 2H] holds each candidate's k at K offsets 0 and H (H = 8 for d <= 8, else
// 16), B [L x 2H] holds z_l split as (z mod 128) at 0 and 128 floor(z / 128) at H, so every entry
// of both is an integer that bf16 represents exactly and D[i, l] = k_i.z_l.  One tcgen05.mma (kind::f16, bf16 inputs, FP32 accumulator in
// tensor memory) per 16 of 2H computes D; while |k.z| < 2^24 every partial sum is an integer
// that FP32 holds exactly.  The epilogue reads a thread's row of D with tcgen05.ld and reduces
// each entry modulo M_l in FP32 (round-to-nearest quotient through the 1.5 * 2^23 shift, exact
// FMA remainder, one correction), then tests the lattice's bit of the non-zero bitmap.
// Operands live in shared memory in the K-major layout without swizzle: core matrices of 8 rows
// x 16 bytes, 128 bytes apart along K, 8-row groups 512 bytes apart along M/N (room for K = 32).
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
    return (size_t)2 * 128 * kTcK * 2 + (size_t)kTcCols * kTcK * 2 + sizeof(float4) * (size_t)L +
           sizeof(uint32_t) * (size_t)nwords + 64;
}

// Two groups of four warps per CTA work on alternate tiles, each with its own A buffer, 64
// tensor-memory columns and mbarrier, so one group's epilogue overlaps the other's MMA; each
// group loads its next tile's candidate rows into registers before waiting for its MMA.  The
// host uses this kernel only for plans with one lattice group and without diagnostics.
constexpr int kTcGroups = 2;

__device__ __forceinline__ void group_sync(int g) {  // named barrier of the 128 threads of group g
    asm volatile("bar.sync %0, 128;" ::"r"(1 + g));
}

__global__ void __launch_bounds__(kTcThreads * kTcGroups) k_hash_count_tc(const InstDesc* __restrict__ insts) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) uint64_t mbar[kTcGroups];
    __shared__ uint32_t tslot;
    __shared__ int gfail[kTcGroups];
    const InstDesc& I = insts[blockIdx.y];
    const int L = I.L, d = I.d, tid = threadIdx.x, warp = tid >> 5;
    const int g = warp >> 2, lt = tid & 127;  // group, thread (= tensor-memory lane) in the group
    const int H = d <= 8 ? 8 : 16;            // K offset of the second copy of k; K = 2 H
    const int nwords = I.nwords;
    unsigned char* sb = tsm;                                           // B [64 x 32] bf16
    unsigned char* sa = sb + kTcCols * kTcK * 2 + g * 128 * kTcK * 2;  // this group's A [128 x 32]
    float4* cst = reinterpret_cast<float4*>(tsm + kTcCols * kTcK * 2 + kTcGroups * 128 * kTcK * 2);
    uint32_t* bits = reinterpret_cast<uint32_t*>(cst + L);
    copy_words_to_smem(bits, I.nzbits, nwords);
    for (int e = tid; e < kTcGroups * 128 * kTcK / 2; e += blockDim.x)
        reinterpret_cast<uint32_t*>(tsm + kTcCols * kTcK * 2)[e] = 0u;
    for (int e = tid; e < kTcCols * kTcK; e += blockDim.x) {
        const int nn = e / kTcK, k = e % kTcK;
        float v = 0.f;
        if (nn < L && (k % H) < d && k < 2 * H) {
            const int z = I.z[nn * d + (k % H)];
            v = k < H ? (float)(z & 127) : (float)(z & ~127);  // z = (z mod 128) + 128 floor(z / 128)
        }
        *reinterpret_cast<__nv_bfloat16*>(sb + kmaj_off(nn, k)) = __float2bfloat16(v);
    }
    for (int l = tid; l < L; l += blockDim.x) {
        const float M = (float)I.Ml[l];
        cst[l] = make_float4(M, 1.0f / M, (float)(I.boff[l] * 32) + kTcMagic, 0.f);
    }
    if (tid < kTcGroups) {
        gfail[tid] = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[tid])));
    }
    if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                     "n"(kTcCols * kTcGroups));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = tslot + (uint32_t)(g * kTcCols);
    const int ks = H / 8;  // K = 16 steps: 2 H / 16
    const int npad = (L + 15) & ~15;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(npad >> 3) << 17) | (8u << 24);
    // base of the bitmap words addressed by (float bits of bit + magic) >> 5: magic's bits are a
    // multiple of 32, so word = bits_base[float_bits >> 5] and the bit is float_bits & 31
    const uint32_t* bits_base = bits - (0x4B400000u >> 5);
    const int64_t n = I.n;
    const int need = I.need;
    const uint32_t* cand8w = reinterpret_cast<const uint32_t*>(I.cand);
    const int32_t* cand32 = reinterpret_cast<const int32_t*>(I.cand);
    const int ld = I.cand_ld, kw = (d + 3) / 4;
    const bool i8 = I.cand_i8 != 0;
    const int64_t ntiles = (n + 127) / 128;
    const int64_t tstep = (int64_t)gridDim.x * kTcGroups;
    // candidate row of tile t in registers (int8 words or int32 entries)
    uint32_t rw[16];
    auto load_row = [&](int64_t t) {
        const int64_t idx = t * 128 + lt;
        if (t >= ntiles || idx >= n) return;
        if (i8) {
#pragma unroll
            for (int w = 0; w < 4; ++w)
                if (w < kw) rw[w] = __ldg(cand8w + idx * (ld >> 2) + w);
        } else {
#pragma unroll
            for (int u = 0; u < 16; ++u)
                if (u < d) rw[u] = (uint32_t)__ldg(cand32 + idx * ld + u);
        }
    };
    uint32_t phase = 0;
    int64_t tile = (int64_t)blockIdx.x * kTcGroups + g;
    load_row(tile);
    for (; tile < ntiles; tile += tstep) {
        const int64_t idx = tile * 128 + lt;
        // ---- A row of this thread's candidate: (k, k) in bf16 (zeros past the end of Gamma)
        // one 16-byte store per core-matrix row chunk of 8 entries, for both copies of k
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (8 * c < H) {
                uint32_t pk[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    uint32_t w2 = 0;
#pragma unroll
                    for (int e2 = 0; e2 < 2; ++e2) {
                        const int u = 8 * c + 2 * h + e2;
                        int k = 0;
                        if (u < d && idx < n) k = i8 ? (int)(int8_t)(rw[u >> 2] >> (8 * (u & 3))) : (int)rw[u];
                        w2 |= (uint32_t)__bfloat16_as_ushort(__float2bfloat16((float)k)) << (16 * e2);
                    }
                    pk[h] = w2;
                }
                const uint4 q4 = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                *reinterpret_cast<uint4*>(sa + kmaj_off(lt, 8 * c)) = q4;
                *reinterpret_cast<uint4*>(sa + kmaj_off(lt, H + 8 * c)) = q4;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        group_sync(g);
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---- D = A B^T in this group's tensor-memory columns
        if (lt == 0) {
            for (int s = 0; s < ks; ++s) {
                const uint64_t ad = smem_desc(smem_u32(sa) + s * 256), bd = smem_desc(smem_u32(sb) + s * 256);
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
                             "l"(ad), "l"(bd), "r"(idesc), "r"(s));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar[g])));
        }
        load_row(tile + tstep);  // the next tile's rows load while the MMA runs
        if (lt == 0) {  // one waiter per group; the others wait at the group barrier
            uint32_t done = 0;
            for (int spin = 0; spin < (1 << 24) && !done; ++spin) {
                asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                             "selp.b32 %0, 1, 0, q;\n\t}"
                             : "=r"(done)
                             : "r"(smem_u32(&mbar[g])), "r"(phase));
            }
            if (!done) gfail[g] = 1;
        }
        phase ^= 1u;
        group_sync(g);
        if (gfail[g]) {  // the MMA never completed: report and stop this group (no hang)
            if (lt == 0) atomicOr((unsigned long long*)&I.cnt[3], (unsigned long long)ERR_TC_TIMEOUT);
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
                : "r"(taddr + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0));
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
        if (idx < n && cnt >= need) mark_detected(I, idx);
        asm volatile("tcgen05.fence::before_thread_sync;");
        group_sync(g);  // tensor memory read and A free before this group's next MMA
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tslot), "n"(kTcCols * kTcGroups));
}

int launch_hash_count_tc(const InstDesc* di, int ninst, int gx, size_t smem, cudaStream_t st) {
    SFFT_TRY(allow_smem((const void*)k_hash_count_tc, 220 * 1024));
    k_hash_count_tc<<<dim3(gx, ninst), kTcThreads * kTcGroups, smem, st>>>(di);
    return launch_check("k_hash_count_tc");
}

}  // namespace sfft
