// Host-side plan object behind the opaque sfft_plan handle, and the argument block of the
// reconstruction stage sequence (shared by single plans and batches).
#pragma once
#include <vector>

#include "common.cuh"

namespace sfft {

// one launch of Bluestein jobs (all in shared memory or all with global scratch)
struct FftLaunch {
    const BlueJob* jobs = nullptr;
    int njobs = 0, maxN = 0;
    int mode = 1;  // work buffer: 0 global scratch, 1 shared memory, 2 two-CTA cluster
    int threads = 0;  // CTA size (0: the transform's largest; autotuned)
    int upair = 0;    // the pass pair of every pass of every job, or 0 (uniform_pair)
};
// one launch of the hash-count kernel over a contiguous range of instances of equal d
struct HashGroup {
    int off = 0, count = 0, d = 0, gx = 1, gx0 = 1, variant = 0;  // gx0: one-wave grid (autotune base)
    int64_t tiles = 1 << 30;                                       // CTA count beyond which CTAs idle
    int l0 = 0, l1 = -1, mode = 3;  // lattice group and first/last flags (see launch_hash_count)
    size_t smem = 0;
    // the tensor-core kernel's launch, when every plan of the group qualifies (the autotuner
    // switches to it if it measures faster)
    bool tc_ok = false;
    int tc_gx0 = 1;
    int64_t tc_tiles = 1;
    size_t tc_smem = 0;
};

// optional per-stage CUDA-event timing of the stage sequence
enum Stage : int {
    ST_CLEAR = 0, ST_FFT_FWD, ST_ZERO_TEST, ST_HASH, ST_COMPACT, ST_DET_HASH, ST_COMBINE,
    ST_LSQ, ST_SCATTER, ST_DELTA, ST_SELECT, ST_COUNT
};
struct StageTimer {
    cudaEvent_t ev[ST_COUNT + 1];
    bool recorded[ST_COUNT + 1];
};

struct PipeArgs {
    StageTimer* timer = nullptr;
    int ninst = 1, nlat = 0, prec = 0;
    int fwd_prec = 0;  // arithmetic of the forward transforms (2 = double-float for FP32 + refinement)
    int64_t maxcap = 0;
    int hybrid = 0, refine = 0, lsq = 0;
    // 0: the whole stage sequence; 1: through the combine, then the detected coefficients summed
    // into FP64 buckets C (a shard's part of the refinement's C); 2: the refinement update on a C
    // given in the buckets, then Algorithm 4 (the second half of a sharded reconstruction)
    int phase = 0;
    InstDesc* d_inst = nullptr;
    const LatDesc* d_lats = nullptr;
    std::vector<FftLaunch> fwd;
    std::vector<HashGroup> hash;
};

struct Plan {
    int d = 0, L = 0, prec = 0, nwords = 0, maxN = 0;
    int64_t n = 0, s = 0, sumM = 0, cap = 0, N_gamma = 0, kmax = 0, last_nout = 0;
    int64_t n_alloc = 0, cap_alloc = 0;  // candidate count and detected capacity the workspace was sized for
    sfft_params p;
    const void* cand = nullptr;  // int32 or int8 rows (p.cand_type, p.cand_ld)
    cudaStream_t st = nullptr;
    std::vector<int64_t> M, z, soff;
    std::vector<int32_t> boff;
    std::vector<FftTables*> tabs;
    std::vector<void*> allocs;
    // device workspace
    uint32_t* nzbits = nullptr;
    void* ghat = nullptr;
    LatStats* stats = nullptr;
    uint32_t* detbits = nullptr;
    int64_t* det = nullptr;
    int64_t* cnt = nullptr;
    c64* coef = nullptr;
    int32_t* H = nullptr;
    uint8_t* sel = nullptr;
    uint8_t* rsel = nullptr;      // refinement's selected lattices (refine plans)
    c64* adj_w = nullptr;         // adjoint cotangents of the detected set
    c64* adj_out = nullptr;       // FP64 sample cotangents of FP32 plans (first backward call)
    int32_t* outpos = nullptr;
    int32_t* coll = nullptr;
    c64* C = nullptr;
    c32* ghat_lo = nullptr;  // low words of the double-float forward transform (FP32 + refinement)
    c64* lsq_work = nullptr; // conjugate-gradient vectors of the least-squares combine
    int32_t* lsq_next = nullptr;
    void* lsq_pairs = nullptr;
    int64_t lsq_pair_cap = 0;
    void* scratch = nullptr;
    double* sop_a = nullptr;
    int32_t* sop_tri = nullptr;
    InstDesc* d_inst = nullptr;
    InstDesc* h_inst = nullptr;  // pinned
    int64_t* h_cnt = nullptr;    // pinned
    LatDesc* d_lats = nullptr;
    std::vector<BlueJob> jobs_fwd, jobs_samp, jobs_adj;
    BlueJob* d_jobs_fwd = nullptr;
    BlueJob *d_jobs_samp = nullptr, *d_jobs_adj = nullptr;
    size_t hash_smem = 0;
    bool packed = false;          // |k| <= 127 and M < 65536: packed dp2a hash kernel
    bool hash_tc = false;         // tensor-core products (hash_tc.cu): one lattice group, |k.z| < 2^24
    size_t tc_smem = 0;
    std::vector<std::pair<int, int>> hgroups;  // lattice groups whose bitmaps fit shared memory
    std::vector<size_t> hsmem;                 // shared memory of each group
    uint8_t* cnt8 = nullptr;
    int* d_minmax = nullptr;      // [2 kMaxD] candidate bounds scratch
    int32_t* d_z = nullptr;       // [L, d] generating vectors on the device
    bool diag_run = false;        // the current reconstruct writes per-candidate diagnostics
    bool have_forward = false;
    bool shard_open = false;      // sfft_reconstruct_shard_begin ran; _end is due
    cudaEvent_t io_ev = nullptr;  // recorded after each upload of h_inst (staging reuse guard)

    int io_begin();               // wait until the previous upload of h_inst has completed
    int io_upload();              // enqueue h_inst -> d_inst and record io_ev

    void release();
    int alloc(void** p, size_t bytes);
    size_t esz() const;
    int fwd_prec() const;           // arithmetic of the forward transform
    bool fits_smem(int tprec) const;
    int buf_mode(int tprec) const;  // work-buffer mode of the transforms in precision tprec
    int build_jobs();
    int prepare_adjoint();
    int hash_grid() const;
    PipeArgs pipe_args();
};

int plan_create(Plan* P, int d, const void* cand, int64_t n, int64_t s, int L, const int64_t* M, const int64_t* z,
                const sfft_params* p, cudaStream_t st);
int run_pipeline(const PipeArgs& a, cudaStream_t st);
int tc_grid(size_t smem, int64_t tiles, int count);
// Bluestein job for the tables of one M; prec: 0 double, 1 float, 2 double-float; dir 0 forward
BlueJob make_blue_job(const FftTables* t, int prec, int dir, double scale);
int upload_jobs(const std::vector<BlueJob>& v, BlueJob** dst, std::vector<void*>* owner);
uint64_t philox_word0(uint64_t key0, uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3);
double philox_u01(uint64_t key, uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3);
bool is_prime(int64_t n);
int64_t next_prime_above(double x);
int L_rule(int rule, int64_t n, double delta, double c);

}  // namespace sfft
