// Launch wrappers of the per-lattice / per-candidate kernels (kernels.cu).
#pragma once
#include "common.cuh"

namespace sfft {
// variant: 0 int32 inner products, 1 packed (int8 k, int16 z, dp2a), 2 packed with diagnostics
// lattice group [l0, l1) (l1 < 0: through the last lattice); mode bit 0: first group (counts start
// at 0, else from cnt8), bit 1: last group (apply the count rule, else store counts in cnt8)
int launch_hash_count(const InstDesc* di, int ninst, int d, int gx, size_t smem, int variant, int l0, int l1, int mode,
                      cudaStream_t st);
size_t hash_smem_bytes(int d, int L, int64_t nwords, bool packed);
// candidates one CTA covers per pass of its grid-stride loop, CTA size and CTAs per SM of the hash
// kernels for a bitmap segment of smem bytes
int64_t hash_tile(bool packed, size_t smem);
int hash_threads(bool packed, size_t smem);
int hash_ctas_per_sm(size_t smem);
int launch_zero_test(const LatDesc* dl, int nlat, InstDesc* di, int prec, double kappa_u, cudaStream_t st);
int launch_compact(InstDesc* di, int ninst, cudaStream_t st);
int launch_det_hashes(const InstDesc* di, int ninst, int64_t maxdet, cudaStream_t st);
int launch_collisions(const InstDesc* di, int ninst, cudaStream_t st);
// mode 0: combine (median / hybrid), 1: refinement update, 2: refinement update on FP32 buckets,
// 3: median combine that also forms (and stores) the hashes of Itilde
int launch_combine(const InstDesc* di, int ninst, int64_t maxdet, int prec, int mode, cudaStream_t st, int zc = 0);
int launch_lsq(InstDesc* di, int ninst, int prec, cudaStream_t st);
int launch_scatter_coef(const InstDesc* di, int ninst, bool f32, cudaStream_t st);
int launch_select(InstDesc* di, int ninst, cudaStream_t st);
int launch_scatter_terms(const InstDesc* di, int ninst, int64_t max_terms_x_L, cudaStream_t st);
// adjoint cotangent of the lattice DFTs into I.C (cleared before), from the output cotangents dcoef
// (NULL: zero) through the optional refinement step and the median (see kernels.cu)
int launch_adjoint_buckets(const InstDesc* di, const c64* dcoef, bool refine, int64_t maxdet, cudaStream_t st);
int launch_points(const InstDesc* di, int32_t* numer, double* x, int64_t tot, cudaStream_t st);
int launch_cand_stats(const void* cand, int i8, int ld, int64_t n, int d, int* mn, int* mx, cudaStream_t st);
int launch_to_c64(const void* src, int prec, c64* dst, int64_t n, cudaStream_t st);
size_t hash_tc_smem_bytes(int L, int64_t nwords);
int launch_hash_count_tc(const InstDesc* di, int ninst, int gx, size_t smem, cudaStream_t st);
int launch_upload(void* dst, const void* pinned_src, size_t bytes, cudaStream_t st);
int launch_clear(InstDesc* di, int ninst, int clear_det, int clear_coll, int clear_C, cudaStream_t st);
// sum-of-products test function (sop.cu)
int launch_sop_coefs(const double* theta, int n_terms, int K, double width, double* a, double* da, cudaStream_t st);
int launch_sop_sample(const InstDesc* di, const int32_t* triples_dev, int n_terms, int K, const double* a, void* out,
                      int prec, cudaStream_t st);
int launch_sop_backward(const InstDesc* di, const int32_t* triples_dev, int n_terms, int K, const double* a,
                        const double* da, const void* dsamples, int prec, double* dtheta, cudaStream_t st);
int launch_sop_eval_points(const double* x, int64_t n, int d, const int32_t* triples_dev, int n_terms, int K,
                           const double* a, double* y, cudaStream_t st);
int launch_sparse_eval_points(const double* x, int64_t n, int d, const int32_t* kvec, const double* coef,
                              int64_t nterms, double* y, cudaStream_t st);
// dimension-incremental driver (dimincr_kernels.cu)
int launch_pairing(const int32_t* prev, int64_t np, int t, const int32_t* cur, int nt, int32_t* out, cudaStream_t st);
int launch_assemble_nodes(const double* xl, int64_t n, int tc, const double* tail, int d, double* X, cudaStream_t st);
int launch_step1_nodes(const double* tail, int d, int t, int K, double* X, cudaStream_t st);
int launch_c64_to_c32(const c64* a, c32* b, int64_t n, cudaStream_t st);
int launch_gather_rows(const int32_t* J, int w, const int64_t* idx, int64_t n, int32_t* rows, cudaStream_t st);
int launch_philox_tail(uint64_t key, uint64_t c1, uint64_t c2, uint64_t c3, int d, double* out, cudaStream_t st);
int launch_step1_select(const c64* ph, int K, int lo, int64_t s_keep, double theta_abs, double theta_rel, int rank_bits,
                        double* mag, uint8_t* mask, cudaStream_t st);
int launch_union_scatter(const int64_t* supp, const c64* coef, int64_t n, uint8_t* flag, c64* acc, cudaStream_t st);
int64_t flag_compact_blocks(int64_t n);  // entries of the counts scratch of launch_flag_compact
int launch_flag_compact(const uint8_t* flag, int64_t n, int64_t* counts, int64_t* out, int64_t* total, cudaStream_t st);
int launch_gather_c64(const c64* v, const int64_t* idx, int64_t n, c64* out, cudaStream_t st);
int launch_positions_to_values(const int64_t* pos, int64_t n, int lo, int32_t* out, cudaStream_t st);
}  // namespace sfft
