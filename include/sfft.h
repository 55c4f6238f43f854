/*
 * sfft.h -- C ABI of a GB300 (sm_103a) implementation of the sparse FFT for arbitrary
 * frequency candidate sets by Kaemmerer, Krahmer and Volkmer (arXiv 2006.13053).
 *
 * Notation follows the paper: Gamma (the candidate set, "cand") is a finite set of integer
 * frequency vectors k in Z^d; the unknown function is sampled along L rank-1 lattices
 * Lambda(z_l, M_l) = { j z_l / M_l mod 1 : j = 0..M_l-1 } (Section 2.1, eq. 2.1); each
 * lattice's samples are transformed by a length-M_l DFT (Algorithm 2); a candidate
 * k is detected when its buckets ghat^(l)_{k.z_l mod M_l} are non-zero for at least nu*L
 * lattices (Algorithm 1; nu = 1/2 in Algorithm 2) and its coefficient is the component-wise
 * median of those L bucket values (Algorithm 2, eq. 2.6).  Algorithm 4 then keeps the
 * s_tilde largest coefficients of modulus >= theta.  Algorithm 3 is the
 * dimension-incremental driver around Algorithm 4.
 *
 * Conventions (every entry point):
 *   - returns an int status: SFFT_OK (0) or one of the SFFT_E* codes below; nothing throws
 *     across the ABI.  sfft_last_error() returns a message for the calling thread's last
 *     failure.
 *   - "device" pointers are CUDA device memory of the current device (e.g. a torch tensor's
 *     data_ptr()); "host" pointers are ordinary host memory.  The caller owns every buffer
 *     it passes; the library never frees them.  A plan owns its own workspace, released by
 *     sfft_plan_destroy().
 *   - complex arrays are interleaved (re, im) pairs.  Arrays documented as "complex in the
 *     plan precision" are float2 for SFFT_FP32 plans and double2 for SFFT_FP64 plans; arrays
 *     documented as "complex double" are always double2.
 *   - samples of all lattices are concatenated in lattice order l = 0..L-1; inside lattice l
 *     the node order is j = 0..M_l-1 (eq. 2.1).  offsets[l] = M_0 + ... + M_{l-1}.
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).  Work is
 *     enqueued on it; entry points that return host-side counts synchronise it.
 */
#ifndef SFFT_H
#define SFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define SFFT_OK 0
#define SFFT_EINVAL 1      /* invalid argument (null pointer, size out of range, even L ...)    */
#define SFFT_ENOTPRIME 2   /* a lattice size M_l is not prime                                  */
#define SFFT_EALIAS 3      /* |Gamma mod M_l| < |Gamma| could not be excluded (M_l <= N_Gamma) */
#define SFFT_EOVERFLOW 4   /* |k.z| bound does not fit the exact 32-bit hash arithmetic        */
#define SFFT_ENOMEM 5      /* device allocation failed                                         */
#define SFFT_ECUDA 6       /* a CUDA runtime call failed                                       */
#define SFFT_ETIMEOUT 7    /* a bounded device-side wait gave up                               */
#define SFFT_ECAPACITY 8   /* a caller- or plan-sized buffer was too small (count still set)   */
#define SFFT_ESTATE 9      /* call out of order (e.g. backward before forward)                 */

/* ---------------------------------------------------------------- parameters */
#define SFFT_FP64 0 /* samples, twiddles and FFT arithmetic in double                         */
#define SFFT_FP32 1 /* samples, twiddles and FFT arithmetic in float (FP32 accumulation);
                       with refine = 1 (or the LSQ combine) the forward lattice DFTs run in
                       the arithmetic that sfft_params.dft selects                            */

/* Arithmetic of the forward lattice DFTs of an FP32 plan with refinement (or the LSQ combine).
 * The refinement's residual spectrum is ghat - C, C the bucket sums of the detected coefficients
 * (eq. 2.3), so its accuracy is that of ghat:
 *   SFFT_DFT_DF64  double-float (float pairs, ~48 bits): coefficients agree with an FP64
 *                  reconstruction to ~1e-12 relative (the default)
 *   SFFT_DFT_FP32  float with FP32 accumulation: each bucket carries the transform's rounding,
 *                  ~1e-7 of the spectrum's rms, so a coefficient of magnitude |c| agrees to
 *                  ~1e-7 rms/|c| (1e-6 class for complex-Gaussian coefficients); ~3x cheaper
 * FP64 plans and FP32 plans without refinement ignore it (their transforms run in the plan's
 * precision).                                                                                 */
#define SFFT_DFT_DF64 0
#define SFFT_DFT_FP32 1

#define SFFT_L_COR26 0    /* L = min odd n >= 4c/((c-2)ln(c-1)) (ln|Gamma| - ln delta), Cor 2.6 */
#define SFFT_L_EQ42 1     /* a quarter of the Cor 2.6 bound, rounded up to odd, eq. (4.2)       */
#define SFFT_L_FALLBACK 2 /* L = ceil(2 ln|Gamma|)+1 rounded up to odd; M_l = L smallest primes >= 4s */

#define SFFT_COMBINE_MEDIAN 0 /* eq. (2.6): component-wise median over the L lattices             */
#define SFFT_COMBINE_HYBRID 1 /* Remark 2.8: mean over collision-free lattices, median fallback    */
#define SFFT_COMBINE_LSQ 2    /* Remark 2.8: least-squares fit of all samples on the detected set, */
                              /* started at the medians (conjugate gradients, FP64)                */

typedef struct sfft_params {
    double c;         /* Cor 2.6 constant (> 1/nu); default 10.33 (Theorem 1.1)                */
    double delta;     /* failure probability in the L rule; default 0.1                        */
    double nu;        /* detection fraction of Algorithm 1, 0 < nu <= 1/2; default 1/2 (Alg 2) */
    double tau_abs;   /* zero test (Remark 2.3): |ghat| > tau_l counts as non-zero, where      */
    double tau_rel;   /*   tau_l = max(tau_abs, tau_rel * max_h |ghat^(l)_h|); default 0, 1e-10 */
    double theta_abs; /* Algorithm 4 threshold theta = max(theta_abs, theta_rel * max|c|)      */
    double theta_rel; /*   defaults 0, 0                                                       */
    int64_t s_tilde;  /* Algorithm 4 output limit; 0 = keep every detected frequency (Alg 2)  */
    int precision;    /* SFFT_FP64 or SFFT_FP32                                                */
    int refine;       /* number of FP64 refinement steps on the detected support (0 or 1)     */
    int L_rule;       /* SFFT_L_* (used when the caller does not fix L)                       */
    int combine;      /* SFFT_COMBINE_*                                                       */
    uint64_t seed;    /* key of the Philox4x64-10 draws of generating vectors                  */
    int64_t detect_cap; /* capacity for |Itilde|; 0 = max(4 s + 4096, 16384)                  */
    int cand_type;    /* element type of the candidate rows: SFFT_CAND_I32 (default) or _I8     */
    int cand_ld;      /* row stride in elements: 0 = d (I32); I8 rows: >= d bytes               */
    int dft;          /* SFFT_DFT_*: forward DFT arithmetic of FP32 plans with refinement      */
    int rank_bits;    /* Algorithm 4 sort by modulus: 0 = exact FP64 order; 1..51 = moduli that  */
                      /* agree when rounded to rank_bits significant bits rank as equal, and    */
                      /* equal ranks keep the lower candidate index (a deterministic rule for   */
                      /* near-ties, e.g. the +-k symmetric coefficients of real functions)      */
} sfft_params;

#define SFFT_CAND_I32 0 /* int32 rows of d entries                                              */
#define SFFT_CAND_I8 1  /* int8 rows (|k_t| <= 127) of stride cand_ld >= d bytes in an array of  */
                        /* n_cand * cand_ld bytes starting 4-byte aligned (it is read as 32-bit */
                        /* words); bytes past d are ignored                                     */

/* Fill *p with the defaults listed above.  Never fails. */
void sfft_params_default(sfft_params* p);

/* ---------------------------------------------------------------- plans (Algorithm 2 / 4) */
typedef struct sfft_plan sfft_plan;

/*
 * Create a plan for candidates Gamma = cand (device, row-major [n_cand] rows of d entries of the
 * type p->cand_type: int32 rows with the pointer 16-byte aligned when d % 4 == 0 and 8-byte
 * aligned when d % 2 == 0 (they are read as vector words), or int8 rows of stride p->cand_ld
 * bytes with the pointer 4-byte aligned; a misaligned pointer returns SFFT_EINVAL before any
 * device work.  Not copied: it must stay valid and unchanged until the plan is destroyed) and
 * sparsity s.
 *   L     > 0: number of lattices (must be odd for the median, Algorithm 2), or 0: take L
 *              from p->L_rule with |Gamma| = n_cand (Corollary 2.6 / eq. 4.2 / fallback).
 *   M     host int64 [L] lattice sizes (each prime), or NULL: M_l = the smallest prime
 *              > c*s (Corollary 2.6), or the fallback primes.  M_l <= N_Gamma (eq. 2.4) is
 *              rejected with SFFT_EALIAS.
 *   z     host int64 [L, d] generating vectors with 0 <= z < M_l, or NULL: drawn as
 *              z_{l,u} = Philox4x64-10(counter=(u, l, 0, 0), key=(seed, 0)).word0 mod M_l.
 * Needs 1 <= d <= 32, n_cand >= 1, s >= 1, |k_t| small enough that d*max|k|*(M-1) < 2^31
 * (else SFFT_EOVERFLOW).  Precomputes chirps and Bluestein filters on `stream`.
 */
int sfft_plan_create(sfft_plan** out, int d, const void* cand, int64_t n_cand, int64_t s, int L,
                     const int64_t* M, const int64_t* z, const sfft_params* p, void* stream);

/*
 * Rebind the plan to another candidate set Gamma' (same row layout, n_cand <= the n_cand the plan was
 * created with, every |k_t| within the plan's creation bound, N_Gamma' < every M_l: then the
 * lattices, tables, hash offsets and kernel choice stay valid).  Nothing is allocated; the rows
 * are scanned for their bounds (synchronises the plan's stream).  Returns SFFT_EINVAL or
 * SFFT_EALIAS when the set does not fit the plan.  Batches created earlier keep the old set.
 * (Repeated experiments on fixed lattices, e.g. the PFP/PFN audit of Section 4.1, use it to
 * reconstruct on a fresh random candidate set per repetition.)
 */
int sfft_plan_set_candidates(sfft_plan* plan, const void* cand, int64_t n_cand);

/*
 * Replace the generating vectors (host int64 [L, d], 0 <= z < M_l; the lattice sizes stay): a new
 * random lattice configuration on the same plan, nothing allocated.  Synchronises the plan's
 * stream first.  Batches containing the plan read the same device array, so their later calls
 * use the new vectors too.  (Section 4.1.3's experiment draws a fresh configuration per
 * repetition on fixed Gamma and I.)
 */
int sfft_plan_set_generators(sfft_plan* plan, const int64_t* z);

/* L, the lattice sizes M (host int64 [L], optional), z (host int64 [L*d], optional) and the
 * total number of samples sum_l M_l (optional). */
int sfft_plan_info(const sfft_plan* plan, int* L, int64_t* M, int64_t* z, int64_t* n_samples);

void sfft_plan_destroy(sfft_plan* plan);

/*
 * Lattice nodes of eq. (2.1): numer_out (device int32 [sum M, d], optional) receives the exact
 * integers (j z_l mod M_l); x_out (device double [sum M, d], optional) receives numer / M_l;
 * offsets (host int64 [L+1], optional) the lattice offsets.
 */
int sfft_sample_points(const sfft_plan* plan, int32_t* numer_out, double* x_out, int64_t* offsets);

/* Optional diagnostics of sfft_reconstruct (any member may be NULL / ignored). */
typedef struct sfft_diag {
    uint8_t* counts;     /* device [n_cand]: n_k = #{l : |ghat^(l)_{h_kl}| > tau_l}          */
    int32_t* hashes;     /* device [n_cand, L]: h_kl = k.z_l mod M_l                         */
    int32_t* collisions; /* device [sum M]: c_l[h] = #{k in Itilde : h_kl = h} (Remark 2.8)  */
    int64_t* detected;   /* device [detect_cap]: Itilde (indices into Gamma, ascending)       */
    double* pcheck;      /* device complex double [detect_cap]: medians of Itilde (eq. 2.6)   */
    double* ghat;        /* device complex double [sum M]: lattice DFTs (Algorithm 2)        */
    double* tau;         /* device double [L]: zero-test thresholds                           */
    int64_t n_detected;  /* out: |Itilde|                                                     */
    int64_t n_guard;     /* out: buckets whose zero test was re-done in FP64                  */
    int64_t lsq_iters;   /* out: conjugate-gradient iterations of the least-squares combine   */
} sfft_diag;

/*
 * Algorithm 2 (nu = 1/2) or 1 on the plan's Gamma, followed by the optional Remark 2.8
 * combine, the optional FP64 refinement step(s) and Algorithm 4's theta filter and
 * top-s_tilde selection.
 *   samples  device complex in the plan precision [sum M]: f at the lattice nodes.
 *   supp_out device int64 [cap]: selected indices into Gamma, ascending.
 *   coef_out device complex double [cap]: their coefficients.
 *   n_out    host: number of selected frequencies (may exceed cap -> SFFT_ECAPACITY).
 * Synchronises the plan's stream.
 */
int sfft_reconstruct(sfft_plan* plan, const void* samples, int64_t* supp_out, double* coef_out, int64_t cap,
                     int64_t* n_out, sfft_diag* diag);

/*
 * Vector-Jacobian product of the last sfft_reconstruct of this plan (median combine, with or
 * without the refinement step), with the selected support and the lattices every median selected
 * held fixed.  The median coefficient is Re ghat^(l_re)_h + i Im ghat^(l_im)_h (eq. 2.6); the
 * refinement adds Re rhat^(m_re)_h + i Im rhat^(m_im)_h with rhat = ghat - C and C the median
 * coefficients summed into their buckets (eq. 2.3), so the map samples -> coefficients is linear
 * and its adjoint is: the cotangents into the refinement's selected buckets, minus their gather
 * over all lattices into the median coefficients of the whole detected set, those into the
 * median's selected buckets, then the adjoint of the 1/M-normalised DFT (an inverse prime-length
 * transform, run in FP64 for every plan precision).
 * dcoef: device complex double [n_out of that call] (dL/dRe + i dL/dIm);
 * dsamples: device complex in the plan precision [sum M] (overwritten).
 * The first call on a plan allocates the adjoint's job list (and, for FP32 plans, an FP64 buffer
 * of sum M complex values); later calls allocate nothing.  Synchronises the plan's stream.
 */
int sfft_reconstruct_backward(sfft_plan* plan, const double* dcoef, void* dsamples);

/*
 * Sharded reconstruction of one instance whose candidate set is split into slices, one plan per
 * slice (one per GPU / process), every plan with the instance's lattices (the same M and z) and
 * the same parameters (median combine, absolute theta: theta_rel = 0).  Every shard transforms
 * the same samples (the lattice DFTs are repeated per shard: sum M is small next to |Gamma|).
 *   begin: Algorithm 2 on the slice (lattice DFTs, zero test, hash + count, median combine),
 *          then C_out (device complex double [sum M]) = the slice's median coefficients summed
 *          into their buckets (eq. 2.3); n_detected (optional host) = the slice's |Itilde|.
 *   The caller sums C over the shards (an all-reduce: the refinement's residual spectrum
 *   ghat - C needs every shard's detected coefficients).
 *   end:   the refinement update with the summed C_sum (plans with refine = 1; others ignore it),
 *          then Algorithm 4's theta filter and top-s_tilde on the slice: supp_out (indices into
 *          the slice, ascending), coef_out (complex double), keys_out (optional device uint64
 *          [cap]: the rank key of each output, see sfft_params.rank_bits).  Merging the shards'
 *          outputs by (key descending, global index ascending) and keeping s_tilde gives the
 *          unsharded selection.
 * Both synchronise the plan's stream; end must follow begin on the same plan.
 */
int sfft_reconstruct_shard_begin(sfft_plan* plan, const void* samples, double* C_out, int64_t* n_detected);
int sfft_reconstruct_shard_end(sfft_plan* plan, const double* C_sum, int64_t* supp_out, double* coef_out,
                               uint64_t* keys_out, int64_t cap, int64_t* n_out);

/* ---------------------------------------------------------------- synthetic test functions */
/*
 * Samples of the sparse trigonometric polynomial p(x) = sum_q coef_q exp(2 pi i kvec_q . x)
 * (eq. 2.2) at the plan's lattice nodes, plus optional additive noise:
 *   kvec  device int32 [n_terms, d];  coef device complex double [n_terms];
 *   noise device complex [sum M] in the plan precision, or NULL;  samples_out device complex
 *   (plan precision).
 * Computed exactly through eq. (2.3): the coefficients are summed into their buckets
 * k.z_l mod M_l and each lattice is inverse-transformed (a transform whose work buffer fits one
 * CTA's shared memory sums its buckets there; the others take a global bucket pass first).  FP32
 * plans form buckets, transform and noise sum in FP32 (samples within a few FP32 ulps of the exact
 * value plus noise).  Bucket sums are formed by atomic additions, so a bucket of three or more
 * terms may round differently from one call to the next.
 * Asynchronous on the plan stream.
 */
int sfft_sample_sparse_poly(const sfft_plan* plan, const int32_t* kvec, const double* coef, int64_t n_terms,
                            const void* noise, void* samples_out);

/*
 * Samples of the sum-of-products function f(x) = sum_m prod_{t in T_m} g_{theta_m}(x_t) with
 * g_theta(x) = sum_{|k| <= K} sinc(pi k / (width theta))^4 exp(2 pi i k x) (real valued).
 *   triples host int32 [n_terms, 3] (dimensions < d); theta device double [n_terms].
 * samples_out device complex (plan precision; imaginary parts are 0).  Asynchronous on the
 * plan stream.
 */
int sfft_sample_sop(const sfft_plan* plan, const int32_t* triples, const double* theta, int n_terms, int K,
                    double width, void* samples_out);

/*
 * Adjoint of sfft_sample_sop with respect to theta: dtheta[m] = sum_j Re(dsamples_j)
 * d f(x_j) / d theta_m, recomputing f's factors at the nodes instead of storing them.
 *   dsamples device complex (plan precision) [sum M]; dtheta device double [n_terms] (overwritten).
 */
int sfft_sample_sop_backward(const sfft_plan* plan, const int32_t* triples, const double* theta, int n_terms,
                             int K, double width, const void* dsamples, double* dtheta);

/*
 * Samples of Section 4.3's test function (eq. 4.3), a sum of products of periodic B-splines,
 *   f(x) = sum_{q < n_terms} prod_{t in dims_q} N_{m_q}(x_t),
 *   N_m(x) = C_m sum_k sinc(pi k/m)^m (-1)^k exp(2 pi i k x),  ||N_m||_{L2(T)} = 1,
 * at the plan's lattice nodes.  dims: host int32 [n_terms, 4], the term's distinct dimensions
 * (< d; a -1 ends a term with fewer than 4); orders: host int32 [n_terms], 1 <= m <= 12;
 * 1 <= n_terms <= 8.  N_m is evaluated in closed form (one scaled cardinal B-spline per period,
 * Cox-de Boor recurrence in FP64), so the samples carry rounding only.  samples_out: device
 * complex in the plan precision (imaginary parts 0).  Asynchronous on the plan stream.
 * Errors: SFFT_EINVAL for a bad term.
 */
int sfft_sample_bspline(const sfft_plan* plan, const int32_t* dims, const int32_t* orders, int n_terms,
                        void* samples_out);

/* ---------------------------------------------------------------- batched reconstruction */
/* The batch calls have no counterpart in the paper: they run the per-plan path of sfft_reconstruct
 * (Algorithm 2, the optional refinement, Algorithm 4) and sfft_sample_sparse_poly (eq. 2.3) for
 * many plans in shared launches, and control and measure those launches. */
typedef struct sfft_batch sfft_batch;

/*
 * Group n_plans plans (same precision) so that sfft_batch_reconstruct runs every stage of all
 * of them in shared launches (one launch per stage for the whole batch).  The plans must
 * outlive the batch.  use_graph != 0 captures the stage sequence into a CUDA graph at the
 * second call on `stream` (which must not be the legacy NULL stream) and replays it on later
 * calls; the per-call buffer addresses are re-read at every replay.
 */
int sfft_batch_create(sfft_batch** out, sfft_plan* const* plans, int n_plans, int use_graph, void* stream);
void sfft_batch_destroy(sfft_batch* b);

/*
 * Run sfft_reconstruct for every plan of the batch.  samples[i], supp_out[i], coef_out[i]:
 * device pointers as in sfft_reconstruct; cap[i] host capacities; n_out_dev device int64
 * [n_plans] receives the counts.  Does not synchronise (counts stay on the device).
 */
int sfft_batch_reconstruct(sfft_batch* b, const void* const* samples, int64_t* const* supp_out,
                           double* const* coef_out, const int64_t* cap, int64_t* n_out_dev);

/*
 * Autotuner: runs sfft_batch_reconstruct on the given buffers (reps timed runs per candidate
 * after one warm-up) for hash-kernel grids of 1/2, 1, 2 and 4 waves of resident CTAs and for
 * lattice transforms of 256, 384, 512 or 576 threads per CTA, and the tensor-core hash kernel
 * (1, 2, 4 waves; plans with one lattice group, d <= 16, L <= 64, |k.z| < 2^24) against the
 * packed one, times the affected stage with CUDA events, keeps the fastest shapes for later
 * calls (a captured graph is re-captured) and reports them (hash_waves, negative when the
 * tensor-core kernel won; fft_threads: optional host outputs).  Synchronises the batch stream.
 */
int sfft_batch_autotune(sfft_batch* b, const void* const* samples, int64_t* const* supp_out, double* const* coef_out,
                        const int64_t* cap, int reps, double* hash_waves, int* fft_threads);

/*
 * Applies launch shapes that sfft_batch_autotune reported (for another batch of the same plans'
 * shapes, e.g. a second batch object alternating with the first on another stream, so that both
 * run the same shapes without tuning twice): hash_waves > 0 sets every packed / int32 hash grid to
 * that many waves of resident CTAs; hash_waves < 0 selects the tensor-core hash kernel with
 * |hash_waves| waves for the launches that qualify (as sfft_batch_select_hash); fft_threads sets
 * the forward transforms' CTA size (0: the largest).  Errors: SFFT_EINVAL for hash_waves = 0 or
 * |hash_waves| > 64, or for hash_waves > 0 once the tensor-core kernel is selected.  A captured
 * graph is re-captured at the next call.  Host only.
 */
int sfft_batch_set_shapes(sfft_batch* b, double hash_waves, int fft_threads);

/*
 * Use the tensor-core hash kernel (tcgen05: the inner products k.z_l of a 128-candidate tile and
 * all lattices as one bf16 GEMM with exact FP32 accumulation) for every hash launch of the batch
 * that qualifies (one lattice group, d <= 16, L <= 64, d max|k| (M-1) < 2^24, |k_t| <= 127,
 * M <= 32768).  tensor = 1 selects it; 0 is accepted only while no launch uses it.  The
 * default is the packed dp2a kernel; sfft_batch_autotune picks whichever measures faster.
 */
int sfft_batch_select_hash(sfft_batch* b, int tensor);

/*
 * Kernel launches that one sfft_batch_reconstruct (reconstruct) and one
 * sfft_batch_sample_sparse_poly with terms (sampler) enqueue in the steady state (descriptor
 * uploads happen only when a call's buffers differ from the previous call's).  Host only.
 */
int sfft_batch_launch_count(sfft_batch* b, int* reconstruct, int* sampler);

/*
 * Status of the last sfft_batch_reconstruct (waits for it): flags host int64 [n_plans] in the
 * caller's plan order, bit 1 = detected set above its capacity, 2 = more uncertain buckets in
 * the FP64 guard band than one lattice can re-test (tau below the working precision's
 * resolution), 4 = output above cap.  Returns SFFT_ECAPACITY if any flag is set.
 */
int sfft_batch_flags(sfft_batch* b, int64_t* flags);

/*
 * sfft_sample_sparse_poly for every plan of the batch in shared launches (one inverse-transform
 * launch per work-buffer mode, plus a clear and a bucket scatter when some transform does not fit
 * one CTA's shared memory).  Arrays are indexed by the caller's plan order: kvec[i]
 * device int32 [n_terms[i], d_i]; coef[i] device complex double; noise NULL or noise[i] device
 * complex [sum M] in the plan precision (may be NULL); samples_out[i] device complex (plan
 * precision).
 * Asynchronous on the batch stream.
 */
int sfft_batch_sample_sparse_poly(sfft_batch* b, const int32_t* const* kvec, const double* const* coef,
                                  const int64_t* n_terms, const void* const* noise, void* const* samples_out);

/*
 * Per-stage GPU time of the batch's stage sequence, measured with CUDA events on the batch
 * stream around each stage of every call since the last reset.  Stage order: clear, lattice
 * DFT (Algorithm 2), zero test, hash + count, compaction, hashes of Itilde (a separate launch
 * only for the hybrid combine; else formed by the combine), combine, least squares (Remark
 * 2.8), refinement scatter, refinement update, Algorithm 4 selection.  ms / launches: host
 * arrays of 11 entries (optional) receive the accumulated milliseconds and the number of timed
 * calls.  mode = 1 enables timing (graph batches then run eagerly), 0 disables it, both reset
 * the totals; mode = -1 only reads.  Returns the number of stages (11) or -1.
 */
int sfft_batch_timing(sfft_batch* b, int mode, double* ms, int64_t* launches);

/* ---------------------------------------------------------------- Algorithm 3 */
/*
 * Black-box function for Algorithm 3: evaluate f at n nodes x (device double [n, d],
 * row-major) into y (device complex double [n]); return 0 on success.
 */
typedef int (*sfft_sample_fn)(void* ctx, const double* x, int64_t n, double* y, void* stream);

typedef struct sfft_dimincr_params {
    int64_t s;         /* sparsity (sets M_l = smallest prime > c s)                        */
    int64_t s_local;   /* Step 1 / Step 2 (t < d) output size; default 2 s                  */
    int r;             /* number of detection iterations; 0 = the theory's choice
                          r = ceil(2 s ln(3 d s / delta)) (Section 3.3)                      */
    double theta_abs;  /* Algorithm 3/4 threshold (absolute) ...                            */
    double theta_rel;  /* ... or relative to the largest modulus of the current call        */
    double delta;      /* eq. (4.2) failure parameter                                       */
    double c;          /* lattice-size constant (10.33)                                      */
    double tau_abs, tau_rel; /* zero test                                                   */
    int precision;     /* SFFT_FP64 / SFFT_FP32                                              */
    int refine;        /* FP64 refinement steps per Algorithm 4 call                          */
    uint64_t seed;     /* Philox key; draws documented in the implementation                 */
    int64_t max_samples; /* 0 = unlimited; otherwise stop with SFFT_ECAPACITY                */
    int rank_bits;     /* near-tie rule of every Algorithm 4 selection (see sfft_params)     */
    int L_rule;        /* lattices per Step-2 call: SFFT_L_EQ42 (default, Section 4.2: eq. 4.2
                          with delta) or SFFT_L_COR26 with the theory's failure probability
                          gamma_A = delta / (3 d r) of Section 3.3                            */
} sfft_dimincr_params;

void sfft_dimincr_params_default(sfft_dimincr_params* p);

/*
 * Algorithm 3 with Algorithm 4 as Algorithm A on Gamma = the box prod_t [box_lo[t], box_hi[t]]
 * (host int32 [d] each).  supp_out host int32 [cap, d] (lexicographic order), coef_out host
 * complex double [cap]; n_out host; n_samples (optional host) = function evaluations used.
 */
int sfft_dim_incremental(int d, const int32_t* box_lo, const int32_t* box_hi, const sfft_dimincr_params* p,
                         sfft_sample_fn f, void* ctx, int32_t* supp_out, double* coef_out, int64_t cap,
                         int64_t* n_out, int64_t* n_samples, void* stream);

/* Built-in black boxes for Algorithm 3 (ctx = a struct owned by the caller):
 *   sfft_fn_sparse_poly: direct FP64 evaluation of sum_q coef_q exp(2 pi i kvec_q . x) (eq. 2.2);
 *       ctx = sfft_fn_sparse_poly_ctx (device kvec int32 [n_terms, d], device coef complex double).
 *   sfft_fn_sop: the sum-of-products function of sfft_sample_sop at arbitrary nodes;
 *       ctx = sfft_fn_sop_ctx (host triples int32 [n_terms*3], device theta double [n_terms],
 *       device work buffer of at least 16 n_terms (K+1) + 12 n_terms bytes). */
typedef struct sfft_fn_sparse_poly_ctx { const int32_t* kvec; const double* coef; int64_t n_terms; int d; } sfft_fn_sparse_poly_ctx;
/*   sfft_fn_bspline: Section 4.3's B-spline sum (eq. 4.3, as in sfft_sample_bspline) at arbitrary
 *       nodes, FP64 closed form; ctx = sfft_fn_bspline_ctx (host dims int32 [n_terms, 4] with -1
 *       ending a term, host orders int32 [n_terms], 1 <= n_terms <= 8, d the node dimension). */
typedef struct sfft_fn_bspline_ctx { const int32_t* dims; const int32_t* orders; int n_terms; int d; } sfft_fn_bspline_ctx;
typedef struct sfft_fn_sop_ctx { const int32_t* triples; const double* theta; int n_terms; int K; double width; int d; void* work; } sfft_fn_sop_ctx;
int sfft_fn_sparse_poly(void* ctx, const double* x, int64_t n, double* y, void* stream);
int sfft_fn_sop(void* ctx, const double* x, int64_t n, double* y, void* stream);
int sfft_fn_bspline(void* ctx, const double* x, int64_t n, double* y, void* stream);

/* ---------------------------------------------------------------- allocation-free detection */
/*
 * The detection step of sfft_reconstruct (zero test, candidate hashing with the count rule
 * "detected iff #{l : |ghat^(l)_{k.z_l mod M_l}| > tau_l} >= nu L", ascending compaction of
 * Itilde) for callers that cannot allocate device memory: code running where cudaMalloc is
 * forbidden or may fail at a bad moment (inside host callbacks, under a custom or capped
 * allocator, in a long-running service that must not grow its footprint).  The paper has no
 * counterpart; it is an interface convenience.
 *   cand   device int32 [n_cand, d], starting 16-byte aligned when d % 4 == 0, 8-byte aligned
 *          when d % 2 == 0 (the rows are read as vector words; else SFFT_EINVAL);
 *   M, z   host int64 [L], [L, d] (z < M);
 *   ghat   device complex double [sum M]: the normalised lattice DFTs (e.g. sfft_diag.ghat);
 *   tau    host double [L]: zero-test thresholds (|ghat| > tau_l counts as non-zero);
 *   nu     count rule: detected iff #{l : non-zero} >= nu L;
 *   detected_out device int64 [cap]: detected indices, ascending; n_detected host (true count).
 * Nothing is allocated: the scratch lives in one fixed 8 MiB device array owned by the library,
 * held by every GPU that loads it until the process exits.  Sizes beyond it (about 6.4e7
 * candidates with small lattices, less with large sum M) return SFFT_ECAPACITY, as does a
 * detected set larger than cap.  Every call looks the array's address up on the current device
 * (cudaGetSymbolAddress), so a device reset between calls is harmless; the first call on a device
 * also loads the library's device code there, so make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents (each call clears what must
 * start at zero): calls that overlap on the GPU race, so serialise them.  Synchronises `stream`.
 */
int sfft_detect_noalloc(int d, const int32_t* cand, int64_t n_cand, int L, const int64_t* M, const int64_t* z,
                        const double* ghat, const double* tau, double nu, int64_t* detected_out, int64_t cap,
                        int64_t* n_detected, void* stream);

/* ---------------------------------------------------------------- host utilities */
/* (the generators' counter-based random numbers and Corollary 2.6 / eq. 4.2 lattice rules of the
 * plan, exposed for checks on the host) */
/* Word 0 of Philox4x64-10 (Salmon et al., SC'11) for counter (c0..c3) and key (key0, 0). */
uint64_t sfft_philox4x64_word0(uint64_t key0, uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3);

/* Smallest prime > x; L of the Cor 2.6 / eq. 4.2 / fallback rules (host, no device work). */
int64_t sfft_next_prime_above(double x);
int sfft_L_rule(int rule, int64_t n_cand, double delta, double c);

/* Message of the calling thread's last failure ("" if none). */
const char* sfft_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SFFT_H */
