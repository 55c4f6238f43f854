// Batched reconstruction and the dimension-incremental driver (Algorithm 3).
#include "common.cuh"
#include "kernels.cuh"
#include "plan.cuh"

using namespace sfft;

extern "C" {

void sfft_dimincr_params_default(sfft_dimincr_params* p) {
    if (!p) return;
    p->s = 1;
    p->s_local = 0;
    p->r = 1;
    p->theta_abs = 1e-12;
    p->theta_rel = 0.0;
    p->delta = 0.9;
    p->c = 10.33;
    p->tau_abs = 0.0;
    p->tau_rel = 1e-10;
    p->precision = SFFT_FP64;
    p->refine = 1;
    p->seed = 0;
    p->max_samples = 0;
}

int sfft_batch_create(sfft_batch** out, sfft_plan* const* plans, int n_plans, int use_graph, void* stream) {
    (void)out; (void)plans; (void)n_plans; (void)use_graph; (void)stream;
    set_error("sfft_batch_create: not available in this build");
    return SFFT_EINVAL;
}
void sfft_batch_destroy(sfft_batch* b) { (void)b; }
int sfft_batch_reconstruct(sfft_batch* b, const void* const* samples, int64_t* const* supp_out, double* const* coef_out,
                           const int64_t* cap, int64_t* n_out_dev) {
    (void)b; (void)samples; (void)supp_out; (void)coef_out; (void)cap; (void)n_out_dev;
    set_error("sfft_batch_reconstruct: not available in this build");
    return SFFT_EINVAL;
}
int sfft_dim_incremental(int d, const int32_t* box_lo, const int32_t* box_hi, const sfft_dimincr_params* p,
                         sfft_sample_fn f, void* ctx, int32_t* supp_out, double* coef_out, int64_t cap, int64_t* n_out,
                         int64_t* n_samples, void* stream) {
    (void)d; (void)box_lo; (void)box_hi; (void)p; (void)f; (void)ctx; (void)supp_out; (void)coef_out; (void)cap;
    (void)n_out; (void)n_samples; (void)stream;
    set_error("sfft_dim_incremental: not available in this build");
    return SFFT_EINVAL;
}
int sfft_fn_sparse_poly(void* ctx, const double* x, int64_t n, double* y, void* stream) {
    auto* c = reinterpret_cast<sfft_fn_sparse_poly_ctx*>(ctx);
    if (!c || !x || !y) return SFFT_EINVAL;
    return launch_sparse_eval_points(x, n, c->d, c->kvec, c->coef, c->n_terms, y, (cudaStream_t)stream);
}
int sfft_fn_sop(void* ctx, const double* x, int64_t n, double* y, void* stream) {
    (void)ctx; (void)x; (void)n; (void)y; (void)stream;
    set_error("sfft_fn_sop: not available in this build");
    return SFFT_EINVAL;
}

}  // extern "C"
