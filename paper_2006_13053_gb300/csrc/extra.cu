// Batched reconstruction (many plans, one launch per stage, optionally replayed from a CUDA
// graph) and the dimension-incremental driver (Algorithm 3).
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "plan.cuh"

namespace sfft {

// output counts and status flags of batch entry i; n_out (optional) in the caller's order
__global__ void k_gather_counts(const InstDesc* __restrict__ insts, int n, int64_t* out, int64_t* flags,
                                const int* __restrict__ order, int64_t* n_out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        out[i] = insts[i].cnt[1];
        flags[i] = insts[i].cnt[3];
        if (n_out) n_out[order[i]] = insts[i].cnt[1];
    }
}

struct Batch {
    std::vector<Plan*> plans;   // batch order (sorted by d)
    std::vector<int> order;     // batch index -> caller's plan index
    cudaStream_t st = nullptr;
    int use_graph = 0, prec = 0;
    InstDesc* d_inst = nullptr;
    InstDesc* h_inst = nullptr;  // pinned descriptors [n]: the current state (a captured graph uploads it)
    // eager calls upload a copy of h_inst from a ring of kStage pinned slots, so that the host can
    // run several calls ahead of the GPU: a slot is rewritten only after its upload kStage calls
    // ago has executed
    static constexpr int kStage = 4;
    InstDesc* h_ring = nullptr;  // pinned [kStage][n]
    cudaEvent_t ring_ev[kStage] = {};
    int ring_next = 0;
    // the descriptors the device holds (kernels never write them): an unchanged call uploads
    // nothing, so repeated calls on the same buffers read no host memory while bulk copies run
    std::vector<InstDesc> h_dev;
    LatDesc* d_lats = nullptr;
    std::vector<void*> allocs;
    PipeArgs args;
    std::vector<FftLaunch> samp;  // sparse-polynomial sampler transforms of every plan
    bool samp_scatter = false;    // some sampler transform needs the global bucket pass (not in shared memory)
    int64_t max_samp_terms_L = 0;
    int64_t* d_counts = nullptr;
    int* d_order = nullptr;     // batch index -> caller's plan index (device copy of order)
    int64_t* graph_nout = nullptr;  // n_out_dev the captured graph writes
    int64_t* d_flags = nullptr;
    cudaEvent_t done = nullptr;    // end of the last enqueued call (results and flags ready)
    cudaEvent_t io_ev = nullptr;   // the last graph launch has read h_inst (h_inst writable)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int calls = 0;
    // stage timing
    bool timing = false, pending = false, timer_made = false;
    StageTimer timer;
    double stage_ms[ST_COUNT] = {0};
    int64_t stage_n[ST_COUNT] = {0};

    int collect() {  // add the elapsed times of the last timed call
        if (!pending) return SFFT_OK;
        SFFT_CU(cudaEventSynchronize(timer.ev[ST_COUNT]));
        for (int s = 0; s < ST_COUNT; ++s) {
            if (!timer.recorded[s]) continue;
            int nx = s + 1;
            while (nx < ST_COUNT && !timer.recorded[nx]) ++nx;
            float ms = 0;
            SFFT_CU(cudaEventElapsedTime(&ms, timer.ev[s], timer.ev[nx]));
            stage_ms[s] += ms;
            stage_n[s] += 1;
        }
        pending = false;
        return SFFT_OK;
    }

    void release() {
        if (done) cudaEventSynchronize(done);
        if (timer_made)
            for (int i = 0; i <= ST_COUNT; ++i) cudaEventDestroy(timer.ev[i]);
        timer_made = false;
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (done) cudaEventDestroy(done);
        if (io_ev) cudaEventDestroy(io_ev);
        io_ev = nullptr;
        for (int k = 0; k < kStage; ++k)
            if (ring_ev[k]) cudaEventDestroy(ring_ev[k]);
        for (void* p : allocs) cudaFree(p);
        if (h_inst) cudaFreeHost(h_inst);
        if (h_ring) cudaFreeHost(h_ring);
        allocs.clear();
        exec = nullptr; graph = nullptr; done = nullptr; h_inst = nullptr; h_ring = nullptr;
    }
    // upload the current descriptors through the next ring slot (eager calls)
    int stage_upload() {
        const int n = (int)plans.size();
        // a byte comparison: h_dev is a byte copy of h_inst, so padding bytes compare equal too
        if (memcmp(h_dev.data(), h_inst, sizeof(InstDesc) * n) == 0) return SFFT_OK;
        memcpy(h_dev.data(), h_inst, sizeof(InstDesc) * n);
        const int k = ring_next;
        ring_next = (k + 1) % kStage;
        SFFT_CU(cudaEventSynchronize(ring_ev[k]));
        InstDesc* slot = h_ring + (size_t)k * n;
        memcpy(slot, h_inst, sizeof(InstDesc) * n);
        SFFT_TRY(launch_upload(d_inst, slot, sizeof(InstDesc) * n, st));
        SFFT_CU(cudaEventRecord(ring_ev[k], st));
        return SFFT_OK;
    }
    int alloc(void** p, size_t bytes) {
        SFFT_CU(cudaMalloc(p, std::max<size_t>(bytes, 16)));
        allocs.push_back(*p);
        return SFFT_OK;
    }
    int enqueue(bool eager, int64_t* n_out) {
        const int n = (int)plans.size();
        if (eager) {
            SFFT_TRY(stage_upload());
        } else {  // graph capture: every launch uploads h_inst as it is then
            SFFT_TRY(launch_upload(d_inst, h_inst, sizeof(InstDesc) * n, st));
        }
        SFFT_TRY(run_pipeline(args, st));
        k_gather_counts<<<(n + 127) / 128, 128, 0, st>>>(d_inst, n, d_counts, d_flags, d_order, n_out);
        return launch_check("k_gather_counts");
    }
};

static int batch_create(Batch* B, sfft_plan* const* plans, int n, int use_graph, cudaStream_t st) {
    SFFT_CHECK(plans && n >= 1, SFFT_EINVAL, "empty batch");
    SFFT_CHECK(!use_graph || st != nullptr, SFFT_EINVAL,
               "graph capture needs a non-default stream (the legacy NULL stream cannot be captured)");
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    for (int i = 0; i < n; ++i) SFFT_CHECK(plans[i] != nullptr, SFFT_EINVAL, "plan %d is NULL", i);
    auto P0 = reinterpret_cast<Plan*>(plans[0]);
    for (int i = 0; i < n; ++i) {
        auto P = reinterpret_cast<Plan*>(plans[i]);
        SFFT_CHECK(P->prec == P0->prec, SFFT_EINVAL, "all plans of a batch need the same precision");
        SFFT_CHECK(P->p.refine == P0->p.refine, SFFT_EINVAL, "all plans of a batch need the same refine setting");
        SFFT_CHECK(P->fwd_prec() == P0->fwd_prec(), SFFT_EINVAL,
                   "all plans of a batch need the same forward-transform arithmetic (refine / least-squares)");
    }
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        return reinterpret_cast<Plan*>(plans[a])->d < reinterpret_cast<Plan*>(plans[b])->d;
    });
    B->st = st;
    B->use_graph = use_graph;
    B->prec = P0->prec;
    B->order = idx;
    for (int i : idx) B->plans.push_back(reinterpret_cast<Plan*>(plans[i]));
    SFFT_CU(cudaMallocHost((void**)&B->h_inst, sizeof(InstDesc) * n));
    SFFT_CU(cudaMallocHost((void**)&B->h_ring, sizeof(InstDesc) * n * Batch::kStage));
    std::vector<LatDesc> lats;
    std::vector<BlueJob> jf[3], js[3];  // by work-buffer mode: global scratch, shared memory, cluster
    int maxN[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    PipeArgs& A = B->args;
    A.ninst = n;
    A.prec = B->prec;
    A.fwd_prec = P0->fwd_prec();
    A.refine = P0->p.refine;
    for (int b = 0; b < n; ++b) {
        Plan* P = B->plans[b];
        B->h_inst[b] = *P->h_inst;
        A.maxcap = std::max<int64_t>(A.maxcap, P->cap);
        A.hybrid |= P->p.combine == SFFT_COMBINE_HYBRID;
        A.lsq |= P->p.combine == SFFT_COMBINE_LSQ;
        for (int l = 0; l < P->L; ++l)
            lats.push_back(LatDesc{b, l, (int)P->M[l], (int)P->tabs[l]->N, P->soff[l], P->boff[l], 0,
                                   (const double*)P->tabs[l]->dft64, P->tabs[l]->dftdf});
        const int sf = P->buf_mode(P->fwd_prec()), sp = P->buf_mode(P->prec);
        B->samp_scatter |= sp != 1;
        for (int l = 0; l < P->L; ++l) {
            BlueJob f = P->jobs_fwd[l], s = P->jobs_samp[l];
            f.inst = b; s.inst = b;
            jf[sf].push_back(f); js[sp].push_back(s);
        }
        maxN[sf][0] = std::max(maxN[sf][0], P->maxN);
        maxN[sp][1] = std::max(maxN[sp][1], P->maxN);
    }
    A.nlat = (int)lats.size();
    SFFT_TRY(B->alloc((void**)&B->d_lats, sizeof(LatDesc) * lats.size()));
    SFFT_CU(cudaMemcpy(B->d_lats, lats.data(), sizeof(LatDesc) * lats.size(), cudaMemcpyHostToDevice));
    SFFT_TRY(B->alloc((void**)&B->d_inst, sizeof(InstDesc) * n));
    SFFT_CU(cudaMemcpy(B->d_inst, B->h_inst, sizeof(InstDesc) * n, cudaMemcpyHostToDevice));
    B->h_dev.assign(B->h_inst, B->h_inst + n);
    A.d_inst = B->d_inst;
    A.d_lats = B->d_lats;
    for (int md : {1, 2, 0}) {
        if (!jf[md].empty()) {
            BlueJob* dj = nullptr;
            SFFT_TRY(upload_jobs(jf[md], &dj, &B->allocs));
            A.fwd.push_back(FftLaunch{dj, (int)jf[md].size(), maxN[md][0], md});
            A.fwd.back().upair = uniform_pair(jf[md].data(), jf[md].size());
        }
        if (!js[md].empty()) {
            BlueJob* dj = nullptr;
            SFFT_TRY(upload_jobs(js[md], &dj, &B->allocs));
            B->samp.push_back(FftLaunch{dj, (int)js[md].size(), maxN[md][1], md});
            B->samp.back().upair = uniform_pair(js[md].data(), js[md].size());
        }
    }
    // hash launches: contiguous runs of single-group plans with equal d and kernel variant share a
    // launch (grid.y = instances); plans with several lattice groups get one launch per group
    for (int b = 0; b < n;) {
        Plan* Pb = B->plans[b];
        if (Pb->hgroups.size() > 1) {
            const int ng = (int)Pb->hgroups.size();
            for (int g = 0; g < ng; ++g) {
                HashGroup h;
                h.off = b; h.count = 1; h.d = Pb->d; h.gx = h.gx0 = Pb->hash_grid(); h.smem = Pb->hsmem[g];
                h.variant = Pb->packed ? 1 : 0;
                h.l0 = Pb->hgroups[g].first;
                h.l1 = g + 1 < ng ? Pb->hgroups[g].second : -1;
                h.mode = (g == 0 ? 1 : 0) | (g + 1 == ng ? 2 : 0);
                A.hash.push_back(h);
            }
            ++b;
            continue;
        }
        int e = b;
        HashGroup h;
        h.off = b;
        h.d = Pb->d;
        int64_t maxn = 0;
        h.tc_ok = true;
        h.tc_tiles = 0;
        while (e < n && B->plans[e]->d == h.d && B->plans[e]->packed == Pb->packed && B->plans[e]->hgroups.size() == 1) {
            h.smem = std::max(h.smem, B->plans[e]->hash_smem);
            maxn = std::max<int64_t>(maxn, B->plans[e]->n);
            h.tc_ok = h.tc_ok && B->plans[e]->hash_tc;
            h.tc_smem = std::max(h.tc_smem, B->plans[e]->tc_smem);
            h.tc_tiles = std::max<int64_t>(h.tc_tiles, (B->plans[e]->n + 127) / 128);
            ++e;
        }
        h.count = e - b;
        h.variant = Pb->packed ? 1 : 0;
        if (h.tc_ok) h.tc_gx0 = tc_grid(h.tc_smem, h.tc_tiles, h.count);
        const int64_t tile = hash_tile(Pb->packed, h.smem), tiles = (maxn + tile - 1) / tile;
        const int per_sm = hash_ctas_per_sm(h.smem);
        h.gx = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (152 * per_sm + h.count - 1) / h.count));
        h.gx0 = h.gx;
        h.tiles = tiles;
        A.hash.push_back(h);
        b = e;
    }
    SFFT_TRY(B->alloc((void**)&B->d_counts, sizeof(int64_t) * n));
    SFFT_TRY(B->alloc((void**)&B->d_order, sizeof(int) * n));
    SFFT_CU(cudaMemcpy(B->d_order, B->order.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    SFFT_TRY(B->alloc((void**)&B->d_flags, sizeof(int64_t) * n));
    SFFT_CU(cudaEventCreateWithFlags(&B->done, cudaEventDisableTiming));
    SFFT_CU(cudaEventCreateWithFlags(&B->io_ev, cudaEventDisableTiming));
    for (int k = 0; k < Batch::kStage; ++k) SFFT_CU(cudaEventCreateWithFlags(&B->ring_ev[k], cudaEventDisableTiming));
    for (int i = 0; i <= ST_COUNT; ++i) SFFT_CU(cudaEventCreate(&B->timer.ev[i]));
    B->timer_made = true;
    return SFFT_OK;
}

}  // namespace sfft

using namespace sfft;

extern "C" {

int sfft_batch_create(sfft_batch** out, sfft_plan* const* plans, int n_plans, int use_graph, void* stream) {
    if (!out) { set_error("out is NULL"); return SFFT_EINVAL; }
    *out = nullptr;
    Batch* B = new Batch();
    int rc = batch_create(B, plans, n_plans, use_graph, (cudaStream_t)stream);
    if (rc != SFFT_OK) {
        B->release();
        delete B;
        return rc;
    }
    *out = reinterpret_cast<sfft_batch*>(B);
    return SFFT_OK;
}

void sfft_batch_destroy(sfft_batch* b) {
    if (!b) return;
    Batch* B = reinterpret_cast<Batch*>(b);
    B->release();
    delete B;
}

int sfft_batch_reconstruct(sfft_batch* b, const void* const* samples, int64_t* const* supp_out, double* const* coef_out,
                           const int64_t* cap, int64_t* n_out_dev) {
    if (!b || !samples || !supp_out || !coef_out || !cap) { set_error("null argument"); return SFFT_EINVAL; }
    Batch* B = reinterpret_cast<Batch*>(b);
    const int n = (int)B->plans.size();
    // a pending graph launch reads h_inst when it runs (eager uploads use the ring)
    SFFT_CU(cudaEventSynchronize(B->io_ev));
    for (int i = 0; i < n; ++i) {
        const int u = B->order[i];  // caller's index of batch entry i
        SFFT_CHECK(samples[u] && (cap[u] == 0 || (supp_out[u] && coef_out[u])), SFFT_EINVAL, "null buffer for plan %d", u);
        InstDesc& I = B->h_inst[i];
        I.samples = samples[u];
        I.supp_out = supp_out[u];
        I.coef_out = reinterpret_cast<c64*>(coef_out[u]);
        I.out_cap = cap[u];
        I.dcounts = nullptr;
        I.dhashes = nullptr;
        I.key_out = nullptr;
        B->plans[i]->have_forward = false;  // batch runs do not keep a backward context
    }
    cudaStream_t st = B->st;
    SFFT_TRY(B->collect());
    B->args.timer = B->timing ? &B->timer : nullptr;
    if (B->timing && B->exec == nullptr && B->use_graph && B->calls >= 1) {
        // the graph is captured without timers; timed runs of a graph batch use the eager path
        SFFT_TRY(B->enqueue(true, n_out_dev));
        B->pending = true;
    } else if (B->use_graph && B->calls >= 1 && !B->timing) {
        if (B->exec && B->graph_nout != n_out_dev) {  // the graph holds the old output pointer
            cudaGraphExecDestroy(B->exec);
            cudaGraphDestroy(B->graph);
            B->exec = nullptr;
            B->graph = nullptr;
        }
        if (!B->exec) {
            SFFT_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            int rc = B->enqueue(false, n_out_dev);
            B->graph_nout = n_out_dev;
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(st, &g);
            if (rc != SFFT_OK) return rc;
            if (e != cudaSuccess) { set_error("graph capture failed: %s", cudaGetErrorString(e)); return SFFT_ECUDA; }
            B->graph = g;
            SFFT_CU(cudaGraphInstantiate(&B->exec, g, 0));
        }
        SFFT_CU(cudaGraphLaunch(B->exec, st));
        memcpy(B->h_dev.data(), B->h_inst, sizeof(InstDesc) * n);  // what the launch uploads
        SFFT_CU(cudaEventRecord(B->io_ev, st));  // the graph reads the staging buffer when it runs
    } else {
        SFFT_TRY(B->enqueue(true, n_out_dev));
        B->pending = B->timing;
    }
    SFFT_CU(cudaEventRecord(B->done, st));
    B->calls++;
    return SFFT_OK;
}

int sfft_batch_sample_sparse_poly(sfft_batch* b, const int32_t* const* kvec, const double* const* coef,
                                  const int64_t* n_terms, const void* const* noise, void* const* samples_out) {
    if (!b || !kvec || !coef || !n_terms || !samples_out) { set_error("null argument"); return SFFT_EINVAL; }
    Batch* B = reinterpret_cast<Batch*>(b);
    const int n = (int)B->plans.size();
    SFFT_CU(cudaEventSynchronize(B->io_ev));  // h_inst writable (see sfft_batch_reconstruct)
    int64_t mx = 0;
    for (int i = 0; i < n; ++i) {
        const int u = B->order[i];
        SFFT_CHECK(samples_out[u] && n_terms[u] >= 0 && (n_terms[u] == 0 || (kvec[u] && coef[u])), SFFT_EINVAL,
                   "bad sampler arguments for plan %d", u);
        InstDesc& I = B->h_inst[i];
        I.samp_kvec = kvec[u];
        I.samp_coef = reinterpret_cast<const c64*>(coef[u]);
        I.samp_nterms = n_terms[u];
        I.samp_out = samples_out[u];
        I.samp_noise = noise ? noise[u] : nullptr;
        mx = std::max<int64_t>(mx, n_terms[u] * B->plans[i]->L);
    }
    cudaStream_t st = B->st;
    SFFT_TRY(B->stage_upload());
    if (B->samp_scatter) {  // transforms in shared memory sum their own buckets
        SFFT_TRY(launch_clear(B->d_inst, n, 0, 0, B->prec ? 2 : 1, st));
        if (mx > 0) SFFT_TRY(launch_scatter_terms(B->d_inst, n, mx, st));
    }
    for (const auto& f : B->samp)
        SFFT_TRY(launch_bluestein(f.jobs, f.njobs, f.maxN, f.mode, B->prec, B->prec, B->prec, +1, EPI_ADDNOISE, B->d_inst,
                                  st, nullptr, nullptr, f.threads, f.upair));
    SFFT_CU(cudaEventRecord(B->done, st));
    return SFFT_OK;
}

int sfft_batch_autotune(sfft_batch* b, const void* const* samples, int64_t* const* supp_out, double* const* coef_out,
                        const int64_t* cap, int reps, double* hash_waves, int* fft_threads) {
    if (!b) { set_error("batch is NULL"); return SFFT_EINVAL; }
    Batch* B = reinterpret_cast<Batch*>(b);
    if (reps < 1) reps = 1;
    const bool was_timing = B->timing;
    // one eager, timed run per candidate; the stage timer isolates the tuned stage
    auto timed = [&](int stage, double* ms) -> int {
        B->timing = true;
        double acc = 0;
        for (int r = 0; r <= reps; ++r) {  // the first run warms up
            double m[ST_COUNT] = {0};
            int64_t nl[ST_COUNT] = {0};
            SFFT_TRY(B->collect());
            for (int s = 0; s < ST_COUNT; ++s) { B->stage_ms[s] = 0; B->stage_n[s] = 0; }
            SFFT_TRY(sfft_batch_reconstruct(b, samples, supp_out, coef_out, cap, nullptr));
            SFFT_TRY(B->collect());
            for (int s = 0; s < ST_COUNT; ++s) { m[s] = B->stage_ms[s]; nl[s] = B->stage_n[s]; }
            if (r > 0) acc += m[stage];
            (void)nl;
        }
        *ms = acc / reps;
        return SFFT_OK;
    };
    // hash kernel: grids of {1/2, 1, 2, 4} waves
    const double mults[4] = {0.5, 1.0, 2.0, 4.0};
    double best = 1e30, bestm = 1.0;
    for (double m : mults) {
        for (auto& h : B->args.hash)
            h.gx = (int)std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(h.tiles, 1), (int64_t)llround(h.gx0 * m)));
        double ms = 0;
        SFFT_TRY(timed(ST_HASH, &ms));
        if (ms < best) { best = ms; bestm = m; }
    }
    for (auto& h : B->args.hash)
        h.gx = (int)std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(h.tiles, 1), (int64_t)llround(h.gx0 * bestm)));
    // the tensor-core hash kernel (groups that qualify), kept only if it measures faster
    bool any_tc = false;
    for (const auto& h : B->args.hash) any_tc |= h.tc_ok;
    if (any_tc) {
        const std::vector<HashGroup> keep = B->args.hash;
        const double mtc[3] = {1.0, 2.0, 4.0};
        double best_tc = 1e30, bmt = 1.0;
        for (double m : mtc) {
            for (auto& h : B->args.hash)
                if (h.tc_ok) {
                    h.variant = 3;
                    h.smem = h.tc_smem;
                    h.gx = (int)std::max<int64_t>(1, std::min<int64_t>(h.tc_tiles, (int64_t)llround(h.tc_gx0 * m)));
                }
            double ms = 0;
            SFFT_TRY(timed(ST_HASH, &ms));
            if (ms < best_tc) { best_tc = ms; bmt = m; }
        }
        if (best_tc < best) {
            for (auto& h : B->args.hash)
                if (h.tc_ok) h.gx = (int)std::max<int64_t>(1, std::min<int64_t>(h.tc_tiles, (int64_t)llround(h.tc_gx0 * bmt)));
            bestm = -bmt;  // reported negative: tensor-core kernel, |value| waves
        } else {
            B->args.hash = keep;
        }
    }
    // lattice transforms: 256 to 576 threads per CTA (sizes above a transform type's largest CTA
    // run at that largest)
    const int ths[4] = {256, 384, 512, 576};
    best = 1e30;
    int bestt = 0;
    for (int th : ths) {
        for (auto& f : B->args.fwd) f.threads = th;
        double ms = 0;
        SFFT_TRY(timed(ST_FFT_FWD, &ms));
        if (ms < best) { best = ms; bestt = th; }
    }
    for (auto& f : B->args.fwd) f.threads = bestt;
    B->timing = was_timing;
    for (int s = 0; s < ST_COUNT; ++s) { B->stage_ms[s] = 0; B->stage_n[s] = 0; }
    // a captured graph holds the old launch shapes
    if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
    if (hash_waves) *hash_waves = bestm;
    if (fft_threads) *fft_threads = bestt;
    return SFFT_OK;
}

int sfft_batch_set_shapes(sfft_batch* b, double hash_waves, int fft_threads) {
    if (!b) { set_error("batch is NULL"); return SFFT_EINVAL; }
    Batch* B = reinterpret_cast<Batch*>(b);
    SFFT_CHECK(hash_waves != 0.0 && fabs(hash_waves) <= 64.0, SFFT_EINVAL, "hash_waves must be non-zero with |hash_waves| <= 64");
    if (hash_waves > 0) {
        for (const auto& h : B->args.hash)
            SFFT_CHECK(h.variant != 3, SFFT_EINVAL, "the tensor-core hash kernel is selected: positive waves need a new batch");
        for (auto& h : B->args.hash)
            h.gx = (int)std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(h.tiles, 1), (int64_t)llround(h.gx0 * hash_waves)));
    } else {
        for (auto& h : B->args.hash)
            if (h.tc_ok) {
                h.variant = 3;
                h.smem = h.tc_smem;
                h.gx = (int)std::max<int64_t>(1, std::min<int64_t>(h.tc_tiles, (int64_t)llround(h.tc_gx0 * -hash_waves)));
            }
    }
    for (auto& f : B->args.fwd) f.threads = fft_threads;
    // a captured graph holds the old launch shapes
    if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
    return SFFT_OK;
}

int sfft_batch_select_hash(sfft_batch* b, int tensor) {
    if (!b) { set_error("batch is NULL"); return SFFT_EINVAL; }
    Batch* B = reinterpret_cast<Batch*>(b);
    int n_tc = 0;
    for (auto& h : B->args.hash) {
        if (tensor && h.tc_ok) {
            h.variant = 3;
            h.smem = h.tc_smem;
            h.gx = h.gx0 = h.tc_gx0;
            ++n_tc;
        } else if (!tensor && h.variant == 3) {
            SFFT_CHECK(false, SFFT_EINVAL, "switching back to the packed hash kernel needs a new batch");
        }
    }
    SFFT_CHECK(!tensor || n_tc > 0, SFFT_EINVAL, "no hash launch of this batch qualifies for the tensor-core kernel");
    if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
    return SFFT_OK;
}

int sfft_batch_launch_count(sfft_batch* b, int* reconstruct, int* sampler) {
    if (!b) { set_error("batch is NULL"); return SFFT_EINVAL; }
    Batch* B = reinterpret_cast<Batch*>(b);
    const PipeArgs& A = B->args;
    // run_pipeline: clear, forward transforms, zero test, hash groups, compaction, combine, select;
    // the hybrid combine adds the hashes of Itilde and the collision counts, least squares four
    // launches, the refinement the scatter and the update (and a clear of its buckets after least
    // squares, which uses them as scratch; otherwise the combine zeroes them); the batch adds the counts
    int n = 1 + (int)A.fwd.size() + 1 + (int)A.hash.size() + 1 + 1 + 1 + 1;
    if (A.hybrid) n += 2;
    if (A.lsq) n += 4;
    if (A.refine) n += A.lsq ? 3 : 2;
    if (reconstruct) *reconstruct = n;
    // clear and bucket scatter (only for transforms outside shared memory), inverse transforms
    if (sampler) *sampler = (B->samp_scatter ? 2 : 0) + (int)B->samp.size();
    return SFFT_OK;
}

int sfft_batch_flags(sfft_batch* b, int64_t* flags) {
    if (!b || !flags) { set_error("null argument"); return SFFT_EINVAL; }
    Batch* B = reinterpret_cast<Batch*>(b);
    const int n = (int)B->plans.size();
    std::vector<int64_t> f(n);
    SFFT_CU(cudaEventSynchronize(B->done));
    SFFT_CU(cudaMemcpy(f.data(), B->d_flags, sizeof(int64_t) * n, cudaMemcpyDeviceToHost));
    int rc = SFFT_OK;
    for (int i = 0; i < n; ++i) {
        flags[B->order[i]] = f[i];
        if (f[i]) rc = SFFT_ECAPACITY;
    }
    if (rc != SFFT_OK)
        set_error("a capacity was exceeded in at least one plan (flags: 1 detected set, 2 FP64 guard band, 4 output)");
    return rc;
}

int sfft_batch_timing(sfft_batch* b, int mode, double* ms, int64_t* launches) {
    if (!b) { set_error("batch is NULL"); return -1; }
    Batch* B = reinterpret_cast<Batch*>(b);
    if (B->collect() != SFFT_OK) return -1;
    if (ms) for (int s = 0; s < ST_COUNT; ++s) ms[s] = B->stage_ms[s];
    if (launches) for (int s = 0; s < ST_COUNT; ++s) launches[s] = B->stage_n[s];
    if (mode >= 0) {
        B->timing = mode > 0;
        for (int s = 0; s < ST_COUNT; ++s) { B->stage_ms[s] = 0; B->stage_n[s] = 0; }
    }
    return ST_COUNT;
}

}  // extern "C"
