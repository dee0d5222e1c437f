// Batched models (hrt_batch_*): many models advance one Lucy iteration per persistent launch.
//
// The device keeps one descriptor per model (its grid, dust, sources, tallies, tables and
// temperature state) and a queue of (model, packet range) chunks ordered largest model first;
// warps of one persistent kernel pull chunks until the queue is empty (event.cu).  Temperature
// update, quantile select and the convergence test run on per-model cell segments, and a model
// that converges drops out of the next launch without any host decision.  The whole iteration
// is captured once as a CUDA graph and replayed; the host reads one small statistics copy per
// iteration.  hrt_batch_tune times a few launch shapes and caches the fastest per problem class.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

#include "ctx_internal.h"

using namespace hrt;

namespace {

constexpr int64_t CHUNK_PACKETS = 8192;
constexpr int64_t SEG_CELLS = 16384;

std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int>, Launch> g_tune_cache;   // (grid type, log2 cells, log2 packets)

}  // namespace

struct hrt_batch {
    std::vector<hrt_ctx*> models;
    int device = 0;
    cudaStream_t stream = nullptr;
    DBuf<BatchModel> d_models;
    DBuf<BatchChunk> d_chunks;
    DBuf<BatchSeg> d_segs;
    DBuf<BatchState> d_state;
    DBuf<unsigned> d_hist, d_chunk_counter, d_report_count;
    DBuf<unsigned long long> d_counters, d_t0;
    DBuf<int32_t> d_abort;
    DBuf<float> d_report;
    BatchState* h_state = nullptr;
    unsigned long long* h_counters = nullptr;
    std::vector<int64_t> packets;
    std::vector<double> eps;
    int nchunks[2] = {0, 0};
    int nsegs = 0;
    int nesc = 0;
    Launch launch;
    bool tuned = false;
    hrt_run_params built_params{};
    bool built = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

int bfail(cudaError_t e) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? HRT_ENOMEM : HRT_ECUDA;
}

#define BCK(call)                                  \
    do {                                           \
        cudaError_t _e = (call);                   \
        if (_e != cudaSuccess) return bfail(_e);   \
    } while (0)

bool same_params(const hrt_run_params& a, const hrt_run_params& b) {
    return a.max_interactions == b.max_interactions && a.quantity == b.quantity && a.p == b.p &&
           a.q_thres == b.q_thres && a.delta_thres == b.delta_thres && a.watchdog_ms == b.watchdog_ms &&
           a.terminate_on_absorb == b.terminate_on_absorb && a.regroup_threshold == b.regroup_threshold &&
           a.blocks_per_sm == b.blocks_per_sm;
}

void release_graph(hrt_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Device descriptors, chunk queue, cell segments and state for the given packet budgets.
int build_batch(hrt_batch* b, const int64_t* n_packets, const hrt_run_params& P) {
    const int n = (int)b->models.size();
    std::vector<BatchModel> desc(n);
    std::vector<BatchState> st(n);
    b->packets.assign(n_packets, n_packets + n);
    b->eps.assign(n, 0.0);
    b->nesc = 0;
    BCK(b->d_counters.alloc((size_t)n * N_COUNTERS));
    BCK(b->d_abort.alloc(1));
    BCK(b->d_t0.alloc(1));
    BCK(b->d_report.alloc(WD_REPORTS * WD_FIELDS));
    BCK(b->d_report_count.alloc(1));
    for (int m = 0; m < n; ++m) {
        hrt_ctx* ctx = b->models[m];
        const int rc = prepare_ctx(ctx);
        if (rc != HRT_OK) return rc;
        BCK(cudaStreamSynchronize(ctx->stream));   // staging ran on the model's stream
        if (n_packets[m] < 1 || n_packets[m] > 0xFFFFFFFFll) return HRT_EINVAL;
        BatchModel& M = desc[m];
        std::memset(&M, 0, sizeof(M));
        M.g = ctx->grid;
        M.d = ctx->dust;
        M.d.emit_row = ctx->d_row.p;
        M.s = ctx->src;
        M.o = ctx->obs;
        M.t.acc = ctx->d_acc.p;
        M.t.sed = ctx->d_sed.p;
        M.t.img = ctx->d_img.p;
        M.t.esc = ctx->d_esc.p;
        M.t.counters = b->d_counters.p + (size_t)m * N_COUNTERS;
        M.t.abort_flag = b->d_abort.p;
        M.t.report = b->d_report.p;
        M.t.report_count = b->d_report_count.p;
        M.t.visits = nullptr;
        RunArgs& A = M.a;
        A.n_packets = n_packets[m];
        A.first_packet = 0;
        A.key0 = (uint32_t)(ctx->seed & 0xFFFFFFFFu);
        A.key1 = (uint32_t)(ctx->seed >> 32);
        A.model_key = ctx->model_id;
        A.eps = ctx->L_tot / (double)n_packets[m];
        A.epsL0 = A.eps * ctx->L0;
        A.max_interactions = P.max_interactions;
        A.peel = 0;
        A.terminate_on_absorb = P.terminate_on_absorb;
        A.budget_ns = P.watchdog_ms > 0 ? (uint64_t)(P.watchdog_ms * 1e6) : 0ull;
        A.smem_sed = 0;
        A.t0 = b->d_t0.p;
        b->eps[m] = A.eps;
        M.va = ctx->d_va.p; M.vb = ctx->d_vb.p; M.vc = ctx->d_vc.p;
        M.E = ctx->d_E.p; M.lnE = ctx->d_lnE.p; M.lnT = ctx->d_lnT.p; M.Tn = ctx->d_Tn.p;
        M.nT = (int)ctx->Tn.size();
        M.quantity = P.quantity;
        M.T = ctx->d_T.p;
        M.adot = ctx->d_adot.p;
        M.emit_row = ctx->d_row.p;
        M.keys = ctx->d_keys.p;
        M.n_dust = ctx->n_dust;
        const int64_t nc = ctx->ncells();
        int64_t k = ctx->n_dust > 0 ? (nc - ctx->n_dust) + (int64_t)std::ceil(P.p * (double)ctx->n_dust) - 1 : 0;
        M.krank = std::max<int64_t>(0, std::min<int64_t>(k, nc - 1));
        b->nesc = std::max(b->nesc, N_ESC_MU * ctx->nsed);
        std::memset(&st[m], 0, sizeof(BatchState));
        st[m].iteration = (uint32_t)ctx->iteration;
        st[m].active = 1;
        st[m].have_Q = ctx->have_Q ? 1 : 0;
        st[m].Q_prev = ctx->Q_prev;
    }
    // chunk queue per grid type, largest packet budgets first
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return n_packets[x] > n_packets[y]; });
    std::vector<BatchChunk> chunks;
    for (int type = 0; type < 2; ++type) {
        const size_t start = chunks.size();
        for (int m : order) {
            if (desc[m].g.type != type) continue;
            for (int64_t p0 = 0; p0 < n_packets[m]; p0 += CHUNK_PACKETS) {
                BatchChunk c;
                c.model = m;
                c.pad = 0;
                c.p0 = p0;
                c.p1 = std::min<int64_t>(p0 + CHUNK_PACKETS, n_packets[m]);
                chunks.push_back(c);
            }
        }
        b->nchunks[type] = (int)(chunks.size() - start);
    }
    std::vector<BatchSeg> segs;
    for (int m = 0; m < n; ++m) {
        const int64_t nc = b->models[m]->ncells();
        for (int64_t c0 = 0; c0 < nc; c0 += SEG_CELLS) {
            BatchSeg sg;
            sg.model = m;
            sg.pad = 0;
            sg.c0 = c0;
            sg.c1 = std::min<int64_t>(c0 + SEG_CELLS, nc);
            segs.push_back(sg);
        }
    }
    b->nsegs = (int)segs.size();
    BCK(b->d_models.upload(desc.data(), n, b->stream));
    BCK(b->d_chunks.upload(chunks.data(), std::max<size_t>(chunks.size(), 1), b->stream));
    BCK(b->d_segs.upload(segs.data(), segs.size(), b->stream));
    BCK(b->d_state.upload(st.data(), n, b->stream));
    BCK(b->d_hist.alloc((size_t)n * 256));
    BCK(b->d_chunk_counter.alloc(2));
    if (!b->h_state) {
        BCK(cudaMallocHost(&b->h_state, sizeof(BatchState) * n));
        BCK(cudaMallocHost(&b->h_counters, sizeof(unsigned long long) * n * N_COUNTERS));
    }
    std::memcpy(b->h_state, st.data(), sizeof(BatchState) * n);
    if (!b->ev0) BCK(cudaEventCreate(&b->ev0));
    if (!b->ev1) BCK(cudaEventCreate(&b->ev1));
    BCK(cudaStreamSynchronize(b->stream));
    b->built_params = P;
    b->built = true;
    release_graph(b);
    return HRT_OK;
}

// The kernels of one batched iteration, in stream order.
int enqueue_iteration(hrt_batch* b, const hrt_run_params& P, bool propagate_only) {
    const int n = (int)b->models.size();
    BCK(cudaMemsetAsync(b->d_abort.p, 0, sizeof(int32_t), b->stream));
    BCK(cudaMemsetAsync(b->d_report_count.p, 0, sizeof(unsigned), b->stream));
    BCK(launch_stamp(b->d_t0.p, b->stream));
    BCK(launch_batch_begin(b->d_models.p, b->d_state.p, n, b->d_segs.p, b->nsegs, b->d_chunk_counter.p, b->d_hist.p,
                           b->nesc, b->stream));
    if (b->nchunks[0] > 0)
        BCK(launch_propagate_batch(GRID_CARTESIAN, b->d_models.p, b->d_chunks.p, b->nchunks[0], b->d_chunk_counter.p,
                                   b->d_state.p, b->launch, b->stream));
    if (b->nchunks[1] > 0)
        BCK(launch_propagate_batch(GRID_SPHERICAL, b->d_models.p, b->d_chunks.p + b->nchunks[0], b->nchunks[1],
                                   b->d_chunk_counter.p + 1, b->d_state.p, b->launch, b->stream));
    if (propagate_only) return HRT_OK;
    BCK(launch_batch_temperature(b->d_models.p, b->d_state.p, b->d_segs.p, b->nsegs, b->stream));
    BCK(launch_batch_select(b->d_models.p, b->d_state.p, n, b->d_segs.p, b->nsegs, b->d_hist.p, b->stream));
    BCK(launch_batch_end(b->d_models.p, b->d_state.p, n, P.q_thres, P.delta_thres, b->stream));
    BCK(cudaMemcpyAsync(b->h_state, b->d_state.p, sizeof(BatchState) * n, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaMemcpyAsync(b->h_counters, b->d_counters.p, sizeof(unsigned long long) * n * N_COUNTERS,
                        cudaMemcpyDeviceToHost, b->stream));
    return HRT_OK;
}

int capture(hrt_batch* b, const hrt_run_params& P) {
    release_graph(b);
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_iteration(b, P, false);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc != HRT_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    BCK(e);
    b->graph = g;
    BCK(cudaGraphInstantiate(&b->exec, g, 0));
    return HRT_OK;
}

Launch launch_from(const hrt_run_params& P, const Launch& tuned) {
    Launch l = tuned;
    if (P.regroup_threshold > 0) l.regroup = P.regroup_threshold;
    if (P.blocks_per_sm > 0) l.blocks_per_sm = P.blocks_per_sm;
    return l;
}

std::tuple<int, int, int> class_key(hrt_batch* b, const int64_t* n_packets) {
    int64_t cells = 0, packets = 0;
    for (size_t m = 0; m < b->models.size(); ++m) {
        cells += b->models[m]->ncells();
        packets += n_packets[m];
    }
    const int type = b->models.empty() ? 0 : b->models[0]->gtype;
    return {type, (int)std::log2((double)std::max<int64_t>(cells, 1)), (int)std::log2((double)std::max<int64_t>(packets, 1))};
}

}  // namespace

extern "C" {

int hrt_batch_create(hrt_batch** out, hrt_ctx* const* models, int n) {
    if (!out || !models || n < 1) return HRT_EINVAL;
    *out = nullptr;
    for (int m = 0; m < n; ++m)
        if (!models[m] || models[m]->device != models[0]->device || models[m]->gtype == GRID_CYLINDRICAL)
            return HRT_EINVAL;          // the batch runs Cartesian and spherical-polar models
    hrt_batch* b = new hrt_batch();
    b->models.assign(models, models + n);
    b->device = models[0]->device;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    // a stream of its own: graph capture is not possible on the legacy default stream
    const cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        delete b;
        return bfail(e);
    }
    *out = b;
    return HRT_OK;
}

int hrt_batch_destroy(hrt_batch* b) {
    if (!b) return HRT_EINVAL;
    cudaStreamSynchronize(b->stream);
    release_graph(b);
    b->d_models.release(); b->d_chunks.release(); b->d_segs.release(); b->d_state.release();
    b->d_hist.release(); b->d_chunk_counter.release(); b->d_report_count.release(); b->d_counters.release();
    b->d_t0.release(); b->d_abort.release(); b->d_report.release();
    if (b->h_state) cudaFreeHost(b->h_state);
    if (b->h_counters) cudaFreeHost(b->h_counters);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return HRT_OK;
}

int hrt_batch_tune(hrt_batch* b, const int64_t* n_packets) {
    if (!b || !n_packets) return HRT_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    hrt_run_params P;
    hrt_default_params(&P);
    const auto key = class_key(b, n_packets);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            b->launch = it->second;
            b->tuned = true;
            release_graph(b);
            if (prev >= 0) cudaSetDevice(prev);
            return HRT_OK;
        }
    }
    // trial launches on at most ~2^24 packets in all (each model's budget scaled alike)
    int64_t total = 0;
    for (size_t m = 0; m < b->models.size(); ++m) total += n_packets[m];
    const double scale = total > ((int64_t)1 << 24) ? (double)((int64_t)1 << 24) / (double)total : 1.0;
    std::vector<int64_t> trial(b->models.size());
    for (size_t m = 0; m < trial.size(); ++m) trial[m] = std::max<int64_t>(1, (int64_t)(n_packets[m] * scale));
    // the caller's device comes back on every exit
    auto done = [&](int code) {
        if (prev >= 0) cudaSetDevice(prev);
        return code;
    };
    int rc = build_batch(b, trial.data(), P);
    if (rc != HRT_OK) return done(rc);
    const int regroups[] = {12, 16, 20, 24};
    const int per_sm[] = {2, 3, 4};
    float best = 1e30f;
    Launch best_l = b->launch;
    for (int bp : per_sm) {
        for (int rg : regroups) {
            b->launch.regroup = rg;
            b->launch.blocks_per_sm = bp;
            for (int rep = 0; rep < 2; ++rep) {     // first run warms up
                cudaEventRecord(b->ev0, b->stream);
                rc = enqueue_iteration(b, P, true);
                if (rc != HRT_OK) return done(rc);
                cudaEventRecord(b->ev1, b->stream);
                if (cudaStreamSynchronize(b->stream) != cudaSuccess) return done(bfail(cudaGetLastError()));
                float ms = 0.f;
                cudaEventElapsedTime(&ms, b->ev0, b->ev1);
                if (rep == 1 && ms < best) {
                    best = ms;
                    best_l = b->launch;
                }
            }
        }
    }
    b->launch = best_l;
    b->tuned = true;
    release_graph(b);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = best_l;
    }
    if (prev >= 0) cudaSetDevice(prev);
    return HRT_OK;
}

int hrt_batch_run(hrt_batch* b, const int64_t* n_packets, int max_iter, const hrt_run_params* params,
                  hrt_iter_stats* per_model_out, int* iterations_run) {
    if (!b || !n_packets || max_iter < 0) return HRT_EINVAL;
    hrt_run_params P;
    if (params) P = *params;
    else hrt_default_params(&P);
    if (!(P.p > 0 && P.p <= 1) || P.max_interactions < 0) return HRT_EINVAL;
    if ((P.quantity != 0 && P.quantity != 1) || (P.block_size != 0 && P.block_size != 256) || P.blocks_per_sm < 0 ||
        P.regroup_threshold < 0 || P.regroup_threshold > 32 || !(P.watchdog_ms >= 0) || !std::isfinite(P.watchdog_ms) ||
        std::isnan(P.q_thres) || std::isnan(P.delta_thres))
        return HRT_EINVAL;
    // Lucy iterations only: the extensions and imaging passes run in single-model calls
    if (P.mrw_gamma != 0 || P.pda_min_visits != 0 || P.raytrace_rays != 0 || P.peel != 0 || !P.update_temperature)
        return HRT_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    const int n = (int)b->models.size();
    bool rebuild = !b->built || !same_params(P, b->built_params);
    for (int m = 0; m < n && !rebuild; ++m) rebuild = b->packets[m] != n_packets[m];
    int rc = HRT_OK;
    if (rebuild) {
        rc = build_batch(b, n_packets, P);
        if (rc != HRT_OK) {
            if (prev >= 0) cudaSetDevice(prev);
            return rc;
        }
    } else {
        // restart the convergence state from the contexts (a new run of the batch)
        std::vector<BatchState> st(n);
        for (int m = 0; m < n; ++m) {
            std::memset(&st[m], 0, sizeof(BatchState));
            st[m].iteration = (uint32_t)b->models[m]->iteration;
            st[m].active = 1;
            st[m].have_Q = b->models[m]->have_Q ? 1 : 0;
            st[m].Q_prev = b->models[m]->Q_prev;
        }
        std::memcpy(b->h_state, st.data(), sizeof(BatchState) * n);
        BCK(cudaMemcpyAsync(b->d_state.p, b->h_state, sizeof(BatchState) * n, cudaMemcpyHostToDevice, b->stream));
    }
    b->launch = launch_from(P, b->launch);
    if (!b->exec) {
        rc = capture(b, P);
        if (rc != HRT_OK) {
            if (prev >= 0) cudaSetDevice(prev);
            return rc;
        }
    }
    int iters = 0;
    bool timed_out = false;
    for (int it = 0; it < max_iter; ++it) {
        bool any = false;
        for (int m = 0; m < n; ++m) any = any || b->h_state[m].active;
        if (!any) break;
        BCK(cudaEventRecord(b->ev0, b->stream));
        BCK(cudaGraphLaunch(b->exec, b->stream));
        BCK(cudaEventRecord(b->ev1, b->stream));
        BCK(cudaStreamSynchronize(b->stream));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, b->ev0, b->ev1);
        ++iters;
        for (int m = 0; m < n; ++m) {
            const BatchState& S = b->h_state[m];
            if (!S.ran) continue;
            const unsigned long long* h = b->h_counters + (size_t)m * N_COUNTERS;
            if (h[C_WATCHDOG]) timed_out = true;
            if (!per_model_out) continue;
            hrt_iter_stats& st = per_model_out[m];
            std::memset(&st, 0, sizeof(st));
            st.iteration = (int32_t)S.iteration - 1;
            st.converged = S.converged;
            st.Q = S.Q;
            st.Delta = S.Delta;
            st.e_emitted = b->models[m]->L_tot;
            st.e_escaped = (double)h[C_ESCAPED] * b->eps[m];
            st.e_killed = (double)h[C_KILLED] * b->eps[m];
            st.e_absorbed = (double)h[C_ABSORBED_TERM] * b->eps[m];
            st.n_packets = b->packets[m];
            st.n_interactions = (int64_t)h[C_INTERACTIONS];
            st.n_scatter = (int64_t)h[C_SCATTER];
            st.n_absorb = (int64_t)h[C_ABSORB];
            st.n_crossings = (int64_t)h[C_CROSSINGS];
            st.n_peel_crossings = (int64_t)h[C_PEEL_CROSSINGS];
            st.n_killed = (int64_t)h[C_KILLED];
            st.clamp_low = (int64_t)S.clamp_low;
            st.clamp_high = (int64_t)S.clamp_high;
            st.ms_total = ms;
            st.ms_propagate = ms;
            st.kernel_launches = 24 + (b->nchunks[0] > 0) + (b->nchunks[1] > 0);
        }
        if (timed_out) break;
    }
    for (int m = 0; m < n; ++m) {
        hrt_ctx* ctx = b->models[m];
        ctx->iteration = (int)b->h_state[m].iteration;
        ctx->Q_prev = b->h_state[m].Q_prev;
        ctx->have_Q = b->h_state[m].have_Q != 0;
        ctx->last_eps = b->eps[m];
        ctx->acc_scale = b->eps[m] * ctx->L0;
    }
    if (iterations_run) *iterations_run = iters;
    if (prev >= 0) cudaSetDevice(prev);
    return timed_out ? HRT_ETIMEDOUT : HRT_OK;
}

}  // extern "C"
