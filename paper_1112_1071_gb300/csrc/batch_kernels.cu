// Kernels of one batched Lucy iteration over many models (all device-resident, so the whole
// iteration is captured once as a CUDA graph and replayed):
//   begin:       per model, zero the tallies and reset the select state; per cell segment, zero
//                the absorbed-energy accumulators and set the re-emission rows from T.
//   temperature: per cell segment, Eqs. 2-3 and the convergence key (temperature.cuh).
//   select:      8 radix passes with per-model histograms -> each model's nearest-rank quantile.
//   end:         per model, Q, Delta (Eq. 6), the convergence flag and the next iteration key;
//                a converged model drops out of later launches.
#include "hrt_internal.h"
#include "temperature.cuh"

namespace hrt {

__global__ void k_batch_begin_models(const BatchModel* __restrict__ models, BatchState* state, int nmodels,
                                     unsigned* chunk_counter, unsigned* hist, int nesc) {
    const int m = blockIdx.x;
    if (m == 0 && threadIdx.x < 2) chunk_counter[threadIdx.x] = 0u;   // one queue per grid type
    if (m >= nmodels) return;
    const BatchModel& M = models[m];
    BatchState& S = state[m];
    const bool act = S.active != 0;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[(int64_t)m * 256 + i] = 0u;
    if (!act) return;
    for (int i = threadIdx.x; i < N_COUNTERS; i += blockDim.x) M.t.counters[i] = 0ull;
    for (int i = threadIdx.x; i < nesc; i += blockDim.x) M.t.esc[i] = 0ull;
    if (threadIdx.x == 0) {
        S.prefix = 0ull;
        S.rank = (unsigned long long)M.krank;
        S.clamp_low = S.clamp_high = 0ull;
    }
}

__global__ void __launch_bounds__(256) k_batch_begin_cells(const BatchModel* __restrict__ models,
                                                           const BatchState* __restrict__ state,
                                                           const BatchSeg* __restrict__ segs, int nsegs) {
    for (int sg = blockIdx.x; sg < nsegs; sg += gridDim.x) {
        const BatchSeg seg = segs[sg];
        if (!state[seg.model].active) continue;
        const BatchModel& M = models[seg.model];
        for (int64_t c = seg.c0 + threadIdx.x; c < seg.c1; c += blockDim.x) {
            M.t.acc[c] = 0.0;
            M.emit_row[c] = nearest_row(M.T[c], M.lnT, M.nT);
        }
    }
}

__global__ void __launch_bounds__(256) k_batch_temperature(const BatchModel* __restrict__ models, BatchState* state,
                                                           const BatchSeg* __restrict__ segs, int nsegs) {
    for (int sg = blockIdx.x; sg < nsegs; sg += gridDim.x) {
        const BatchSeg seg = segs[sg];
        BatchState& S = state[seg.model];
        if (!S.active) continue;
        const BatchModel& M = models[seg.model];
        const bool first = S.have_Q == 0 && M.quantity != 0;
        unsigned long long lo_c = 0, hi_c = 0;
        for (int64_t c = seg.c0 + threadIdx.x; c < seg.c1; c += blockDim.x) {
            const int i = (int)(c % M.g.n1);
            const int jj = (int)((c / M.g.n1) % M.g.n2);
            const int k = (int)(c / ((int64_t)M.g.n1 * M.g.n2));
            int cl;
            double T = M.T[c], A = M.adot[c];
            int32_t row;
            M.keys[c] = temperature_cell(M.t.acc[c] * M.a.epsL0, M.va[i] * M.vb[jj] * M.vc[k], M.g.rhoL[c] > 0.f, M.quantity,
                                         first, M.E, M.lnE, M.lnT, M.Tn, M.nT, T, A, row, cl);
            M.T[c] = T;
            M.adot[c] = A;
            M.emit_row[c] = row;
            lo_c += cl < 0;
            hi_c += cl > 0;
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo_c += __shfl_down_sync(0xffffffffu, lo_c, o);
            hi_c += __shfl_down_sync(0xffffffffu, hi_c, o);
        }
        if ((threadIdx.x & 31) == 0) {
            if (lo_c) atomicAdd(&S.clamp_low, lo_c);
            if (hi_c) atomicAdd(&S.clamp_high, hi_c);
        }
    }
}

__global__ void __launch_bounds__(256) k_batch_hist(const BatchModel* __restrict__ models,
                                                    const BatchState* __restrict__ state,
                                                    const BatchSeg* __restrict__ segs, int nsegs, int shift,
                                                    unsigned* hist) {
    __shared__ unsigned int h[256];
    const unsigned long long himask = (shift >= 56) ? 0ull : (~0ull << (shift + 8));
    for (int sg = blockIdx.x; sg < nsegs; sg += gridDim.x) {
        const BatchSeg seg = segs[sg];
        const BatchState& S = state[seg.model];
        if (!S.active || models[seg.model].n_dust == 0) continue;   // block-uniform
        h[threadIdx.x] = 0u;
        __syncthreads();
        const unsigned long long prefix = S.prefix;
        const unsigned long long* keys = models[seg.model].keys;
        for (int64_t c = seg.c0 + threadIdx.x; c < seg.c1; c += blockDim.x) {
            const unsigned long long key = keys[c];
            if ((key & himask) == (prefix & himask)) atomicAdd(&h[(key >> shift) & 255ull], 1u);
        }
        __syncthreads();
        if (h[threadIdx.x]) atomicAdd(hist + (int64_t)seg.model * 256 + threadIdx.x, h[threadIdx.x]);
        __syncthreads();
    }
}

__global__ void k_batch_pick(const BatchModel* __restrict__ models, BatchState* state, int nmodels, int shift,
                             unsigned* hist) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmodels) return;
    BatchState& S = state[m];
    if (!S.active || models[m].n_dust == 0) return;
    unsigned* hm = hist + (int64_t)m * 256;
    unsigned long long k = S.rank, cum = 0;
    int b = 0;
    for (; b < 255; ++b) {
        if (cum + hm[b] > k) break;
        cum += hm[b];
    }
    S.prefix |= ((unsigned long long)b) << shift;
    S.rank = k - cum;
    for (int i = 0; i < 256; ++i) hm[i] = 0u;
}

__global__ void k_batch_end(const BatchModel* __restrict__ models, BatchState* state, int nmodels, double q_thres,
                            double delta_thres) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmodels) return;
    BatchState& S = state[m];
    S.ran = S.active;
    if (!S.active) return;
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    double Q = inf;
    if (models[m].n_dust > 0) Q = __longlong_as_double((long long)S.prefix);
    const double D = (S.have_Q && isfinite(S.Q_prev) && isfinite(Q)) ? fmax(S.Q_prev / Q, Q / S.Q_prev) : inf;
    S.Q = Q;
    S.Delta = D;
    S.converged = (Q < q_thres) && (D < delta_thres || isinf(delta_thres));
    S.Q_prev = Q;
    S.have_Q = models[m].n_dust > 0 ? 1 : S.have_Q;
    S.iteration += 1u;
    if (S.converged) S.active = 0;
}

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

cudaError_t launch_batch_begin(const BatchModel* models, BatchState* state, int nmodels, const BatchSeg* segs,
                               int nsegs, unsigned* chunk_counter, unsigned* hist, int nesc, cudaStream_t s) {
    k_batch_begin_models<<<nmodels, 128, 0, s>>>(models, state, nmodels, chunk_counter, hist, nesc);
    const int grid = nsegs < sm_count() * 8 ? nsegs : sm_count() * 8;
    k_batch_begin_cells<<<grid > 0 ? grid : 1, 256, 0, s>>>(models, state, segs, nsegs);
    return cudaGetLastError();
}

cudaError_t launch_batch_temperature(const BatchModel* models, BatchState* state, const BatchSeg* segs, int nsegs,
                                     cudaStream_t s) {
    const int grid = nsegs < sm_count() * 8 ? nsegs : sm_count() * 8;
    k_batch_temperature<<<grid > 0 ? grid : 1, 256, 0, s>>>(models, state, segs, nsegs);
    return cudaGetLastError();
}

cudaError_t launch_batch_select(const BatchModel* models, BatchState* state, int nmodels, const BatchSeg* segs,
                                int nsegs, unsigned* hist, cudaStream_t s) {
    const int grid = nsegs < sm_count() * 8 ? nsegs : sm_count() * 8;
    for (int shift = 56; shift >= 0; shift -= 8) {
        k_batch_hist<<<grid > 0 ? grid : 1, 256, 0, s>>>(models, state, segs, nsegs, shift, hist);
        k_batch_pick<<<(nmodels + 127) / 128, 128, 0, s>>>(models, state, nmodels, shift, hist);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_end(const BatchModel* models, BatchState* state, int nmodels, double q_thres,
                             double delta_thres, cudaStream_t s) {
    k_batch_end<<<(nmodels + 127) / 128, 128, 0, s>>>(models, state, nmodels, q_thres, delta_thres);
    return cudaGetLastError();
}

}  // namespace hrt
