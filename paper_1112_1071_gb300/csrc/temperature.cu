// Temperature update and convergence statistic of a Lucy iteration (FP64).
//
// Sect. 2.3, Eqs. 2-3: per cell Adot = acc/(V dt) and T from the tabulated E(T) (temperature.cuh).
// Sect. 2.4, Eqs. 4-5: R = delta(prev, new) per cell with dust; the p-quantile Q is the exact
//   nearest-rank order statistic, found by an 8-pass radix select on the IEEE-754 bit patterns
//   of R (positive doubles sort like their bit patterns).
#include "hrt_internal.h"
#include "temperature.cuh"

namespace hrt {

constexpr int MAX_T_SMEM = 1024;   // four FP64 tables: 32 KB of static shared memory

__global__ void __launch_bounds__(256) k_temperature(TemperatureJob j) {
    __shared__ double sE[MAX_T_SMEM], slnE[MAX_T_SMEM], slnT[MAX_T_SMEM], sT[MAX_T_SMEM];
    const bool use_s = j.nT <= MAX_T_SMEM;
    if (use_s) {
        for (int i = threadIdx.x; i < j.nT; i += blockDim.x) {
            sE[i] = j.E[i]; slnE[i] = j.lnE[i]; slnT[i] = j.lnT[i]; sT[i] = j.Tn[i];
        }
    }
    __syncthreads();
    const double* E = use_s ? sE : j.E;
    const double* lnE = use_s ? slnE : j.lnE;
    const double* lnT = use_s ? slnT : j.lnT;
    const double* Tn = use_s ? sT : j.Tn;
    unsigned long long lo_c = 0, hi_c = 0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < j.ncells; c += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(c % j.n1);
        const int jj = (int)((c / j.n1) % j.n2);
        const int k = (int)(c / ((int64_t)j.n1 * j.n2));
        int cl;
        double T = j.T[c], A = j.adot[c];
        int32_t row;
        j.keys[c] = temperature_cell(j.acc[c] * j.acc_scale, j.va[i] * j.vb[jj] * j.vc[k], j.rhoL[c] > 0.f, j.quantity, j.first != 0,
                                     E, lnE, lnT, Tn, j.nT, T, A, row, cl);
        j.T[c] = T;
        j.adot[c] = A;
        j.emit_row[c] = row;
        lo_c += cl < 0;
        hi_c += cl > 0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo_c += __shfl_down_sync(0xffffffffu, lo_c, o);
        hi_c += __shfl_down_sync(0xffffffffu, hi_c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (lo_c) atomicAdd(j.counters + 0, lo_c);
        if (hi_c) atomicAdd(j.counters + 1, hi_c);
    }
}

static int grid_for(int64_t n, int block) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (n + block - 1) / block;
    const int64_t cap = (int64_t)sms * 8;
    return (int)(need < 1 ? 1 : (need < cap ? need : cap));
}

cudaError_t launch_temperature(const TemperatureJob& j, cudaStream_t s, int* launched) {
    k_temperature<<<grid_for(j.ncells, 256), 256, 0, s>>>(j);
    *launched += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------- radix select
// state[0] = prefix of the answer found so far, state[1] = rank still to find within it
__global__ void __launch_bounds__(256) k_radix_hist(const unsigned long long* __restrict__ keys, int64_t n, int shift,
                                                    const unsigned long long* __restrict__ state,
                                                    unsigned int* __restrict__ hist) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const unsigned long long prefix = state[0];
    const unsigned long long himask = (shift >= 56) ? 0ull : (~0ull << (shift + 8));
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[c];
        if ((key & himask) == (prefix & himask)) atomicAdd(&h[(key >> shift) & 255ull], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(hist + threadIdx.x, h[threadIdx.x]);
}

__global__ void k_radix_pick(int shift, unsigned long long* state, unsigned int* hist, unsigned long long* out) {
    if (threadIdx.x != 0) return;
    unsigned long long k = state[1];
    unsigned long long cum = 0;
    int b = 0;
    for (; b < 256; ++b) {
        if (cum + hist[b] > k) break;
        cum += hist[b];
    }
    if (b == 256) b = 255;   // unreachable for k < n
    state[0] |= ((unsigned long long)b) << shift;
    state[1] = k - cum;
    for (int i = 0; i < 256; ++i) hist[i] = 0u;
    if (shift == 0) *out = state[0];
}

__global__ void k_radix_init(unsigned long long* state, unsigned int* hist, unsigned long long k) {
    state[0] = 0ull;
    state[1] = k;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0u;
}

cudaError_t launch_select_kth(const unsigned long long* keys, int64_t n, unsigned long long k, unsigned int* d_hist,
                              unsigned long long* d_state, unsigned long long* d_out, cudaStream_t s, int* launched) {
    k_radix_init<<<1, 256, 0, s>>>(d_state, d_hist, k);
    const int grid = grid_for(n, 256);
    for (int shift = 56; shift >= 0; shift -= 8) {
        k_radix_hist<<<grid, 256, 0, s>>>(keys, n, shift, d_state, d_hist);
        k_radix_pick<<<1, 32, 0, s>>>(shift, d_state, d_hist, d_out);
    }
    *launched += 17;
    return cudaGetLastError();
}

// ---------------------------------------------------------------- single-step helpers
__global__ void k_invert(const double* adot, double* T, int64_t n, const double* E, const double* lnE,
                         const double* lnT, const double* Tn, int nT) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        int cl;
        T[c] = invert_E(adot[c], E, lnE, lnT, Tn, nT, cl);
    }
}

cudaError_t launch_invert_temperature(const double* adot, double* T, int64_t n, const double* E, const double* lnE,
                                      const double* lnT, const double* Tn, int nT, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_invert<<<grid_for(n, 256), 256, 0, s>>>(adot, T, n, E, lnE, lnT, Tn, nT);
    return cudaGetLastError();
}

__global__ void k_emit_rows(const double* T, int32_t* rows, int64_t n, const double* lnT, int nT) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        rows[c] = nearest_row(T[c], lnT, nT);
}

cudaError_t launch_emit_rows(const double* T, int32_t* rows, int64_t n, const double* lnT, int nT, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_emit_rows<<<grid_for(n, 256), 256, 0, s>>>(T, rows, n, lnT, nT);
    return cudaGetLastError();
}

}  // namespace hrt
