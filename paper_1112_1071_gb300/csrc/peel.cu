// The peel pass of an imaging pass (Sect. 2.6.2): the propagation kernel queues every event
// whose peel-off rays need a walk (a scattering, a re-emission, an emission from a cell) and
// carries on with its packet; this pass walks the rays from the queued events to every
// observer, one ray per thread.
//
// The events are first ordered by cell (a counting sort: histogram, exclusive scan, scatter of
// event indices), and rays are assigned observer-major in that order, so the 32 rays of a warp
// share their direction and start in the same or neighbouring cells: they cross nearly the same
// walls and stay converged.  Each ray is walked to the grid edge or PEEL_TAU_STOP with the same
// steps as the propagation kernel's own peel rays, and eps p exp(-tau) is tallied into the SED
// (and image) bins; only the order of the FP64 additions differs from walking them inline.
#include "propagate_common.cuh"

namespace hrt {

constexpr int USCAN_BLOCK = 1024;
constexpr int PEEL_MINB = 4;       // blocks of 256 per SM the registers are budgeted for (measured)

namespace {

__device__ __forceinline__ unsigned long long queued_events(const RunArgs& a) {
    const unsigned long long nq = *a.peel_n;
    return nq < (unsigned long long)a.peel_cap ? nq : (unsigned long long)a.peel_cap;
}

// bucket of an event: its cell, or ncells for an event located along each observer direction
__device__ __forceinline__ int64_t peel_key(const PeelEvent& e, int64_t ncells) {
    return e.ci < 0 ? ncells : (int64_t)e.ci;
}

__device__ __forceinline__ uint32_t block_inclusive_scan(uint32_t v, uint32_t* warp_sums) {
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if ((int)lane >= o) v += y;
    }
    if (lane == 31) warp_sums[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < blockDim.x / 32 ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if ((int)lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    return v + (warp > 0 ? warp_sums[warp - 1] : 0u);
}

}  // namespace

__global__ void k_peel_hist(RunArgs a, int64_t ncells, uint32_t* __restrict__ hist) {
    const unsigned long long n = queued_events(a);
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (unsigned long long)gridDim.x * blockDim.x)
        atomicAdd(hist + peel_key(a.peel_q[e], ncells), 1u);
}

// exclusive scan of x[0 .. n-1] in place: per-block scans, a scan of the block totals by one block,
// and the block offsets added
__global__ void __launch_bounds__(USCAN_BLOCK) k_uscan_blocks(uint32_t* x, int64_t n, uint32_t* sums) {
    __shared__ uint32_t ws[32];
    const int64_t c = (int64_t)blockIdx.x * USCAN_BLOCK + threadIdx.x;
    const uint32_t v = c < n ? x[c] : 0u;
    const uint32_t incl = block_inclusive_scan(v, ws);
    if (c < n) x[c] = incl - v;
    if (threadIdx.x == USCAN_BLOCK - 1) sums[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(USCAN_BLOCK) k_uscan_sums(uint32_t* sums, int nb) {
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry_s;
    if (threadIdx.x == 0) carry_s = 0u;
    __syncthreads();
    for (int base = 0; base < nb; base += USCAN_BLOCK) {
        const int b = base + threadIdx.x;
        const uint32_t v = b < nb ? sums[b] : 0u;
        const uint32_t incl = block_inclusive_scan(v, ws);
        const uint32_t carry = carry_s;
        if (b < nb) sums[b] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == USCAN_BLOCK - 1) carry_s = carry + incl;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(USCAN_BLOCK) k_uscan_add(uint32_t* x, int64_t n, const uint32_t* sums) {
    const int64_t c = (int64_t)blockIdx.x * USCAN_BLOCK + threadIdx.x;
    if (c < n) x[c] += sums[blockIdx.x];
}

__global__ void k_peel_scatter(RunArgs a, int64_t ncells, uint32_t* __restrict__ offs, uint32_t* __restrict__ order) {
    const unsigned long long n = queued_events(a);
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (unsigned long long)gridDim.x * blockDim.x)
        order[atomicAdd(offs + peel_key(a.peel_q[e], ncells), 1u)] = (uint32_t)e;
}

template <int G>
__global__ void __launch_bounds__(256, PEEL_MINB)
    k_peel_rays(DevGrid g, DevDust d, DevSources s, DevObs o, RunArgs a, Tallies t, const uint32_t* __restrict__ order) {
    const SharedTallies st = shared_tallies(o, a);
    __shared__ unsigned long long cnt_sh[8][N_COUNTERS];
    LocalCounters lc;
    lc.init(cnt_sh[threadIdx.x >> 5]);
    const unsigned long long n_ev = queued_events(a);
    const unsigned long long total = n_ev * (unsigned long long)o.nobs;
    unsigned check = 0;
    for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        if (((++check) & 63u) == 0 && past_deadline(a, t)) {
            lc.inc(C_WATCHDOG);
            break;
        }
        const int ob = (int)(q / n_ev);
        const PeelEvent e = a.peel_q[order[q - (unsigned long long)ob * n_ev]];
        const float3 n = make_float3(__ldg(o.n + 3 * ob), __ldg(o.n + 3 * ob + 1), __ldg(o.n + 3 * ob + 2));
        // the packet's extinction and SED bin, recomputed from its frequency by the same functions
        const float nu = fabsf(e.nu);
        const int sbin = sed_bin(o, nu);
        if (sbin < 0) continue;                             // (never queued)
        const float chi = dust_at(d, nu).chi;
        Ray r;
        r.p = make_float3(e.px, e.py, e.pz);
        r.ci = e.ci;
        if (e.ci >= 0) {
            r.i = e.ci % g.n1;
            r.j = (e.ci / g.n1) % g.n2;
            r.k = e.ci / (g.n1 * g.n2);
        }
        set_dir(r, n);
        float tau = 0.f;
        if (e.ci >= 0 || grid_locate<G>(g, r)) {
            // stops past PEEL_TAU_STOP (< 4e-18 of the weight remains); F_INF: stuck, dropped
            tau = tau_to_edge<G>(g, r, chi, lc.peel_cross, PEEL_TAU_STOP);
            if (tau == F_INF) lc.inc(C_STUCK);
        }
        const float prob = (e.nu < 0.f) ? hg_phase(d.g, dot3(make_float3(e.ux, e.uy, e.uz), n)) : (0.25f / CUDART_PI_F);
        const double w = a.eps * (double)(prob * expf(-tau));
        if (st.sed) atomicAdd(st.sed + ob * o.nsed + sbin, w);
        else atomicAdd(t.sed + (int64_t)ob * o.nsed + sbin, w);
        if (o.nimg > 0) {
            const float px = e.px * __ldg(o.ex + 3 * ob) + e.py * __ldg(o.ex + 3 * ob + 1) + e.pz * __ldg(o.ex + 3 * ob + 2);
            const float py = e.px * __ldg(o.ey + 3 * ob) + e.py * __ldg(o.ey + 3 * ob + 1) + e.pz * __ldg(o.ey + 3 * ob + 2);
            const int ix = (int)floorf((px + o.img_half) * o.img_scale);
            const int iy = (int)floorf((py + o.img_half) * o.img_scale);
            if (ix >= 0 && ix < o.img_nx && iy >= 0 && iy < o.img_ny)
                for (int l = 0; l < o.nimg; ++l)
                    if (__ldg(o.img_bin + l) == sbin)
                        atomicAdd(t.img + (((int64_t)ob * o.nimg + l) * o.img_ny + iy) * o.img_nx + ix, w);
        }
    }
    flush_counters(lc, t.counters);
    flush_shared(o, a, t, st);
}

template <int G>
static cudaError_t launch_rays(const PropagateJob& j, const uint32_t* order, int sms, cudaStream_t s) {
    const size_t smem = shared_bytes(j);
    cudaError_t e = cudaFuncSetAttribute(k_peel_rays<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peel_rays<G>, 256, smem);
    if (e != cudaSuccess) return e;
    k_peel_rays<G><<<sms * (per_sm > 0 ? per_sm : 1), 256, smem, s>>>(j.grid, j.dust, j.src, j.obs, j.args, j.tal, order);
    return cudaGetLastError();
}

// hist: ncells + 1 entries, sums: (ncells + USCAN_BLOCK) / USCAN_BLOCK entries, order: peel_cap
cudaError_t launch_peel_pass(const PropagateJob& j, uint32_t* hist, uint32_t* sums, uint32_t* order, cudaStream_t s,
                             int* launched) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t nk = j.grid.ncells + 1;
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)nk * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_peel_hist<<<sms * 4, 256, 0, s>>>(j.args, j.grid.ncells, hist);
    const int nb = (int)((nk + USCAN_BLOCK - 1) / USCAN_BLOCK);
    k_uscan_blocks<<<nb, USCAN_BLOCK, 0, s>>>(hist, nk, sums);
    k_uscan_sums<<<1, USCAN_BLOCK, 0, s>>>(sums, nb);
    k_uscan_add<<<nb, USCAN_BLOCK, 0, s>>>(hist, nk, sums);
    k_peel_scatter<<<sms * 4, 256, 0, s>>>(j.args, j.grid.ncells, hist, order);
    *launched += 6;
    if (j.grid.type == GRID_CARTESIAN) return launch_rays<GRID_CARTESIAN>(j, order, sms, s);
    if (j.grid.type == GRID_CYLINDRICAL) return launch_rays<GRID_CYLINDRICAL>(j, order, sms, s);
    return launch_rays<GRID_SPHERICAL>(j, order, sms, s);
}

}  // namespace hrt
