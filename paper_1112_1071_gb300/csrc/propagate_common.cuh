// Helpers shared by the propagation kernels: per-block shared-memory SED and escape tallies,
// the watchdog test and the persistent launch shape.
#pragma once
#include "hrt_internal.h"
#include "packet.cuh"

namespace hrt {

struct SharedTallies {
    double* sed;        // [nobs][nsed] or null (then global atomics)
    unsigned* esc;      // [10][nsed] or null
};

__device__ __forceinline__ SharedTallies shared_tallies(const DevObs& o, const RunArgs& a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SharedTallies st{nullptr, nullptr};
    if (a.smem_sed) {
        st.sed = reinterpret_cast<double*>(smem_raw);
        st.esc = reinterpret_cast<unsigned*>(smem_raw + sizeof(double) * (size_t)o.nobs * o.nsed);
        for (int i = threadIdx.x; i < o.nobs * o.nsed; i += blockDim.x) st.sed[i] = 0.0;
        for (int i = threadIdx.x; i < N_ESC_MU * o.nsed; i += blockDim.x) st.esc[i] = 0u;
    }
    __syncthreads();
    return st;
}

__device__ __forceinline__ void flush_shared(const DevObs& o, const RunArgs& a, const Tallies& t,
                                             const SharedTallies& st) {
    __syncthreads();
    if (!a.smem_sed) return;
    for (int i = threadIdx.x; i < o.nobs * o.nsed; i += blockDim.x)
        if (st.sed[i] != 0.0) atomicAdd(t.sed + i, st.sed[i]);
    for (int i = threadIdx.x; i < N_ESC_MU * o.nsed; i += blockDim.x)
        if (st.esc[i]) atomicAdd(t.esc + i, (unsigned long long)st.esc[i]);
}

// Watchdog: a kernel past its time budget raises the abort flag and every thread stops at its
// next check (no trap; the host reports HRT_ETIMEDOUT and the context stays usable).
__device__ __forceinline__ bool past_deadline(const RunArgs& a, const Tallies& t) {
    if (a.budget_ns == 0) return false;
    if (*(volatile int32_t*)t.abort_flag) return true;
    if (global_ns() > *a.t0 + a.budget_ns) {
        atomicExch(t.abort_flag, 1);
        return true;
    }
    return false;
}

// L2 eviction priorities for the walk (per-access cache policies, `createpolicy`): the FP64
// reductions into the accumulators are marked evict_last and the density loads evict_first, so
// that where the two arrays together exceed L2 (the 256^3 cloud: 128 + 64 MiB against 126 MB)
// the accumulator sectors -- whose misses cost a read and a write-back -- are the ones that stay.
struct L2Hints {
    uint64_t keep, stream;
};
__device__ __forceinline__ L2Hints make_l2_hints() {
    L2Hints h;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(h.keep));
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(h.stream));
    return h;
}
__device__ __forceinline__ float ld_hint(const float* p, uint64_t pol) {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(__cvta_generic_to_global(p)), "l"(pol));
    return v;
}
template <bool HINT>
__device__ __forceinline__ void add_acc(double* a, double v, uint64_t pol) {
    if constexpr (HINT)
        asm volatile("red.global.add.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(__cvta_generic_to_global(a)), "d"(v),
                     "l"(pol)
                     : "memory");
    else
        atomicAdd(a, v);
}

// Deposit of one lane: merged while the packet stays in one cell, flushed on a cell change.
// With WAGG, the flushes of all lanes at one step are grouped by cell (match.any) and each
// group adds its sum (formed in FP64) with one FP64 atomic.  Each flushed run is one packet entry of the cell,
// counted into `visits` when the diffusion approximation needs it.
template <bool WAGG, bool HINT = false>
__device__ __forceinline__ void flush_deposit(double* acc, uint32_t* visits, bool flushing, int32_t ci, float v,
                                              uint64_t pol = 0) {
    if constexpr (WAGG) {
        const unsigned lane = threadIdx.x & 31u;
        const int key = flushing ? ci : -1 - (int)lane;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (!flushing) return;
        if (__popc(peers) == 1) {
            add_acc<HINT>(acc + ci, widen(v), pol);
            if (visits) atomicAdd(visits + ci, 1u);
            return;
        }
        // the group's sum in FP64 (exact widening, then FP64 adds): the result does not depend
        // on which packets happen to share a warp step, to FP64 rounding
        double sum = 0.0;
        for (unsigned m = peers; m; m &= m - 1) sum += widen(__shfl_sync(peers, v, __ffs(m) - 1));
        if (lane == (unsigned)(__ffs(peers) - 1)) {
            add_acc<HINT>(acc + ci, sum, pol);
            if (visits) atomicAdd(visits + ci, (uint32_t)__popc(peers));
        }
    } else {
        if (flushing) {
            add_acc<HINT>(acc + ci, widen(v), pol);
            if (visits) atomicAdd(visits + ci, 1u);
        }
    }
}

// End of a lane's run outside the walk step (packet end, watchdog, kernel end).
template <bool HINT = false>
__device__ __forceinline__ void flush_run(const Tallies& t, int32_t ci, float v, uint64_t pol = 0) {
    if (ci < 0) return;
    if (v != 0.f) add_acc<HINT>(t.acc + ci, widen(v), pol);
    if (t.visits) atomicAdd(t.visits + ci, 1u);
}

// Optical depth beyond which a peel-off ray stops: exp(-40) = 4e-18 of its weight remains.
constexpr float PEEL_TAU_STOP = 40.f;

inline size_t shared_bytes(const PropagateJob& job) {
    if (!job.args.smem_sed) return 0;
    return sizeof(double) * (size_t)job.obs.nobs * job.obs.nsed + sizeof(unsigned) * (size_t)N_ESC_MU * job.obs.nsed;
}

// Persistent launch: blocks_per_sm (or the occupancy limit) blocks on every SM, fewer when
// there are fewer packets than threads.
template <typename K>
inline cudaError_t launch_persistent(K kernel, const PropagateJob& job, const Launch& l, cudaStream_t s) {
    const size_t smem = shared_bytes(job);
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, l.block, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (l.blocks_per_sm > 0 && l.blocks_per_sm < per_sm) per_sm = l.blocks_per_sm;
    int blocks = l.blocks > 0 ? l.blocks : per_sm * sms;
    const int64_t need = (job.args.n_packets + l.block - 1) / l.block;
    if (need < blocks) blocks = (int)(need > 0 ? need : 1);
    kernel<<<blocks, l.block, smem, s>>>(job.grid, job.dust, job.src, job.obs, job.args, job.tal);
    return cudaGetLastError();
}

}  // namespace hrt
