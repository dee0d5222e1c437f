// Propagation kernels of one Lucy iteration (Sect. 2.2, Eq. 2, Sect. 2.6.2).
//
// k_plain: one thread per packet history, grid-stride over packets, every deposit a plain FP64
//          atomic.  The reference GPU formulation ("plain GPU").
// k_event: persistent warps in which every lane runs a small state machine (emit, walk,
//          interact, peel ray) and refills itself from a global packet counter; the walk phase
//          runs while at least `regroup` lanes are walking, so packets in different states
//          are regrouped into long converged walk loops; deposits are merged per lane while the
//          packet stays in one cell and across lanes of a warp that hit the same cell.
#include <cooperative_groups.h>

#include "hrt_internal.h"
#include "packet.cuh"

namespace hrt {

// ---------------------------------------------------------------- shared tallies
struct SharedTallies {
    double* sed;        // [nobs][nsed] or null
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

__global__ void k_stamp(unsigned long long* t0) { *t0 = global_ns(); }

cudaError_t launch_stamp(unsigned long long* t0, cudaStream_t s) {
    k_stamp<<<1, 1, 0, s>>>(t0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- plain kernel
// Walk to optical depth tau (extinction) or escape; each segment in a cell with dust adds
// eps * kappa * l to the cell (Eq. 2's numerator).
template <int G>
__device__ __forceinline__ int walk_plain(const DevGrid& g, const RunArgs& a, const Tallies& t, Packet& pk,
                                          float tau, LocalCounters& lc) {
    const float chi = pk.dust.chi;
    const double dep = a.epsL0 * (double)pk.dust.kappa;
    unsigned check = 0;
    int zero_run = 0;
    for (;;) {
        int axis, dir;
        const float l = cell_exit<G>(g, pk.r, axis, dir);
        if constexpr (G == GRID_SPHERICAL) {
            if (!tiny_step(pk.r, l)) zero_run = 0;
            else if (++zero_run > ZERO_RUN_LIMIT) { nudge(pk.r); zero_run = 0; }
        }
        if (check >= MAX_WALK_STEPS) {
            lc.v[C_STUCK]++;
            return EV_STUCK;
        }
        const float rho = __ldg(g.rhoL + pk.r.ci);
        const float k = rho * chi;
        const float dtau = k * l;
        if (tau < dtau) {
            const float lp = tau / k;
            atomicAdd(t.acc + pk.r.ci, dep * (double)lp);
            pk.r.p.x += lp * pk.r.u.x;
            pk.r.p.y += lp * pk.r.u.y;
            pk.r.p.z += lp * pk.r.u.z;
            return EV_INTERACT;
        }
        if (rho > 0.f) atomicAdd(t.acc + pk.r.ci, dep * (double)l);
        tau -= dtau;
        lc.v[C_CROSSINGS]++;
        if (cell_step<G>(g, pk.r, l, axis, dir)) return EV_ESCAPE;
        if (((++check) & 1023u) == 0 && past_deadline(a, t)) return EV_ABORT;
    }
}

template <int G>
__global__ void __launch_bounds__(256) k_plain(DevGrid g, DevDust d, DevSources s, DevObs o, RunArgs a, Tallies t) {
    const SharedTallies st = shared_tallies(o, a);
    LocalCounters lc;
    lc.zero();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < a.n_packets; q += stride) {
        if (past_deadline(a, t)) {
            lc.v[C_WATCHDOG]++;
            break;
        }
        Packet pk;
        if (!emit_packet<G>(g, d, s, o, a, t, st.sed, a.first_packet + q, pk, lc)) {
            lc.v[C_ESCAPED]++;
            lc.v[C_PACKETS_DONE]++;
            continue;
        }
        for (;;) {
            const float tau = -logf(pk.rng.next());
            const int ev = walk_plain<G>(g, a, t, pk, tau, lc);
            if (ev == EV_ESCAPE) {
                lc.v[C_ESCAPED]++;
                tally_escape(o, t, pk, st.esc);
                break;
            }
            if (ev == EV_ABORT) {
                lc.v[C_WATCHDOG]++;
                break;
            }
            if (ev == EV_STUCK) {
                lc.v[C_KILLED]++;
                break;
            }
            if (++pk.nint > a.max_interactions) {
                lc.v[C_KILLED]++;
                break;
            }
            if (!interact<G>(g, d, o, a, t, st.sed, pk, lc)) break;
        }
        lc.v[C_PACKETS_DONE]++;
    }
    flush_counters(lc, t.counters);
    flush_shared(o, a, t, st);
}

static size_t shared_bytes(const PropagateJob& job) {
    if (!job.args.smem_sed) return 0;
    return sizeof(double) * (size_t)job.obs.nobs * job.obs.nsed + sizeof(unsigned) * (size_t)N_ESC_MU * job.obs.nsed;
}

template <typename K>
static cudaError_t launch_persistent(K kernel, const PropagateJob& job, const Launch& l, cudaStream_t s) {
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

cudaError_t launch_propagate_plain(const PropagateJob& job, const Launch& l, cudaStream_t s, int* launched) {
    if (job.args.n_packets <= 0) return cudaSuccess;
    Launch ll = l;
    ll.block = 256;
    *launched += 1;
    if (job.grid.type == GRID_CARTESIAN) return launch_persistent(k_plain<GRID_CARTESIAN>, job, ll, s);
    return launch_persistent(k_plain<GRID_SPHERICAL>, job, ll, s);
}

// ---------------------------------------------------------------- event kernel
enum LaneMode : int32_t { M_NEED = 0, M_WALK, M_PEEL, M_INTERACT, M_ESCAPED, M_PEEL_DONE, M_KILLED, M_DONE };

// Deposit of one lane: merged while the packet stays in one cell, flushed on a cell change.
// With WAGG, the flushes of all lanes at one step are grouped by cell (match.any) and each
// group adds its sum with one FP64 atomic.
template <bool WAGG>
__device__ __forceinline__ void flush_deposit(double* acc, bool flushing, int32_t ci, double v) {
    if constexpr (WAGG) {
        const unsigned lane = threadIdx.x & 31u;
        const int key = flushing ? ci : -1 - (int)lane;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (!flushing) return;
        if (__popc(peers) == 1) {
            atomicAdd(acc + ci, v);
            return;
        }
        double sum = 0.0;
        for (unsigned m = peers; m; m &= m - 1) sum += __shfl_sync(peers, v, __ffs(m) - 1);
        if (lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(acc + ci, sum);
    } else {
        if (flushing) atomicAdd(acc + ci, v);
    }
}

template <int G, bool WAGG>
__global__ void __launch_bounds__(256, 2) k_event(DevGrid g, DevDust d, DevSources s, DevObs o, RunArgs a, Tallies t) {
    const SharedTallies st = shared_tallies(o, a);
    LocalCounters lc;
    lc.zero();
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;

    Packet pk;                 // the packet; pk.r is the ray currently walked (packet or peel ray)
    Ray saved;                 // packet ray while its peel rays are walked
    float3 porg = make_float3(0.f, 0.f, 0.f);   // origin of the peel rays (event position)
    float3 uin = make_float3(0.f, 0.f, 1.f);    // incoming direction at a scattering (HG peel)
    float tau = 0.f;           // optical depth left (packet) or accumulated (peel ray)
    int32_t mode = M_NEED;
    int32_t pobs = 0, pkind = PEEL_ISO, prelocate = 0;
    int32_t dep_ci = -1;
    double dep_val = 0.0, dep_rate = 0.0;
    int zero_run = 0;
    unsigned ray_steps = 0;    // crossings of the current ray since it started or last interacted
    bool aborted = false;

    // start peel ray `ob` from porg (cell of `saved`, or located along the observer direction)
    auto start_peel = [&](int ob) {
        pk.r = saved;
        pk.r.p = porg;
        set_dir(pk.r, make_float3(__ldg(o.n + 3 * ob), __ldg(o.n + 3 * ob + 1), __ldg(o.n + 3 * ob + 2)));
        tau = 0.f;
        ray_steps = 0;
        zero_run = 0;
        mode = M_PEEL;
        if (prelocate && !grid_locate<G>(g, pk.r)) mode = M_PEEL_DONE;
    };
    // after an emission or interaction: peel (if wanted) then draw a new optical depth
    auto after_event = [&](int kind, int relocate) {
        if (a.peel && pk.sbin >= 0 && o.nobs > 0) {
            saved = pk.r;
            pkind = kind;
            prelocate = relocate;
            pobs = 0;
            start_peel(0);
        } else {
            tau = -logf(pk.rng.next());
            dep_rate = a.epsL0 * (double)pk.dust.kappa;
            ray_steps = 0;
            zero_run = 0;
            mode = M_WALK;
        }
    };
    // Watchdog (warp-uniform call): past the time budget, every live lane stops, records its
    // state in the report buffer (first WD_REPORTS lanes) and is counted; nothing traps.
    unsigned rounds = 0;
    auto watchdog = [&](unsigned where) {
        bool ab = false;
        if (lane == 0) ab = past_deadline(a, t);
        if (!__shfl_sync(FULL, ab ? 1 : 0, 0)) return;
        aborted = true;
        if (mode == M_DONE) return;
        lc.v[C_WATCHDOG]++;
        const unsigned slot = atomicAdd(t.report_count, 1u);
        if (slot < (unsigned)WD_REPORTS) {
            float* r = t.report + slot * WD_FIELDS;
            r[0] = (float)mode; r[1] = (float)pk.rng.pkt; r[2] = (float)pk.nint; r[3] = tau;
            r[4] = pk.r.p.x; r[5] = pk.r.p.y; r[6] = pk.r.p.z;
            r[7] = pk.r.u.x; r[8] = pk.r.u.y; r[9] = pk.r.u.z;
            r[10] = (float)pk.r.i; r[11] = (float)pk.r.j; r[12] = (float)pk.r.k;
            r[13] = pk.nu; r[14] = (float)pobs; r[15] = (float)where;
        }
        if (dep_ci >= 0 && dep_val != 0.0) atomicAdd(t.acc + dep_ci, dep_val);
        dep_ci = -1;
        mode = M_DONE;
    };
    auto end_packet = [&]() {
        if (dep_ci >= 0 && dep_val != 0.0) atomicAdd(t.acc + dep_ci, dep_val);
        dep_ci = -1;
        dep_val = 0.0;
        lc.v[C_PACKETS_DONE]++;
        mode = M_NEED;
    };

    for (;;) {
        // ------------------------------------------------------------ event phase
        if (mode == M_KILLED) {
            end_packet();
        } else if (mode == M_ESCAPED) {
            lc.v[C_ESCAPED]++;
            tally_escape(o, t, pk, st.esc);
            end_packet();
        } else if (mode == M_INTERACT) {
            if (++pk.nint > a.max_interactions) {
                lc.v[C_KILLED]++;
                end_packet();
            } else {
                lc.v[C_INTERACTIONS]++;
                const float z = pk.rng.next();
                if (z > pk.dust.albedo) {
                    lc.v[C_ABSORB]++;
                    if (a.terminate_on_absorb) {
                        lc.v[C_ABSORBED_TERM]++;
                        end_packet();
                    } else {
                        const float u1 = pk.rng.next(), u2 = pk.rng.next();
                        set_dir(pk.r, isotropic_dir(u1, u2));
                        const int row = __ldg(d.emit_row + pk.r.ci);
                        set_frequency(pk, d, o, sample_table(d.nu, d.cdf_emit + (int64_t)row * d.nnu, d.nnu, pk.rng.next()));
                        porg = pk.r.p;
                        after_event(PEEL_ISO, 0);
                    }
                } else {
                    lc.v[C_SCATTER]++;
                    const float mu = hg_mu(d.g, pk.rng.next());
                    const float u2 = pk.rng.next();
                    uin = pk.r.u;
                    set_dir(pk.r, scatter_dir(uin, mu, u2));
                    porg = pk.r.p;
                    after_event(PEEL_HG, 0);
                }
            }
        } else if (mode == M_PEEL_DONE) {
            const float3 n = pk.r.u;
            const float prob = (pkind == PEEL_HG) ? hg_phase(d.g, dot3(uin, n)) : (0.25f / CUDART_PI_F);
            const double w = a.eps * (double)(prob * expf(-tau));
            if (st.sed) atomicAdd(st.sed + pobs * o.nsed + pk.sbin, w);
            else atomicAdd(t.sed + (int64_t)pobs * o.nsed + pk.sbin, w);
            if (o.nimg > 0) {
                const float px = porg.x * __ldg(o.ex + 3 * pobs) + porg.y * __ldg(o.ex + 3 * pobs + 1) + porg.z * __ldg(o.ex + 3 * pobs + 2);
                const float py = porg.x * __ldg(o.ey + 3 * pobs) + porg.y * __ldg(o.ey + 3 * pobs + 1) + porg.z * __ldg(o.ey + 3 * pobs + 2);
                const int ix = (int)floorf((px + o.img_half) * o.img_scale);
                const int iy = (int)floorf((py + o.img_half) * o.img_scale);
                if (ix >= 0 && ix < o.img_nx && iy >= 0 && iy < o.img_ny)
                    for (int l = 0; l < o.nimg; ++l)
                        if (__ldg(o.img_bin + l) == pk.sbin)
                            atomicAdd(t.img + (((int64_t)pobs * o.nimg + l) * o.img_ny + iy) * o.img_nx + ix, w);
            }
            if (++pobs < o.nobs) {
                start_peel(pobs);
            } else {
                pk.r = saved;
                tau = -logf(pk.rng.next());
                dep_rate = a.epsL0 * (double)pk.dust.kappa;
                ray_steps = 0;
                zero_run = 0;
                mode = M_WALK;
            }
        }
        // refill: lanes without a packet take the next ids from the global counter
        const unsigned need = __ballot_sync(FULL, mode == M_NEED);
        if (need) {
            if (!aborted && past_deadline(a, t)) aborted = true;
            unsigned long long base = 0;
            const int leader = __ffs(need) - 1;
            if ((int)lane == leader) base = atomicAdd(a.work_counter, (unsigned long long)__popc(need));
            base = __shfl_sync(FULL, base, leader);
            if (mode == M_NEED) {
                const unsigned long long q = base + __popc(need & lt_mask);
                if (aborted || q >= (unsigned long long)a.n_packets) {
                    if (aborted && q < (unsigned long long)a.n_packets) lc.v[C_WATCHDOG]++;
                    mode = M_DONE;
                } else {
                    if (!emit_packet<G>(g, d, s, o, a, t, st.sed, a.first_packet + (int64_t)q, pk, lc, false)) {
                        lc.v[C_ESCAPED]++;
                        lc.v[C_PACKETS_DONE]++;
                    } else {
                        porg = pk.last_origin;
                        after_event(PEEL_ISO, pk.emit_relocate);
                    }
                }
            }
        }
        unsigned live = __ballot_sync(FULL, mode != M_DONE);
        if (live == 0) break;
        // ------------------------------------------------------------ walk phase
        const int thr = min(a.regroup, __popc(live));
        unsigned steps = 0;
        for (;;) {
            const unsigned walkers = __ballot_sync(FULL, mode == M_WALK || mode == M_PEEL);
            if (walkers == 0 || (__popc(walkers) < thr && walkers != live)) break;
            bool flushing = false;
            int32_t fci = 0;
            double fval = 0.0;
            if (mode == M_WALK || mode == M_PEEL) {
                int axis, dir;
                const float l = cell_exit<G>(g, pk.r, axis, dir);
                const float rho = __ldg(g.rhoL + pk.r.ci);
                const float k = rho * pk.dust.chi;
                bool stop = false;
                if (mode == M_WALK) {
                    const float dtau = k * l;
                    float seg = l;
                    if (tau < dtau) {
                        seg = tau / k;
                        stop = true;
                    } else {
                        tau -= dtau;
                    }
                    if (rho > 0.f) {
                        const double v = dep_rate * (double)seg;
                        if (pk.r.ci == dep_ci) {
                            dep_val += v;
                        } else {
                            flushing = dep_ci >= 0;
                            fci = dep_ci;
                            fval = dep_val;
                            dep_ci = pk.r.ci;
                            dep_val = v;
                        }
                    }
                    if (stop) {
                        pk.r.p.x += seg * pk.r.u.x;
                        pk.r.p.y += seg * pk.r.u.y;
                        pk.r.p.z += seg * pk.r.u.z;
                        mode = M_INTERACT;
                    } else {
                        lc.v[C_CROSSINGS]++;
                    }
                } else {
                    tau += k * l;
                    lc.v[C_PEEL_CROSSINGS]++;
                }
                if (!stop) {
                    if (cell_step<G>(g, pk.r, l, axis, dir)) mode = (mode == M_WALK) ? M_ESCAPED : M_PEEL_DONE;
                    if constexpr (G == GRID_SPHERICAL) {
                        if (!tiny_step(pk.r, l)) zero_run = 0;
                        else if (++zero_run > ZERO_RUN_LIMIT) { nudge(pk.r); zero_run = 0; }
                    }
                    if (++ray_steps > MAX_WALK_STEPS && (mode == M_WALK || mode == M_PEEL)) {
                        lc.v[C_STUCK]++;
                        if (mode == M_WALK) {
                            lc.v[C_KILLED]++;
                            mode = M_KILLED;
                        } else {
                            tau = F_INF;           // the peel ray is dropped (zero weight)
                            mode = M_PEEL_DONE;
                        }
                    }
                } else {
                    ray_steps = 0;
                }
            }
            flush_deposit<WAGG>(t.acc, flushing, fci, fval);
            if (((++steps) & 4095u) == 0) watchdog(steps);
        }
        if (((++rounds) & 255u) == 0) watchdog(rounds);
    }
    if (dep_ci >= 0 && dep_val != 0.0) atomicAdd(t.acc + dep_ci, dep_val);
    flush_counters(lc, t.counters);
    flush_shared(o, a, t, st);
}

cudaError_t launch_propagate_event(const PropagateJob& job, const Launch& l, cudaStream_t s, int* launched) {
    if (job.args.n_packets <= 0) return cudaSuccess;
    Launch ll = l;
    ll.block = 256;
    PropagateJob j = job;
    j.args.regroup = l.regroup > 0 ? (l.regroup > 32 ? 32 : l.regroup) : 12;
    *launched += 1;
    const bool wagg = true;
    if (job.grid.type == GRID_CARTESIAN)
        return wagg ? launch_persistent(k_event<GRID_CARTESIAN, true>, j, ll, s)
                    : launch_persistent(k_event<GRID_CARTESIAN, false>, j, ll, s);
    return wagg ? launch_persistent(k_event<GRID_SPHERICAL, true>, j, ll, s)
                : launch_persistent(k_event<GRID_SPHERICAL, false>, j, ll, s);
}

}  // namespace hrt
