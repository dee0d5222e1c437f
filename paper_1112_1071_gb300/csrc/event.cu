// Event-based persistent propagation (Sect. 2.2, Eq. 2, Sect. 2.6.2).
//
// Every lane of a persistent warp runs a small state machine: it takes a packet, emits it,
// walks it to its next event (interaction or escape), handles the event (scatter, or absorb
// and re-emit), and takes the next packet when the history ends.
// A round has two phases:
//   * event phase: lanes with a finished walk handle their event (short, divergent code);
//   * walk phase: all walking lanes take cell crossings together while at least `regroup`
//     lanes are walking, so the walk -- where nearly all time goes -- runs in long converged
//     loops.
// In an imaging pass each event's peel-off rays are queued (one record per event) and walked
// afterwards by a separate pass, one ray per thread (peel.cu); only events past the queue's
// capacity are peeled by the lane itself, so the walk loop is the Lucy iterations' own.
// Lanes that need a packet draw consecutive packet ids with one atomic per warp.  Packet p
// always draws from its own Philox stream, so the histories do not depend on which lane or
// launch shape runs them.  Deposits are the FP32 products kappa * l (scaled length), merged
// in registers while the packet stays in one cell; at each step, lanes of a warp that flush
// into the same cell add one FP64 atomic.  The FP64 accumulators therefore hold sum kappa l,
// and the temperature update multiplies by eps L0 (Eq. 2) in FP64.
//
// The same loop serves the batched launch: warps pull (model, packet range) chunks of many
// models from one queue (largest models first) -- the device-side form of the paper's chunked
// packet scheduling (Sect. 3).
#include "propagate_common.cuh"

namespace hrt {

enum LaneMode : int32_t { M_NEED = 0, M_WALK = 1, M_INTERACT = 3, M_ESCAPED = 4, M_KILLED = 6, M_DONE = 7, M_MRW = 8 };


// The persistent lane state machine.  `fetch(need, lt_mask)` is called by the whole warp when
// `need` (ballot) lanes want a packet and returns this lane's packet id, or -1 when none is left.
template <int G, bool WAGG, bool PEEL, bool MRW, class Fetch>
__device__ __forceinline__ void event_loop(const DevGrid& g, const DevDust& d, const DevSources& s, const DevObs& o,
                                           const RunArgs& a, const Tallies& t, const SharedTallies& st,
                                           LocalCounters& lc, Fetch&& fetch) {
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;

    Packet pk;                 // the packet
    float3 porg = make_float3(0.f, 0.f, 0.f);   // origin of the peel rays (event position)
    float3 uin = make_float3(0.f, 0.f, 1.f);    // incoming direction at a scattering (HG peel)
    float tau = 0.f;           // optical depth left to the next interaction
    int32_t mode = M_NEED;
    int32_t dep_ci = -1;
    float dep_val = 0.f;       // kappa * l (scaled length) merged while the packet stays in one cell
    int zero_run = 0;
    unsigned ray_steps = 0;    // crossings of the packet since it started or last interacted
    bool aborted = false;
    // the walk's look-ahead: the density of the current cell, loaded one crossing ahead (when the
    // ray entered the cell), and (Cartesian) the next wall of every axis; `fresh` marks a ray that
    // starts (or starts again) and needs both loaded
    bool fresh = true;
    float rho_nx = 0.f;
    float3 wn = make_float3(0.f, 0.f, 0.f);
    const L2Hints l2 = make_l2_hints();

    auto start_walk = [&]() {
        if constexpr (MRW) {
            if (a.mrw_gamma > 0.f) {       // the event phase tries modified-random-walk steps first
                mode = M_MRW;
                return;
            }
        }
        tau = -logf(pk.rng.next());
        ray_steps = 0;
        zero_run = 0;
        fresh = true;
        mode = M_WALK;
    };
    // after an emission or interaction: peel off (if wanted), then draw a new optical depth.
    // raytraced: point-source emission or re-emission, which an a.rt pass raytraces instead.
    // Peel rays that need a walk go to the queue of the peel pass while it has room; emission
    // from a point source with precomputed columns, and events past the queue's capacity, are
    // peeled here, one ray per observer (the lane's packet waits meanwhile; no random number is
    // drawn, so the histories do not depend on which path peels)
    auto after_event = [&](int kind, int relocate, bool raytraced) {
        if constexpr (PEEL) {
            if (a.peel && pk.sbin >= 0 && o.nobs > 0 && !(raytraced && a.rt)) {
                const bool cols = relocate && s.col;
                unsigned long long slot = ~0ull;
                if (a.peel_q && !cols) slot = atomicAdd(a.peel_n, 1ull);
                if (slot < (unsigned long long)a.peel_cap) {
                    PeelEvent e;
                    e.px = porg.x; e.py = porg.y; e.pz = porg.z;
                    e.ci = relocate ? -1 : pk.r.ci;
                    e.ux = uin.x; e.uy = uin.y; e.uz = uin.z;
                    e.nu = kind == PEEL_HG ? -pk.nu : pk.nu;
                    a.peel_q[slot] = e;
                } else {
                    Ray at = pk.r;
                    at.p = porg;
                    peel_event<G>(g, d, o, a, t, st.sed, at, uin, kind, relocate != 0, pk.dust.chi, pk.sbin, lc,
                                  cols ? s.col + (int64_t)pk.src * o.nobs : nullptr, PEEL_TAU_STOP);
                }
            }
        }
        start_walk();
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
        lc.inc(C_WATCHDOG);
        const unsigned slot = atomicAdd(t.report_count, 1u);
        if (slot < (unsigned)WD_REPORTS) {
            float* r = t.report + slot * WD_FIELDS;
            r[0] = (float)mode; r[1] = (float)pk.rng.pkt; r[2] = (float)pk.nint; r[3] = tau;
            r[4] = pk.r.p.x; r[5] = pk.r.p.y; r[6] = pk.r.p.z;
            r[7] = pk.r.u.x; r[8] = pk.r.u.y; r[9] = pk.r.u.z;
            r[10] = (float)pk.r.i; r[11] = (float)pk.r.j; r[12] = (float)pk.r.k;
            r[13] = pk.nu; r[14] = 0.f; r[15] = (float)where;
        }
        flush_run<true>(t, dep_ci, dep_val, l2.keep);
        dep_ci = -1;
        mode = M_DONE;
    };
    auto end_packet = [&]() {
        flush_run<true>(t, dep_ci, dep_val, l2.keep);
        dep_ci = -1;
        dep_val = 0.f;
        lc.inc(C_PACKETS_DONE);
        mode = M_NEED;
    };

    // modified random walk (Sect. 2.2) at the start of a flight: one step per event phase while the
    // packet sits deep in a thick cell (each one interaction against the cap and an isotropic
    // re-emission at its end, peeled off like one; the lane stays in M_MRW for the next phase, so a
    // long chain never holds up its warp), else a new optical depth and the walk
    auto mrw_steps = [&]() {
        const float R0 = mrw_sphere<G>(g, a, pk.r);
        if (R0 < 0.f) {
            tau = -logf(pk.rng.next());
            ray_steps = 0;
            zero_run = 0;
            fresh = true;
            mode = M_WALK;
            return;
        }
        if (++pk.nint > a.max_interactions) {
            lc.inc(C_KILLED);
            end_packet();
            return;
        }
        lc.inc(C_MRW);
        const float v = mrw_take(d, o, a, pk, R0);
        if (pk.r.ci == dep_ci) {
            dep_val += v;
        } else {
            flush_run<true>(t, dep_ci, dep_val, l2.keep);
            dep_ci = pk.r.ci;
            dep_val = v;
        }
        porg = pk.r.p;
        if constexpr (PEEL) {
            if (a.peel && pk.sbin >= 0 && o.nobs > 0 && !a.rt) after_event(PEEL_ISO, 0, true);
        }
    };

    for (;;) {
        // ------------------------------------------------------------ event phase
        if (mode == M_KILLED) {
            end_packet();
        } else if (mode == M_ESCAPED) {
            lc.inc(C_ESCAPED);
            tally_escape(o, t, pk, st.esc);
            end_packet();
        } else if (mode == M_INTERACT) {
            if (++pk.nint > a.max_interactions) {
                lc.inc(C_KILLED);
                end_packet();
            } else {
                lc.inc(C_INTERACTIONS);
                const float z = pk.rng.next();
                if (z > pk.dust.albedo) {
                    lc.inc(C_ABSORB);
                    if (a.terminate_on_absorb) {
                        lc.inc(C_ABSORBED_TERM);
                        end_packet();
                    } else {
                        const float u1 = pk.rng.next(), u2 = pk.rng.next();
                        set_dir(pk.r, isotropic_dir(u1, u2));
                        const int row = min(max(__ldg(d.emit_row + pk.r.ci), 0), d.nT - 1);   // bounds check
                        set_frequency(pk, d, o, sample_table(d.nu, d.cdf_emit + (int64_t)row * d.nnu, d.nnu, pk.rng.next()));
                        porg = pk.r.p;
                        after_event(PEEL_ISO, 0, true);
                    }
                } else {
                    lc.inc(C_SCATTER);
                    const float mu = hg_mu(d.g, pk.rng.next());
                    const float u2 = pk.rng.next();
                    uin = pk.r.u;
                    set_dir(pk.r, scatter_dir(uin, mu, u2));
                    porg = pk.r.p;
                    after_event(PEEL_HG, 0, false);
                }
            }
        }
        if (MRW && mode == M_MRW) mrw_steps();
        // refill: lanes without a packet take the next ids
        const unsigned need = __ballot_sync(FULL, mode == M_NEED);
        if (need) {
            if (!aborted && past_deadline(a, t)) aborted = true;
            const long long q = fetch(need, lt_mask);
            if (mode == M_NEED) {
                if (aborted || q < 0) {
                    if (aborted && q >= 0) lc.inc(C_WATCHDOG);
                    mode = M_DONE;
                } else if (!emit_packet<G>(g, d, s, o, a, t, st.sed, (int64_t)q, pk, lc, false)) {
                    lc.inc(C_ESCAPED);
                    lc.inc(C_PACKETS_DONE);
                } else if (pk.src >= s.npoint && pk.src < s.npoint + s.next) {
                    start_walk();               // external field: background, not peeled off
                } else {
                    porg = pk.last_origin;
                    after_event(PEEL_ISO, pk.emit_relocate, pk.src < s.npoint);
                }
                if (MRW && mode == M_MRW) mrw_steps();
            }
        }
        const unsigned live = __ballot_sync(FULL, mode != M_DONE);
        if (live == 0) break;
        // ------------------------------------------------------------ walk phase
        const int thr = min(a.regroup, __popc(live));
        unsigned steps = 0;
        for (;;) {
            const unsigned walkers = __ballot_sync(FULL, mode == M_WALK);
            if (walkers == 0 || (__popc(walkers) < thr && walkers != live)) break;
            bool flushing = false;
            int32_t fci = 0;
            float fval = 0.f;
            if (mode == M_WALK) {
                int axis, dir = 0;
                float l;
                if constexpr (G == GRID_CARTESIAN) {
                    if (fresh) wn = cart_next_walls(g, pk.r);
                    l = cart_exit_w(pk.r, wn, axis);
                } else {
                    l = cell_exit<G>(g, pk.r, axis, dir);
                }
                const float rho = fresh ? ld_hint(g.rhoL + pk.r.ci, l2.stream) : rho_nx;
                fresh = false;
                const float k = rho * pk.dust.chi;
                const float dtau = k * l;
                float seg = l;
                bool stop = false;
                if (tau < dtau) {
                    seg = tau / k;
                    stop = true;
                } else {
                    tau -= dtau;
                }
                if (rho > 0.f) {
                    const float v = pk.dust.kappa * seg;
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
                    lc.inc(C_CROSSINGS);
                }
                if (!stop) {
                    bool out;
                    if constexpr (G == GRID_CARTESIAN) out = cart_step_w(g, pk.r, wn, l, axis);
                    else out = cell_step<G>(g, pk.r, l, axis, dir);
                    if (out) mode = M_ESCAPED;
                    else rho_nx = ld_hint(g.rhoL + pk.r.ci, l2.stream);      // the next crossing's density, ahead of use
                    if constexpr (G != GRID_CARTESIAN) {
                        if (!tiny_step(pk.r, l)) zero_run = 0;
                        else if (++zero_run > ZERO_RUN_LIMIT) { nudge(pk.r); zero_run = 0; }
                    }
                    if (++ray_steps > MAX_WALK_STEPS && mode == M_WALK) {
                        lc.inc(C_STUCK);
                        lc.inc(C_KILLED);
                        mode = M_KILLED;
                    }
                } else {
                    ray_steps = 0;
                }
            }
            flush_deposit<WAGG, true>(t.acc, t.visits, flushing, fci, fval, l2.keep);
            if (((++steps) & 4095u) == 0) watchdog(steps);
        }
        if (((++rounds) & 255u) == 0) watchdog(rounds);
    }
    flush_run<true>(t, dep_ci, dep_val, l2.keep);
}

// ---------------------------------------------------------------- one model
// MINB = resident blocks per SM the registers are budgeted for (2: 128 registers, 3: 80, 4: 64);
// PEEL = imaging pass (peel-off events queued, or peeled in place), compiled out of the Lucy
// iterations' kernel.
template <int G, bool WAGG, int MINB, bool PEEL, bool MRW>
__global__ void __launch_bounds__(256, MINB) k_event(DevGrid g, DevDust d, DevSources s, DevObs o, RunArgs a, Tallies t) {
    const SharedTallies st = shared_tallies(o, a);
    __shared__ unsigned long long cnt_sh[8][N_COUNTERS];
    LocalCounters lc;
    lc.init(cnt_sh[threadIdx.x >> 5], MRW ? CNT_REG : CNT_GROUPED);
    const unsigned lane = threadIdx.x & 31u;
    auto fetch = [&](unsigned need, unsigned lt_mask) -> long long {
        unsigned long long base = 0;
        const int leader = __ffs(need) - 1;
        if ((int)lane == leader) base = atomicAdd(a.work_counter, (unsigned long long)__popc(need));
        base = __shfl_sync(0xffffffffu, base, leader);
        const unsigned long long q = base + __popc(need & lt_mask);
        return q < (unsigned long long)a.n_packets ? (long long)(a.first_packet + (int64_t)q) : -1ll;
    };
    event_loop<G, WAGG, PEEL, MRW>(g, d, s, o, a, t, st, lc, fetch);
    flush_counters(lc, t.counters);
    flush_shared(o, a, t, st);
}

// MRW = modified random walk compiled in (runs with mrw_gamma > 0; 3 blocks per SM only)
// WAGG (deposits of a warp's lanes grouped by cell before the atomic) on Cartesian grids only:
// measured on GB300, it saves 10 % of a Lucy iteration on the 256^3 cloud (large accumulator
// array beyond L2, fewer reductions) and costs 13 % on the disk (accumulators in L2, where the
// grouping's match.any per crossing outweighs the atomics it saves).
template <int G, bool PEEL>
static cudaError_t launch_event_shape(const PropagateJob& j, const Launch& l, int bps, cudaStream_t s) {
    constexpr bool WAGG = G == GRID_CARTESIAN;
    if (j.args.mrw_gamma > 0.f) return launch_persistent(k_event<G, WAGG, 3, PEEL, true>, j, l, s);
    if constexpr (!PEEL) {
        if (bps >= 4) return launch_persistent(k_event<G, WAGG, 4, PEEL, false>, j, l, s);
    }
    if (bps >= 3) return launch_persistent(k_event<G, WAGG, 3, PEEL, false>, j, l, s);
    return launch_persistent(k_event<G, WAGG, 2, PEEL, false>, j, l, s);
}

cudaError_t launch_propagate_event(const PropagateJob& job, const Launch& l, cudaStream_t s, int* launched) {
    if (job.args.n_packets <= 0) return cudaSuccess;
    Launch ll = l;
    ll.block = 256;
    PropagateJob j = job;
    const bool peel = job.args.peel != 0;
    // default shapes (measured on GB300): Lucy iterations at 4 blocks of 256 per SM (64
    // registers; with the L2 hints 5 % faster than 3 on the 256^3 cloud, 7 % on the disk despite
    // some spilling there, 20 % on the cylindrical ISRF cloud, within 1 % on the cylindrical
    // disk); imaging passes at 3 (80 registers: 6-8 % faster than 2 on the disk and the cloud).
    // Warps stay in the walk phase while at least 20 lanes walk (Lucy on curvilinear grids; 19
    // on Cartesian runs of >= 4M packets: 1 % faster than 20 on the cloud), 16 (imaging: 7 %
    // faster than 20 on the cloud), 12 for Cartesian Lucy runs of < 4M packets, whose tail
    // dominates
    int rg_default = DEFAULT_REGROUP;
    if (peel) rg_default = 16;
    else if (job.grid.type != GRID_CARTESIAN) rg_default = 20;
    else if (job.args.n_packets >= (int64_t)1 << 22) rg_default = 19;
    j.args.regroup = l.regroup > 0 ? (l.regroup > 32 ? 32 : l.regroup) : rg_default;
    *launched += 1;
    const int bps = l.blocks_per_sm > 0 ? l.blocks_per_sm : (peel ? 3 : 4);
    cudaError_t e;
    if (job.grid.type == GRID_CARTESIAN)
        e = peel ? launch_event_shape<GRID_CARTESIAN, true>(j, ll, bps, s)
                 : launch_event_shape<GRID_CARTESIAN, false>(j, ll, bps, s);
    else if (job.grid.type == GRID_CYLINDRICAL)
        e = peel ? launch_event_shape<GRID_CYLINDRICAL, true>(j, ll, bps, s)
                 : launch_event_shape<GRID_CYLINDRICAL, false>(j, ll, bps, s);
    else
        e = peel ? launch_event_shape<GRID_SPHERICAL, true>(j, ll, bps, s)
                 : launch_event_shape<GRID_SPHERICAL, false>(j, ll, bps, s);
    return e;
}

// ---------------------------------------------------------------- many models, one launch
template <int G, bool WAGG, int MINB>
__global__ void __launch_bounds__(256, MINB) k_event_batch(const BatchModel* __restrict__ models,
                                                        const BatchChunk* __restrict__ chunks, int nchunks,
                                                        unsigned* chunk_counter, const BatchState* __restrict__ state,
                                                        int regroup) {
    const unsigned lane = threadIdx.x & 31u;
    const SharedTallies st{nullptr, nullptr};
    __shared__ unsigned long long cnt_sh[8][N_COUNTERS];
    for (;;) {
        int c = 0;
        if (lane == 0) c = (int)atomicAdd(chunk_counter, 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= nchunks) break;
        const BatchChunk ch = chunks[c];
        if (!state[ch.model].active || models[ch.model].g.type != G) continue;
        const BatchModel& M = models[ch.model];
        RunArgs a = M.a;
        a.iter_key = state[ch.model].iteration;
        a.regroup = regroup;
        long long cursor = ch.p0;
        const long long end = ch.p1;
        auto fetch = [&](unsigned need, unsigned lt_mask) -> long long {
            const long long q = cursor + __popc(need & lt_mask);
            cursor += __popc(need);
            return q < end ? q : -1ll;
        };
        LocalCounters lc;
        lc.init(cnt_sh[threadIdx.x >> 5]);
        event_loop<G, WAGG, false, false>(M.g, M.d, M.s, M.o, a, M.t, st, lc, fetch);
        flush_counters(lc, M.t.counters);
    }
}

// deposit aggregation as for one model: on Cartesian grids only
template <int G, int MINB>
static void launch_batch_shape(const BatchModel* models, const BatchChunk* chunks, int nchunks, unsigned* chunk_counter,
                               const BatchState* state, int want_per_sm, int regroup, int sms, cudaStream_t s) {
    constexpr bool WAGG = G == GRID_CARTESIAN;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_event_batch<G, WAGG, MINB>, 256, 0);
    if (want_per_sm > 0 && want_per_sm < per_sm) per_sm = want_per_sm;
    k_event_batch<G, WAGG, MINB><<<sms * (per_sm > 0 ? per_sm : 1), 256, 0, s>>>(models, chunks, nchunks, chunk_counter,
                                                                                 state, regroup);
}

// Default shape as for one model's Lucy iteration: 4 blocks of 256 per SM, regroup 20; the
// autotuner times others (2-4 blocks).
cudaError_t launch_propagate_batch(int gtype, const BatchModel* models, const BatchChunk* chunks, int nchunks,
                                   unsigned* chunk_counter, const BatchState* state, const Launch& l, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int regroup = l.regroup > 0 ? (l.regroup > 32 ? 32 : l.regroup) : 20;
    const int bps = l.blocks_per_sm > 0 ? l.blocks_per_sm : 4;
    if (gtype == GRID_CARTESIAN) {
        if (bps >= 4) launch_batch_shape<GRID_CARTESIAN, 4>(models, chunks, nchunks, chunk_counter, state, bps, regroup, sms, s);
        else if (bps == 3) launch_batch_shape<GRID_CARTESIAN, 3>(models, chunks, nchunks, chunk_counter, state, bps, regroup, sms, s);
        else launch_batch_shape<GRID_CARTESIAN, 2>(models, chunks, nchunks, chunk_counter, state, bps, regroup, sms, s);
    } else {
        if (bps >= 4) launch_batch_shape<GRID_SPHERICAL, 4>(models, chunks, nchunks, chunk_counter, state, bps, regroup, sms, s);
        else if (bps == 3) launch_batch_shape<GRID_SPHERICAL, 3>(models, chunks, nchunks, chunk_counter, state, bps, regroup, sms, s);
        else launch_batch_shape<GRID_SPHERICAL, 2>(models, chunks, nchunks, chunk_counter, state, bps, regroup, sms, s);
    }
    return cudaGetLastError();
}

}  // namespace hrt
