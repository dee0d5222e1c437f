// Event-based propagation with the live packets regrouped by state across the warps of a block
// (Sect. 2.2, Eq. 2, Sect. 2.6.2; the device-side form of the chunked scheduling of Sect. 3).
//
// A block of 256 threads runs seven walker warps and one service warp.
//  * Walker lanes only walk: each walks one packet, held in registers, to its next event.  The
//    stopped packet goes into one of the lane's two shared-memory slots, tagged with its state --
//    SCATTER, ABSORB (absorb and re-emit) or NEED (its history ended by escape, the interaction
//    cap or terminate-on-absorb: a new packet is wanted) -- and the lane takes the packet waiting in
//    its other slot.  A walker warp stays in its walk phase while at least `regroup` lanes walk,
//    then hands over and takes up all its stopped lanes at once.
//  * The service warp moves the handed-over slots from the walker warps' queues into one list
//    per state and runs one state at a time in batches of up to 32 slots, so that its lanes
//    execute the same event code together: Henyey-Greenstein scattering, absorption with isotropic
//    re-emission at a frequency from the cell's emissivity row, emission of new packets (one
//    atomic per batch for their ids), the peel-off of each event and the next optical depth.  A
//    list runs as soon as it holds 32 slots, or, when nothing new has arrived for a while, the
//    largest list runs as it is.
// Packet p draws from its own Philox stream in the order of the warp-local kernel (event.cu):
// the interaction's first uniform (absorb or scatter) is drawn by the walker lane, the rest by
// the service lane, so every history equals k_event's.  Every wait is bounded in time: past the
// watchdog budget, or after RG_STALL_NS without progress, the block stops and the call returns
// HRT_ETIMEDOUT.  Modified-random-walk runs use k_event.
//
// Measured on GB300 against the warp-local kernel (same histories): 910 against 315 ms for a
// 1e8-packet Lucy iteration of the 256^3 cloud, 107 against 59 ms for 1e7 packets on the disk,
// insensitive to the batch and hand-over thresholds.  The parked packets take 58 KB of shared
// memory per block, which at 2-3 blocks per SM leaves the walk a third of the L1 capacity it has
// otherwise, while events are rare (one per ~60 cell crossings on these workloads) so that even
// free event handling would save at most a tenth of the instructions.  The library therefore
// runs the warp-local kernel by default (HRT_KERNEL_EVENT) and this one on request.
#include "propagate_common.cuh"

namespace hrt {
namespace {

constexpr int RG_WALKERS = 7;                   // walker warps per block; warp 7 serves
constexpr int RG_LANES = RG_WALKERS * 32;       // 224 walker lanes
constexpr int RG_SLOTS = 2 * RG_LANES;          // two slots per walker lane: lane l owns l and l + 224
constexpr int RG_RING = 64;                     // a walker warp's queue: its 64 slots fit
constexpr int RG_LIST = 512;                    // a service list: every slot fits
constexpr uint64_t RG_STALL_NS = 30ull * 1000000000ull;
constexpr int RG_QUIET_POLLS = 4;               // polls without arrivals before a partial batch
constexpr int RG_BATCH_MIN = 32;                // a list this long runs at once
constexpr int RG_SWAP_MIN = 1;                  // below the threshold, stopped lanes that end a walk phase

enum RgCode : int32_t { RG_SCATTER = 0, RG_ABSORB = 1, RG_NEED = 2 };
enum RgFlag : int32_t { RG_FREE = 0, RG_PENDING = 1, RG_READY = 2, RG_DONE = 3 };
enum RgLane : int32_t { L_WALK = 0, L_INTERACT, L_ESCAPED, L_KILLED, L_IDLE, L_DONE };

// A packet between two walks; 29 words, odd, so that lanes reading consecutive slots hit
// distinct shared-memory banks.
struct RgSlot {
    float px, py, pz, ux, uy, uz, vx, vy, vz;   // position, direction, 1 / direction
    int32_t i, j, k, ci;
    float nu, chi, kappa, albedo;
    int32_t sbin, nint;
    uint32_t pkt, rn, b0, b1, b2, b3;           // Philox stream: packet id, draws made, cached block
    float tau, dep_val;
    int32_t dep_ci, pad;
};

struct RgShared {
    RgSlot slot[RG_SLOTS];
    int32_t flag[RG_SLOTS];
    int32_t ring[RG_WALKERS][RG_RING];          // (slot << 2) | code
    int32_t tail[RG_WALKERS];                   // entries published by each walker warp
    uint16_t list[3][RG_LIST];                  // the service's slots per state
    int32_t exited;                             // walker warps that have finished
    int32_t abort;                              // the block stops (watchdog, stall)
};

constexpr size_t RG_TALLY_OFFSET = (sizeof(RgShared) + 15) & ~(size_t)15;

__device__ __forceinline__ void pack(RgSlot& s, const Packet& pk, float tau, int32_t dep_ci, float dep_val) {
    s.px = pk.r.p.x; s.py = pk.r.p.y; s.pz = pk.r.p.z;
    s.ux = pk.r.u.x; s.uy = pk.r.u.y; s.uz = pk.r.u.z;
    s.vx = pk.r.inv.x; s.vy = pk.r.inv.y; s.vz = pk.r.inv.z;
    s.i = pk.r.i; s.j = pk.r.j; s.k = pk.r.k; s.ci = pk.r.ci;
    s.nu = pk.nu; s.chi = pk.dust.chi; s.kappa = pk.dust.kappa; s.albedo = pk.dust.albedo;
    s.sbin = pk.sbin;
    s.nint = (int32_t)pk.nint;
    s.pkt = pk.rng.pkt; s.rn = pk.rng.n;
    s.b0 = pk.rng.buf.x; s.b1 = pk.rng.buf.y; s.b2 = pk.rng.buf.z; s.b3 = pk.rng.buf.w;
    s.tau = tau; s.dep_val = dep_val; s.dep_ci = dep_ci;
}

__device__ __forceinline__ void unpack(const RgSlot& s, const RunArgs& a, Packet& pk, float& tau, int32_t& dep_ci,
                                       float& dep_val) {
    pk.r.p = make_float3(s.px, s.py, s.pz);
    pk.r.u = make_float3(s.ux, s.uy, s.uz);
    pk.r.inv = make_float3(s.vx, s.vy, s.vz);
    pk.r.i = s.i; pk.r.j = s.j; pk.r.k = s.k; pk.r.ci = s.ci;
    pk.nu = s.nu; pk.dust.chi = s.chi; pk.dust.kappa = s.kappa; pk.dust.albedo = s.albedo;
    pk.sbin = s.sbin;
    pk.nint = s.nint;
    pk.rng.key = make_uint2(a.key0, a.key1);
    pk.rng.pkt = s.pkt; pk.rng.iter = a.iter_key; pk.rng.model = a.model_key; pk.rng.n = s.rn;
    pk.rng.buf = make_uint4(s.b0, s.b1, s.b2, s.b3);
    tau = s.tau; dep_val = s.dep_val; dep_ci = s.dep_ci;
}

__device__ __forceinline__ int32_t vload(const int32_t* p) { return *(const volatile int32_t*)p; }
__device__ __forceinline__ void vstore(int32_t* p, int32_t v) { *(volatile int32_t*)p = v; }

// ---------------------------------------------------------------- walker warps
template <int G, bool WAGG>
__device__ void rg_walker(const DevGrid& g, const DevDust& d, const DevObs& o, const RunArgs& a, const Tallies& t,
                          const SharedTallies& st, RgShared& sh, int w, LocalCounters& lc) {
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int sl[2] = {w * 32 + (int)lane, w * 32 + (int)lane + RG_LANES};

    Packet pk;
    float tau = 0.f;
    int32_t dep_ci = -1;
    float dep_val = 0.f;
    int32_t mode = L_IDLE;
    int32_t code = RG_NEED;
    int cur = 0;               // the slot to take next
    int inflight = 2;          // this lane's slots with the service
    int zero_run = 0;
    unsigned ray_steps = 0;
    bool fresh = true;         // walls and density of a ray that (re)starts need loading
    float rho_nx = 0.f;
    float3 wn = make_float3(0.f, 0.f, 0.f);

    // both slots ask for packets
    sh.flag[sl[0]] = RG_PENDING;
    sh.flag[sl[1]] = RG_PENDING;
    sh.ring[w][2 * lane] = (sl[0] << 2) | RG_NEED;
    sh.ring[w][2 * lane + 1] = (sl[1] << 2) | RG_NEED;
    __syncwarp();
    __threadfence_block();
    if (lane == 0) vstore(&sh.tail[w], 64);
    int tail = 64;

    const int thr = a.regroup;
    unsigned steps = 0, polls = 0;
    uint64_t idle_since = 0;
    for (;;) {
        // ------------------------------------------------------------ walk phase
        // below the threshold (of the lanes still live), leave as soon as a lane has stopped, or
        // every 16 steps to look for packets the service has made ready
        const int thr_eff = min(thr, __popc(__ballot_sync(FULL, mode != L_DONE)));
        unsigned below = 0;
        for (;;) {
            const unsigned walkers = __ballot_sync(FULL, mode == L_WALK);
            if (walkers == 0) break;
            if (__popc(walkers) < thr_eff) {
                const unsigned stopped = __ballot_sync(FULL, mode == L_INTERACT || mode == L_ESCAPED || mode == L_KILLED);
                if (__popc(stopped) >= RG_SWAP_MIN || ++below >= 16) break;
            }
            bool flushing = false;
            int32_t fci = 0;
            float fval = 0.f;
            if (mode == L_WALK) {
                int axis, dir = 0;
                float l;
                if constexpr (G == GRID_CARTESIAN) {
                    if (fresh) wn = cart_next_walls(g, pk.r);
                    l = cart_exit_w(pk.r, wn, axis);
                } else {
                    l = cell_exit<G>(g, pk.r, axis, dir);
                }
                const float rho = fresh ? __ldg(g.rhoL + pk.r.ci) : rho_nx;
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
                    mode = L_INTERACT;
                } else {
                    lc.inc(C_CROSSINGS);
                    bool out;
                    if constexpr (G == GRID_CARTESIAN) out = cart_step_w(g, pk.r, wn, l, axis);
                    else out = cell_step<G>(g, pk.r, l, axis, dir);
                    if (out) mode = L_ESCAPED;
                    else rho_nx = __ldg(g.rhoL + pk.r.ci);      // the next crossing's density, ahead of use
                    if constexpr (G != GRID_CARTESIAN) {
                        if (!tiny_step(pk.r, l)) zero_run = 0;
                        else if (++zero_run > ZERO_RUN_LIMIT) { nudge(pk.r); zero_run = 0; }
                    }
                    if (++ray_steps > MAX_WALK_STEPS && mode == L_WALK) {
                        lc.inc(C_STUCK);
                        lc.inc(C_KILLED);
                        mode = L_KILLED;
                    }
                }
            }
            flush_deposit<WAGG>(t.acc, t.visits, flushing, fci, fval);
            if (((++steps) & 4095u) == 0) {
                bool ab = false;
                if (lane == 0) ab = vload(&sh.abort) != 0 || past_deadline(a, t);
                if (__shfl_sync(FULL, ab ? 1 : 0, 0)) {
                    if (lane == 0) {
                        vstore(&sh.abort, 1);
                        lc.inc(C_WATCHDOG);
                    }
                    break;
                }
            }
        }
        if (__shfl_sync(FULL, lane == 0 ? vload(&sh.abort) : 0, 0)) break;

        // ------------------------------------------------------------ hand over stopped packets
        if (mode == L_INTERACT) {
            ray_steps = 0;
            if (++pk.nint > a.max_interactions) {
                lc.inc(C_KILLED);
                flush_run(t, dep_ci, dep_val);
                lc.inc(C_PACKETS_DONE);
                code = RG_NEED;
            } else {
                lc.inc(C_INTERACTIONS);
                const float z = pk.rng.next();
                if (z > pk.dust.albedo) {
                    lc.inc(C_ABSORB);
                    code = RG_ABSORB;
                } else {
                    lc.inc(C_SCATTER);
                    code = RG_SCATTER;
                }
            }
        } else if (mode == L_ESCAPED) {
            lc.inc(C_ESCAPED);
            tally_escape(o, t, pk, st.esc);
            flush_run(t, dep_ci, dep_val);
            lc.inc(C_PACKETS_DONE);
            code = RG_NEED;
        } else if (mode == L_KILLED) {
            flush_run(t, dep_ci, dep_val);
            lc.inc(C_PACKETS_DONE);
            code = RG_NEED;
        }
        const bool push = mode == L_INTERACT || mode == L_ESCAPED || mode == L_KILLED;
        const unsigned pm = __ballot_sync(FULL, push);
        if (pm) {
            if (push) {
                // the free slot: the one not queued to be taken next
                const int fs = sl[inflight == 0 ? cur : (cur ^ 1)];
                if (code != RG_NEED) pack(sh.slot[fs], pk, tau, dep_ci, dep_val);
                sh.flag[fs] = RG_PENDING;
                sh.ring[w][(tail + __popc(pm & lt_mask)) & (RG_RING - 1)] = (fs << 2) | code;
                ++inflight;
                dep_ci = -1;
                dep_val = 0.f;
                mode = L_IDLE;
            }
            __syncwarp();
            __threadfence_block();
            tail += __popc(pm);
            if (lane == 0) vstore(&sh.tail[w], tail);
        }
        // ------------------------------------------------------------ take up waiting packets
        bool took = false;
        if (mode == L_IDLE) {
            if (inflight > 0) {
                const int s = sl[cur];
                const int32_t f = vload(&sh.flag[s]);
                if (f == RG_READY) {
                    __threadfence_block();
                    unpack(sh.slot[s], a, pk, tau, dep_ci, dep_val);
                    sh.flag[s] = RG_FREE;
                    --inflight;
                    cur ^= 1;
                    mode = L_WALK;
                    fresh = true;
                    zero_run = 0;
                    ray_steps = 0;
                    took = true;
                } else if (f == RG_DONE) {
                    sh.flag[s] = RG_FREE;
                    --inflight;
                    cur ^= 1;
                    took = true;
                    if (inflight == 0) mode = L_DONE;
                }
            } else {
                mode = L_DONE;
            }
        }
        if (__ballot_sync(FULL, mode != L_DONE) == 0) break;
        // nothing walks and nothing was ready: wait a little for the service (bounded in time)
        if (__ballot_sync(FULL, mode == L_WALK || took) == 0) {
            if (idle_since == 0) idle_since = global_ns();
            __nanosleep(200);
            if (((++polls) & 63u) == 0) {
                bool ab = false;
                if (lane == 0)
                    ab = vload(&sh.abort) != 0 || past_deadline(a, t) || global_ns() - idle_since > RG_STALL_NS;
                if (__shfl_sync(FULL, ab ? 1 : 0, 0)) {
                    if (lane == 0) {
                        vstore(&sh.abort, 1);
                        lc.inc(C_WATCHDOG);
                    }
                    break;
                }
            }
        } else {
            idle_since = 0;
        }
    }
    // stopped by the watchdog or a stall: lanes that still hold a packet record it and stop
    const bool aborted = __shfl_sync(FULL, lane == 0 ? vload(&sh.abort) : 0, 0) != 0;
    if (aborted && mode != L_DONE && mode != L_IDLE) {
        lc.inc(C_WATCHDOG);
        const unsigned slot = atomicAdd(t.report_count, 1u);
        if (slot < (unsigned)WD_REPORTS) {
            float* r = t.report + slot * WD_FIELDS;
            r[0] = 1.f; r[1] = (float)pk.rng.pkt; r[2] = (float)pk.nint; r[3] = tau;
            r[4] = pk.r.p.x; r[5] = pk.r.p.y; r[6] = pk.r.p.z;
            r[7] = pk.r.u.x; r[8] = pk.r.u.y; r[9] = pk.r.u.z;
            r[10] = (float)pk.r.i; r[11] = (float)pk.r.j; r[12] = (float)pk.r.k;
            r[13] = pk.nu; r[14] = 0.f; r[15] = (float)steps;
        }
        flush_run(t, dep_ci, dep_val);
    }
    if (aborted && lane == 0) atomicExch(t.abort_flag, 1);
    __syncwarp();
    if (lane == 0) atomicAdd(&sh.exited, 1);
}

// ---------------------------------------------------------------- the service warp
template <int G, bool PEEL>
__device__ void rg_service(const DevGrid& g, const DevDust& d, const DevSources& s, const DevObs& o,
                           const RunArgs& a, const Tallies& t, const SharedTallies& st, RgShared& sh,
                           LocalCounters& lc) {
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;
    int head[RG_WALKERS];
#pragma unroll
    for (int w = 0; w < RG_WALKERS; ++w) head[w] = 0;
    int lh[3] = {0, 0, 0}, lt[3] = {0, 0, 0};
    int quiet = 0;
    unsigned polls = 0;
    uint64_t last = global_ns();

    // append this lane's slot (if any) to list c: one ballot per list
    auto append = [&](bool has, int code, int slot) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const unsigned m = __ballot_sync(FULL, has && code == c);
            if (has && code == c) sh.list[c][(lt[c] + __popc(m & lt_mask)) & (RG_LIST - 1)] = (uint16_t)slot;
            lt[c] += __popc(m);
        }
    };
    // peel-off of an event (Sect. 2.6.2): point-source emission from its precomputed columns,
    // other events queued for the peel pass (or walked here when the queue is full)
    auto peel = [&](const Packet& pk, float3 porg, float3 uin, int kind, int relocate, bool raytraced) {
        if constexpr (PEEL) {
            if (a.peel && pk.sbin >= 0 && o.nobs > 0 && !(raytraced && a.rt)) {
                Ray at = pk.r;
                at.p = porg;
                if (relocate && s.col) {
                    peel_event<G>(g, d, o, a, t, st.sed, at, uin, kind, true, pk.dust.chi, pk.sbin, lc,
                                  s.col + (int64_t)pk.src * o.nobs);
                    return;
                }
                if (a.peel_q) {
                    const unsigned long long q = atomicAdd(a.peel_n, 1ull);
                    if (q < (unsigned long long)a.peel_cap) {
                        PeelEvent e;
                        e.px = porg.x; e.py = porg.y; e.pz = porg.z;
                        e.ci = relocate ? -1 : pk.r.ci;
                        e.ux = uin.x; e.uy = uin.y; e.uz = uin.z;
                        e.nu = kind == PEEL_HG ? -pk.nu : pk.nu;
                        a.peel_q[q] = e;
                        return;
                    }
                }
                peel_event<G>(g, d, o, a, t, st.sed, at, uin, kind, relocate != 0, pk.dust.chi, pk.sbin, lc, nullptr,
                              PEEL_TAU_STOP);
            }
        }
    };

    for (;;) {
        // ------------------------------------------------------------ gather handed-over slots
        int arrived = 0;
#pragma unroll
        for (int w = 0; w < RG_WALKERS; ++w) {
            int tl = 0;
            if (lane == 0) tl = vload(&sh.tail[w]);
            tl = __shfl_sync(FULL, tl, 0);
            const int n = tl - head[w];
            if (n > 0) {
                __threadfence_block();
                for (int k0 = 0; k0 < n; k0 += 32) {
                    const bool has = k0 + (int)lane < n;
                    const int e = has ? sh.ring[w][(head[w] + k0 + (int)lane) & (RG_RING - 1)] : 0;
                    append(has, e & 3, e >> 2);
                }
                head[w] = tl;
                arrived += n;
            }
        }
        __syncwarp();                           // list entries written by one lane, read by another
        int best = 0, bn = lt[0] - lh[0];
        if (lt[1] - lh[1] > bn) best = 1, bn = lt[1] - lh[1];
        if (lt[2] - lh[2] > bn) best = 2, bn = lt[2] - lh[2];
        quiet = arrived ? 0 : quiet + 1;
        if (bn >= RG_BATCH_MIN || (bn > 0 && quiet >= RG_QUIET_POLLS)) {
            // ------------------------------------------------------------ one batch of one state
            last = global_ns();
            const int nb = bn < 32 ? bn : 32;
            const bool act = (int)lane < nb;
            const int slot = act ? (int)sh.list[best][(lh[best] + (int)lane) & (RG_LIST - 1)] : 0;
            lh[best] += nb;
            Packet pk;
            float tau = 0.f, dep_val = 0.f;
            int32_t dep_ci = -1;
            bool again = false;                 // the slot wants a new packet (another NEED round)
            int32_t result = RG_READY;
            if (best == RG_NEED) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(a.work_counter, (unsigned long long)nb);
                base = __shfl_sync(FULL, base, 0);
                if (act) {
                    const unsigned long long q = base + lane;
                    if (q >= (unsigned long long)a.n_packets) {
                        result = RG_DONE;
                    } else if (!emit_packet<G>(g, d, s, o, a, t, st.sed, a.first_packet + (int64_t)q, pk, lc, false)) {
                        lc.inc(C_ESCAPED);                   // starts outside the grid
                        lc.inc(C_PACKETS_DONE);
                        again = true;
                    } else {
                        if (!(pk.src >= s.npoint && pk.src < s.npoint + s.next))    // external field: not peeled
                            peel(pk, pk.last_origin, pk.r.u, PEEL_ISO, pk.emit_relocate, pk.src < s.npoint);
                        tau = -logf(pk.rng.next());
                    }
                }
            } else if (act) {
                unpack(sh.slot[slot], a, pk, tau, dep_ci, dep_val);
                if (best == RG_SCATTER) {
                    const float mu = hg_mu(d.g, pk.rng.next());
                    const float u2 = pk.rng.next();
                    const float3 uin = pk.r.u;
                    set_dir(pk.r, scatter_dir(uin, mu, u2));
                    peel(pk, pk.r.p, uin, PEEL_HG, 0, false);
                    tau = -logf(pk.rng.next());
                } else if (a.terminate_on_absorb) {
                    lc.inc(C_ABSORBED_TERM);
                    flush_run(t, dep_ci, dep_val);
                    lc.inc(C_PACKETS_DONE);
                    again = true;
                } else {
                    const float u1 = pk.rng.next(), u2 = pk.rng.next();
                    set_dir(pk.r, isotropic_dir(u1, u2));
                    const int row = min(max(__ldg(d.emit_row + pk.r.ci), 0), d.nT - 1);   // bounds check
                    set_frequency(pk, d, o, sample_table(d.nu, d.cdf_emit + (int64_t)row * d.nnu, d.nnu, pk.rng.next()));
                    peel(pk, pk.r.p, pk.r.u, PEEL_ISO, 0, true);
                    tau = -logf(pk.rng.next());
                }
            }
            if (act && !again) {
                if (result == RG_READY) pack(sh.slot[slot], pk, tau, dep_ci, dep_val);
                __threadfence_block();
                vstore(&sh.flag[slot], result);
            }
            append(act && again, RG_NEED, slot);
            __syncwarp();
        } else if (!arrived) {
            // ------------------------------------------------------------ nothing to do
            if (__shfl_sync(FULL, lane == 0 ? vload(&sh.exited) : 0, 0) >= RG_WALKERS) break;
            __nanosleep(100);
            if (((++polls) & 63u) == 0) {
                bool ab = false;
                if (lane == 0) ab = vload(&sh.abort) != 0 || past_deadline(a, t) || global_ns() - last > RG_STALL_NS;
                if (__shfl_sync(FULL, ab ? 1 : 0, 0)) {
                    if (lane == 0) {
                        vstore(&sh.abort, 1);
                        lc.inc(C_WATCHDOG);
                    }
                    break;
                }
            }
        } else {
            last = global_ns();
        }
        if (__shfl_sync(FULL, lane == 0 ? vload(&sh.abort) : 0, 0)) break;
    }
    if (lane == 0 && vload(&sh.abort)) atomicExch(t.abort_flag, 1);
}

template <int G, bool WAGG, bool PEEL, int MINB>
__global__ void __launch_bounds__(256, MINB) k_event_rg(DevGrid g, DevDust d, DevSources s, DevObs o, RunArgs a,
                                                        Tallies t) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RgShared& sh = *reinterpret_cast<RgShared*>(smem_raw);
    SharedTallies st{nullptr, nullptr};
    if (a.smem_sed) {
        st.sed = reinterpret_cast<double*>(smem_raw + RG_TALLY_OFFSET);
        st.esc = reinterpret_cast<unsigned*>(smem_raw + RG_TALLY_OFFSET + sizeof(double) * (size_t)o.nobs * o.nsed);
        for (int i = threadIdx.x; i < o.nobs * o.nsed; i += blockDim.x) st.sed[i] = 0.0;
        for (int i = threadIdx.x; i < N_ESC_MU * o.nsed; i += blockDim.x) st.esc[i] = 0u;
    }
    for (int i = threadIdx.x; i < RG_SLOTS; i += blockDim.x) sh.flag[i] = RG_FREE;
    if (threadIdx.x < RG_WALKERS) sh.tail[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        sh.exited = 0;
        sh.abort = 0;
    }
    __syncthreads();
    __shared__ unsigned long long cnt_sh[8][N_COUNTERS];
    LocalCounters lc;
    lc.init(cnt_sh[threadIdx.x >> 5]);
    const int w = threadIdx.x >> 5;
    if (w < RG_WALKERS) rg_walker<G, WAGG>(g, d, o, a, t, st, sh, w, lc);
    else rg_service<G, PEEL>(g, d, s, o, a, t, st, sh, lc);
    flush_counters(lc, t.counters);
    flush_shared(o, a, t, st);
}

template <int G, bool PEEL, int MINB>
cudaError_t launch_rg(const PropagateJob& j, int bps_cap, cudaStream_t s) {
    constexpr bool WAGG = G == GRID_CARTESIAN;       // as in k_event (measured per grid type)
    auto kernel = k_event_rg<G, WAGG, PEEL, MINB>;
    const size_t smem = RG_TALLY_OFFSET + shared_bytes(j);
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem)) != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (bps_cap > 0 && bps_cap < per_sm) per_sm = bps_cap;
    int blocks = per_sm * sms;
    const int64_t need = (j.args.n_packets + RG_LANES - 1) / RG_LANES;
    if (need < blocks) blocks = (int)(need > 0 ? need : 1);
    kernel<<<blocks, 256, smem, s>>>(j.grid, j.dust, j.src, j.obs, j.args, j.tal);
    return cudaGetLastError();
}

template <int G, bool PEEL>
cudaError_t launch_rg_shape(const PropagateJob& j, int bps, cudaStream_t s) {
    if (bps >= 3) return launch_rg<G, PEEL, 3>(j, bps, s);
    return launch_rg<G, PEEL, 2>(j, bps, s);
}

}  // namespace

bool regroup_supported(const PropagateJob& job) {
    return job.args.mrw_gamma <= 0.f && job.args.max_interactions < (int64_t)0x7FFFFFFF &&
           RG_TALLY_OFFSET + shared_bytes(job) <= (size_t)200 * 1024;
}

// Lucy iterations at 3 blocks per SM, imaging passes at 2 (as for k_event); regroup threshold
// as k_event's defaults unless given.
cudaError_t launch_propagate_regroup(const PropagateJob& job, const Launch& l, cudaStream_t s, int* launched) {
    if (job.args.n_packets <= 0) return cudaSuccess;
    PropagateJob j = job;
    const bool peel = job.args.peel != 0;
    int rg_default = DEFAULT_REGROUP;
    if (job.grid.type != GRID_CARTESIAN) rg_default = 24;
    else if (job.args.n_packets >= (int64_t)1 << 22) rg_default = 20;
    j.args.regroup = l.regroup > 0 ? (l.regroup > 32 ? 32 : l.regroup) : rg_default;
    const int bps = l.blocks_per_sm > 0 ? l.blocks_per_sm : (peel ? 2 : 3);
    *launched += 1;
    if (job.grid.type == GRID_CARTESIAN)
        return peel ? launch_rg_shape<GRID_CARTESIAN, true>(j, bps, s) : launch_rg_shape<GRID_CARTESIAN, false>(j, bps, s);
    if (job.grid.type == GRID_CYLINDRICAL)
        return peel ? launch_rg_shape<GRID_CYLINDRICAL, true>(j, bps, s)
                    : launch_rg_shape<GRID_CYLINDRICAL, false>(j, bps, s);
    return peel ? launch_rg_shape<GRID_SPHERICAL, true>(j, bps, s) : launch_rg_shape<GRID_SPHERICAL, false>(j, bps, s);
}

}  // namespace hrt
