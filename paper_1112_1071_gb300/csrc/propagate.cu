// Plain propagation kernel of one Lucy iteration (Sect. 2.2, Eq. 2, Sect. 2.6.2): one thread
// per packet history, grid-stride over packets, every deposit a plain FP64 atomic, peel-off rays
// walked inline.  The straightforward GPU formulation the event kernel (event.cu) is measured
// against.
#include "propagate_common.cuh"

namespace hrt {

__global__ void k_stamp(unsigned long long* t0) { *t0 = global_ns(); }

cudaError_t launch_stamp(unsigned long long* t0, cudaStream_t s) {
    k_stamp<<<1, 1, 0, s>>>(t0);
    return cudaGetLastError();
}

// Walk to optical depth tau (extinction) or escape; each segment in a cell with dust adds
// eps * kappa * l to the cell (Eq. 2's numerator).
template <int G>
__device__ __forceinline__ int walk_plain(const DevGrid& g, const RunArgs& a, const Tallies& t, Packet& pk,
                                          float tau, LocalCounters& lc) {
    const float chi = pk.dust.chi;
    const float kap = pk.dust.kappa;   // deposits are kappa * l; eps L0 is applied in the T update
    unsigned check = 0;
    int zero_run = 0;
    for (;;) {
        int axis, dir;
        const float l = cell_exit<G>(g, pk.r, axis, dir);
        if constexpr (G != GRID_CARTESIAN) {
            if (!tiny_step(pk.r, l)) zero_run = 0;
            else if (++zero_run > ZERO_RUN_LIMIT) { nudge(pk.r); zero_run = 0; }
        }
        if (check >= MAX_WALK_STEPS) {
            lc.inc(C_STUCK);
            return EV_STUCK;
        }
        const float rho = __ldg(g.rhoL + pk.r.ci);
        const float k = rho * chi;
        const float dtau = k * l;
        if (rho > 0.f && t.visits && pk.r.ci != pk.run_ci) {    // a new run: one packet entry
            atomicAdd(t.visits + pk.r.ci, 1u);
            pk.run_ci = pk.r.ci;
        }
        if (tau < dtau) {
            const float lp = tau / k;
            atomicAdd(t.acc + pk.r.ci, (double)(kap * lp));
            pk.r.p.x += lp * pk.r.u.x;
            pk.r.p.y += lp * pk.r.u.y;
            pk.r.p.z += lp * pk.r.u.z;
            return EV_INTERACT;
        }
        if (rho > 0.f) atomicAdd(t.acc + pk.r.ci, (double)(kap * l));
        tau -= dtau;
        lc.inc(C_CROSSINGS);
        if (cell_step<G>(g, pk.r, l, axis, dir)) return EV_ESCAPE;
        if (((++check) & 1023u) == 0 && past_deadline(a, t)) return EV_ABORT;
    }
}

template <int G>
__global__ void __launch_bounds__(256) k_plain(DevGrid g, DevDust d, DevSources s, DevObs o, RunArgs a, Tallies t) {
    const SharedTallies st = shared_tallies(o, a);
    __shared__ unsigned long long cnt_sh[8][N_COUNTERS];
    LocalCounters lc;
    lc.init(cnt_sh[threadIdx.x >> 5]);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < a.n_packets; q += stride) {
        if (past_deadline(a, t)) {
            lc.inc(C_WATCHDOG);
            break;
        }
        Packet pk;
        if (!emit_packet<G>(g, d, s, o, a, t, st.sed, a.first_packet + q, pk, lc)) {
            lc.inc(C_ESCAPED);
            lc.inc(C_PACKETS_DONE);
            continue;
        }
        for (;;) {
            // modified random walk (Sect. 2.2) while the packet sits deep in a thick cell: each step
            // one interaction against the cap and an isotropic re-emission at its end
            bool killed = false;
            while (a.mrw_gamma > 0.f) {
                const float R0 = mrw_sphere<G>(g, a, pk.r);
                if (R0 < 0.f) break;
                if (++pk.nint > a.max_interactions) {
                    killed = true;
                    break;
                }
                lc.inc(C_MRW);
                const float v = mrw_take(d, o, a, pk, R0);
                atomicAdd(t.acc + pk.r.ci, widen(v));
                if (t.visits && pk.r.ci != pk.run_ci) {
                    atomicAdd(t.visits + pk.r.ci, 1u);
                    pk.run_ci = pk.r.ci;
                }
                if (a.peel && !a.rt)
                    peel_event<G>(g, d, o, a, t, st.sed, pk.r, pk.r.u, PEEL_ISO, false, pk.dust.chi, pk.sbin, lc);
            }
            if (killed) {
                lc.inc(C_KILLED);
                break;
            }
            const float tau = -logf(pk.rng.next());
            const int ev = walk_plain<G>(g, a, t, pk, tau, lc);
            if (ev == EV_ESCAPE) {
                lc.inc(C_ESCAPED);
                tally_escape(o, t, pk, st.esc);
                break;
            }
            if (ev == EV_ABORT) {
                lc.inc(C_WATCHDOG);
                break;
            }
            if (ev == EV_STUCK) {
                lc.inc(C_KILLED);
                break;
            }
            if (++pk.nint > a.max_interactions) {
                lc.inc(C_KILLED);
                break;
            }
            if (!interact<G>(g, d, o, a, t, st.sed, pk, lc)) break;
        }
        lc.inc(C_PACKETS_DONE);
    }
    flush_counters(lc, t.counters);
    flush_shared(o, a, t, st);
}

// Columns sum rhoL l from each point source to the grid edge along each observer direction (-1
// for a source outside the grid, which emits no packets into it): the
// peel-off rays of every packet emitted by a point source start at the source and run along the
// observer direction, so their optical depth is chi(nu) times this column (Sect. 2.6.2).
template <int G>
__global__ void k_source_columns(DevGrid g, DevSources s, DevObs o, float* col) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= s.npoint * o.nobs) return;
    const int src = q / o.nobs, ob = q % o.nobs;
    Ray r;
    r.p = make_float3(s.pos[3 * src], s.pos[3 * src + 1], s.pos[3 * src + 2]);
    set_dir(r, make_float3(o.n[3 * ob], o.n[3 * ob + 1], o.n[3 * ob + 2]));
    float sum = -1.f;                  // -1: the source lies outside the grid
    unsigned long long ncross = 0;
    if (grid_locate<G>(g, r)) sum = tau_to_edge<G>(g, r, 1.f, ncross, F_INF);
    col[q] = sum;
}

cudaError_t launch_source_columns(const DevGrid& g, const DevSources& src, const DevObs& o, float* col,
                                  cudaStream_t s) {
    const int n = src.npoint * o.nobs;
    if (n <= 0) return cudaSuccess;
    const int blocks = (n + 127) / 128;
    if (g.type == GRID_CARTESIAN) k_source_columns<GRID_CARTESIAN><<<blocks, 128, 0, s>>>(g, src, o, col);
    else if (g.type == GRID_CYLINDRICAL) k_source_columns<GRID_CYLINDRICAL><<<blocks, 128, 0, s>>>(g, src, o, col);
    else k_source_columns<GRID_SPHERICAL><<<blocks, 128, 0, s>>>(g, src, o, col);
    return cudaGetLastError();
}

cudaError_t launch_propagate_plain(const PropagateJob& job, const Launch& l, cudaStream_t s, int* launched) {
    if (job.args.n_packets <= 0) return cudaSuccess;
    Launch ll = l;
    ll.block = 256;
    *launched += 1;
    if (job.grid.type == GRID_CARTESIAN) return launch_persistent(k_plain<GRID_CARTESIAN>, job, ll, s);
    if (job.grid.type == GRID_CYLINDRICAL) return launch_persistent(k_plain<GRID_CYLINDRICAL>, job, ll, s);
    return launch_persistent(k_plain<GRID_SPHERICAL>, job, ll, s);
}

}  // namespace hrt
