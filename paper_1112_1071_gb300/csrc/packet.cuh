// Packet-level steps shared by the propagation kernels: emission (Sect. 2.1.1, 2.2), the walk
// to a sampled optical depth with Lucy deposits (Sect. 2.2, Eq. 2), interactions (scatter or
// absorb and re-emit, Sect. 2.2 and 2.1.3) and peeling-off (Sect. 2.6.2).
#pragma once
#include "device_grid.cuh"
#include "mrw.cuh"

namespace hrt {

// Per-thread tallies of a propagation kernel.  The two per-crossing counts live in registers;
// the per-event counts (escapes, interactions, ...: one per tens of crossings) go, in the default
// mode, by shared-memory atomics to the warp's slot, so a thread holds 4 registers of counters
// instead of 2 per counter.  `slot` is this warp's row of a kernel's __shared__ unsigned long long
// [8][N_COUNTERS] (blocks of <= 256 threads).  Modes (a constant of each kernel):
//   CNT_GROUPED: the lanes that reach one call site together add their count with one shared
//     atomic (a thick model's events come in whole warps; 32 atomics on one address serialise);
//   CNT_LANE: one shared atomic per lane;
//   CNT_REG: every count in registers, as for the modified-random-walk kernels, whose steps are
//     events and which run at 3 blocks per SM anyway (measured: grouped 45-49 % and per-lane
//     atomics 2-15 % slower there).
enum CounterMode : int { CNT_GROUPED = 0, CNT_LANE = 1, CNT_REG = 2 };

struct LocalCounters {
    unsigned long long cross, peel_cross;
    unsigned long long* slot;
    int mode;
    unsigned long long v[N_COUNTERS];      // CNT_REG
    __device__ __forceinline__ void init(unsigned long long* warp_slot, int m = CNT_GROUPED) {
        cross = peel_cross = 0ull;
        slot = warp_slot;
        mode = m;
        if (mode == CNT_REG) {
#pragma unroll
            for (int i = 0; i < N_COUNTERS; ++i) v[i] = 0ull;
        }
        const unsigned lane = threadIdx.x & 31u;
        if (lane < (unsigned)N_COUNTERS) slot[lane] = 0ull;
        __syncwarp();
    }
    __device__ __forceinline__ void add(int c, unsigned long long x) {
        if (c == C_CROSSINGS) cross += x;
        else if (c == C_PEEL_CROSSINGS) peel_cross += x;
        else if (mode == CNT_REG) v[c] += x;
        else atomicAdd(slot + c, x);
    }
    __device__ __forceinline__ void inc(int c) {
        if (c == C_CROSSINGS) {
            ++cross;
        } else if (c == C_PEEL_CROSSINGS) {
            ++peel_cross;
        } else if (mode == CNT_REG) {
            ++v[c];
        } else if (mode == CNT_GROUPED) {
            const unsigned m = __activemask();
            if ((threadIdx.x & 31u) == (unsigned)(__ffs(m) - 1)) atomicAdd(slot + c, (unsigned long long)__popc(m));
        } else {
            atomicAdd(slot + c, 1ull);
        }
    }
};

// Whole warp: add the warp's counts to the global tallies (one atomic per warp and counter) and
// start again from zero.
__device__ __forceinline__ void flush_counters(LocalCounters& lc, unsigned long long* g) {
    const unsigned lane = threadIdx.x & 31u;
    unsigned long long x = lc.cross, y = lc.peel_cross;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
    }
    if (lane == 0 && x) atomicAdd(g + C_CROSSINGS, x);
    if (lane == 0 && y) atomicAdd(g + C_PEEL_CROSSINGS, y);
    if (lc.mode == CNT_REG) {
#pragma unroll
        for (int i = 0; i < N_COUNTERS; ++i) {
            if (i == C_CROSSINGS || i == C_PEEL_CROSSINGS) continue;
            unsigned long long z = lc.v[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) z += __shfl_down_sync(0xffffffffu, z, o);
            if (lane == 0 && z) atomicAdd(g + i, z);
            lc.v[i] = 0ull;
        }
    }
    __syncwarp();
    if (lane < (unsigned)N_COUNTERS && lane != (unsigned)C_CROSSINGS && lane != (unsigned)C_PEEL_CROSSINGS) {
        const unsigned long long z = lc.slot[lane];
        if (z) atomicAdd(g + lane, z);
        lc.slot[lane] = 0ull;
    }
    __syncwarp();
    lc.cross = lc.peel_cross = 0ull;
}

// SED bin of a frequency: floor(nsed ln(lambda/lambda_min) / ln(lambda_max/lambda_min)), -1 outside.
// The bin is decided by x = sed_a - sed_b ln nu in FP64.  An FP32 pass screens it first: the
// rounding of sed_a, sed_b, logf (<= 1 ulp), the product and the difference together stay
// below 2^-22 (|sed_a| + |sed_b ln nu| + |x|); only when x_f lies within 1e-6 of that sum of
// an integer (a bin edge, 0 or nsed) does the FP64 value decide, so the result is always the
// FP64 one while the FP64 pipe is used on a small fraction of frequencies.
__device__ __forceinline__ int sed_bin(const DevObs& o, float nu) {
    const float t = o.sed_bf * logf(nu);
    const float xf = o.sed_af - t;
    const float guard = 1e-6f * (fabsf(o.sed_af) + fabsf(t) + fabsf(xf));
    const float fl = floorf(xf);
    if (xf - fl > guard && fl + 1.f - xf > guard) {
        if (!(fl >= 0.f) || fl >= (float)o.nsed) return -1;
        return (int)fl;
    }
    const double x = o.sed_a - o.sed_b * log((double)nu);
    if (!(x >= 0.0) || x >= (double)o.nsed) return -1;
    return (int)x;
}

struct Packet {
    Ray r;
    float nu;
    DustAt dust;
    int32_t sbin;
    int64_t nint;
    PacketRng rng;
    float3 last_origin;      // emission position (before any hole crossing)
    int32_t emit_relocate;   // 1: emission peel rays must locate their cell along the observer
    int32_t src;             // emitting source
    int32_t run_ci;          // cell of the current run of deposits (plain kernel's entry count)
};

__device__ __forceinline__ void set_frequency(Packet& pk, const DevDust& d, const DevObs& o, float nu) {
    pk.nu = nu;
    pk.dust = dust_at(d, nu);
    pk.sbin = sed_bin(o, nu);
}

enum PeelKind : int32_t { PEEL_ISO = 0, PEEL_HG = 1 };

// Peel-off towards every observer from position r.p: weight eps p exp(-tau_obs).  With
// relocate, the starting cell is found along each observer direction (emission from a point
// source, which may sit on walls or in the spherical hole); otherwise the packet's cell is used.
// With col (emission from a point source whose columns were precomputed), tau_obs = chi col[ob]:
// every packet of that source peels along the same rays, so they are walked once per pass.  A ray
// stops once its optical depth passes tau_stop (its weight is then below exp(-tau_stop)).
template <int G>
__device__ void peel_event(const DevGrid& g, const DevDust& d, const DevObs& o, const RunArgs& a,
                           const Tallies& t, double* sed_s, const Ray& at, float3 uin, int kind, bool relocate,
                           float chi, int sbin, LocalCounters& lc, const float* col = nullptr,
                           float tau_stop = F_INF) {
    if (sbin < 0) return;
    for (int ob = 0; ob < o.nobs; ++ob) {
        const float3 n = make_float3(__ldg(o.n + 3 * ob), __ldg(o.n + 3 * ob + 1), __ldg(o.n + 3 * ob + 2));
        const float prob = (kind == PEEL_HG) ? hg_phase(d.g, dot3(uin, n)) : (0.25f / CUDART_PI_F);
        Ray pr = at;
        set_dir(pr, n);
        float tau = 0.f;
        bool inside = true;
        if (col) tau = chi * fmaxf(__ldg(col + ob), 0.f);
        else {
            if (relocate) inside = grid_locate<G>(g, pr);
            if (inside) {
                tau = tau_to_edge<G>(g, pr, chi, lc.peel_cross, tau_stop);
                if (tau == F_INF) lc.inc(C_STUCK);
            }
        }
        const double w = a.eps * (double)(prob * expf(-tau));
        if (sed_s) atomicAdd(sed_s + ob * o.nsed + sbin, w);
        else atomicAdd(t.sed + (int64_t)ob * o.nsed + sbin, w);
        if (o.nimg > 0) {
            const float px = at.p.x * __ldg(o.ex + 3 * ob) + at.p.y * __ldg(o.ex + 3 * ob + 1) + at.p.z * __ldg(o.ex + 3 * ob + 2);
            const float py = at.p.x * __ldg(o.ey + 3 * ob) + at.p.y * __ldg(o.ey + 3 * ob + 1) + at.p.z * __ldg(o.ey + 3 * ob + 2);
            const int ix = (int)floorf((px + o.img_half) * o.img_scale);
            const int iy = (int)floorf((py + o.img_half) * o.img_scale);
            if (ix >= 0 && ix < o.img_nx && iy >= 0 && iy < o.img_ny) {
                for (int l = 0; l < o.nimg; ++l) {
                    if (__ldg(o.img_bin + l) != sbin) continue;
                    atomicAdd(t.img + (((int64_t)ob * o.nimg + l) * o.img_ny + iy) * o.img_nx + ix, w);
                }
            }
        }
    }
}

// Cell c and a point uniform in its volume from three uniforms (Cartesian: each coordinate;
// spherical: r^3, cos(theta) and phi uniform; cylindrical: R^2, z and phi uniform), as for
// emission from a cell.
template <int G>
__device__ __forceinline__ void place_in_cell(const DevGrid& g, int64_t c, float f0, float f1, float f2, Ray& r) {
    r.i = (int)(c % g.n1);
    r.j = (int)((c / g.n1) % g.n2);
    r.k = (int)(c / ((int64_t)g.n1 * g.n2));
    r.ci = (int32_t)c;
    if constexpr (G == GRID_CARTESIAN) {
        const float x0 = __ldg(g.w1 + r.i), y0 = __ldg(g.w2 + r.j), z0 = __ldg(g.w3 + r.k);
        r.p = make_float3(x0 + f0 * (__ldg(g.w1 + r.i + 1) - x0), y0 + f1 * (__ldg(g.w2 + r.j + 1) - y0),
                          z0 + f2 * (__ldg(g.w3 + r.k + 1) - z0));
    } else if constexpr (G == GRID_CYLINDRICAL) {     // R^2, z, phi uniform
        const double R0 = __ldg(g.rwd + r.i), R1 = __ldg(g.rwd + r.i + 1);
        const float R = (float)sqrt(R0 * R0 + (double)f0 * (R1 * R1 - R0 * R0));
        const float z0 = __ldg(g.w2 + r.j);
        const float ph0 = __ldg(g.phw + r.k);
        const float ph = ph0 + f2 * (__ldg(g.phw + r.k + 1) - ph0);
        float sp, cp;
        sincosf(ph, &sp, &cp);
        r.p = make_float3(R * cp, R * sp, z0 + f1 * (__ldg(g.w2 + r.j + 1) - z0));
    } else {
        const double r0 = __ldg(g.rwd + r.i), r1 = __ldg(g.rwd + r.i + 1);
        const double rad = cbrt(r0 * r0 * r0 + (double)f0 * (r1 * r1 * r1 - r0 * r0 * r0));
        const double c0 = __ldg(g.cthd + r.j), c1 = __ldg(g.cthd + r.j + 1);
        const double ct = c0 + (double)f1 * (c1 - c0);
        const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
        const float ph0 = __ldg(g.phw + r.k);
        const float ph = ph0 + f2 * (__ldg(g.phw + r.k + 1) - ph0);
        float sp, cp;
        sincosf(ph, &sp, &cp);
        r.p = make_float3((float)(rad * st) * cp, (float)(rad * st) * sp, (float)(rad * ct));
    }
}

// Emission: source by luminosity CDF, then position (cell sources), direction, frequency.
// Returns false when the packet starts outside the grid (counted as escaped).
template <int G>
__device__ bool emit_packet(const DevGrid& g, const DevDust& d, const DevSources& s, const DevObs& o,
                            const RunArgs& a, const Tallies& t, double* sed_s, int64_t pid, Packet& pk,
                            LocalCounters& lc, bool inline_peel = true) {
    pk.rng.init(make_uint2(a.key0, a.key1), (uint32_t)pid, a.iter_key, a.model_key);
    pk.nint = 0;
    const int src = (int)select_cdf<double>(s.cdf, s.nsrc, (double)pk.rng.next());
    pk.src = src;
    pk.run_ci = -1;
    if (src < s.npoint) {
        pk.r.p = make_float3(__ldg(s.pos + 3 * src), __ldg(s.pos + 3 * src + 1), __ldg(s.pos + 3 * src + 2));
        const float u1 = pk.rng.next(), u2 = pk.rng.next();
        set_dir(pk.r, isotropic_dir(u1, u2));
        set_frequency(pk, d, o, sample_table(s.spec_nu, s.spec_cdf + (int64_t)src * s.nspec, s.nspec, pk.rng.next()));
        const Ray at = pk.r;
        pk.last_origin = at.p;
        pk.emit_relocate = 1;
        if (!grid_locate<G>(g, pk.r)) return false;
        if (a.peel && !a.rt && inline_peel)     // raytraced instead when a.rt (Sect. 2.6.3)
            peel_event<G>(g, d, o, a, t, sed_s, at, pk.r.u, PEEL_ISO, true, pk.dust.chi, pk.sbin, lc,
                          s.col ? s.col + (int64_t)src * o.nobs : nullptr);
    } else if (src < s.npoint + s.next) {
        // external isotropic source (Sect. 2.1.1): a point uniform on its sphere, a direction into
        // it with the cosine-weighted distribution of an isotropic intensity (cos = sqrt(u) about
        // the inward normal, azimuth in the normal's fixed frame); the packet travels through
        // vacuum to the grid and enters it 1e-6 L0 deep, or escapes; no peel-off (background)
        const int e = src - s.npoint;
        const float u1 = pk.rng.next(), u2 = pk.rng.next();
        const float3 nh = isotropic_dir(u1, u2);
        const float R = __ldg(s.ext_R + e);
        const float3 p = make_float3(__ldg(s.ext_c + 3 * e) + R * nh.x, __ldg(s.ext_c + 3 * e + 1) + R * nh.y,
                                     __ldg(s.ext_c + 3 * e + 2) + R * nh.z);
        const float u3 = pk.rng.next(), u4 = pk.rng.next();
        float3 e1 = fabsf(nh.z) < 0.99999f ? make_float3(-nh.y, nh.x, 0.f) : make_float3(nh.z, 0.f, -nh.x);
        const float ie = rsqrtf(e1.x * e1.x + e1.y * e1.y + e1.z * e1.z);
        e1.x *= ie; e1.y *= ie; e1.z *= ie;
        const float3 e2 = make_float3(nh.y * e1.z - nh.z * e1.y, nh.z * e1.x - nh.x * e1.z, nh.x * e1.y - nh.y * e1.x);
        const float ct = sqrtf(u3), st = sqrtf(1.f - u3);
        float sp, cp;
        sincospif(2.f * u4, &sp, &cp);
        float3 u = make_float3(-ct * nh.x + st * (cp * e1.x + sp * e2.x), -ct * nh.y + st * (cp * e1.y + sp * e2.y),
                               -ct * nh.z + st * (cp * e1.z + sp * e2.z));
        const float iu = rsqrtf(u.x * u.x + u.y * u.y + u.z * u.z);
        u.x *= iu; u.y *= iu; u.z *= iu;
        set_frequency(pk, d, o, sample_table(s.spec_nu, s.spec_cdf + (int64_t)src * s.nspec, s.nspec, pk.rng.next()));
        pk.emit_relocate = 0;
        const float t = grid_entry<G>(g, p, u);
        if (t < 0.f) return false;
        const float te = t + 1e-6f;
        pk.r.p = make_float3(p.x + te * u.x, p.y + te * u.y, p.z + te * u.z);
        set_dir(pk.r, u);
        pk.last_origin = pk.r.p;
        if (!grid_locate_entry<G>(g, pk.r)) return false;
    } else {
        pk.emit_relocate = 0;
        const int64_t c = select_cdf<double>(s.cell_cdf, g.ncells, (double)pk.rng.next());
        const float f0 = pk.rng.next(), f1 = pk.rng.next(), f2 = pk.rng.next();
        place_in_cell<G>(g, c, f0, f1, f2, pk.r);
        const float u1 = pk.rng.next(), u2 = pk.rng.next();
        set_dir(pk.r, isotropic_dir(u1, u2));
        set_frequency(pk, d, o, sample_table(s.spec_nu, s.spec_cdf + (int64_t)src * s.nspec, s.nspec, pk.rng.next()));
        pk.last_origin = pk.r.p;
        if (a.peel && inline_peel) peel_event<G>(g, d, o, a, t, sed_s, pk.r, pk.r.u, PEEL_ISO, false, pk.dust.chi, pk.sbin, lc);
    }
    return true;
}

// Interaction at the packet's position (Sect. 2.2): absorbed when zeta > albedo, then
// re-emitted isotropically with a frequency from the cell's emissivity row; otherwise scattered.
// Returns false when the packet ends (terminate-on-absorb test mode).
template <int G>
__device__ __forceinline__ bool interact(const DevGrid& g, const DevDust& d, const DevObs& o, const RunArgs& a,
                                         const Tallies& t, double* sed_s, Packet& pk, LocalCounters& lc) {
    lc.inc(C_INTERACTIONS);
    const float z = pk.rng.next();
    if (z > pk.dust.albedo) {
        lc.inc(C_ABSORB);
        if (a.terminate_on_absorb) {
            lc.inc(C_ABSORBED_TERM);
            return false;
        }
        const float u1 = pk.rng.next(), u2 = pk.rng.next();
        set_dir(pk.r, isotropic_dir(u1, u2));
        const int row = min(max(__ldg(d.emit_row + pk.r.ci), 0), d.nT - 1);   // bounds check
        set_frequency(pk, d, o, sample_table(d.nu, d.cdf_emit + (int64_t)row * d.nnu, d.nnu, pk.rng.next()));
        if (a.peel && !a.rt) peel_event<G>(g, d, o, a, t, sed_s, pk.r, pk.r.u, PEEL_ISO, false, pk.dust.chi, pk.sbin, lc);
    } else {
        lc.inc(C_SCATTER);
        const float mu = hg_mu(d.g, pk.rng.next());
        const float u2 = pk.rng.next();
        const float3 uin = pk.r.u;
        set_dir(pk.r, scatter_dir(uin, mu, u2));
        if (a.peel) peel_event<G>(g, d, o, a, t, sed_s, pk.r, uin, PEEL_HG, false, pk.dust.chi, pk.sbin, lc);
    }
    return true;
}

// Modified random walk (Sect. 2.2).  mrw_sphere: radius R0 of the step's sphere at the
// packet's position (MRW_SHRINK times the distance to the nearest wall of its cell), or -1 when
// the cell has no dust or the sphere is fewer than a.mrw_gamma transport mean free paths in
// radius.  mrw_take: the step itself, drawing (in this order) the path length, the exit point
// on the sphere and the isotropic re-emission (direction, then frequency from the cell's
// emissivity row); returns the deposit kappa_P(T) s (scaled length; Eq. 2 with the Planck-mean
// absorption coefficient of the thermalised field).  The packet stays in its cell.
template <int G>
__device__ __forceinline__ float mrw_sphere(const DevGrid& g, const RunArgs& a, const Ray& r) {
    const float k = __ldg(a.mrw_k + r.ci);
    if (!(k > 0.f)) return -1.f;
    const float R0 = MRW_SHRINK * wall_distance<G>(g, r);
    return (k * R0 >= a.mrw_gamma) ? R0 : -1.f;
}

__device__ __forceinline__ float mrw_take(const DevDust& d, const DevObs& o, const RunArgs& a, Packet& pk, float R0) {
    const float tau0 = __ldg(a.mrw_k + pk.r.ci) * R0;
    // the packet cannot reach the sphere's surface along a path shorter than R0
    const float s = R0 * fmaxf(mrw_path(tau0, pk.rng.next()), 1.f);
    const float u1 = pk.rng.next(), u2 = pk.rng.next();
    const float3 n = isotropic_dir(u1, u2);
    pk.r.p.x = fmaf(R0, n.x, pk.r.p.x);
    pk.r.p.y = fmaf(R0, n.y, pk.r.p.y);
    pk.r.p.z = fmaf(R0, n.z, pk.r.p.z);
    const float u3 = pk.rng.next(), u4 = pk.rng.next();
    set_dir(pk.r, isotropic_dir(u3, u4));
    const int row = min(max(__ldg(d.emit_row + pk.r.ci), 0), d.nT - 1);   // bounds check
    set_frequency(pk, d, o, sample_table(d.nu, d.cdf_emit + (int64_t)row * d.nnu, d.nnu, pk.rng.next()));
    return __ldg(a.mrw_kp + pk.r.ci) * s;
}

__device__ __forceinline__ void tally_escape(const DevObs& o, const Tallies& t, const Packet& pk, unsigned* esc_s) {
    if (pk.sbin < 0) return;
    int bm = (int)floorf((pk.r.u.z + 1.f) * 0.5f * N_ESC_MU);
    bm = bm < 0 ? 0 : (bm >= N_ESC_MU ? N_ESC_MU - 1 : bm);
    if (esc_s) atomicAdd(esc_s + bm * o.nsed + pk.sbin, 1u);
    else atomicAdd(t.esc + (int64_t)bm * o.nsed + pk.sbin, 1ull);
}

}  // namespace hrt
