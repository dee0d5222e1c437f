// Plain structs handed to the kernels by value: device views of the problem (grid, dust,
// sources, observers), the per-call arguments and the output tallies.  Lengths are in the
// scaled unit L0 (the grid's largest |coordinate| or outer radius), so positions are O(1).
#pragma once
#include <cstdint>

namespace hrt {

enum GridType : int32_t { GRID_CARTESIAN = 0, GRID_SPHERICAL = 1, GRID_CYLINDRICAL = 2 };

struct DevGrid {
    int32_t type;
    int32_t n1, n2, n3;            // cells per axis (x,y,z), (r,theta,phi) or (R,z,phi)
    int64_t ncells;
    const float* rhoL;             // [ncells] rho * L0 (so dtau = rhoL * chi * l)
    // Cartesian walls (scaled); cylindrical: w2 holds the z walls
    const float* w1;
    const float* w2;
    const float* w3;
    // spherical: radii (scaled) and squares, polar walls (angle, cos, sin), azimuthal walls;
    // cylindrical: the cylinder radii R in rw/r2w/r2wl/rwd and the azimuthal walls
    const float* rw;               // [n1+1]
    const float* r2w;              // [n1+1] r^2 rounded to FP32
    const float* r2wl;             // [n1+1] r^2 - r2w (the FP32 pair holds r^2 to ~2^-48)
    const double* rwd;             // [n1+1] FP64 radii for small-r and grazing solves
    const float* thw;              // [n2+1]
    const float* cth;              // [n2+1] cos, exactly 0 for the midplane wall
    const float* sth;
    const double* cthd;            // FP64 copies for near-axis cones
    const double* sthd;
    const float* phw;              // [n3+1]
    const float* cph;
    const float* sph;
    float r0;                      // inner radius (scaled), 0 without a hole
    float r_fp64;                  // sphere coefficients for walls below this radius in FP64
    float sin_fp64;                // cone coefficients for walls with sin(theta) below this in FP64
    int32_t poles;                 // spherical: bit 0 theta_0 = 0, bit 1 theta_n = pi (the polar axis,
                                   // which bounds no cell)
};

struct DevDust {
    int32_t nnu;
    int32_t nT;
    const float* lnu;              // [nnu] ln nu
    const float* inv_dlnu;         // [nnu-1] 1/(ln nu_{j+1} - ln nu_j)
    const float* lchi;             // [nnu] ln chi
    const float* alb;              // [nnu]
    const float* nu;               // [nnu]
    const float* cdf_emit;         // [nT][nnu] cumulative emissivity rows
    const int32_t* emit_row;       // [ncells] row used for re-emission in this iteration
    float g;
    int32_t pad0;
};

struct DevSources {
    int32_t npoint;
    int32_t nsrc;                  // npoint + (cell source ? 1 : 0)
    int32_t nspec;                 // spectrum nodes per source
    int32_t pad0;
    const float* pos;              // [npoint][3] scaled
    const double* cdf;             // [nsrc] cumulative luminosity
    const float* spec_nu;          // [nspec]
    const float* spec_cdf;         // [nsrc][nspec]
    const double* cell_cdf;        // [ncells] cumulative cell luminosity or null
    int32_t next;                  // external isotropic sources: indices npoint .. npoint+next-1
    int32_t pad_ext;
    const float* ext_c;            // [next][3] sphere centres (scaled)
    const float* ext_R;            // [next] sphere radii (scaled)
    const float* col;              // [npoint][nobs] sum of rhoL l from each point source along each
                                   // observer direction (imaging passes), or null
};

struct DevObs {
    int32_t nobs;
    int32_t nsed;
    int32_t img_nx, img_ny, nimg;
    int32_t pad0;
    const float* n;                // [nobs][3]
    const float* ex;               // [nobs][3]
    const float* ey;               // [nobs][3]
    double sed_a, sed_b;           // SED bin = floor(sed_a - sed_b * ln nu)
    float sed_af, sed_bf;          // the same coefficients rounded to FP32 (screening pass)
    float img_scale;               // nx / (2 * half extent) in scaled units
    float img_half;                // scaled half extent
    const int32_t* img_bin;        // [nimg] SED bin per image wavelength
};

struct Tallies {
    double* acc;                   // [ncells] sum eps kappa l (cgs)
    double* sed;                   // [nobs][nsed]
    double* img;                   // [nobs][nimg][ny][nx]
    unsigned long long* esc;       // [10][nsed] escaping packet counts (x eps = energy)
    unsigned long long* counters;  // [N_COUNTERS]
    int32_t* abort_flag;           // set by the watchdog
    float* report;                 // [WD_REPORTS][WD_FIELDS] state of lanes stopped by the watchdog
    unsigned* report_count;
    uint32_t* visits;              // [ncells] packet entries (runs of one packet's segments in the
                                   // cell), counted for the diffusion approximation; null = off
};

constexpr int WD_REPORTS = 32;
constexpr int WD_FIELDS = 16;

enum Counter {
    C_ESCAPED = 0,
    C_KILLED,
    C_ABSORBED_TERM,
    C_INTERACTIONS,
    C_SCATTER,
    C_ABSORB,
    C_CROSSINGS,
    C_PEEL_CROSSINGS,
    C_PACKETS_DONE,
    C_WATCHDOG,
    C_STUCK,          // rays ended after MAX_WALK_STEPS crossings without reaching an event
    C_MRW,            // modified-random-walk steps
    N_COUNTERS
};

constexpr int N_ESC_MU = 10;

// A peel-off event queued by the propagation kernel of an imaging pass (Sect. 2.6.2): the peel
// rays from it to every observer are walked by a separate pass, one ray per thread.  The record
// is 32 bytes, one memory sector: the per-axis cell indices follow from the linear index, and the
// extinction and SED bin from the frequency, through the same functions the packet used.
struct __align__(16) PeelEvent {
    float px, py, pz;              // event position (scaled)
    int32_t ci;                    // its cell (linear), or -1: locate the cell along each observer direction
    float ux, uy, uz;              // incoming direction (Henyey-Greenstein scattering)
    float nu;                      // packet frequency; negated for a scattering (Henyey-Greenstein weight)
};

struct RunArgs {
    int64_t n_packets;
    int64_t first_packet;
    uint32_t key0, key1;
    uint32_t iter_key, model_key;
    double eps;                    // packet energy (erg)
    double epsL0;                  // eps * L0 (deposit per unit scaled length per kappa)
    int64_t max_interactions;
    int32_t peel;
    int32_t terminate_on_absorb;
    int32_t rt;                    // 1: point-source emission and re-emission are raytraced, not peeled
    float mrw_gamma;               // > 0: modified random walk where the sphere to the nearest wall is
                                   // at least this many transport mean free paths in radius
    const float* mrw_k;            // [ncells] rhoL chi_t(T): inverse transport mean free path (scaled)
    const float* mrw_kp;           // [ncells] Planck-mean absorption coefficient kappa_P(T)
    PeelEvent* peel_q;             // imaging pass, event kernel: queue of peel-off events, or null
    unsigned long long* peel_n;    // events queued (may pass peel_cap: those were peeled inline)
    int64_t peel_cap;
    uint64_t budget_ns;            // watchdog budget after the launch stamp, 0 = none
    int32_t regroup;               // event kernel: leave walk phase below this many walkers
    int32_t smem_sed;              // 1: SED tallies in shared memory
    unsigned long long* work_counter;   // event kernel: next packet to start
    const unsigned long long* t0;  // globaltimer stamp written just before the launch
};

constexpr int DEFAULT_REGROUP = 12;

// ---------------------------------------------------------------- batched models
// Device descriptor of one model of a batch: its problem views, tallies and run arguments, and
// what the temperature update and the convergence select need.
struct BatchModel {
    DevGrid g;
    DevDust d;
    DevSources s;
    DevObs o;
    Tallies t;
    RunArgs a;
    const double* va;              // per-axis volume factors
    const double* vb;
    const double* vc;
    const double* E;               // [nT] emission table, its log, log T nodes, T nodes
    const double* lnE;
    const double* lnT;
    const double* Tn;
    int32_t nT;
    int32_t quantity;              // 0 T, 1 Adot
    double* T;
    double* adot;
    int32_t* emit_row;
    unsigned long long* keys;
    int64_t n_dust;                // cells with dust
    int64_t krank;                 // rank of the quantile among all keys (cells without dust key 0)
};

struct BatchChunk {                // packets [p0, p1) of one model
    int32_t model;
    int32_t pad;
    int64_t p0, p1;
};

struct BatchSeg {                  // cells [c0, c1) of one model
    int32_t model;
    int32_t pad;
    int64_t c0, c1;
};

// Per-model iteration state kept on the device between graph launches.
struct BatchState {
    uint32_t iteration;            // keys the random streams of the next iteration
    int32_t active;                // 0 once converged
    int32_t have_Q;
    int32_t ran;                   // ran in the last launch
    int32_t converged;
    int32_t pad;
    double Q, Q_prev, Delta;
    unsigned long long prefix, rank;   // radix select of the quantile
    unsigned long long clamp_low, clamp_high;
};

}  // namespace hrt
