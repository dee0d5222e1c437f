/*
 * hrt.h - C ABI of the GB300 Monte-Carlo dust continuum radiative transfer library (libhrt).
 *
 * The library computes the iterative LTE dust temperature of Robitaille (2011), HYPERION,
 * Sects. 2.2-2.6: photon packets are emitted from point, cell and external isotropic sources
 * (Sect. 2.1.1), propagated through a Cartesian, spherical-polar or cylindrical-polar grid of
 * constant-density cells (Sect. 2.1.2) to a sampled optical depth, scattered
 * (Henyey-Greenstein) or absorbed and re-emitted, and the path lengths they travel give the
 * absorbed energy rate of every cell (Eq. 2); the cell temperatures follow from the
 * Planck-mean balance (Eq. 3), the iteration is repeated until the percentile test of
 * Sect. 2.4 (Eqs. 4-6) passes, and SEDs and images are formed by peeling-off (Sect. 2.6.2).
 * Optional parts of the method on the same path: the modified random walk in optically thick
 * cells (Sect. 2.2), the partial diffusion approximation for poorly sampled cells (App. A) and
 * raytracing of source and dust emission (Sect. 2.6.3); all are selected in hrt_run_params.
 *
 * Conventions (all entry points)
 *   - Every function returns 0 (HRT_OK) or a negative hrt_status; hrt_last_error() holds a
 *     one-line message for the last failure on that context.
 *   - Units are cgs: lengths cm, angles rad, frequencies Hz, luminosities erg/s, densities
 *     g/cm^3, opacities cm^2/g, temperatures K.  The emission time step is dt = 1 s.
 *   - Cell arrays are C-ordered [n3][n2][n1]: Cartesian [z][y][x], spherical [phi][theta][r],
 *     cylindrical [phi][z][R].
 *   - Host input arrays are copied; the caller keeps ownership and may free them on return.
 *     Host output arrays are caller-owned and must hold at least the stated count n
 *     (HRT_EINVAL otherwise).  *_device variants take device pointers and are ordered on the
 *     context's stream.
 *   - All device memory the context needs is allocated and owned by the context and freed by
 *     hrt_destroy().  `stream` arguments are cudaStream_t values passed as void*.
 *   - The context is not thread-safe; use one context per host thread.
 */
#ifndef HRT_H
#define HRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HRT_OK = 0,
    HRT_EINVAL = -1,     /* bad argument (size, NaN, ordering, range) */
    HRT_ENOMEM = -2,     /* device or host allocation failed */
    HRT_ESTATE = -3,     /* call order: e.g. run before grid/density/dust/sources are set */
    HRT_ECUDA = -4,      /* a CUDA runtime call failed (message holds cudaGetErrorString) */
    HRT_ETIMEDOUT = -5,  /* the propagation watchdog expired; results of the call are partial */
    HRT_ERANGE = -6      /* a value beyond a table (strict mode) */
} hrt_status;

typedef struct hrt_ctx hrt_ctx;
typedef struct hrt_batch hrt_batch;

/* ------------------------------------------------------------------ lifetime */

/* Create a context on CUDA device `device`.  `seed` keys the Philox4x32-10 streams of all
 * packets (Salmon et al. 2011): packet p of iteration i draws from counters
 * (draw block, p, i, model id) under key (seed low 32 bits, seed high 32 bits).
 * `stream` (cudaStream_t, may be NULL = legacy default stream) orders all device work. */
int hrt_create(hrt_ctx** out, int device, uint64_t seed, void* stream);
int hrt_destroy(hrt_ctx* ctx);
const char* hrt_last_error(const hrt_ctx* ctx);
int hrt_set_stream(hrt_ctx* ctx, void* stream);
/* Library version string, e.g. "hrt 0.1 sm_103a". */
const char* hrt_version(void);

/* ------------------------------------------------------------------ problem (Sect. 2.1) */

/* Cartesian grid (Sect. 2.1.2): nx+1, ny+1, nz+1 strictly increasing wall coordinates (cm).
 * Resetting the grid discards density, temperatures and cell sources. */
int hrt_set_grid_cartesian(hrt_ctx* ctx, int nx, int ny, int nz,
                           const double* xw, const double* yw, const double* zw);

/* Spherical-polar grid (Sect. 2.1.2): radii rw[0..nr] (rw[0] >= 0; rw[0] > 0 leaves an empty
 * inner hole that packets cross without interacting), polar walls tw[0..nt] with tw[0] = 0 and
 * tw[nt] = pi, azimuthal walls pw[0..np] with pw[0] = 0, pw[np] = 2 pi and every cell at most
 * pi wide.  All strictly increasing. */
int hrt_set_grid_spherical(hrt_ctx* ctx, int nr, int nt, int np,
                           const double* rw, const double* tw, const double* pw);

/* Cylindrical-polar grid (Sect. 2.1.2): cylinder radii Rw[0..nR] about the z axis (Rw[0] >= 0;
 * Rw[0] > 0 leaves an empty inner cylinder that packets cross without interacting), planes
 * zw[0..nz] (cm), azimuthal walls pw[0..np] with pw[0] = 0, pw[np] = 2 pi and every cell at most
 * pi wide.  All strictly increasing.  Cells are ordered [phi][z][R].  Not accepted by the batch
 * (hrt_batch_create); the diffusion approximation stays spherical-polar. */
int hrt_set_grid_cylindrical(hrt_ctx* ctx, int nR, int nz, int np,
                             const double* Rw, const double* zw, const double* pw);

/* Dust density per cell (g/cm^3), n = number of cells, finite and >= 0.  Cells of zero density
 * hold no dust: packets cross them without interacting or depositing. */
int hrt_set_density(hrt_ctx* ctx, const float* rho, int64_t n);

/* One dust type (Sect. 2.1.3): nnu strictly increasing frequencies nu (Hz) with mass
 * extinction chi (cm^2/g, > 0) and albedo in [0,1]; Henyey-Greenstein asymmetry g in (-1,1).
 * Between nodes chi is interpolated log-log and the albedo linearly in log nu.  nT strictly
 * increasing temperature nodes (K) span the emissivity table: the library tabulates
 * E(T) = 4 pi int kappa_nu B_nu(T) dnu (Eq. 3, kappa = (1 - albedo) chi, trapezoid rule over
 * the nodes) and the cumulative emissivity kappa_nu B_nu(T) of each node for re-emission. */
int hrt_set_dust(hrt_ctx* ctx, int nnu, const double* nu, const double* chi, const double* albedo,
                 double g, int nT, const double* T);

/* Isotropic point source (Sect. 2.1.1) at x[3] (cm, inside the grid or its inner hole) with
 * luminosity L (erg/s) and a blackbody spectrum of temperature Teff, tabulated on 1000
 * log-spaced frequencies over the dust band and renormalised to carry all of L. */
int hrt_add_point_source(hrt_ctx* ctx, const double x[3], double L, double Teff);

/* External isotropic source (Sect. 2.1.1: an interstellar radiation field): the sphere of
 * centre c[3] and radius R (cm) emits L (erg/s) inwards, from points uniform on it, with the
 * cosine-weighted directions of an isotropic intensity and a blackbody spectrum of temperature
 * Teff; inside it (and without dust) the mean intensity is J = L / (4 pi^2 R^2).  Packets travel
 * through vacuum to the grid and enter it (or escape if they miss it); they are not peeled off
 * at emission (background).  L, R, Teff > 0, c finite; HRT_ESTATE before a grid is set. */
int hrt_add_external_source(hrt_ctx* ctx, const double c[3], double radius, double L, double Teff);

/* Point source (Sect. 2.1.1) at x[3] with luminosity L and a spectrum of its own: f_nu (>= 0,
 * any normalisation) at n >= 2 strictly increasing frequencies nu (Hz).  Between two nodes f_nu
 * is interpolated as a power law (log-log), linearly where either value is zero, and it is zero
 * outside the nodes; it is tabulated on the 1000 log-spaced frequencies of the source grid over
 * the dust band, and the in-band part carries all of L.  HRT_EINVAL for a non-finite or negative
 * value or non-increasing frequencies; the other checks are those of hrt_add_point_source.  A
 * spectrum with no flux at any frequency of that grid has nothing to carry L: the next
 * hrt_run_iteration returns HRT_EINVAL. */
int hrt_add_point_source_spectrum(hrt_ctx* ctx, const double x[3], double L, int n,
                                  const double* nu, const double* fnu);

/* Diffuse source (Sect. 2.1.1): luminosity per cell Lcell[n] (erg/s, >= 0) emitted from a
 * position uniform in the cell volume with an isotropic direction and a blackbody spectrum of
 * temperature Teff.  Replaces any previous cell source. */
int hrt_set_cell_source(hrt_ctx* ctx, const double* Lcell, int64_t n, double Teff);
int hrt_clear_sources(hrt_ctx* ctx);

/* Observers for peeling-off (Sect. 2.6.2): nobs directions given by inclination incl[o] and
 * azimuth az[o] (rad), observer unit vector n = (sin i cos az, sin i sin az, cos i).  SEDs have
 * nsed log-spaced wavelength bins over [lam_min_um, lam_max_um] (microns) and hold
 * erg/s/sr per bin.  Images (img_nx > 0) are img_nx x img_ny pixels over +-img_half_extent_cm
 * on the sky plane (axes e_x = (-sin az, cos az, 0), e_y = n x e_x) at the nimg wavelengths
 * img_lam_um, each collecting the packets of the SED bin holding that wavelength. */
int hrt_set_peeloff(hrt_ctx* ctx, int nobs, const double* incl, const double* az, int nsed,
                    double lam_min_um, double lam_max_um, int img_nx, int img_ny,
                    double img_half_extent_cm, int nimg, const double* img_lam_um);

/* ------------------------------------------------------------------ iteration (Sects. 2.2-2.4) */

/* Propagation kernels; all three draw packet p from the same Philox stream in the same order, so
 * their histories are the same.  HRT_KERNEL_EVENT: persistent event-based propagation in which
 * each warp's lanes walk together and handle their events in a short event phase (the default,
 * and the fastest on the benchmark workloads).  HRT_KERNEL_PLAIN: one thread per packet
 * history, the plain-GPU comparison.  HRT_KERNEL_REGROUP: the event-based form with the live
 * packets regrouped by state across the warps of a block -- walker warps hand stopped packets to
 * a service warp through shared-memory queues, and it runs each kind of event (scattering,
 * absorption and re-emission, new packets) in same-state batches; modified-random-walk runs
 * use HRT_KERNEL_EVENT instead. */
typedef enum { HRT_KERNEL_EVENT = 0, HRT_KERNEL_PLAIN = 1, HRT_KERNEL_REGROUP = 2 } hrt_kernel;

typedef struct {
    int64_t max_interactions;    /* per packet; a packet beyond it is killed and its energy tallied */
    int32_t peel;                /* 1: peel-off into the SED/image bins (zeroed at the start of the call) */
    int32_t update_temperature;  /* 1: Lucy iteration (Eqs. 2-6); 0: imaging pass, temperatures kept */
    int32_t terminate_on_absorb; /* test mode: an absorbed packet ends instead of being re-emitted */
    int32_t quantity;            /* convergence quantity: 0 temperature, 1 Adot (the paper's choice) */
    double p;                    /* percentile of Sect. 2.4 (e.g. 0.99) */
    double q_thres;              /* Q threshold (e.g. 1.02 on T, 2 on Adot) */
    double delta_thres;          /* Delta threshold (INFINITY disables the Delta test) */
    int32_t kernel;              /* hrt_kernel */
    int32_t block_size;          /* threads per block: 0 or 256 (the propagation kernels are compiled
                                    for 256-thread blocks) */
    int32_t blocks_per_sm;       /* persistent blocks per SM, 0 = tuned default (>= 0) */
    int32_t regroup_threshold;   /* event kernel: a warp leaves the walk phase when fewer lanes
                                    than this are still walking (1..32, 0 = tuned default) */
    double watchdog_ms;          /* > 0: the propagation kernel stops after this long and the call
                                    returns HRT_ETIMEDOUT (the context stays usable) */
    int64_t first_packet;        /* the call runs packet ids first_packet .. first_packet + n_packets - 1
                                    of the iteration (each id has its own Philox stream); default 0 */
    int64_t n_total;             /* packets of the whole iteration, eps = L_total dt / n_total; 0 (default)
                                    = n_packets.  With n_total > n_packets the call runs one share of an
                                    iteration (Sect. 3: packet chunks are independent and their
                                    accumulators add): a shard of a partitioned run, or a sample that
                                    can be checked packet by packet.  Needs first_packet >= 0 and
                                    first_packet + n_packets <= n_total <= 2^32 (else HRT_EINVAL). */
    int64_t pda_min_visits;      /* partial diffusion approximation (App. A), spherical-polar grids, Lucy
                                    iterations: cells with dust entered by fewer than this many packets
                                    (a packet's consecutive path segments in a cell count once) take T
                                    from the discrete diffusion equation of App. A, with well-sampled
                                    neighbours as boundary values; 0 (default) = off; < 2^32 */
    int64_t raytrace_rays;       /* imaging passes (update_temperature 0, peel 1): > 0 raytraces the
                                    point-source and dust emission into the SED and image bins
                                    (Sect. 2.6.3) instead of peeling it off: each source along its one
                                    ray, the dust by this many rays that start at points drawn in
                                    proportion to the cells' emission m E(T), each carrying
                                    L_dust / raytrace_rays over all bins at once; scattered light is
                                    still peeled off.  0 (default) = off; < 2^32 */
    double mrw_gamma;            /* modified random walk (Sect. 2.2, in the published diffusion form the
                                    paper refers to): > 0 lets a packet in a cell with dust cross, in
                                    one step, the sphere of radius 0.99 x its distance to the nearest
                                    wall of the cell whenever that sphere is at least mrw_gamma
                                    transport mean free paths (1 / rho chi_t, chi_t the Rosseland mean
                                    of chi_nu (1 - albedo g) at the cell's temperature) in radius.
                                    The step's path length s solves the diffusion survival probability
                                    (at least the radius), deposits kappa_P(T) s (Eq. 2 with the
                                    Planck-mean absorption coefficient), and ends with an isotropic
                                    re-emission from a point uniform on the sphere (frequency from the
                                    cell's emissivity row; peeled off like a re-emission); each step
                                    counts as one interaction against max_interactions.  Single-model
                                    runs only (a batch returns HRT_EINVAL).  0 (default) = off;
                                    finite, >= 0 */
    int64_t peel_queue_events;   /* imaging passes with the event kernel queue their peel-off events for
                                    a separate peel pass (48 bytes each); this caps the queue (0 =
                                    default: 2 per packet, at least 2^20, at most 2^27); events past
                                    the cap are peeled inline by the propagation kernel (same
                                    results, slower); >= 0 */
} hrt_run_params;

typedef struct {
    int32_t iteration;           /* index of the iteration that ran (0-based) */
    int32_t converged;           /* Q < q_thres and Delta < delta_thres */
    double Q;                    /* Eq. 5-6: p-quantile of delta(prev, new) over cells with dust */
    double Delta;                /* Eq. 6: delta(Q_prev, Q); INFINITY on the first iteration */
    double e_emitted, e_escaped, e_killed, e_absorbed;   /* erg over dt = 1 s */
    int64_t n_packets, n_interactions, n_scatter, n_absorb;
    int64_t n_crossings;         /* propagation cell crossings */
    int64_t n_peel_crossings;    /* peel-off ray cell crossings */
    int64_t n_killed;
    int64_t clamp_low, clamp_high;   /* cells (with dust) whose Adot fell outside E(T) */
    double ms_propagate;         /* device time of the propagation kernel */
    double ms_total;             /* device time of the whole call */
    int64_t kernel_launches;     /* kernels the call launched */
    int64_t n_pda;               /* cells whose T came from the diffusion approximation */
    int64_t pda_iterations;      /* conjugate-gradient iterations of its solve */
    double pda_residual;         /* |b - A x| / |b| at the end of the solve */
    int64_t n_mrw;               /* modified-random-walk steps */
} hrt_iter_stats;

/* Defaults: max_interactions 1e6, peel 0, update_temperature 1, p 0.99, q_thres 1.02 on T,
 * delta_thres INFINITY, event kernel, tuned launch shape, no watchdog. */
void hrt_default_params(hrt_run_params* p);

/* Run one iteration with n_packets packets of energy eps = L_total dt / n_packets.  In a Lucy
 * iteration the absorbed-energy accumulators are zeroed, packets propagate with the
 * temperatures of the previous iteration (10 K before the first), then Adot = acc/(V dt)
 * (Eq. 2) and T from Eq. 3 (table clamps counted) replace the previous values and Q, Delta
 * are formed (Eqs. 4-6).  Blocks until the statistics are on the host.  `out` may be NULL. */
int hrt_run_iteration(hrt_ctx* ctx, int64_t n_packets, const hrt_run_params* params, hrt_iter_stats* out);

/* ------------------------------------------------------------------ read-out / state */

int hrt_get_temperature(hrt_ctx* ctx, double* out, int64_t n);        /* K, [cells] */
int hrt_get_specific_energy(hrt_ctx* ctx, double* out, int64_t n);    /* Adot, erg/s/g, [cells] */
int hrt_get_absorbed(hrt_ctx* ctx, double* out, int64_t n);           /* raw sum eps kappa l, [cells] */
int hrt_get_sed(hrt_ctx* ctx, double* out, int64_t n);                /* [nobs][nsed] erg/s/sr */
int hrt_get_image(hrt_ctx* ctx, double* out, int64_t n);              /* [nobs][nimg][ny][nx] erg/s/sr per pixel */
int hrt_get_escape(hrt_ctx* ctx, double* out, int64_t n);             /* [10 cos(theta) bins][nsed] erg/s, all
                                                                         escaping packets of the last call (Sect. 2.6.1) */
int hrt_get_temperature_device(hrt_ctx* ctx, double* d_out, int64_t n);
int hrt_get_sed_device(hrt_ctx* ctx, double* d_out, int64_t n);
int64_t hrt_num_cells(const hrt_ctx* ctx);

/* After an HRT_ETIMEDOUT: the state of up to 32 packets the watchdog stopped, 16 floats each
 * (lane mode, packet id, interactions, optical depth, position[3] and direction[3] in the
 * scaled unit, cell index[3], frequency, peel observer, step or round count).  `out` must hold
 * 512 floats.  Returns the number of records (>= 0) or a negative hrt_status. */
int hrt_get_watchdog_report(hrt_ctx* ctx, float* out, int64_t n);

/* Warm start / resume: replace the temperatures (K, > 0) used by the next iteration. */
int hrt_set_temperature(hrt_ctx* ctx, const double* T, int64_t n);
int hrt_set_temperature_device(hrt_ctx* ctx, const double* d_T, int64_t n);
/* Set the iteration counter (it keys the random streams, so a resumed run repeats them). */
int hrt_set_iteration(hrt_ctx* ctx, int iteration);
/* Resume: the rest of the state the next iteration starts from.  A Lucy iteration i reads the
 * temperatures after iteration i-1 (hrt_set_temperature), the iteration counter
 * (hrt_set_iteration), the specific energies Adot after iteration i-1 (Eq. 2, erg s^-1 g^-1,
 * [ncells] C order, finite >= 0; read by the convergence statistic when it is taken on Adot,
 * quantity 1) and the previous percentile Q^{i-1} with whether it exists (Eqs. 5-6: Delta =
 * max(Q^{i-1}/Q^i, Q^i/Q^{i-1})).  Save them with hrt_get_temperature, hrt_get_specific_energy and
 * hrt_get_convergence_state after iteration i-1 and set all four to repeat iteration i exactly
 * (Q, Delta and the converged flag included).  Inputs are copied.  Q_prev >= 1 or +inf when
 * have_Q != 0 (else HRT_EINVAL); have_Q = 0 forgets Q^{i-1} (Delta is then +inf).  Setting the
 * grid clears the convergence state; a new grid starts with Adot = 0. */
int hrt_set_specific_energy(hrt_ctx* ctx, const double* adot, int64_t n);
int hrt_set_convergence_state(hrt_ctx* ctx, int have_Q, double Q_prev);
int hrt_get_convergence_state(hrt_ctx* ctx, int* have_Q, double* Q_prev);
int hrt_set_model_id(hrt_ctx* ctx, uint32_t model_id);

/* ------------------------------------------------------------------ single steps (test hooks)
 * Each runs one step of the method on n independent inputs in device memory with given
 * uniform deviates, so that it can be compared element by element with a CPU reference. */

/* Philox4x32-10: out[4i..4i+3] = philox(ctr[4i..4i+3], key[2i..2i+1]). */
int hrt_step_philox(int64_t n, const uint32_t* d_ctr, const uint32_t* d_key, uint32_t* d_out, void* stream);

/* Cell exit along the context grid (Sect. 2.2): pos/dir [n][3] (cm, unit), cell [n][3]
 * (per-axis indices); writes the distance to the exit (cm) and axis*2 + (sense > 0). */
int hrt_step_cell_exit(hrt_ctx* ctx, int64_t n, const float* d_pos, const float* d_dir,
                       const int32_t* d_cell, float* d_dist, int32_t* d_exit);

/* Extinction optical depth from pos along dir to the grid boundary at frequency nu[n]
 * (the peel-off ray of Sect. 2.6.2). */
int hrt_step_tau_to_edge(hrt_ctx* ctx, int64_t n, const float* d_pos, const float* d_dir,
                         const float* d_nu, float* d_tau);

/* Modified random walk (Sect. 2.2): distance (cm) from pos [n][3] (cm, inside cell [n][3]) to
 * the nearest wall bounding the cell; the polar axis, r = 0, R = 0 and the phi walls of a
 * single-phi-cell grid bound nothing. */
int hrt_step_wall_distance(hrt_ctx* ctx, int64_t n, const float* d_pos, const int32_t* d_cell, float* d_dist);

/* Modified random walk (Sect. 2.2): path length / R0 at which the diffusion survival probability
 * 2 sum_{n>=1} (-1)^{n+1} exp(-n^2 pi^2 s / (3 tau0 R0)) equals zeta[n] in (0, 1], for spheres of
 * tau0[n] transport mean free paths in radius (0 for zeta = 1; no lower bound applied). */
int hrt_step_mrw_path(int64_t n, const float* d_tau0, const float* d_zeta, float* d_out, void* stream);

/* Henyey-Greenstein scattering: new direction from dir_in [n][3] and uniforms u1 (cos theta)
 * and u2 (azimuth). */
int hrt_step_hg_scatter(hrt_ctx* ctx, int64_t n, const float* d_dir_in, const float* d_u1,
                        const float* d_u2, float* d_dir_out);

/* Re-emission frequency from emissivity row[n] (temperature node) with uniform u[n]. */
int hrt_step_sample_emission(hrt_ctx* ctx, int64_t n, const int32_t* d_row, const float* d_u, float* d_nu);

/* Source spectrum frequency of source src[n] with uniform u[n]. */
int hrt_step_sample_source(hrt_ctx* ctx, int64_t n, const int32_t* d_src, const float* d_u, float* d_nu);

/* Temperature from Adot (Eq. 3 inversion on the library's table). */
int hrt_step_temperature(hrt_ctx* ctx, int64_t n, const double* d_adot, double* d_T);

/* Tabulated E(T) [nT] and emissivity cdf [nT][nnu] as built on the device (copied to host). */
int hrt_get_tables(hrt_ctx* ctx, double* E, int64_t nE, float* cdf, int64_t ncdf);

/* Rosseland mean extinction chi_R(T_m) [nT] (cm^2/g) of the dust on the temperature nodes, as
 * used by the diffusion approximation (App. A): int dB/dT dnu / int chi^-1 dB/dT dnu, trapezoid
 * rule over the dust nodes.  n >= nT. */
int hrt_get_rosseland(hrt_ctx* ctx, double* out, int64_t n);

/* Packet entries per cell [cells] counted by the last Lucy iteration that ran with
 * pda_min_visits > 0 (HRT_ESTATE otherwise).  n must equal the number of cells. */
int hrt_get_visits(hrt_ctx* ctx, uint32_t* out, int64_t n);

/* ------------------------------------------------------------------ learned warm start
 * Not in the paper: a 3-D convolutional encoder-decoder (U-Net) trained on temperature fields
 * that the Monte-Carlo iteration itself produced, used only to start the iteration closer to its
 * fixed point; the Lucy iteration and its convergence test (Sect. 2.3-2.4) decide the result.
 * Levels L (1-4), base width c (multiple of 32): per level two 3x3x3 conv+ReLU and 2x average
 * pooling, a bottleneck of width c 2^L, a mirrored decoder (2x nearest upsampling concatenated
 * with the encoder skip, two conv+ReLU) and a 1x1x1 head.  Weights are FP32 masters (Adam) with
 * BF16 copies; activations BF16; every convolution runs on the tensor cores with FP32
 * accumulation.  Tensors are channels-last [N][D][H][W][C] float32 on the device.
 * Inputs: 2 channels, (log10 rho[g/cm^3] + 21.5) / 1 and log10(F[erg/s/cm^2]) / 2 with F the
 * summed point-source flux L/(4 pi (d^2 + (dx/2)^2)) at the cell centre (hrt_net_features).
 * Output: y = (log10 T[K] - 1.5) / 0.5.  D, H, W must be multiples of 2^L. */
typedef struct hrt_net hrt_net;
int hrt_net_create(hrt_net** out, int device, int base_channels, int levels, uint64_t seed, void* stream);
/* The same network with the width of every level given: widths[0..levels] (multiples of 32, at
 * most 512), e.g. {32, 64, 192} at 2 levels (2.19M parameters).  HRT_EINVAL otherwise. */
int hrt_net_create_widths(hrt_net** out, int device, const int* widths, int levels, uint64_t seed, void* stream);
int hrt_net_destroy(hrt_net* net);
/* Parameters in packed order: per conv layer W[27][Cin][Cout] (tap = 9 dz + 3 dy + dx) then
 * b[Cout]; then the head w[c], b[1].  */
int64_t hrt_net_num_params(const hrt_net* net);
int hrt_net_get_params(hrt_net* net, float* host_out, int64_t n);
int hrt_net_set_params(hrt_net* net, const float* host_in, int64_t n);
/* d_out[N][D][H][W] = network(d_in[N][D][H][W][2]); blocks until done. */
int hrt_net_forward(hrt_net* net, int N, int D, int H, int W, const float* d_in, float* d_out);
/* Loss 0.5 mean((y - target)^2) and its gradient (packed order, host buffer). */
int hrt_net_gradients(hrt_net* net, int N, int D, int H, int W, const float* d_in, const float* d_target,
                      float* host_grad, int64_t n, double* loss);
/* One Adam step (beta 0.9, 0.999) on that loss; *loss (may be NULL) is the loss before the step. */
int hrt_net_train_step(hrt_net* net, int N, int D, int H, int W, const float* d_in, const float* d_target, float lr,
                       double* loss);
/* Input features of a Cartesian context (2 floats per cell, device). */
int hrt_net_features(hrt_ctx* ctx, float* d_out, int64_t n);
/* Training target of a context: its current temperatures as y (1 float per cell, device). */
int hrt_net_temperature_target(hrt_ctx* ctx, float* d_out, int64_t n);
/* Replace the context's temperatures by the network's prediction (clamped to the T table). */
int hrt_net_warm_start(hrt_net* net, hrt_ctx* ctx);
/* Single-layer hooks on FP32 device tensors (converted to BF16 inside): 'same' 3x3x3 conv with
 * bias and optional ReLU (Cin % 16 == 0, Cout % 32 == 0), and its input, weight and bias
 * gradients for an output gradient dy (Cin, Cout % 32 == 0).  Weights [27][Cin][Cout].  The
 * convolutions run on the tcgen05 tensor cores (accumulator in tensor memory); HRT_ETIMEDOUT if
 * one of their bounded waits gave up.  That is a last resort (a wait of seconds that a healthy
 * GPU never reaches): the block that gave up frees its tensor memory while its own MMAs may
 * still be running, so treat the outputs of that call, and of any later tensor-core call in the
 * process, as invalid; the network calls (hrt_net_*) return the same code and leave the weights
 * of a failed training step unchanged, and the caller should recompute or stop.
 * hrt_nn_conv3d runs the TMA-fed pipelined kernel (persistent CTAs; operand stages -- the halo by
 * TMA, the weights, packed per output-channel tile, by bulk copies -- overlap the MMAs);
 * hrt_nn_conv3d_phased the same convolution loading each phase's operands with
 * cp.async before its MMAs; hrt_nn_conv3d_mma the same with warp-level mma.sync, the baseline the
 * tcgen05 kernels are measured against. */
int hrt_nn_conv3d(int N, int D, int H, int W, int Cin, int Cout, const float* d_x, const float* d_w, const float* d_b,
                  int relu, float* d_y, void* stream);
int hrt_nn_conv3d_phased(int N, int D, int H, int W, int Cin, int Cout, const float* d_x, const float* d_w,
                         const float* d_b, int relu, float* d_y, void* stream);
int hrt_nn_conv3d_mma(int N, int D, int H, int W, int Cin, int Cout, const float* d_x, const float* d_w,
                      const float* d_b, int relu, float* d_y, void* stream);
int hrt_nn_conv3d_backward(int N, int D, int H, int W, int Cin, int Cout, const float* d_x, const float* d_w,
                           const float* d_dy, float* d_dx, float* d_dw, float* d_db, void* stream);

/* ------------------------------------------------------------------ allocation-free quantile
 * The paper has no counterpart: this is a convenience for callers of the library that cannot
 * allocate device memory, such as a host framework whose allocator already owns the device's
 * memory, or latency-bound code that cannot afford the device-wide synchronisation that
 * cudaMalloc / cudaFree can impose.  It computes the same statistic as the Q of
 * hrt_run_iteration: the nearest-rank p-quantile of max(prev/cur, cur/prev) over the cells
 * whose density rho is > 0, written as one double to d_out (NaN when no cell holds dust).
 * d_prev, d_cur (n doubles), d_rho (n floats) and d_out are caller-owned device pointers;
 * the work is ordered on `stream` (cudaStream_t as void*) and the call does not wait for it.
 *
 * It allocates nothing: its only scratch is a fixed 1,056-byte array in the library's static
 * device memory, held by every GPU that loads the library until the process exits.  The first call on
 * a device looks up that array's device address (with that device current), so make the first
 * call on each device before any stream capture.  Every call on a device uses the same array
 * and clears it at its start: calls that overlap on the GPU (different streams, or host
 * threads) race and give wrong results; serialise them.
 *
 * Limit: 1 <= n <= HRT_NOALLOC_MAX_CELLS (2^31 - 1, the range of its 32-bit bin counts).
 * Returns HRT_OK; HRT_EINVAL (n out of range, a null pointer, p outside (0, 1]); HRT_ESTATE when
 * a CUDA error from earlier work on the calling thread is already pending (nothing is launched
 * and that error is left in place for the caller to read with cudaGetLastError); or HRT_ECUDA
 * when the device query or one of its own launches fails (that launch error is cleared).  A
 * sticky error (a fault in any earlier kernel of the process) makes it return HRT_ESTATE or
 * HRT_ECUDA as well.  It has no context, so hrt_last_error() does not describe its failures. */
#define HRT_NOALLOC_MAX_CELLS 2147483647LL
int hrt_quantile_ratio_noalloc(int64_t n, const double* d_prev, const double* d_cur, const float* d_rho,
                               double p, double* d_out, void* stream);

/* ------------------------------------------------------------------ batched models (Sect. 3 analogue)
 * Many contexts on the same device run each Lucy iteration in one persistent launch whose
 * blocks pull (model, packet chunk) work items from a device queue (largest first), the
 * device-side form of the paper's dynamic chunk scheduling.  Each model keeps its own
 * seed, tables and convergence state; a converged model drops out of later iterations. */
int hrt_batch_create(hrt_batch** out, hrt_ctx* const* models, int n);
int hrt_batch_destroy(hrt_batch* b);
/* Run up to max_iter Lucy iterations for every unconverged model, n_packets[m] packets each,
 * one persistent launch per iteration (captured as a CUDA graph after the first).  Writes the
 * last stats of every model to per_model_out[n] (may be NULL) and the number of iterations run
 * to *iterations_run (may be NULL).  Models are Cartesian or spherical-polar (hrt_batch_create
 * returns HRT_EINVAL for others).  params: the convergence settings, max_interactions,
 * terminate_on_absorb and watchdog_ms apply; peel-off, imaging passes, the PDA, raytracing and
 * the modified random walk run in single-model calls (mrw_gamma != 0, pda_min_visits != 0,
 * raytrace_rays != 0, peel != 0 or update_temperature == 0 return HRT_EINVAL). */
int hrt_batch_run(hrt_batch* b, const int64_t* n_packets, int max_iter, const hrt_run_params* params,
                  hrt_iter_stats* per_model_out, int* iterations_run);
/* Time a few launch shapes on one iteration's worth of work and keep the fastest. */
int hrt_batch_tune(hrt_batch* b, const int64_t* n_packets);

#ifdef __cplusplus
}
#endif
#endif /* HRT_H */
