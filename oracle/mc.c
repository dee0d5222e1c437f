/*
 * FP64 CPU ORACLE of the Monte-Carlo photon-packet propagation (HYPERION, Robitaille 2011).
 *
 * Test infrastructure only: a plain, slow, single-precision-free (FP64) restatement of the
 * method, written to be checked against the paper by eye.  Nothing in the CUDA library
 * uses this file; only the test-suite, the smoke check and the CPU baseline of the bench
 * load it.
 *
 * What it follows:
 *   Sect. 2.1.1  sources: point sources (a blackbody of Teff or a spectrum of their own, both
 *              tabulated by the caller), a diffuse source whose cells emit in proportion to
 *              their luminosity from points uniform in their volume, external isotropic
 *              fields emitted inwards from an enclosing sphere.
 *   Sect. 2.1.2  grids: Cartesian, spherical-polar (with an empty inner hole) and
 *              cylindrical-polar (with an empty inner cylinder), walls given by the caller.
 *   Sect. 2.2  packet life: emission by source luminosity PDF, tau = -ln(zeta), propagation
 *              to the sampled optical depth or escape, absorb if zeta > albedo else scatter,
 *              new tau after every interaction.
 *   Sect. 2.3, Eq. 2  path-length (Lucy) estimator: every segment of length l in a cell
 *              adds eps * kappa_nu * l to that cell (divided by V dt by the caller).
 *   Sect. 2.1.3  LTE re-emission j_nu = kappa_nu B_nu(T): frequency drawn from a
 *              cumulative emissivity row chosen by the cell temperature of the previous
 *              iteration (the caller passes the row index per cell).
 *   Sect. 2.6.2  peeling-off: at emission, scattering and re-emission every observer gets
 *              eps * p * exp(-tau_obs).
 *   Sect. 2.6.1  photon binning of escaping packets by viewing angle (escape tally).
 *   Sect. 2.2  modified random walk in optically thick cells (the published form the paper
 *              refers to; see the section below).
 *   Sect. 3     packets within an iteration are independent; the threaded mode splits the
 *              packet range and sums per-thread accumulators at the end of the iteration.
 * Scattering uses a Henyey-Greenstein phase function (the synthetic workloads' dust).
 *
 * Random numbers: Philox4x32-10 (Salmon et al. 2011), key = 64-bit seed, counter =
 * (draw block, packet id, iteration key, model id); draw n of a packet is word n mod 4 of
 * block n / 4, mapped to u = ((x >> 8) + 1) 2^-24 in (0, 1].
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define OR_C_LIGHT 2.99792458e10

/* ------------------------------------------------------------------ Philox4x32-10 */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof(c));
}

typedef struct {
    uint32_t key[2];
    uint32_t pkt, iter, model;
    uint32_t n;        /* next draw index */
    uint32_t blk;      /* block held in buf */
    int have;
    uint32_t buf[4];
} rng_t;

static double uniform(rng_t* r) {
    uint32_t b = r->n >> 2;
    if (!r->have || b != r->blk) {
        uint32_t c[4] = {b, r->pkt, r->iter, r->model};
        or_philox4x32_10(c, r->key, r->buf);
        r->blk = b;
        r->have = 1;
    }
    uint32_t x = r->buf[r->n & 3u];
    r->n++;
    return ((double)(x >> 8) + 1.0) * (1.0 / 16777216.0);
}

double or_uniform_from_word(uint32_t x) { return ((double)(x >> 8) + 1.0) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------ model description */
typedef struct {
    int32_t gtype;            /* 0 cartesian (x,y,z); 1 spherical-polar (r, theta, phi);
                                 2 cylindrical-polar (R, z, phi) */
    int32_t n[3];             /* cells per axis */
    const double* w[3];       /* walls per axis: cm, or rad for theta and phi */
    const double* rho;        /* [n3][n2][n1] g/cm^3 */
    /* dust */
    int32_t nnu;
    const double* nu;         /* increasing */
    const double* chi;        /* mass extinction, cm^2/g */
    const double* albedo;
    double g;                 /* HG asymmetry */
    /* re-emission */
    int32_t nT;
    const double* cdf_emit;   /* [nT][nnu] cumulative emissivity per temperature node */
    const int32_t* emit_row;  /* [Ncells] row of cdf_emit for each cell (previous T) */
    /* sources: point sources first, optional cell source last */
    int32_t npoint;
    const double* src_pos;    /* [npoint][3] cm */
    int32_t nsrc;             /* npoint + (cell source ? 1 : 0) */
    const double* src_cdf;    /* [nsrc] cumulative luminosity fraction, last = 1 */
    int32_t nspec;
    const double* spec_nu;    /* [nspec] source spectrum frequency nodes */
    const double* spec_cdf;   /* [nsrc][nspec] */
    const double* cell_cdf;   /* [Ncells] cumulative cell luminosity (cell source), or NULL */
    /* observers and output bins */
    int32_t nobs;
    const double* obs_n;      /* [nobs][3] unit vectors to the observer */
    const double* obs_ex;     /* [nobs][3] sky-plane x axis */
    const double* obs_ey;     /* [nobs][3] sky-plane y axis */
    int32_t nsed;
    double lam_min, lam_max;  /* cm */
    int32_t img_nx, img_ny, nimg;
    double img_half;          /* cm */
    const int32_t* img_bin;   /* [nimg] SED bin of each image wavelength */
    /* external isotropic sources (after the point sources in the source list, before a cell
     * source): spheres of centre ext_c and radius ext_R emitting inwards */
    int32_t next;
    const double* ext_c;      /* [next][3] cm */
    const double* ext_R;      /* [next] cm */
    double L0;                /* grid scale (cm): the entry nudge of external packets is 1e-6 L0 */
    /* modified random walk (used when or_params.mrw_gamma > 0), per cell at the temperatures the
     * pass started from */
    const double* mrw_k;      /* [Ncells] rho chi_tR(T): inverse transport mean free path (cm^-1) */
    const double* mrw_kp;     /* [Ncells] Planck-mean absorption coefficient kappa_P(T) (cm^2/g) */
} or_model;

typedef struct {
    int64_t n_packets;
    int64_t first_packet;     /* packet ids first_packet .. first_packet + n_packets - 1 */
    uint32_t key[2];
    uint32_t iter_key;
    uint32_t model_key;
    double eps;               /* packet energy (erg), L_tot * dt / N_total */
    int64_t max_interactions;
    int32_t peel;
    int32_t terminate_on_absorb;
    int32_t nthreads;
    int32_t raytrace;         /* 1: point-source emission and dust re-emission reach the SEDs and
                                 images by raytracing (Sect. 2.6.3), so they are not peeled off */
    double mrw_gamma;         /* > 0: modified random walk where the sphere to the nearest wall is at
                                 least mrw_gamma transport mean free paths in radius (Sect. 2.2) */
} or_params;

typedef struct {
    double* acc;              /* [Ncells] sum of eps kappa l (erg cm^-1 ... per g) */
    double* sed;              /* [nobs][nsed] erg/s/sr per bin */
    double* img;              /* [nobs][nimg][ny][nx] */
    double* esc;              /* [10][nsed] escape photon binning (cos theta bins x SED bins) */
    double e_escaped, e_killed, e_absorbed;
    int64_t n_interactions, n_scatter, n_absorb, n_crossings, n_peel_crossings, n_killed;
    int64_t* visits;          /* [Ncells] packet entries (runs of one packet's consecutive deposits in
                                 the cell): how many packets sampled the cell's estimate (App. A) */
    int64_t n_mrw;            /* modified-random-walk steps */
} or_result;

#define N_ESC_MU 10

static int64_t ncells(const or_model* m) { return (int64_t)m->n[0] * m->n[1] * m->n[2]; }
static int64_t cell_index(const or_model* m, const int c[3]) {
    return ((int64_t)c[2] * m->n[1] + c[1]) * m->n[0] + c[0];
}
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------ dust at a frequency */
/* chi: log-log interpolation between table nodes; albedo: linear in log(nu). */
static void dust_at(const or_model* m, double nu, double* chi, double* albedo) {
    int n = m->nnu;
    int j;
    if (nu <= m->nu[0]) j = 0;
    else if (nu >= m->nu[n - 1]) j = n - 2;
    else {
        int lo = 0, hi = n - 1; /* nu[lo] <= nu < nu[hi] */
        while (hi - lo > 1) {
            int mid = (lo + hi) / 2;
            if (m->nu[mid] <= nu) lo = mid; else hi = mid;
        }
        j = lo;
    }
    double t = log(nu / m->nu[j]) / log(m->nu[j + 1] / m->nu[j]);
    if (t < 0) t = 0;
    if (t > 1) t = 1;
    *chi = exp((1 - t) * log(m->chi[j]) + t * log(m->chi[j + 1]));
    *albedo = (1 - t) * m->albedo[j] + t * m->albedo[j + 1];
}

/* ------------------------------------------------------------------ table sampling */
/* Pick the interval j with cdf[j] < u <= cdf[j+1] (the largest j with cdf[j] < u) and
 * place x linearly inside it: a piecewise-constant pdf on each interval. */
double or_sample_table(int n, const double* x, const double* cdf, double u) {
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (cdf[mid] < u) lo = mid; else hi = mid;
    }
    int j = lo;
    double f = (u - cdf[j]) / (cdf[j + 1] - cdf[j]);
    return x[j] + f * (x[j + 1] - x[j]);
}

/* smallest index s with cdf[s] >= u */
static int64_t select_cdf(int64_t n, const double* cdf, double u) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (cdf[mid] >= u) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* ------------------------------------------------------------------ directions */
void or_isotropic(double u1, double u2, double out[3]) {
    double mu = 2.0 * u1 - 1.0;
    double ph = 2.0 * OR_PI * u2;
    double s = sqrt(fmax(0.0, 1.0 - mu * mu));
    out[0] = s * cos(ph);
    out[1] = s * sin(ph);
    out[2] = mu;
}

/* Henyey-Greenstein: inverse of the cumulative distribution of cos(Theta). */
double or_hg_mu(double g, double u) {
    if (g == 0.0) return 2.0 * u - 1.0;
    double a = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
    double mu = (1.0 + g * g - a * a) / (2.0 * g);
    if (mu > 1) mu = 1;
    if (mu < -1) mu = -1;
    return mu;
}

double or_hg_phase(double g, double mu) {
    double d = 1.0 + g * g - 2.0 * g * mu;
    return (1.0 - g * g) / (4.0 * OR_PI * d * sqrt(d));
}

/* New direction at scattering angle acos(mu) and azimuth psi about u.  Frame: e1 = unit(z x u)
 * unless |u_z| >= 0.99999, then e1 = unit(y x u); e2 = u x e1. */
void or_scatter_dir(const double u[3], double mu, double psi, double out[3]) {
    double e1[3], e2[3];
    if (fabs(u[2]) < 0.99999) {
        e1[0] = -u[1]; e1[1] = u[0]; e1[2] = 0.0;
    } else {
        e1[0] = u[2]; e1[1] = 0.0; e1[2] = -u[0];
    }
    double n1 = sqrt(dot3(e1, e1));
    e1[0] /= n1; e1[1] /= n1; e1[2] /= n1;
    e2[0] = u[1] * e1[2] - u[2] * e1[1];
    e2[1] = u[2] * e1[0] - u[0] * e1[2];
    e2[2] = u[0] * e1[1] - u[1] * e1[0];
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double cp = cos(psi), sp = sin(psi);
    for (int a = 0; a < 3; ++a) out[a] = mu * u[a] + st * (cp * e1[a] + sp * e2[a]);
}

/* ------------------------------------------------------------------ cartesian grid */
/* Cell along one axis holding coordinate x; a point on a wall belongs to the cell the
 * direction points into (u > 0: upper, else lower).  -1 when outside. */
static int locate_axis(const double* w, int n, double x, double u) {
    if (x < w[0] || x > w[n]) return -1;
    int lo = 0, hi = n; /* w[lo] <= x <= w[hi] */
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (w[mid] <= x) lo = mid; else hi = mid;
    }
    int i = lo;
    if (x == w[hi] && hi == n) i = n; /* on the last wall */
    if (x == w[i]) {
        if (!(u > 0)) i = i - 1;
    }
    if (i < 0 || i >= n) return -1;
    return i;
}

static double cart_exit(const or_model* m, const double p[3], const double u[3], const int c[3],
                        int* axis, int* dir) {
    double best = INFINITY;
    *axis = -1;
    *dir = 0;
    for (int a = 0; a < 3; ++a) {
        double d;
        int s;
        if (u[a] > 0) { d = (m->w[a][c[a] + 1] - p[a]) / u[a]; s = 1; }
        else if (u[a] < 0) { d = (m->w[a][c[a]] - p[a]) / u[a]; s = -1; }
        else continue;
        if (d < 0) d = 0;
        if (d < best) { best = d; *axis = a; *dir = s; }
    }
    return best;
}

/* ------------------------------------------------------------------ spherical-polar grid */
static double wrap_phi(double ph) {
    double t = fmod(ph, 2.0 * OR_PI);
    if (t < 0) t += 2.0 * OR_PI;
    return t;
}

/* Direction of travel of r, theta and phi at point p: +1 increasing, -1 decreasing, 0 none. */
static double drds(const double p[3], const double u[3]) { return dot3(p, u); }
static double dthds(const double p[3], const double u[3]) {
    /* theta = acos(z / r) increases when u_z r^2 - z (p.u) < 0 */
    return -(u[2] * dot3(p, p) - p[2] * dot3(p, u));
}
static double dphids(const double p[3], const double u[3]) { return p[0] * u[1] - p[1] * u[0]; }

/* Locate the cell of point p with direction u.  Returns 0 inside the grid, 1 inside the
 * inner hole (r < r_0), -1 outside. */
static int sph_locate(const or_model* m, const double p[3], const double u[3], int c[3]) {
    const double* rw = m->w[0];
    const double* tw = m->w[1];
    const double* pw = m->w[2];
    double r = sqrt(dot3(p, p));
    double th, ph, vt, vp;
    if (r == 0.0) {
        th = acos(fmax(-1.0, fmin(1.0, u[2])));
        ph = wrap_phi(atan2(u[1], u[0]));
        vt = 0.0; vp = 0.0;
        if (rw[0] > 0) { c[0] = -1; }
        else c[0] = 0;
    } else {
        double vr = drds(p, u);
        if (r < rw[0] || (r == rw[0] && !(vr > 0))) c[0] = -1;
        else {
            int i = locate_axis(rw, m->n[0], r, vr);
            if (i < 0) return -1;
            c[0] = i;
        }
        th = acos(fmax(-1.0, fmin(1.0, p[2] / r)));
        double R = sqrt(p[0] * p[0] + p[1] * p[1]);
        if (R == 0.0) { ph = wrap_phi(atan2(u[1], u[0])); vp = 0.0; }
        else { ph = wrap_phi(atan2(p[1], p[0])); vp = dphids(p, u); }
        vt = dthds(p, u);
    }
    int j = locate_axis(tw, m->n[1], th, vt);
    if (j < 0) j = (th <= tw[0]) ? 0 : m->n[1] - 1;
    c[1] = j;
    int k;
    if (m->n[2] == 1) k = 0;
    else {
        if (ph == 0.0 && !(vp > 0)) k = m->n[2] - 1;
        else {
            k = locate_axis(pw, m->n[2], ph, vp);
            if (k < 0) k = m->n[2] - 1;
        }
    }
    c[2] = k;
    return c[0] < 0 ? 1 : 0;
}

/* Smallest admissible root of the cone theta_w crossing in the given sense.
 * The cone is z sin(theta_w) - R cos(theta_w) = 0 (R the cylindrical radius); squared, it
 * is A s^2 + 2 B s + C = 0.  A root is admissible when it lies on the cone's own nappe
 * and f = z sin - R cos changes with the required sign there (sense = +1: f increasing,
 * i.e. theta decreasing through the wall; -1: theta increasing). */
static double cone_root(const double p[3], const double u[3], double th_w, int sense, double tol) {
    double cw = cos(th_w), sw = sin(th_w);
    if (fabs(cw) < 1e-12) { /* the plane z = 0 */
        if (u[2] == 0.0) return INFINITY;
        /* f = z: increasing when u_z > 0 */
        if ((sense > 0) != (u[2] > 0)) return INFINITY;
        double s = -p[2] / u[2];
        return s < -tol ? INFINITY : fmax(s, 0.0);
    }
    double uR2 = u[0] * u[0] + u[1] * u[1];
    double pu = p[0] * u[0] + p[1] * u[1];
    double R2 = p[0] * p[0] + p[1] * p[1];
    double A = u[2] * u[2] * sw * sw - uR2 * cw * cw;
    double B = p[2] * u[2] * sw * sw - pu * cw * cw;
    double C = p[2] * p[2] * sw * sw - R2 * cw * cw;
    double roots[2];
    int nr = 0;
    if (fabs(A) < 1e-300) {
        if (B != 0.0) roots[nr++] = -C / (2.0 * B);
    } else {
        double disc = B * B - A * C;
        if (disc < 0) return INFINITY;
        double sq = sqrt(disc);
        roots[nr++] = (-B - sq) / A;
        roots[nr++] = (-B + sq) / A;
    }
    double best = INFINITY;
    for (int t = 0; t < nr; ++t) {
        double s = roots[t];
        if (!(s >= -tol)) continue;
        double q[3] = {p[0] + s * u[0], p[1] + s * u[1], p[2] + s * u[2]};
        if (!(q[2] * cw > 0)) continue;           /* other nappe (or apex) */
        double Rq = sqrt(q[0] * q[0] + q[1] * q[1]);
        if (Rq == 0.0) continue;
        double dfds = u[2] * sw - cw * (q[0] * u[0] + q[1] * u[1]) / Rq;
        if (sense > 0 ? !(dfds > 0) : !(dfds < 0)) continue;
        double sc = fmax(s, 0.0);
        if (sc < best) best = sc;
    }
    return best;
}

/* Half-plane phi_w = {(cos phi_w, sin phi_w) . (x, y) > 0, (-sin phi_w, cos phi_w) . (x,y) = 0}
 * crossed in the given sense (+1: phi increasing, -1 decreasing). */
static double phi_root(const double p[3], const double u[3], double ph_w, int sense, double tol) {
    double nx = -sin(ph_w), ny = cos(ph_w);
    double nu_ = nx * u[0] + ny * u[1];
    if (nu_ == 0.0) return INFINITY;
    if ((sense > 0) != (nu_ > 0)) return INFINITY;
    double s = -(nx * p[0] + ny * p[1]) / nu_;
    if (!(s >= -tol)) return INFINITY;
    double qx = p[0] + s * u[0], qy = p[1] + s * u[1];
    if (!(cos(ph_w) * qx + sin(ph_w) * qy > 0)) return INFINITY;
    return fmax(s, 0.0);
}

static double sph_exit(const or_model* m, const double p[3], const double u[3], const int c[3],
                       int* axis, int* dir) {
    const double* rw = m->w[0];
    const double* tw = m->w[1];
    const double* pw = m->w[2];
    double rr = dot3(p, p);
    double b = dot3(p, u);
    double tol = 1e-9 * rw[m->n[0]];
    double best;
    /* outer sphere: the larger root, always ahead of a point inside */
    {
        double R = rw[c[0] + 1];
        double cc = rr - R * R;
        double disc = b * b - cc;
        double s = -b + sqrt(fmax(disc, 0.0));
        best = fmax(s, 0.0);
        *axis = 0;
        *dir = 1;
    }
    /* inner sphere, entered only while moving inwards */
    if (rw[c[0]] > 0 && b < 0) {
        double R = rw[c[0]];
        double cc = rr - R * R;
        double disc = b * b - cc;
        if (disc >= 0) {
            double s = cc / (-b + sqrt(disc));
            s = fmax(s, 0.0);
            if (s < best) { best = s; *axis = 0; *dir = -1; }
        }
    }
    /* cones: lower wall left with theta decreasing, upper wall with theta increasing */
    if (c[1] > 0) {
        double s = cone_root(p, u, tw[c[1]], +1, tol);
        if (s < best) { best = s; *axis = 1; *dir = -1; }
    }
    if (c[1] + 1 < m->n[1]) {
        double s = cone_root(p, u, tw[c[1] + 1], -1, tol);
        if (s < best) { best = s; *axis = 1; *dir = 1; }
    }
    /* azimuthal half-planes */
    if (m->n[2] > 1) {
        double s = phi_root(p, u, pw[c[2]], -1, tol);
        if (s < best) { best = s; *axis = 2; *dir = -1; }
        s = phi_root(p, u, pw[c[2] + 1], +1, tol);
        if (s < best) { best = s; *axis = 2; *dir = 1; }
    }
    return best;
}

/* Cross the inner vacuum hole: from a point on (or inside) the sphere r_0 to the far side. */
static void sph_cross_hole(const or_model* m, double p[3], const double u[3], int c[3]) {
    double r0 = m->w[0][0];
    double b = dot3(p, u);
    double cc = dot3(p, p) - r0 * r0;
    double s = -b + sqrt(fmax(b * b - cc, 0.0));
    if (s < 0) s = 0;
    for (int a = 0; a < 3; ++a) p[a] += s * u[a];
    /* on the sphere r_0, moving outwards */
    int cc3[3];
    sph_locate(m, p, u, cc3);
    c[0] = 0;
    c[1] = cc3[1];
    c[2] = cc3[2];
}

/* ------------------------------------------------------------------ cylindrical-polar grid */
/* Walls: cylinders R_i about the z axis (R_0 > 0: an inner vacuum hole), planes z_j and
 * half-planes phi_k.  Index order [phi][z][R]. */
static int cyl_locate(const or_model* m, const double p[3], const double u[3], int c[3]) {
    const double* Rw = m->w[0];
    double R = sqrt(p[0] * p[0] + p[1] * p[1]);
    double vR = p[0] * u[0] + p[1] * u[1];
    int j = locate_axis(m->w[1], m->n[1], p[2], u[2]);
    if (j < 0) return -1;
    c[1] = j;
    double ph, vp;
    if (R == 0.0) { ph = wrap_phi(atan2(u[1], u[0])); vp = 0.0; }
    else { ph = wrap_phi(atan2(p[1], p[0])); vp = dphids(p, u); }
    int k;
    if (m->n[2] == 1) k = 0;
    else if (ph == 0.0 && !(vp > 0)) k = m->n[2] - 1;
    else {
        k = locate_axis(m->w[2], m->n[2], ph, vp);
        if (k < 0) k = m->n[2] - 1;
    }
    c[2] = k;
    if (R < Rw[0] || (R == Rw[0] && Rw[0] > 0 && !(vR > 0))) { c[0] = -1; return 1; }
    /* without a hole the axis R = 0 lies inside the innermost ring (it is not a wall) */
    int i = (R == 0.0 && Rw[0] == 0.0) ? 0 : locate_axis(Rw, m->n[0], R, vR);
    if (i < 0) return -1;
    c[0] = i;
    return 0;
}

static double cyl_exit(const or_model* m, const double p[3], const double u[3], const int c[3],
                       int* axis, int* dir) {
    const double* Rw = m->w[0];
    const double* zw = m->w[1];
    const double* pw = m->w[2];
    double a = u[0] * u[0] + u[1] * u[1];
    double b = p[0] * u[0] + p[1] * u[1];
    double R2 = p[0] * p[0] + p[1] * p[1];
    double tol = 1e-9 * Rw[m->n[0]];
    double best = INFINITY;
    *axis = -1;
    *dir = 0;
    if (a > 0) {
        /* outer cylinder: the far root, always ahead of a point inside (a s^2 + 2 b s + cc = 0) */
        double cc = R2 - Rw[c[0] + 1] * Rw[c[0] + 1];
        double sq = sqrt(fmax(b * b - a * cc, 0.0));
        double s = b > 0 ? -cc / (b + sq) : (-b + sq) / a;
        best = fmax(s, 0.0);
        *axis = 0;
        *dir = 1;
        /* inner cylinder, entered only while moving inwards */
        if (Rw[c[0]] > 0 && b < 0) {
            double ci = R2 - Rw[c[0]] * Rw[c[0]];
            double disc = b * b - a * ci;
            if (disc >= 0) {
                double si = fmax(ci / (-b + sqrt(disc)), 0.0);
                if (si < best) { best = si; *dir = -1; }
            }
        }
    }
    /* z planes */
    if (u[2] != 0) {
        double s = u[2] > 0 ? (zw[c[1] + 1] - p[2]) / u[2] : (zw[c[1]] - p[2]) / u[2];
        s = fmax(s, 0.0);
        if (s < best) { best = s; *axis = 1; *dir = u[2] > 0 ? 1 : -1; }
    }
    if (m->n[2] > 1) {
        double s = phi_root(p, u, pw[c[2]], -1, tol);
        if (s < best) { best = s; *axis = 2; *dir = -1; }
        s = phi_root(p, u, pw[c[2] + 1], +1, tol);
        if (s < best) { best = s; *axis = 2; *dir = 1; }
    }
    return best;
}

/* Cross the inner vacuum cylinder to its far side; returns 1 when the ray leaves the grid
 * through a z plane on the way (or runs along the axis), 0 with c set in the shell R_0. */
static int cyl_cross_hole(const or_model* m, double p[3], const double u[3], int c[3]) {
    double a = u[0] * u[0] + u[1] * u[1];
    if (!(a > 0)) return 1;
    double R0 = m->w[0][0];
    double b = p[0] * u[0] + p[1] * u[1];
    double cc = p[0] * p[0] + p[1] * p[1] - R0 * R0;
    double sq = sqrt(fmax(b * b - a * cc, 0.0));
    double s = b > 0 ? -cc / (b + sq) : (-b + sq) / a;
    if (s < 0) s = 0;
    for (int q = 0; q < 3; ++q) p[q] += s * u[q];
    int c3[3];
    if (cyl_locate(m, p, u, c3) < 0) return 1;
    c[0] = 0;
    c[1] = c3[1];
    c[2] = c3[2];
    return 0;
}

/* ------------------------------------------------------------------ generic grid API */
/* 0 inside, -1 outside.  Spherical points in the hole are moved through it. */
static int grid_locate(const or_model* m, double p[3], const double u[3], int c[3]) {
    if (m->gtype == 0) {
        for (int a = 0; a < 3; ++a) {
            c[a] = locate_axis(m->w[a], m->n[a], p[a], u[a]);
            if (c[a] < 0) return -1;
        }
        return 0;
    }
    if (m->gtype == 2) {
        int st = cyl_locate(m, p, u, c);
        if (st < 0) return -1;
        if (st == 1 && cyl_cross_hole(m, p, u, c)) return -1;
        return 0;
    }
    int st = sph_locate(m, p, u, c);
    if (st < 0) return -1;
    if (st == 1) {
        /* inside the hole: travel to the sphere r_0 */
        double r0 = m->w[0][0];
        double b = dot3(p, u);
        double cc = dot3(p, p) - r0 * r0;
        double s = -b + sqrt(fmax(b * b - cc, 0.0));
        for (int a = 0; a < 3; ++a) p[a] += s * u[a];
        int c3[3];
        sph_locate(m, p, u, c3);
        c[0] = 0; c[1] = c3[1]; c[2] = c3[2];
    }
    return 0;
}

static double grid_exit(const or_model* m, const double p[3], const double u[3], const int c[3],
                        int* axis, int* dir) {
    if (m->gtype == 2) return cyl_exit(m, p, u, c, axis, dir);
    return m->gtype == 0 ? cart_exit(m, p, u, c, axis, dir) : sph_exit(m, p, u, c, axis, dir);
}

/* Move the cell index across the wall found by grid_exit.  Returns 1 on escape. */
static int grid_step(const or_model* m, double p[3], const double u[3], int c[3], int axis, int dir) {
    c[axis] += dir;
    if (m->gtype == 0) return (c[axis] < 0 || c[axis] >= m->n[axis]) ? 1 : 0;
    if (m->gtype == 2) {
        if (axis == 0) {
            if (c[0] >= m->n[0]) return 1;
            if (c[0] < 0) return cyl_cross_hole(m, p, u, c);
            return 0;
        }
        if (axis == 1) return (c[1] < 0 || c[1] >= m->n[1]) ? 1 : 0;
        if (c[2] < 0) c[2] += m->n[2];
        if (c[2] >= m->n[2]) c[2] -= m->n[2];
        return 0;
    }
    if (axis == 0) {
        if (c[0] >= m->n[0]) return 1;
        if (c[0] < 0) sph_cross_hole(m, p, u, c);
        return 0;
    }
    if (axis == 2) {
        if (c[2] < 0) c[2] += m->n[2];
        if (c[2] >= m->n[2]) c[2] -= m->n[2];
    }
    return 0;
}

/* ------------------------------------------------------------------ exported single steps */
/* Distance to the exit of cell c along u, with the crossed axis and sense. */
double or_cell_exit(const or_model* m, const double p[3], const double u[3], const int32_t c[3],
                    int32_t* axis, int32_t* dir) {
    int ci[3] = {c[0], c[1], c[2]}, a, d;
    double s = grid_exit(m, p, u, ci, &a, &d);
    *axis = a;
    *dir = d;
    return s;
}

int or_locate(const or_model* m, const double p_in[3], const double u[3], double p_out[3], int32_t c[3]) {
    double p[3] = {p_in[0], p_in[1], p_in[2]};
    int ci[3];
    int st = grid_locate(m, p, u, ci);
    for (int a = 0; a < 3; ++a) { c[a] = ci[a]; p_out[a] = p[a]; }
    return st;
}

/* Walk a ray from p (cell located with u) to the grid boundary, recording every segment
 * (cell index, length).  Returns the number of segments (<= maxseg), -1 if p is outside. */
int64_t or_trace(const or_model* m, const double p_in[3], const double u[3], int64_t maxseg,
                 int64_t* seg_cell, double* seg_len) {
    double p[3] = {p_in[0], p_in[1], p_in[2]};
    int c[3];
    if (grid_locate(m, p, u, c) < 0) return -1;
    int64_t n = 0;
    for (;;) {
        int axis, dir;
        double l = grid_exit(m, p, u, c, &axis, &dir);
        if (n < maxseg) { seg_cell[n] = cell_index(m, c); seg_len[n] = l; }
        n++;
        for (int a = 0; a < 3; ++a) p[a] += l * u[a];
        if (grid_step(m, p, u, c, axis, dir)) break;
        if (n > 100000000) break;
    }
    return n;
}

/* ------------------------------------------------------------------ packet walks */
/* Propagate to optical depth tau (extinction) or escape, depositing eps*kappa*l per segment
 * into cells holding dust.  Returns 1 on escape, 0 at an interaction point. */
/* Walk to optical depth tau; *run is the cell of the packet's current run of deposits (-1 at
 * emission): a deposit in another cell starts a new run, one packet entry of that cell. */
static int walk_to_tau(const or_model* m, double p[3], const double u[3], int c[3], double tau,
                       double chi_nu, double dep, double* acc, int64_t* visits, int64_t* run, int64_t* ncross) {
    for (;;) {
        int64_t ci = cell_index(m, c);
        int axis, dir;
        double l = grid_exit(m, p, u, c, &axis, &dir);
        double rho = m->rho[ci];
        double dtau = rho * chi_nu * l;
        if (tau < dtau) {
            double lp = tau / (rho * chi_nu);
            acc[ci] += dep * lp;
            if (*run != ci) { visits[ci]++; *run = ci; }
            for (int a = 0; a < 3; ++a) p[a] += lp * u[a];
            return 0;
        }
        if (rho > 0) {
            acc[ci] += dep * l;
            if (*run != ci) { visits[ci]++; *run = ci; }
        }
        tau -= dtau;
        for (int a = 0; a < 3; ++a) p[a] += l * u[a];
        (*ncross)++;
        if (grid_step(m, p, u, c, axis, dir)) return 1;
    }
}

/* Extinction optical depth from p (in cell c) to the boundary along u. */
static double tau_to_edge(const or_model* m, const double p0[3], const double u[3], const int c0[3],
                          double chi_nu, int64_t* ncross) {
    double p[3] = {p0[0], p0[1], p0[2]};
    int c[3] = {c0[0], c0[1], c0[2]};
    double tau = 0.0;
    for (;;) {
        int64_t ci = cell_index(m, c);
        int axis, dir;
        double l = grid_exit(m, p, u, c, &axis, &dir);
        tau += m->rho[ci] * chi_nu * l;
        for (int a = 0; a < 3; ++a) p[a] += l * u[a];
        (*ncross)++;
        if (grid_step(m, p, u, c, axis, dir)) return tau;
    }
}

double or_tau_to_edge(const or_model* m, const double p[3], const double u[3], double chi_nu) {
    double q[3] = {p[0], p[1], p[2]};
    int c[3];
    int64_t nc = 0;
    if (grid_locate(m, q, u, c) < 0) return 0.0;
    return tau_to_edge(m, q, u, c, chi_nu, &nc);
}

static int sed_bin(const or_model* m, double nu) {
    double lam = OR_C_LIGHT / nu;
    if (lam < m->lam_min || lam >= m->lam_max) return -1;
    int b = (int)floor(m->nsed * log(lam / m->lam_min) / log(m->lam_max / m->lam_min));
    if (b < 0 || b >= m->nsed) return -1;
    return b;
}

int or_sed_bin(const or_model* m, double nu) { return sed_bin(m, nu); }

enum { PEEL_EMIT = 0, PEEL_SCATTER = 1, PEEL_REEMIT = 2 };

/* Peeling-off (Sect. 2.6.2): weight eps * p * exp(-tau_obs) towards every observer. */
static void peel(const or_model* m, const double p[3], const int c[3], const double uin[3], double nu,
                 double eps, int kind, or_result* R) {
    int b = sed_bin(m, nu);
    if (b < 0) return;
    double chi, alb;
    dust_at(m, nu, &chi, &alb);
    for (int o = 0; o < m->nobs; ++o) {
        const double* n = m->obs_n + 3 * o;
        double prob = (kind == PEEL_SCATTER) ? or_hg_phase(m->g, dot3(uin, n)) : 1.0 / (4.0 * OR_PI);
        double tau;
        if (kind == PEEL_EMIT) {
            double q[3] = {p[0], p[1], p[2]};
            int cq[3];
            if (grid_locate(m, q, n, cq) < 0) tau = 0.0;
            else tau = tau_to_edge(m, q, n, cq, chi, &R->n_peel_crossings);
        } else {
            tau = tau_to_edge(m, p, n, c, chi, &R->n_peel_crossings);
        }
        double w = eps * prob * exp(-tau);
        R->sed[(int64_t)o * m->nsed + b] += w;
        if (m->nimg > 0) {
            const double* ex = m->obs_ex + 3 * o;
            const double* ey = m->obs_ey + 3 * o;
            double px = dot3(p, ex), py = dot3(p, ey);
            int ix = (int)floor((px + m->img_half) / (2.0 * m->img_half) * m->img_nx);
            int iy = (int)floor((py + m->img_half) / (2.0 * m->img_half) * m->img_ny);
            if (ix >= 0 && ix < m->img_nx && iy >= 0 && iy < m->img_ny) {
                for (int l = 0; l < m->nimg; ++l) {
                    if (m->img_bin[l] != b) continue;
                    int64_t off = (((int64_t)o * m->nimg + l) * m->img_ny + iy) * m->img_nx + ix;
                    R->img[off] += w;
                }
            }
        }
    }
}

/* A point uniform in the volume of cell c from three uniforms (Cartesian: each coordinate;
 * spherical: r^3, cos(theta), phi uniform; cylindrical: R^2, z, phi uniform). */
static void place_in_cell(const or_model* m, const int c[3], double f0, double f1, double f2, double p[3]) {
    if (m->gtype == 0) {
        double f[3] = {f0, f1, f2};
        for (int a = 0; a < 3; ++a) p[a] = m->w[a][c[a]] + f[a] * (m->w[a][c[a] + 1] - m->w[a][c[a]]);
    } else if (m->gtype == 1) {
        double r0 = m->w[0][c[0]], r1 = m->w[0][c[0] + 1];
        double r = cbrt(r0 * r0 * r0 + f0 * (r1 * r1 * r1 - r0 * r0 * r0));
        double ct0 = cos(m->w[1][c[1]]), ct1 = cos(m->w[1][c[1] + 1]);
        double ct = ct0 + f1 * (ct1 - ct0);
        double ph = m->w[2][c[2]] + f2 * (m->w[2][c[2] + 1] - m->w[2][c[2]]);
        double st = sqrt(fmax(0.0, 1.0 - ct * ct));
        p[0] = r * st * cos(ph); p[1] = r * st * sin(ph); p[2] = r * ct;
    } else {
        double R0 = m->w[0][c[0]], R1 = m->w[0][c[0] + 1];
        double R = sqrt(R0 * R0 + f0 * (R1 * R1 - R0 * R0));
        double z = m->w[1][c[1]] + f1 * (m->w[1][c[1] + 1] - m->w[1][c[1]]);
        double ph = m->w[2][c[2]] + f2 * (m->w[2][c[2] + 1] - m->w[2][c[2]]);
        p[0] = R * cos(ph); p[1] = R * sin(ph); p[2] = z;
    }
}

/* Test hook: the point place_in_cell gives for cell c[3] and fractions f[3] in (0, 1]. */
void or_place_in_cell(const or_model* m, const int32_t c[3], const double f[3], double p[3]) {
    int ci[3] = {c[0], c[1], c[2]};
    place_in_cell(m, ci, f[0], f[1], f[2], p);
}

/* Parameter t >= 0 at which the ray p + t u first enters the grid's outer boundary (0 when p is
 * already inside), or -1 when it misses the grid. */
static double grid_entry(const or_model* m, const double p[3], const double u[3]) {
    double tmin = -INFINITY, tmax = INFINITY;
    if (m->gtype == 1) {
        double ro = m->w[0][m->n[0]];
        double b = dot3(p, u), c = dot3(p, p) - ro * ro;
        if (c <= 0) return 0.0;
        double disc = b * b - c;
        if (disc < 0 || b >= 0) return -1.0;
        return c / (-b + sqrt(disc));
    }
    if (m->gtype == 0) {
        for (int a = 0; a < 3; ++a) {
            double lo = m->w[a][0], hi = m->w[a][m->n[a]];
            if (u[a] == 0) {
                if (p[a] < lo || p[a] > hi) return -1.0;
                continue;
            }
            double t1 = (lo - p[a]) / u[a], t2 = (hi - p[a]) / u[a];
            tmin = fmax(tmin, fmin(t1, t2));
            tmax = fmin(tmax, fmax(t1, t2));
        }
    } else {
        double Ro = m->w[0][m->n[0]];
        double a = u[0] * u[0] + u[1] * u[1];
        double b = p[0] * u[0] + p[1] * u[1];
        double c = p[0] * p[0] + p[1] * p[1] - Ro * Ro;
        if (a == 0) {
            if (c > 0) return -1.0;
        } else {
            double disc = b * b - a * c;
            if (disc < 0) return -1.0;
            double sq = sqrt(disc);
            tmin = (-b - sq) / a;
            tmax = (-b + sq) / a;
        }
        double lo = m->w[1][0], hi = m->w[1][m->n[1]];
        if (u[2] == 0) {
            if (p[2] < lo || p[2] > hi) return -1.0;
        } else {
            double t1 = (lo - p[2]) / u[2], t2 = (hi - p[2]) / u[2];
            tmin = fmax(tmin, fmin(t1, t2));
            tmax = fmin(tmax, fmax(t1, t2));
        }
    }
    if (tmax < fmax(tmin, 0.0)) return -1.0;
    return fmax(tmin, 0.0);
}

/* ------------------------------------------------------------------ raytracing (Sect. 2.6.3) */
/* Dust-emission rays: ray k draws from its own Philox stream (key, counter (draw/4, k, iter_key,
 * model)): u0 picks the cell from the cumulative emitted luminosity cdf_L (smallest index with
 * cdf >= u0), u1..u3 place it uniformly in the cell's volume (as a cell source).  For every
 * observer the column sum rho l from that point to the grid edge is returned (chi = 1). */
int or_raytrace_rays(const or_model* m, const or_params* P, int64_t n_rays, const double* cdf_L,
                     int64_t* cells, double* pos, double* col) {
    for (int64_t k = 0; k < n_rays; ++k) {
        rng_t rng;
        memset(&rng, 0, sizeof(rng));
        rng.key[0] = P->key[0];
        rng.key[1] = P->key[1];
        rng.pkt = (uint32_t)k;
        rng.iter = P->iter_key;
        rng.model = P->model_key;
        int64_t ci = select_cdf(ncells(m), cdf_L, uniform(&rng));
        int c[3];
        c[0] = (int)(ci % m->n[0]);
        c[1] = (int)((ci / m->n[0]) % m->n[1]);
        c[2] = (int)(ci / ((int64_t)m->n[0] * m->n[1]));
        double f0 = uniform(&rng), f1 = uniform(&rng), f2 = uniform(&rng);
        double p[3];
        place_in_cell(m, c, f0, f1, f2, p);
        cells[k] = ci;
        for (int a = 0; a < 3; ++a) pos[3 * k + a] = p[a];
        for (int o = 0; o < m->nobs; ++o) {
            int64_t nc = 0;
            int cc[3] = {c[0], c[1], c[2]};
            col[k * m->nobs + o] = tau_to_edge(m, p, m->obs_n + 3 * o, cc, 1.0, &nc);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ modified random walk
 * Sect. 2.2: deep inside a cell of large optical depth, a packet crosses a sphere that lies
 * inside the cell in one step from the diffusion approximation, instead of the many
 * absorptions and scatterings it would take there.  The paper states the idea and refers to its
 * published form (Min et al. 2009, with the variant of Robitaille 2010); what the steps below
 * compute is that form:
 *   a packet starting at the centre of a sphere of radius R0 with constant density, diffusing
 *   with coefficient D = 1 / (3 rho chi) per unit path length, is still inside after path length
 *   s with probability P(s) = 2 sum_{n>=1} (-1)^{n+1} exp(-n^2 pi^2 D s / R0^2);
 *   s is drawn from P, the packet deposits eps kappa_P s (Eq. 2 with the Planck-mean absorption
 *   coefficient of the thermalised field) and leaves from a point uniform on the sphere,
 *   re-emitted isotropically with a frequency from the cell's emissivity row.
 * chi is the Rosseland mean of the transport extinction chi_nu (1 - albedo g), the
 * diffusion coefficient of anisotropically scattering dust. */

#define MRW_SHRINK 0.99      /* sphere radius / distance to the nearest wall */
#define MRW_POLE_TOL 1e-12   /* theta walls within this of 0 or pi are the polar axis */

/* Distance from p (inside cell c) to the nearest wall bounding c: planes of a Cartesian cell;
 * spheres, cones and half-planes of a spherical-polar cell; cylinders, planes and half-planes of
 * a cylindrical cell.  The polar axis (theta = 0 or pi), r = 0 and R = 0 bound nothing (the
 * cell continues through them), nor do the phi walls of a grid with a single phi cell.  The
 * distance to a cone or half-plane is r sin(angle) within a quarter turn, else the distance to
 * its edge (the origin or the axis). */
double or_wall_distance(const or_model* m, const double p[3], const int32_t c[3]) {
    double d = INFINITY;
    if (m->gtype == 0) {
        for (int a = 0; a < 3; ++a) {
            d = fmin(d, p[a] - m->w[a][c[a]]);
            d = fmin(d, m->w[a][c[a] + 1] - p[a]);
        }
        return d;
    }
    const double R = sqrt(p[0] * p[0] + p[1] * p[1]);
    if (m->n[2] > 1) {
        const double ph = wrap_phi(atan2(p[1], p[0]));
        const double a1 = fabs(ph - m->w[2][c[2]]), a2 = fabs(m->w[2][c[2] + 1] - ph);
        d = fmin(d, a1 < 0.5 * OR_PI ? R * sin(a1) : R);
        d = fmin(d, a2 < 0.5 * OR_PI ? R * sin(a2) : R);
    }
    const double lo = m->w[0][c[0]], hi = m->w[0][c[0] + 1];
    if (m->gtype == 1) {
        const double r = sqrt(dot3(p, p));
        if (lo > 0) d = fmin(d, r - lo);
        d = fmin(d, hi - r);
        const double th = atan2(R, p[2]);
        const double t0 = m->w[1][c[1]], t1 = m->w[1][c[1] + 1];
        if (t0 > MRW_POLE_TOL) {
            const double a = fabs(th - t0);
            d = fmin(d, a < 0.5 * OR_PI ? r * sin(a) : r);
        }
        if (t1 < OR_PI - MRW_POLE_TOL) {
            const double a = fabs(t1 - th);
            d = fmin(d, a < 0.5 * OR_PI ? r * sin(a) : r);
        }
    } else {
        if (lo > 0) d = fmin(d, R - lo);
        d = fmin(d, hi - R);
        d = fmin(d, p[2] - m->w[1][c[1]]);
        d = fmin(d, m->w[1][c[1] + 1] - p[2]);
    }
    return d;
}

/* P at x = pi^2 D s / R0^2: the alternating series summed until its terms are negligible. */
static double mrw_survival(double x) {
    if (!(x > 0)) return 1.0;
    double sum = 0.0;
    for (int n = 1;; ++n) {
        const double t = exp(-(double)n * (double)n * x);
        sum += (n & 1) ? t : -t;
        if (t < 1e-20) break;
    }
    return 2.0 * sum;
}

/* Path length s / R0 at which P(s) = zeta, for a sphere of tau0 = rho chi R0 transport mean free
 * paths in radius (bisection on x; s = 3 tau0 R0 x / pi^2).  zeta = 1 gives 0. */
double or_mrw_path(double tau0, double zeta) {
    if (zeta >= 1.0) return 0.0;
    double lo = 0.0, hi = 1.0;
    while (mrw_survival(hi) > zeta) hi *= 2.0;
    for (int k = 0; k < 200 && hi - lo > 1e-16 * hi; ++k) {
        const double mid = 0.5 * (lo + hi);
        if (mrw_survival(mid) > zeta) lo = mid; else hi = mid;
    }
    return 3.0 * tau0 * (0.5 * (lo + hi)) / (OR_PI * OR_PI);
}

/* ------------------------------------------------------------------ one packet history */
static void run_packet(const or_model* m, const or_params* P, int64_t pid, or_result* R) {
    rng_t rng;
    memset(&rng, 0, sizeof(rng));
    rng.key[0] = P->key[0];
    rng.key[1] = P->key[1];
    rng.pkt = (uint32_t)pid;
    rng.iter = P->iter_key;
    rng.model = P->model_key;
    double eps = P->eps;

    /* emission (Sect. 2.2, 2.1.1) */
    double p[3], u[3], nu;
    int c[3];
    int64_t run = -1;      /* cell of the packet's current run of deposits */
    int s = (int)select_cdf(m->nsrc, m->src_cdf, uniform(&rng));
    if (s < m->npoint) {
        p[0] = m->src_pos[3 * s]; p[1] = m->src_pos[3 * s + 1]; p[2] = m->src_pos[3 * s + 2];
        double u1 = uniform(&rng), u2 = uniform(&rng);
        or_isotropic(u1, u2, u);
        nu = or_sample_table(m->nspec, m->spec_nu, m->spec_cdf + (int64_t)s * m->nspec, uniform(&rng));
        double p0[3] = {p[0], p[1], p[2]};
        if (grid_locate(m, p, u, c) < 0) { R->e_escaped += eps; return; }
        if (P->peel && !P->raytrace) peel(m, p0, c, u, nu, eps, PEEL_EMIT, R);
    } else if (s < m->npoint + m->next) {
        /* external isotropic source (Sect. 2.1.1): a point uniform on the sphere, a direction
         * into it with the cosine-weighted (isotropic-intensity) distribution about the inward
         * normal, cos = sqrt(u), in the fixed frame of the normal; no peel-off (background) */
        int e = s - m->npoint;
        double nh[3], u1 = uniform(&rng), u2 = uniform(&rng);
        or_isotropic(u1, u2, nh);
        for (int a = 0; a < 3; ++a) p[a] = m->ext_c[3 * e + a] + m->ext_R[e] * nh[a];
        double u3 = uniform(&rng), u4 = uniform(&rng);
        double e1[3], e2[3];
        if (fabs(nh[2]) < 0.99999) { e1[0] = -nh[1]; e1[1] = nh[0]; e1[2] = 0.0; }
        else { e1[0] = nh[2]; e1[1] = 0.0; e1[2] = -nh[0]; }
        double n1 = sqrt(dot3(e1, e1));
        for (int a = 0; a < 3; ++a) e1[a] /= n1;
        e2[0] = nh[1] * e1[2] - nh[2] * e1[1];
        e2[1] = nh[2] * e1[0] - nh[0] * e1[2];
        e2[2] = nh[0] * e1[1] - nh[1] * e1[0];
        double ct = sqrt(u3), st = sqrt(1.0 - u3), cp = cos(2.0 * OR_PI * u4), sp = sin(2.0 * OR_PI * u4);
        for (int a = 0; a < 3; ++a) u[a] = -ct * nh[a] + st * (cp * e1[a] + sp * e2[a]);
        double un = sqrt(dot3(u, u));
        for (int a = 0; a < 3; ++a) u[a] /= un;
        nu = or_sample_table(m->nspec, m->spec_nu, m->spec_cdf + (int64_t)s * m->nspec, uniform(&rng));
        /* travel through vacuum to the grid; a packet that misses it escapes */
        double t = grid_entry(m, p, u);
        if (t < 0) { R->e_escaped += eps; return; }
        for (int a = 0; a < 3; ++a) p[a] += (t + 1e-6 * m->L0) * u[a];
        if (grid_locate(m, p, u, c) < 0) { R->e_escaped += eps; return; }
    } else {
        int64_t ci = select_cdf(ncells(m), m->cell_cdf, uniform(&rng));
        c[0] = (int)(ci % m->n[0]);
        c[1] = (int)((ci / m->n[0]) % m->n[1]);
        c[2] = (int)(ci / ((int64_t)m->n[0] * m->n[1]));
        double f0 = uniform(&rng), f1 = uniform(&rng), f2 = uniform(&rng);
        place_in_cell(m, c, f0, f1, f2, p);
        double u1 = uniform(&rng), u2 = uniform(&rng);
        or_isotropic(u1, u2, u);
        nu = or_sample_table(m->nspec, m->spec_nu, m->spec_cdf + (int64_t)s * m->nspec, uniform(&rng));
        if (P->peel) peel(m, p, c, u, nu, eps, PEEL_REEMIT, R); /* isotropic, from inside cell c */
    }

    double chi, alb;
    dust_at(m, nu, &chi, &alb);
    int64_t nint = 0;
    for (;;) {
        /* modified random walk: steps while the packet sits deep enough in a thick cell; each
         * counts as one interaction against the cap */
        while (P->mrw_gamma > 0) {
            const int64_t ci = cell_index(m, c);
            if (!(m->rho[ci] > 0)) break;
            const double R0 = MRW_SHRINK * or_wall_distance(m, p, c);
            const double tau0 = m->mrw_k[ci] * R0;
            if (!(tau0 >= P->mrw_gamma)) break;
            nint++;
            if (nint > P->max_interactions) { R->e_killed += eps; R->n_killed++; return; }
            R->n_mrw++;
            /* the packet cannot reach the surface along a path shorter than R0 */
            const double s = R0 * fmax(or_mrw_path(tau0, uniform(&rng)), 1.0);
            R->acc[ci] += eps * m->mrw_kp[ci] * s;
            if (run != ci) { R->visits[ci]++; run = ci; }
            double n[3], u1 = uniform(&rng), u2 = uniform(&rng);
            or_isotropic(u1, u2, n);
            for (int a = 0; a < 3; ++a) p[a] += R0 * n[a];
            u1 = uniform(&rng);
            u2 = uniform(&rng);
            or_isotropic(u1, u2, u);
            nu = or_sample_table(m->nnu, m->nu, m->cdf_emit + (int64_t)m->emit_row[ci] * m->nnu, uniform(&rng));
            dust_at(m, nu, &chi, &alb);
            if (P->peel && !P->raytrace) peel(m, p, c, u, nu, eps, PEEL_REEMIT, R);
        }
        double tau = -log(uniform(&rng));
        double dep = eps * (1.0 - alb) * chi;   /* eps * kappa_nu */
        if (walk_to_tau(m, p, u, c, tau, chi, dep, R->acc, R->visits, &run, &R->n_crossings)) {
            R->e_escaped += eps;
            int b = sed_bin(m, nu);
            int bm = (int)floor((u[2] + 1.0) * 0.5 * N_ESC_MU);
            if (bm >= N_ESC_MU) bm = N_ESC_MU - 1;
            if (bm < 0) bm = 0;
            if (b >= 0) R->esc[(int64_t)bm * m->nsed + b] += eps;
            return;
        }
        nint++;
        if (nint > P->max_interactions) { R->e_killed += eps; R->n_killed++; return; }
        R->n_interactions++;
        double z = uniform(&rng);
        if (z > alb) {
            /* absorbed, re-emitted isotropically at a frequency drawn from the cell emissivity */
            R->n_absorb++;
            if (P->terminate_on_absorb) { R->e_absorbed += eps; return; }
            double u1 = uniform(&rng), u2 = uniform(&rng);
            or_isotropic(u1, u2, u);
            int row = m->emit_row[cell_index(m, c)];
            nu = or_sample_table(m->nnu, m->nu, m->cdf_emit + (int64_t)row * m->nnu, uniform(&rng));
            dust_at(m, nu, &chi, &alb);
            if (P->peel && !P->raytrace) peel(m, p, c, u, nu, eps, PEEL_REEMIT, R);
        } else {
            R->n_scatter++;
            double mu = or_hg_mu(m->g, uniform(&rng));
            double psi = 2.0 * OR_PI * uniform(&rng);
            double uin[3] = {u[0], u[1], u[2]};
            or_scatter_dir(uin, mu, psi, u);
            if (P->peel) peel(m, p, c, uin, nu, eps, PEEL_SCATTER, R);
        }
    }
}

/* ------------------------------------------------------------------ packet loops */
typedef struct {
    const or_model* m;
    const or_params* P;
    int64_t lo, hi;
    or_result R;
} shard_t;

static void* shard_main(void* arg) {
    shard_t* sh = (shard_t*)arg;
    for (int64_t k = sh->lo; k < sh->hi; ++k) run_packet(sh->m, sh->P, sh->P->first_packet + k, &sh->R);
    return NULL;
}

static int64_t sed_len(const or_model* m) { return (int64_t)m->nobs * m->nsed; }
static int64_t img_len(const or_model* m) { return (int64_t)m->nobs * m->nimg * m->img_nx * m->img_ny; }
static int64_t esc_len(const or_model* m) { return (int64_t)N_ESC_MU * m->nsed; }

/* Run P->n_packets packet histories.  Result arrays must be zeroed by the caller; they are
 * accumulated into.  nthreads > 1 shards the packet range over threads with private
 * accumulators summed at the end (Sect. 3). */
int or_run_packets(const or_model* m, const or_params* P, or_result* R) {
    int nt = P->nthreads > 1 ? P->nthreads : 1;
    if (nt == 1) {
        for (int64_t k = 0; k < P->n_packets; ++k) run_packet(m, P, P->first_packet + k, R);
        return 0;
    }
    shard_t* sh = (shard_t*)calloc((size_t)nt, sizeof(shard_t));
    pthread_t* th = (pthread_t*)calloc((size_t)nt, sizeof(pthread_t));
    if (!sh || !th) return -1;
    int64_t per = (P->n_packets + nt - 1) / nt;
    for (int t = 0; t < nt; ++t) {
        sh[t].m = m;
        sh[t].P = P;
        sh[t].lo = (int64_t)t * per;
        sh[t].hi = sh[t].lo + per > P->n_packets ? P->n_packets : sh[t].lo + per;
        if (sh[t].lo > sh[t].hi) sh[t].lo = sh[t].hi;
        sh[t].R.acc = (double*)calloc((size_t)ncells(m), sizeof(double));
        sh[t].R.sed = (double*)calloc((size_t)(sed_len(m) + 1), sizeof(double));
        sh[t].R.img = (double*)calloc((size_t)(img_len(m) + 1), sizeof(double));
        sh[t].R.esc = (double*)calloc((size_t)(esc_len(m) + 1), sizeof(double));
        sh[t].R.visits = (int64_t*)calloc((size_t)ncells(m), sizeof(int64_t));
        pthread_create(&th[t], NULL, shard_main, &sh[t]);
    }
    for (int t = 0; t < nt; ++t) {
        pthread_join(th[t], NULL);
        or_result* r = &sh[t].R;
        for (int64_t i = 0; i < ncells(m); ++i) R->acc[i] += r->acc[i];
        for (int64_t i = 0; i < sed_len(m); ++i) R->sed[i] += r->sed[i];
        for (int64_t i = 0; i < img_len(m); ++i) R->img[i] += r->img[i];
        for (int64_t i = 0; i < esc_len(m); ++i) R->esc[i] += r->esc[i];
        for (int64_t i = 0; i < ncells(m); ++i) R->visits[i] += r->visits[i];
        R->e_escaped += r->e_escaped;
        R->e_killed += r->e_killed;
        R->e_absorbed += r->e_absorbed;
        R->n_interactions += r->n_interactions;
        R->n_scatter += r->n_scatter;
        R->n_absorb += r->n_absorb;
        R->n_crossings += r->n_crossings;
        R->n_peel_crossings += r->n_peel_crossings;
        R->n_killed += r->n_killed;
        R->n_mrw += r->n_mrw;
        free(r->acc); free(r->sed); free(r->img); free(r->esc); free(r->visits);
    }
    free(sh);
    free(th);
    return 0;
}
