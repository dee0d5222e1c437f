"""Seeded synthetic inputs for the Monte-Carlo dust-temperature solve.

This module only *describes problems*: grid walls, densities, the dust table
values (frequencies, extinction, albedo, HG asymmetry), the temperature nodes of
the emissivity table, sources, observers and packet budgets.  It holds none of
the method's arithmetic (no Planck function, no emissivity tables, no sampling,
no walking); both the FP64 oracle and the CUDA library build those themselves
from these arrays.

The problems stand in for the paper's benchmarks, whose dust optical constants
and reference results are not available here (Sect. 4: the Pascucci et al. disk,
Eq. 9; the Pinte et al. disk; Sect. 5: the star-forming cloud):

* ``tiny_sphere``      - Cartesian 32^3, uniform sphere, one 5800 K star.
* ``flared_disk``      - spherical-polar 200x128x1 flared disk (Eq. 9 shape).
* ``batched_disks``    - many uneven disk models for one batched launch.
* ``turbulent_cloud``  - Cartesian 256^3 log-normal cloud with 20 stars.
* ``warmstart_cloud``  - 128^3 clouds with 1-8 stars (learned warm start).

Every array is produced from a ``numpy.random.default_rng(seed)`` stream so the
same call gives bit-identical inputs to both implementations.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# cgs constants used only to *state* the inputs (wavelength nodes -> frequency,
# lengths in AU / pc, luminosities in Lsun).
C_LIGHT = 2.99792458e10          # cm/s (exact, SI definition)
AU = 1.495978707e13              # cm (IAU 2012)
PC = 3.0856775814913673e18       # cm (IAU 2015)
LSUN = 3.828e33                  # erg/s (IAU 2015 nominal)
MICRON = 1e-4                    # cm

# Dust law of the synthetic workloads: chi_nu = CHI_1UM * (nu / nu(1 um))^BETA_DUST
CHI_1UM = 1.0e4                  # cm^2/g, arbitrary normalisation (temperatures do not depend on it)
BETA_DUST = 1.7
ALBEDO = 0.5
G_HG = 0.6


@dataclass
class Workload:
    """A complete problem statement (the input of Sect. 2: density, dust, sources, outputs)."""

    name: str
    grid_type: str                      # "cartesian", "spherical" or "cylindrical"
    walls: list                         # [w1, w2, w3] float64 arrays: (x, y, z), (r, theta, phi) or
                                        # (R, z, phi); cm, rad for the angles
    rho: np.ndarray                     # float32, C-order [n3][n2][n1], g/cm^3
    nu: np.ndarray                      # dust table frequencies, strictly increasing (Hz)
    chi: np.ndarray                     # mass extinction coefficient at nu (cm^2/g)
    albedo: np.ndarray                  # single-scattering albedo at nu
    g: float                            # Henyey-Greenstein asymmetry parameter
    T_nodes: np.ndarray                 # temperature nodes of the emissivity / Planck-mean table (K)
    sources: list = field(default_factory=list)   # dicts: pos (cm, 3), L (erg/s), Teff (K) or a
                                        # spectrum of its own, "spectrum": (nu Hz, f_nu any scale)
    cell_source: dict | None = None     # {"L": float64 [Nc] erg/s, "Teff": K}
    external_sources: list = field(default_factory=list)  # dicts: center (cm, 3), radius (cm), L, Teff
    obs_incl: np.ndarray = field(default_factory=lambda: np.zeros(0))  # rad
    obs_az: np.ndarray = field(default_factory=lambda: np.zeros(0))    # rad
    nsed: int = 250
    lam_min_um: float = 0.1
    lam_max_um: float = 1000.0
    img_nx: int = 0
    img_ny: int = 0
    img_half_extent: float = 0.0        # cm
    img_lam_um: np.ndarray = field(default_factory=lambda: np.zeros(0))
    n_packets: int = 100_000
    n_iter: int = 5
    seed: int = 1

    @property
    def shape(self):
        return tuple(len(w) - 1 for w in self.walls)  # (n1, n2, n3)

    @property
    def n_cells(self):
        n1, n2, n3 = self.shape
        return n1 * n2 * n3


def dust_table(n_nu: int = 100, lam_min_um: float = 0.1, lam_max_um: float = 1000.0,
               beta: float = BETA_DUST, albedo: float = ALBEDO, g: float = G_HG):
    """Log-spaced wavelength nodes lambda_k = lam_min * (lam_max/lam_min)^(k/(n-1)),
    returned as increasing frequencies with chi = CHI_1UM (nu/nu_1um)^beta."""
    k = np.arange(n_nu, dtype=np.float64)
    lam_um = lam_min_um * (lam_max_um / lam_min_um) ** (k / (n_nu - 1))
    nu = (C_LIGHT / (lam_um * MICRON))[::-1].copy()
    nu_1um = C_LIGHT / MICRON
    chi = CHI_1UM * (nu / nu_1um) ** beta
    alb = np.full(n_nu, albedo)
    return nu, chi, alb, g


def chi_at_lambda_um(lam_um: float, beta: float = BETA_DUST) -> float:
    """Extinction of the synthetic dust law at a wavelength (used to normalise densities)."""
    return CHI_1UM * (1.0 / lam_um) ** beta


def temperature_nodes(n: int = 1000, t_min: float = 1.0, t_max: float = 2000.0) -> np.ndarray:
    """Log-spaced temperature nodes T_m = t_min (t_max/t_min)^(m/(n-1))."""
    m = np.arange(n, dtype=np.float64)
    return t_min * (t_max / t_min) ** (m / (n - 1))


def disk_theta_walls(n_theta: int) -> np.ndarray:
    """Polar walls concentrated at the midplane: theta_j = pi/2 (1 - s_j |s_j|), s_j = 1 - 2j/n."""
    j = np.arange(n_theta + 1, dtype=np.float64)
    s = 1.0 - 2.0 * j / n_theta
    th = 0.5 * math.pi * (1.0 - s * np.abs(s))
    th[0] = 0.0
    th[-1] = math.pi
    return th


# ----------------------------------------------------------------------------- tiny sphere
def tiny_sphere(n: int = 32, half_extent_au: float = 100.0, radius_au: float = 80.0,
                tau_1um: float = 1.0, n_packets: int = 100_000, n_iter: int = 5, seed: int = 1,
                n_nu: int = 100) -> Workload:
    """Cartesian n^3 over +-half_extent, uniform sphere of radius R with radial optical depth
    tau at 1 um (cells included by their centre), central 5800 K 1 Lsun point source,
    SEDs at 12.5, 42.5 and 77.5 degrees (the Pascucci et al. inclinations)."""
    h = half_extent_au * AU
    w = np.linspace(-h, h, n + 1)
    w[n // 2] = 0.0 if n % 2 == 0 else w[n // 2]
    xc = 0.5 * (w[1:] + w[:-1])
    zz, yy, xx = np.meshgrid(xc, xc, xc, indexing="ij")
    r = np.sqrt(xx * xx + yy * yy + zz * zz)
    rho0 = tau_1um / (chi_at_lambda_um(1.0) * radius_au * AU)
    rho = np.where(r < radius_au * AU, rho0, 0.0).astype(np.float32)
    nu, chi, alb, g = dust_table(n_nu)
    return Workload(
        name="tiny_sphere", grid_type="cartesian", walls=[w.copy(), w.copy(), w.copy()], rho=rho,
        nu=nu, chi=chi, albedo=alb, g=g, T_nodes=temperature_nodes(),
        sources=[dict(pos=(0.0, 0.0, 0.0), L=LSUN, Teff=5800.0)],
        obs_incl=np.radians([12.5, 42.5, 77.5]), obs_az=np.zeros(3),
        n_packets=n_packets, n_iter=n_iter, seed=seed)


# ----------------------------------------------------------------------------- flared disk
def flared_disk(n_r: int = 200, n_theta: int = 128, n_phi: int = 1, r_in_au: float = 1.0,
                r_out_au: float = 1000.0, tau_550: float = 100.0, h100_au: float = 10.0,
                alpha: float = 1.0, flaring: float = 1.125, Teff: float = 5800.0,
                L_lsun: float = 1.0, n_packets: int = 10_000_000, n_iter: int = 10,
                seed: int = 2, n_obs: int = 10) -> Workload:
    """Flared disk of Eq. 9 shape on a spherical-polar grid.

    rho = rho0 (R/100 AU)^-alpha exp(-z^2 / 2 h^2), h = h100 (R/100 AU)^flaring, evaluated at
    cell centres (arithmetic-mid r and theta).  rho0 is set from the analytic midplane
    integral so that the radial 550 nm extinction optical depth is tau_550.
    Observers: cos i = 0.05 ... 0.95 in steps of 0.1 (the Pinte et al. inclinations)."""
    r_w = r_in_au * AU * (r_out_au / r_in_au) ** (np.arange(n_r + 1) / n_r)
    r_w[0] = r_in_au * AU
    r_w[-1] = r_out_au * AU
    th_w = disk_theta_walls(n_theta)
    ph_w = np.linspace(0.0, 2.0 * math.pi, n_phi + 1)
    rc = 0.5 * (r_w[1:] + r_w[:-1])
    thc = 0.5 * (th_w[1:] + th_w[:-1])
    TH, RC = np.meshgrid(thc, rc, indexing="ij")          # [theta][r]
    R = RC * np.sin(TH)
    z = RC * np.cos(TH)
    h = h100_au * AU * (R / (100 * AU)) ** flaring
    r0 = 100 * AU
    if abs(alpha - 1.0) < 1e-12:
        integral = r0 * math.log(r_out_au / r_in_au)
    else:
        integral = r0 / (1 - alpha) * ((r_out_au / 100) ** (1 - alpha) - (r_in_au / 100) ** (1 - alpha))
    rho0 = tau_550 / (chi_at_lambda_um(0.55) * integral)
    rho2 = rho0 * (R / r0) ** (-alpha) * np.exp(-0.5 * (z / h) ** 2)
    rho = np.broadcast_to(rho2, (n_phi, n_theta, n_r)).astype(np.float32).copy()
    nu, chi, alb, g = dust_table()
    cosi = 0.05 + 0.1 * np.arange(n_obs)
    return Workload(
        name="flared_disk", grid_type="spherical", walls=[r_w, th_w, ph_w], rho=rho,
        nu=nu, chi=chi, albedo=alb, g=g, T_nodes=temperature_nodes(),
        sources=[dict(pos=(0.0, 0.0, 0.0), L=L_lsun * LSUN, Teff=Teff)],
        obs_incl=np.arccos(cosi), obs_az=np.zeros(n_obs),
        n_packets=n_packets, n_iter=n_iter, seed=seed)


# ----------------------------------------------------------------------------- batched disks
def batched_disks(n_models: int = 512, seed: int = 3, packet_scale: float = 1.0,
                  size_scale: float = 1.0):
    """Uneven disk models for one batched launch: tau_550 log-uniform 1-1e4, inner radius
    log-uniform 0.1-5 AU, flaring 1.0-1.25, stellar Teff 3000-10000 K, nr 50-400,
    ntheta 32-200, nphi 1-64 (axisymmetric density replicated in phi), packet budgets
    log-uniform 1e5-1e7.  ``size_scale``/``packet_scale`` shrink the set for tests."""
    rng = np.random.default_rng(seed)
    models = []
    for m in range(n_models):
        tau = 10 ** rng.uniform(0, 4)
        r_in = 10 ** rng.uniform(math.log10(0.1), math.log10(5.0))
        beta = rng.uniform(1.0, 1.25)
        teff = rng.uniform(3000, 10000)
        nr = int(rng.integers(50, 401))
        nt = int(rng.integers(32, 201))
        npf = int(rng.integers(1, 65))
        npk = int(10 ** rng.uniform(5, 7))
        nr = max(4, int(nr * size_scale))
        nt = max(4, int(nt * size_scale)) // 2 * 2
        npf = max(1, int(npf * size_scale))
        npk = max(1000, int(npk * packet_scale))
        wl = flared_disk(n_r=nr, n_theta=nt, n_phi=npf, r_in_au=r_in, tau_550=tau, flaring=beta,
                         Teff=teff, n_packets=npk, n_iter=10, seed=seed * 100000 + m)
        wl.name = f"disk{m}"
        models.append(wl)
    return models


# ----------------------------------------------------------------------------- turbulent cloud
def gaussian_random_field(n: int, slope: float, rng) -> np.ndarray:
    """Unit-variance Gaussian random field with power spectrum |k|^slope (k = 0 removed)."""
    white = rng.standard_normal((n, n, n))
    f = np.fft.rfftn(white)
    kx = np.fft.fftfreq(n)[:, None, None]
    ky = np.fft.fftfreq(n)[None, :, None]
    kz = np.fft.rfftfreq(n)[None, None, :]
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(k)
    nz = k > 0
    amp[nz] = k[nz] ** (slope / 2.0)
    g = np.fft.irfftn(f * amp, s=(n, n, n), axes=(0, 1, 2))
    g -= g.mean()
    g /= g.std()
    return g


def turbulent_cloud(n: int = 256, box_pc: float = 0.65, sigma_lnrho: float = 1.5,
                    tau_mean_550: float = 10.0, n_sources: int = 20, n_packets: int = 100_000_000,
                    n_iter: int = 10, seed: int = 4, img_n: int = 512,
                    img_lam_um=(1.25, 3.6, 8.0, 70.0, 250.0, 500.0), t_range=(3000.0, 20000.0),
                    l_range=(0.1, 100.0)) -> Workload:
    """Cartesian n^3 log-normal cloud rho ~ exp(sigma G), G a k^-11/3 Gaussian random field,
    scaled to a mean 550 nm optical depth across the box; point sources uniform in the box
    with Teff uniform and L log-uniform; images at (theta, phi) = (45, 45) degrees."""
    rng = np.random.default_rng(seed)
    side = box_pc * PC
    w = np.linspace(-side / 2, side / 2, n + 1)
    G = gaussian_random_field(n, -11.0 / 3.0, rng)
    rho = np.exp(sigma_lnrho * G)
    rho *= tau_mean_550 / (rho.mean() * chi_at_lambda_um(0.55) * side)
    srcs = []
    for _ in range(n_sources):
        pos = tuple(float(v) for v in rng.uniform(-side / 2, side / 2, 3) * 0.999)
        teff = float(rng.uniform(*t_range))
        L = float(10 ** rng.uniform(math.log10(l_range[0]), math.log10(l_range[1]))) * LSUN
        srcs.append(dict(pos=pos, L=L, Teff=teff))
    nu, chi, alb, g = dust_table()
    return Workload(
        name="turbulent_cloud", grid_type="cartesian", walls=[w.copy(), w.copy(), w.copy()],
        rho=rho.astype(np.float32), nu=nu, chi=chi, albedo=alb, g=g, T_nodes=temperature_nodes(),
        sources=srcs, obs_incl=np.radians([45.0]), obs_az=np.radians([45.0]),
        img_nx=img_n, img_ny=img_n, img_half_extent=side / 2,
        img_lam_um=np.asarray(img_lam_um, dtype=np.float64),
        n_packets=n_packets, n_iter=n_iter, seed=seed)


def warmstart_cloud(seed: int, n: int = 128, n_packets: int = 4_000_000, n_iter: int = 12,
                    tau_mean_550: float = 10.0) -> Workload:
    """128^3 cloud as ``turbulent_cloud`` with 1-8 sources (training / held-out fields)."""
    rng = np.random.default_rng(seed)
    ns = int(rng.integers(1, 9))
    wl = turbulent_cloud(n=n, n_sources=ns, n_packets=n_packets, n_iter=n_iter, seed=seed, img_n=0,
                         img_lam_um=(), tau_mean_550=tau_mean_550)
    wl.name = f"warmstart{seed}"
    return wl


def slab(n_layers: int = 10, tau_total: float = 1.0, albedo: float = 0.0, n_xy: int = 1,
         half_width_au: float = 1e4, thickness_au: float = 1.0, n_packets: int = 20000,
         seed: int = 11, source_z_au: float | None = None) -> Workload:
    """A plane-parallel slab of n_layers Cartesian layers (z) with total vertical extinction
    optical depth tau_total at every frequency (grey dust), laterally much wider than thick.
    The point source sits just inside the bottom face; used for first-flight closed forms."""
    hw = half_width_au * AU
    t = thickness_au * AU
    wxy = np.linspace(-hw, hw, n_xy + 1)
    wz = np.linspace(0.0, t, n_layers + 1)
    nu, _, _, g = dust_table(20)
    chi = np.full_like(nu, 1.0)
    alb = np.full_like(nu, albedo)
    rho = np.full((n_layers, n_xy, n_xy), tau_total / (chi[0] * t), dtype=np.float32)
    z0 = 1e-6 * t if source_z_au is None else source_z_au * AU
    return Workload(
        name="slab", grid_type="cartesian", walls=[wxy, wxy.copy(), wz], rho=rho,
        nu=nu, chi=chi, albedo=alb, g=0.0, T_nodes=temperature_nodes(),
        sources=[dict(pos=(0.0, 0.0, z0), L=LSUN, Teff=5800.0)],
        obs_incl=np.radians([0.0, 30.0, 60.0]), obs_az=np.zeros(3),
        n_packets=n_packets, n_iter=1, seed=seed)


def random_rays(n: int, rng, extent: float, inside: float = 0.95):
    """Random origins inside a cube of half-size extent*inside and isotropic unit directions."""
    x = rng.uniform(-extent * inside, extent * inside, (n, 3))
    mu = rng.uniform(-1, 1, n)
    ph = rng.uniform(0, 2 * math.pi, n)
    s = np.sqrt(1 - mu * mu)
    u = np.stack([s * np.cos(ph), s * np.sin(ph), mu], axis=1)
    return x, u


def uniforms(n: int, rng) -> np.ndarray:
    """Uniform deviates in (0, 1] with 24-bit resolution, the same lattice both
    implementations map their Philox words onto."""
    k = rng.integers(0, 1 << 24, n, dtype=np.int64)
    return (k + 1).astype(np.float64) * 2.0 ** -24


SIGMA_SB = 5.670374419e-5      # erg cm^-2 s^-1 K^-4


def isrf_luminosity(radius_cm: float, dilution: float, T_rad: float) -> float:
    """Luminosity an external sphere of radius R must emit inwards for an isotropic field of mean
    intensity J = W B(T_rad) inside it: L = 4 pi R^2 * pi J = 4 pi R^2 W sigma T^4."""
    return 4.0 * math.pi * radius_cm ** 2 * dilution * SIGMA_SB * T_rad ** 4


def isrf_cloud(grid_type: str = "cartesian", n: int = 8, half_extent_au: float = 1e4, tau_550: float = 0.01,
               dilution: float = 1e-14, T_rad: float = 6000.0, n_packets: int = 200_000, seed: int = 12,
               r_ext_factor: float = 1.8) -> Workload:
    """A uniform cloud inside an external isotropic radiation field (Sect. 2.1.1): the external
    sphere (radius r_ext_factor x the cloud's half extent, centred on it) emits inwards with a
    diluted blackbody spectrum; no point sources.  grid_type "cartesian" (n^3 box), "spherical"
    (n shells x n cones x 4 wedges) or "cylindrical" (n x n x 4, |z| <= half extent)."""
    h = half_extent_au * AU
    if grid_type == "cartesian":
        w = np.linspace(-h, h, n + 1)
        walls = [w, w.copy(), w.copy()]
        size = 2 * h
    elif grid_type == "spherical":
        walls = [np.linspace(0.0, h, n + 1), np.linspace(0.0, math.pi, n + 1), np.linspace(0.0, 2 * math.pi, 5)]
        size = h
    else:
        walls = [np.linspace(0.0, h, n + 1), np.linspace(-h, h, n + 1), np.linspace(0.0, 2 * math.pi, 5)]
        size = 2 * h
    shape = tuple(len(x) - 1 for x in walls)
    rho0 = tau_550 / (chi_at_lambda_um(0.55) * size)
    rho = np.full(shape[::-1], rho0, dtype=np.float32)
    nu, chi, alb, g = dust_table()
    R = r_ext_factor * h * (math.sqrt(3.0) if grid_type == "cartesian" else math.sqrt(2.0))
    ext = [dict(center=(0.0, 0.0, 0.0), radius=R, L=isrf_luminosity(R, dilution, T_rad), Teff=T_rad)]
    return Workload(name=f"isrf_{grid_type}", grid_type=grid_type, walls=walls, rho=rho, nu=nu, chi=chi,
                    albedo=alb, g=g, T_nodes=temperature_nodes(), sources=[], external_sources=ext,
                    obs_incl=np.radians([30.0]), obs_az=np.zeros(1), n_packets=n_packets, seed=seed)


def cylindrical_disk(n_R: int = 120, n_z: int = 96, n_phi: int = 1, r_in_au: float = 1.0,
                     r_out_au: float = 300.0, tau_550: float = 100.0, h100_au: float = 10.0,
                     flaring: float = 1.125, n_packets: int = 1_000_000, seed: int = 13,
                     isrf_dilution: float = 0.0) -> Workload:
    """The flared disk of Eq. 9's shape on a cylindrical-polar grid (R log-spaced, z uniform over
    +-4 scale heights at r_out), a 5800 K 1 Lsun star at the centre and, with isrf_dilution > 0,
    an external isotropic field of a diluted 6000 K blackbody around it (Sect. 2.1.1)."""
    Rw = r_in_au * AU * (r_out_au / r_in_au) ** (np.arange(n_R + 1) / n_R)
    zmax = 4 * h100_au * AU * (r_out_au / 100.0) ** flaring
    zw = np.linspace(-zmax, zmax, n_z + 1)
    pw = np.linspace(0.0, 2.0 * math.pi, n_phi + 1)
    Rc = 0.5 * (Rw[1:] + Rw[:-1])
    zc = 0.5 * (zw[1:] + zw[:-1])
    ZZ, RR = np.meshgrid(zc, Rc, indexing="ij")
    hh = h100_au * AU * (RR / (100 * AU)) ** flaring
    rho0 = tau_550 / (chi_at_lambda_um(0.55) * 100 * AU * math.log(r_out_au / r_in_au))
    rho2 = rho0 * (RR / (100 * AU)) ** -1.0 * np.exp(-0.5 * (ZZ / hh) ** 2)
    rho = np.broadcast_to(rho2, (n_phi, n_z, n_R)).astype(np.float32).copy()
    nu, chi, alb, g = dust_table()
    ext = []
    if isrf_dilution > 0:
        R = 1.01 * math.hypot(r_out_au * AU, zmax)
        ext = [dict(center=(0.0, 0.0, 0.0), radius=R, L=isrf_luminosity(R, isrf_dilution, 6000.0), Teff=6000.0)]
    cosi = 0.05 + 0.1 * np.arange(10)
    return Workload(name="cylindrical_disk", grid_type="cylindrical", walls=[Rw, zw, pw], rho=rho, nu=nu,
                    chi=chi, albedo=alb, g=g, T_nodes=temperature_nodes(),
                    sources=[dict(pos=(0.0, 0.0, 0.0), L=LSUN, Teff=5800.0)], external_sources=ext,
                    obs_incl=np.arccos(cosi), obs_az=np.zeros(10), n_packets=n_packets, seed=seed)


def embedded_envelope(n_r: int = 60, n_theta: int = 8, tau_550: float = 1e5, r_in_au: float = 1.0,
                      r_out_au: float = 1000.0, power: float = 1.5, n_packets: int = 100_000,
                      seed: int = 14) -> Workload:
    """A star embedded in an optically thick envelope, rho ∝ r^-power (an infalling envelope),
    on a spherical-polar grid (r log-spaced r_in to r_out, n_theta uniform cones, one phi cell)
    with an empty inner cavity, normalised to a radial tau_550 at cell centres: the regime where
    packets re-emitted deep inside need the modified random walk (Sect. 2.2)."""
    rw = r_in_au * AU * (r_out_au / r_in_au) ** (np.arange(n_r + 1) / n_r)
    walls = [rw, np.linspace(0.0, math.pi, n_theta + 1), np.array([0.0, 2.0 * math.pi])]
    rc = 0.5 * (rw[1:] + rw[:-1])
    rho0 = tau_550 / (chi_at_lambda_um(0.55) * np.sum((rc / AU) ** -power * np.diff(rw)))
    rho = np.broadcast_to(rho0 * (rc / AU) ** -power, (1, n_theta, n_r)).astype(np.float32).copy()
    nu, chi, alb, g = dust_table()
    cosi = 0.05 + 0.1 * np.arange(10)
    return Workload(name="embedded_envelope", grid_type="spherical", walls=walls, rho=rho, nu=nu, chi=chi,
                    albedo=alb, g=g, T_nodes=temperature_nodes(),
                    sources=[dict(pos=(0.0, 0.0, 0.0), L=LSUN, Teff=5800.0)], obs_incl=np.arccos(cosi),
                    obs_az=np.zeros(10), n_packets=n_packets, seed=seed)


def thick_grey(kind: str = "cartesian", n_packets: int = 3000, tau_cell: float | None = None) -> Workload:
    """Optically thick grey models whose cells are many transport mean free paths across (the
    modified random walk's regime, Sect. 2.2): grey dust (chi = 1 cm^2/g, albedo 0.5, g = 0.6).
    "cartesian": 4^3 cells over +-100 AU, 60 extinction mean free paths per cell (tau_cell), a
    5800 K 1 Lsun star off-centre; "spherical": r walls 5, 20, 45, 80, 100 AU (a hole), 4 cones,
    3 wedges, tau_cell per 20 AU (default 50); "cylindrical": R walls 0, 20, 45, 80, 100 AU, z
    walls -60, -20, 20, 60 AU, one phi cell, tau_cell per 20 AU (default 50); stars at the origin
    except for the cube."""
    nu, chi, alb, g = dust_table()
    chi = np.full_like(nu, 1.0)
    alb = np.full_like(nu, 0.5)
    src = [dict(pos=(0.0, 0.0, 0.0), L=LSUN, Teff=5800.0)]
    if kind == "cartesian":
        w = np.linspace(-100 * AU, 100 * AU, 5)
        walls = [w, w.copy(), w.copy()]
        rho = np.float32((60.0 if tau_cell is None else tau_cell) / (50 * AU))
        src = [dict(pos=(AU, 2 * AU, 3 * AU), L=LSUN, Teff=5800.0)]
    elif kind == "spherical":
        walls = [np.array([5.0, 20.0, 45.0, 80.0, 100.0]) * AU, np.array([0.0, 0.9, math.pi / 2, 2.2, math.pi]),
                 np.array([0.0, 2.0, 4.0, 2 * math.pi])]
        rho = np.float32((50.0 if tau_cell is None else tau_cell) / (20 * AU))
    elif kind == "cylindrical":
        walls = [np.array([0.0, 20.0, 45.0, 80.0, 100.0]) * AU, np.array([-60.0, -20.0, 20.0, 60.0]) * AU,
                 np.array([0.0, 2 * math.pi])]
        rho = np.float32((50.0 if tau_cell is None else tau_cell) / (20 * AU))
    else:
        raise ValueError(kind)
    shape = tuple(len(x) - 1 for x in walls)[::-1]
    return Workload(name=f"thick_{kind}", grid_type=kind, walls=walls, rho=np.full(shape, rho, np.float32), nu=nu,
                    chi=chi, albedo=alb, g=g, T_nodes=temperature_nodes(), sources=src,
                    obs_incl=np.radians([30.0]), obs_az=np.zeros(1), n_packets=n_packets, seed=21)


WORKLOADS = {
    "tiny_sphere": tiny_sphere,
    "flared_disk": flared_disk,
    "turbulent_cloud": turbulent_cloud,
}
