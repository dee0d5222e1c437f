"""FP64 ORACLE: dust tables, temperature inversion and convergence statistic (numpy).

Test infrastructure only: this module, with ``mc.c``, is the plain CPU restatement of the
method that the CUDA library is checked against.  Only tests, the smoke check and the CPU
baseline of the bench use it.  It shares no code with the CUDA library.

* Sect. 2.1.3: LTE emissivity j_nu = kappa_nu B_nu(T) with kappa_nu = (1 - albedo) chi_nu;
  mean opacities and emissivities are pre-computed on a table.
* Sect. 2.3, Eq. 2: Adot = eps / (V dt) sum(l kappa_nu), dt = 1 s.
* Sect. 2.3, Eq. 3: 4 pi kappa_P(T) B(T) = Adot with B = (sigma/pi) T^4, i.e.
  Adot = E(T) = 4 pi int kappa_nu B_nu(T) dnu, inverted on the tabulated E.
* Sect. 2.4, Eqs. 4-6: delta(x1, x2) = max(x1/x2, x2/x1); R_j = delta over cells; the
  p-th percentile Q and its change Delta.
* Sect. 2.1.1: source spectra on a log-spaced grid over the dust band (a blackbody of Teff, or
  the source's own f_nu interpolated log-log between its nodes), renormalised so that the
  in-band part carries all of the luminosity.
* App. A and Sect. 2.2 (modified random walk): Rosseland means of the extinction and of the
  transport extinction, and the Planck-mean absorption coefficient, on the temperature nodes.
"""
from __future__ import annotations

import math

import numpy as np

# CODATA 2018 (exact SI definitions converted to cgs)
H_PLANCK = 6.62607015e-27      # erg s
K_BOLTZ = 1.380649e-16         # erg/K
C_LIGHT = 2.99792458e10        # cm/s
SIGMA_SB = 2.0 * math.pi ** 5 * K_BOLTZ ** 4 / (15.0 * H_PLANCK ** 3 * C_LIGHT ** 2)  # erg/cm^2/s/K^4


def planck_bnu(nu, T):
    """B_nu(T) = (2 h nu^3 / c^2) / (exp(h nu / k T) - 1)  [erg/s/cm^2/Hz/sr]."""
    nu = np.asarray(nu, dtype=np.float64)
    x = H_PLANCK * nu / (K_BOLTZ * T)
    with np.errstate(over="ignore"):
        return 2.0 * H_PLANCK * nu ** 3 / C_LIGHT ** 2 / np.expm1(x)


def planck_dbdt(nu, T):
    """dB_nu/dT = (2 h nu^3 / c^2) (x / T) e^x / (e^x - 1)^2, x = h nu / k T, written with
    e^x / (e^x - 1)^2 = 1 / (4 sinh^2(x / 2))  [erg/s/cm^2/Hz/sr/K]."""
    nu = np.asarray(nu, dtype=np.float64)
    x = H_PLANCK * nu / (K_BOLTZ * T)
    with np.errstate(over="ignore"):
        return 2.0 * H_PLANCK * nu ** 3 / C_LIGHT ** 2 * (x / T) / (4.0 * np.sinh(0.5 * x) ** 2)


def rosseland_mean(nu, chi, T_nodes):
    """Rosseland mean extinction chi_R(T) = int dB/dT dnu / int chi_nu^-1 dB/dT dnu (the
    diffusion coefficient D = 1 / (3 rho chi_R) of App. A), trapezoid rule over the dust nodes."""
    nu = np.asarray(nu, dtype=np.float64)
    chi = np.asarray(chi, dtype=np.float64)
    T_nodes = np.asarray(T_nodes, dtype=np.float64)
    w = planck_dbdt(nu[None, :], T_nodes[:, None])
    return trapezoid_pieces(nu, w).sum(axis=-1) / trapezoid_pieces(nu, w / chi[None, :]).sum(axis=-1)


def transport_rosseland_mean(nu, chi, albedo, g, T_nodes):
    """Rosseland mean of the transport extinction chi_nu (1 - albedo_nu g) (Henyey-Greenstein
    scattering removes only the share 1 - g of the momentum): the diffusion coefficient
    D = 1 / (3 rho chi) of the modified random walk (Sect. 2.2)."""
    chi_t = np.asarray(chi, dtype=np.float64) * (1.0 - np.asarray(albedo, dtype=np.float64) * float(g))
    return rosseland_mean(nu, chi_t, T_nodes)


def planck_mean_kappa(nu, kappa, T_nodes):
    """Planck-mean absorption coefficient int kappa_nu B_nu dnu / int B_nu dnu over the dust
    nodes (trapezoid rule): the absorption per unit path length of a field thermalised at T."""
    nu = np.asarray(nu, dtype=np.float64)
    T_nodes = np.asarray(T_nodes, dtype=np.float64)
    b = planck_bnu(nu[None, :], T_nodes[:, None])
    kb = np.asarray(kappa, dtype=np.float64)[None, :] * b
    return trapezoid_pieces(nu, kb).sum(axis=-1) / trapezoid_pieces(nu, b).sum(axis=-1)


def interp_loglog(x, x_nodes, y_nodes):
    """y(x) linear in log-log between table nodes, clamped to the end values."""
    lx = np.log(np.asarray(x_nodes, dtype=np.float64))
    ly = np.log(np.asarray(y_nodes, dtype=np.float64))
    return np.exp(np.interp(np.log(np.asarray(x, dtype=np.float64)), lx, ly))


def kappa_abs(chi, albedo):
    """Mass absorption coefficient kappa_nu = (1 - albedo) chi_nu."""
    return (1.0 - np.asarray(albedo)) * np.asarray(chi)


def trapezoid_pieces(x, f):
    """Areas of the trapezoids of f over consecutive nodes x."""
    return 0.5 * (f[..., 1:] + f[..., :-1]) * np.diff(x)


def cumulative_cdf(x, f):
    """Normalised cumulative trapezoid integral of f over x: cdf[0] = 0, cdf[-1] = 1."""
    pieces = trapezoid_pieces(x, f)
    c = np.concatenate([np.zeros(pieces.shape[:-1] + (1,)), np.cumsum(pieces, axis=-1)], axis=-1)
    total = c[..., -1:]
    c = c / total
    c[..., -1] = 1.0
    return c


class DustTables:
    """Emission table E(T_m) = 4 pi int kappa_nu B_nu(T_m) dnu and the normalised cumulative
    emissivity rows used to draw re-emission frequencies (trapezoid rule over the dust nodes)."""

    def __init__(self, nu, chi, albedo, T_nodes):
        self.nu = np.asarray(nu, dtype=np.float64)
        self.chi = np.asarray(chi, dtype=np.float64)
        self.albedo = np.asarray(albedo, dtype=np.float64)
        self.T = np.asarray(T_nodes, dtype=np.float64)
        self.kappa = kappa_abs(self.chi, self.albedo)
        jnu = self.kappa[None, :] * planck_bnu(self.nu[None, :], self.T[:, None])   # [nT][nnu]
        self.E = 4.0 * math.pi * trapezoid_pieces(self.nu, jnu).sum(axis=-1)
        self.cdf = cumulative_cdf(self.nu, jnu)

    def kappa_planck(self):
        """kappa_P(T_m) from Eq. 3: E = 4 pi kappa_P (sigma/pi) T^4."""
        return self.E / (4.0 * SIGMA_SB * self.T ** 4)


def temperature_from_adot(adot, T_nodes, E):
    """Invert E(T) = Adot (Eq. 3): find E_m <= Adot < E_{m+1}, interpolate log T linearly in
    log E; clamp to the table ends.  Returns (T, n_low_clamps, n_high_clamps)."""
    adot = np.asarray(adot, dtype=np.float64)
    T_nodes = np.asarray(T_nodes, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    T = np.empty_like(adot)
    low = adot <= E[0]
    high = adot >= E[-1]
    mid = ~(low | high)
    m = np.searchsorted(E, adot[mid], side="right") - 1
    lt = np.log(T_nodes)
    le = np.log(E)
    f = (np.log(adot[mid]) - le[m]) / (le[m + 1] - le[m])
    T[mid] = np.exp(lt[m] + f * (lt[m + 1] - lt[m]))
    T[low] = T_nodes[0]
    T[high] = T_nodes[-1]
    return T, int(low.sum()), int(high.sum())


def emission_row(T, T_nodes):
    """Table row for re-emission from a cell at temperature T: the nearest node in log T
    (ties go to the lower node)."""
    T = np.asarray(T, dtype=np.float64)
    lt = np.log(np.asarray(T_nodes, dtype=np.float64))
    x = np.log(T)
    m = np.clip(np.searchsorted(lt, x, side="right") - 1, 0, len(lt) - 2)
    up = (lt[m + 1] - x) < (x - lt[m])
    row = np.where(up, m + 1, m)
    row = np.where(x <= lt[0], 0, row)
    row = np.where(x >= lt[-1], len(lt) - 1, row)
    return row.astype(np.int32)


def delta(x1, x2):
    """Eq. 4: delta(x1, x2) = max(x1/x2, x2/x1)."""
    x1 = np.asarray(x1, dtype=np.float64)
    x2 = np.asarray(x2, dtype=np.float64)
    return np.maximum(x1 / x2, x2 / x1)


def percentile_nearest_rank(values, p):
    """Nearest-rank p-quantile: sorted(values)[ceil(p n) - 1]."""
    v = np.sort(np.asarray(values, dtype=np.float64))
    n = len(v)
    if n == 0:
        return float("nan")
    k = int(math.ceil(p * n)) - 1
    k = min(max(k, 0), n - 1)
    return float(v[k])


def convergence(prev, cur, mask, p, Q_prev=None):
    """Eqs. 5-6: Q = p-quantile of delta(prev, cur) over the masked cells; Delta = delta(Q_prev, Q)
    (infinite when there is no previous quantile)."""
    R = delta(prev[mask], cur[mask])
    Q = percentile_nearest_rank(R, p)
    D = float("inf") if Q_prev is None or not np.isfinite(Q_prev) else float(delta(Q_prev, Q))
    return Q, D


def cell_volumes(grid_type, walls):
    """Cell volumes [n3][n2][n1] (cm^3)."""
    w1, w2, w3 = (np.asarray(w, dtype=np.float64) for w in walls)
    if grid_type == "cartesian":
        return (np.diff(w3)[:, None, None] * np.diff(w2)[None, :, None] * np.diff(w1)[None, None, :])
    if grid_type == "cylindrical":       # (R, z, phi): (R_1^2 - R_0^2) / 2 dz dphi
        return (np.diff(w3)[:, None, None] * np.diff(w2)[None, :, None] * (0.5 * np.diff(w1 ** 2))[None, None, :])
    dr3 = np.diff(w1 ** 3) / 3.0
    dcos = -np.diff(np.cos(w2))
    dph = np.diff(w3)
    return dph[:, None, None] * dcos[None, :, None] * dr3[None, None, :]


def source_spectrum(nu_min, nu_max, Teff, n=1000):
    """Blackbody source spectrum on n log-spaced frequencies over the dust band, as (nodes,
    cdf); the cdf renormalises the in-band part to carry all of the luminosity."""
    k = np.arange(n, dtype=np.float64)
    nu = nu_min * (nu_max / nu_min) ** (k / (n - 1))
    nu[0] = nu_min
    nu[-1] = nu_max
    return nu, cumulative_cdf(nu, planck_bnu(nu, Teff))


def user_spectrum_at(v, unu, ufnu):
    """A source's own spectrum f_nu, given at its nodes unu (strictly increasing, f >= 0),
    evaluated at frequency v: a power law between two nodes (log-log interpolation), a straight
    line where either of the two values is zero, and zero outside the nodes."""
    if v < unu[0] or v > unu[-1]:
        return 0.0
    j = min(int(np.searchsorted(unu, v, side="right")) - 1, len(unu) - 2)
    a, b = float(ufnu[j]), float(ufnu[j + 1])
    if a > 0 and b > 0:
        t = math.log(v / unu[j]) / math.log(unu[j + 1] / unu[j])
        return math.exp((1 - t) * math.log(a) + t * math.log(b))
    return a + (b - a) * (v - unu[j]) / (unu[j + 1] - unu[j])


def user_source_spectrum(nu_min, nu_max, unu, ufnu, n=1000):
    """A source with its own spectrum on the n log-spaced frequencies of the source grid over the
    dust band, as (nodes, cdf); the cdf renormalises the in-band part to carry all of the
    luminosity (Sect. 2.1.1: a source has a luminosity and a spectrum)."""
    k = np.arange(n, dtype=np.float64)
    nu = nu_min * (nu_max / nu_min) ** (k / (n - 1))
    nu[0] = nu_min
    nu[-1] = nu_max
    unu = np.asarray(unu, dtype=np.float64)
    ufnu = np.asarray(ufnu, dtype=np.float64)
    f = np.array([user_spectrum_at(v, unu, ufnu) for v in nu])
    return nu, cumulative_cdf(nu, f)


def observer_frames(incl, az):
    """Observer unit vectors n = (sin i cos phi, sin i sin phi, cos i) and sky axes
    e_x = (-sin phi, cos phi, 0), e_y = n x e_x."""
    incl = np.asarray(incl, dtype=np.float64)
    az = np.asarray(az, dtype=np.float64)
    n = np.stack([np.sin(incl) * np.cos(az), np.sin(incl) * np.sin(az), np.cos(incl)], axis=1)
    ex = np.stack([-np.sin(az), np.cos(az), np.zeros_like(az)], axis=1)
    ey = np.cross(n, ex)
    return n, ex, ey


def sed_bin_of_lambda(lam_cm, nsed, lam_min_cm, lam_max_cm):
    """Log-spaced SED bin holding a wavelength (-1 outside)."""
    b = int(math.floor(nsed * math.log(lam_cm / lam_min_cm) / math.log(lam_max_cm / lam_min_cm)))
    return b if 0 <= b < nsed else -1
