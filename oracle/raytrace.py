"""FP64 ORACLE of raytracing the source and dust emission into SEDs and images (Sect. 2.6.3).

Test infrastructure only (tests, the smoke check, the bench's CPU legs); the CUDA library
never imports it.  After the temperatures have converged, the thermal emission reaches each
observer without a random walk: for emission at a point with column Sigma = int rho ds to the
grid edge along the observer direction, the energy per unit solid angle arriving in SED bin b is

    L / (4 pi) * int_bin p(nu) exp(-chi(nu) Sigma) dnu,

p the normalised spectrum of the emission (the same piecewise-constant pdf the packets sample:
the source spectrum for a point source, the emissivity row kappa_nu B_nu(T) of the cell for
dust) and chi(nu) the extinction, log-log between the dust nodes.  Point sources contribute
their luminosity along the one ray from the source.  Dust emission is sampled by rays: ray k
picks a cell with probability proportional to its emitted luminosity m E(T) (Eq. 3: the cell
emits 4 pi kappa_P B(T) per unit mass, which equals the absorbed Adot once the temperatures have
converged) and a position uniform in the cell; each ray carries L_dust / n_rays.  Images take the same weights at the projected position of the emission point,
in the bins holding the image wavelengths.

Readings where the paper is silent: the bin integral is evaluated by 8-point Gauss-Legendre
quadrature on each piece of the bin between consecutive nodes of p and of chi; the emission row
of a cell is the one the re-emission of the same pass uses (nearest node in log T); dust rays
draw from Philox streams keyed by 2^30 + iteration.
"""
from __future__ import annotations

import math

import numpy as np

from . import tables as T

RAYTRACE_KEY = 0x40000000
_GL_X, _GL_W = np.polynomial.legendre.leggauss(8)


def bin_edges_nu(nsed, lam_min_cm, lam_max_cm):
    """[nsed][2] (nu_lo, nu_hi) of the SED bins (log-spaced in wavelength)."""
    lam = lam_min_cm * (lam_max_cm / lam_min_cm) ** (np.arange(nsed + 1) / nsed)
    nu = T.C_LIGHT / lam
    return np.stack([nu[1:], nu[:-1]], axis=1)


def quadrature(p_nodes, chi_nodes, edges):
    """Quadrature nodes for every bin: (nu_q, w_q, bin_q, j_q), j_q the interval of p_nodes
    holding nu_q.  Each bin is cut at the nodes of p and of chi."""
    nus, ws, bins = [], [], []
    brk = np.union1d(p_nodes, chi_nodes)
    for b, (lo, hi) in enumerate(edges):
        cuts = np.concatenate([[lo], brk[(brk > lo) & (brk < hi)], [hi]])
        for a, c in zip(cuts[:-1], cuts[1:]):
            x = 0.5 * (a + c) + 0.5 * (c - a) * _GL_X
            nus.append(x)
            ws.append(0.5 * (c - a) * _GL_W)
            bins.append(np.full(x.size, b))
    nu_q = np.concatenate(nus)
    j_q = np.clip(np.searchsorted(p_nodes, nu_q, side="right") - 1, 0, len(p_nodes) - 2)
    return nu_q, np.concatenate(ws), np.concatenate(bins), j_q


def chi_at(nu, dust_nu, dust_chi):
    """Extinction log-log between the dust nodes (clamped at the ends)."""
    return np.exp(np.interp(np.log(nu), np.log(dust_nu), np.log(dust_chi)))


def pdf_pieces(x, cdf):
    """Piecewise-constant pdf of a cumulative table: p_j = (cdf_{j+1} - cdf_j) / (x_{j+1} - x_j)."""
    x = np.asarray(x, dtype=np.float64)
    cdf = np.asarray(cdf, dtype=np.float64)
    return np.diff(cdf, axis=-1) / np.diff(x)


def _accumulate(om, weight, sigma, pdf_q, quad, pos, sed, img):
    """Add weight/(4 pi) * sum_q w_q p_q exp(-chi_q Sigma) to the SED bins of every observer, and
    to the image pixels of pos.  weight [n], sigma [n][nobs], pdf_q [n][Q]."""
    nu_q, w_q, bin_q, _ = quad
    chi_q = chi_at(nu_q, om.nu, om.chi)
    nsed = om.wl.nsed
    for o in range(om.nobs):
        att = np.exp(-np.outer(sigma[:, o], chi_q))             # [n][Q]
        contrib = (weight[:, None] / (4 * math.pi)) * pdf_q * w_q[None, :] * att
        per_bin = np.zeros((len(weight), nsed))
        np.add.at(per_bin.T, bin_q, contrib.T)
        sed[o] += per_bin.sum(axis=0)
        if om.nimg > 0:
            ex, ey = om.obs_ex[3 * o:3 * o + 3], om.obs_ey[3 * o:3 * o + 3]
            h = float(om.wl.img_half_extent)
            ix = np.floor((pos @ ex + h) / (2 * h) * om.wl.img_nx).astype(np.int64)
            iy = np.floor((pos @ ey + h) / (2 * h) * om.wl.img_ny).astype(np.int64)
            ok = (ix >= 0) & (ix < om.wl.img_nx) & (iy >= 0) & (iy < om.wl.img_ny)
            for l, b in enumerate(om.img_bin):
                if 0 <= b < nsed:
                    np.add.at(img[o, l], (iy[ok], ix[ok]), per_bin[ok, b])


def sources(om, sed, img):
    """Point-source emission along the ray from each source (inside the grid) to each observer.
    Needs om.struct() built."""
    edges = bin_edges_nu(om.wl.nsed, om.lam_min, om.lam_max)
    quad = quadrature(om.spec_nu, om.nu, edges)
    npt = len(om.wl.sources)
    if npt == 0:
        return
    from . import mc as M
    pos = om.src_pos.reshape(npt, 3)
    sigma = np.zeros((npt, om.nobs))
    inside = np.ones(npt, dtype=bool)
    out = np.zeros(3)
    c = np.zeros(3, np.int32)
    for s in range(npt):
        if M.lib().or_locate(om._struct, M._ptr(pos[s]), M._ptr(om.obs_n[0:3]), M._ptr(out), M._ptr(c, M._ip)) < 0:
            inside[s] = False
            continue
        for o in range(om.nobs):
            sigma[s, o] = M.lib().or_tau_to_edge(om._struct, M._ptr(pos[s]), M._ptr(om.obs_n[3 * o:3 * o + 3]), 1.0)
    Ls = np.array([float(src["L"]) for src in om.wl.sources])
    pdf = pdf_pieces(om.spec_nu, om.spec_cdf[:npt])             # [npt][nspec-1]
    pdf_q = pdf[:, quad[3]]
    _accumulate(om, np.where(inside, Ls, 0.0), sigma, pdf_q, quad, pos, sed, img)


def raytrace(om, n_rays, iter_key):
    """SED and image contributions of the point sources and of n_rays dust-emission rays at the
    model's current temperatures; also returns the rays' cells."""
    from . import mc as M
    L_c = om.rho * om.vol * T.interp_loglog(om.T, om.T_nodes, om.dust.E)
    cdf = np.cumsum(L_c)
    L_dust = cdf[-1]
    if not (L_dust > 0):
        n_rays = 0
    else:
        cdf = cdf / L_dust
        cdf[-1] = 1.0
    cells = np.zeros(n_rays, np.int64)
    pos = np.zeros((n_rays, 3))
    col = np.zeros((n_rays, om.nobs))
    rows = T.emission_row(om.T, om.T_nodes)
    m = om.struct(rows)
    P = M.ORParams()
    P.key = (M.C.c_uint32 * 2)(om.seed & 0xFFFFFFFF, (om.seed >> 32) & 0xFFFFFFFF)
    P.iter_key = int(iter_key) & 0xFFFFFFFF
    P.model_key = int(om.model_key) & 0xFFFFFFFF
    if n_rays > 0:
        M.lib().or_raytrace_rays(M.C.byref(m), M.C.byref(P), n_rays, M._ptr(np.ascontiguousarray(cdf)),
                                 M._ptr(cells, M._lp), M._ptr(pos), M._ptr(col))
    edges = bin_edges_nu(om.wl.nsed, om.lam_min, om.lam_max)
    quad = quadrature(om.nu, om.nu, edges)
    pdf = pdf_pieces(om.nu, om.cdf_emit)                         # [nT][nnu-1]
    sed = np.zeros((om.nobs, om.wl.nsed))
    img = np.zeros((om.nobs, om.nimg, om.wl.img_ny, om.wl.img_nx))
    sources(om, sed, img)
    w = np.full(n_rays, L_dust / max(n_rays, 1))
    for a in range(0, n_rays, 4096):
        sl = slice(a, min(n_rays, a + 4096))
        _accumulate(om, w[sl], col[sl], pdf[rows[cells[sl]]][:, quad[3]], quad, pos[sl], sed, img)
    return sed, img, cells
