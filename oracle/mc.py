"""FP64 ORACLE driver: builds ``mc.c`` with gcc and runs Lucy iterations on the CPU.

Test infrastructure only (tests, the smoke check and the bench's CPU baseline).  The CUDA
library never imports it, and it never imports the CUDA library.

``OracleModel`` follows the iteration of Sect. 2 (the overview paragraph before Sect. 2.1):
propagate packets (Sect. 2.2), form Adot per cell (Eq. 2), convert to temperature (Eq. 3),
test convergence (Eqs. 4-6), and after convergence compute SEDs and images by peeling-off
(Sect. 2.6.2) in one more pass whose absorbed energy is not used.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

from . import tables as T

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libhrt_oracle.so")
_lock = threading.Lock()
_lib = None

N_ESC_MU = 10
IMAGING_KEY = 0x80000000


def build(force: bool = False) -> str:
    """Compile mc.c into a shared library (plain gcc -O2, no target-specific flags)."""
    src = os.path.join(_HERE, "mc.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)


class ORModel(C.Structure):
    _fields_ = [
        ("gtype", C.c_int32), ("n", C.c_int32 * 3), ("w", _dp * 3), ("rho", _dp),
        ("nnu", C.c_int32), ("nu", _dp), ("chi", _dp), ("albedo", _dp), ("g", C.c_double),
        ("nT", C.c_int32), ("cdf_emit", _dp), ("emit_row", _ip),
        ("npoint", C.c_int32), ("src_pos", _dp), ("nsrc", C.c_int32), ("src_cdf", _dp),
        ("nspec", C.c_int32), ("spec_nu", _dp), ("spec_cdf", _dp), ("cell_cdf", _dp),
        ("nobs", C.c_int32), ("obs_n", _dp), ("obs_ex", _dp), ("obs_ey", _dp),
        ("nsed", C.c_int32), ("lam_min", C.c_double), ("lam_max", C.c_double),
        ("img_nx", C.c_int32), ("img_ny", C.c_int32), ("nimg", C.c_int32),
        ("img_half", C.c_double), ("img_bin", _ip),
        ("next", C.c_int32), ("ext_c", _dp), ("ext_R", _dp), ("L0", C.c_double),
        ("mrw_k", _dp), ("mrw_kp", _dp),
    ]


class ORParams(C.Structure):
    _fields_ = [
        ("n_packets", C.c_int64), ("first_packet", C.c_int64), ("key", C.c_uint32 * 2),
        ("iter_key", C.c_uint32), ("model_key", C.c_uint32), ("eps", C.c_double),
        ("max_interactions", C.c_int64), ("peel", C.c_int32), ("terminate_on_absorb", C.c_int32),
        ("nthreads", C.c_int32), ("raytrace", C.c_int32), ("mrw_gamma", C.c_double),
    ]


class ORResult(C.Structure):
    _fields_ = [
        ("acc", _dp), ("sed", _dp), ("img", _dp), ("esc", _dp),
        ("e_escaped", C.c_double), ("e_killed", C.c_double), ("e_absorbed", C.c_double),
        ("n_interactions", C.c_int64), ("n_scatter", C.c_int64), ("n_absorb", C.c_int64),
        ("n_crossings", C.c_int64), ("n_peel_crossings", C.c_int64), ("n_killed", C.c_int64),
        ("visits", _lp), ("n_mrw", C.c_int64),
    ]


def _declare(L):
    L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
    L.or_philox4x32_10.restype = None
    L.or_uniform_from_word.argtypes = [C.c_uint32]
    L.or_uniform_from_word.restype = C.c_double
    L.or_sample_table.argtypes = [C.c_int, _dp, _dp, C.c_double]
    L.or_sample_table.restype = C.c_double
    L.or_isotropic.argtypes = [C.c_double, C.c_double, _dp]
    L.or_isotropic.restype = None
    L.or_hg_mu.argtypes = [C.c_double, C.c_double]
    L.or_hg_mu.restype = C.c_double
    L.or_hg_phase.argtypes = [C.c_double, C.c_double]
    L.or_hg_phase.restype = C.c_double
    L.or_scatter_dir.argtypes = [_dp, C.c_double, C.c_double, _dp]
    L.or_scatter_dir.restype = None
    L.or_cell_exit.argtypes = [C.POINTER(ORModel), _dp, _dp, _ip, _ip, _ip]
    L.or_cell_exit.restype = C.c_double
    L.or_locate.argtypes = [C.POINTER(ORModel), _dp, _dp, _dp, _ip]
    L.or_locate.restype = C.c_int
    L.or_trace.argtypes = [C.POINTER(ORModel), _dp, _dp, C.c_int64, _lp, _dp]
    L.or_trace.restype = C.c_int64
    L.or_raytrace_rays.argtypes = [C.POINTER(ORModel), C.POINTER(ORParams), C.c_int64, _dp, _lp, _dp, _dp]
    L.or_raytrace_rays.restype = C.c_int
    L.or_tau_to_edge.argtypes = [C.POINTER(ORModel), _dp, _dp, C.c_double]
    L.or_tau_to_edge.restype = C.c_double
    L.or_sed_bin.argtypes = [C.POINTER(ORModel), C.c_double]
    L.or_sed_bin.restype = C.c_int
    L.or_wall_distance.argtypes = [C.POINTER(ORModel), _dp, _ip]
    L.or_wall_distance.restype = C.c_double
    L.or_place_in_cell.argtypes = [C.POINTER(ORModel), _ip, _dp, _dp]
    L.or_place_in_cell.restype = None
    L.or_mrw_path.argtypes = [C.c_double, C.c_double]
    L.or_mrw_path.restype = C.c_double
    L.or_run_packets.argtypes = [C.POINTER(ORModel), C.POINTER(ORParams), C.POINTER(ORResult)]
    L.or_run_packets.restype = C.c_int


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t) if a is not None else None


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform_from_word(x):
    return lib().or_uniform_from_word(int(x) & 0xFFFFFFFF)


def sample_table(x, cdf, u):
    x = np.ascontiguousarray(x, dtype=np.float64)
    cdf = np.ascontiguousarray(cdf, dtype=np.float64)
    return lib().or_sample_table(len(x), _ptr(x), _ptr(cdf), float(u))


def isotropic(u1, u2):
    o = (C.c_double * 3)()
    lib().or_isotropic(float(u1), float(u2), o)
    return np.array(o[:])


def hg_mu(g, u):
    return lib().or_hg_mu(float(g), float(u))


def hg_phase(g, mu):
    return lib().or_hg_phase(float(g), float(mu))


def scatter_dir(u, mu, psi):
    ui = (C.c_double * 3)(*[float(v) for v in u])
    o = (C.c_double * 3)()
    lib().or_scatter_dir(ui, float(mu), float(psi), o)
    return np.array(o[:])


class OracleModel:
    """A workload held by the oracle: derived tables plus the iteration state."""

    def __init__(self, wl, t_init: float = 10.0):
        self.wl = wl
        self.gtype = {"cartesian": 0, "spherical": 1, "cylindrical": 2}[wl.grid_type]
        self.walls = [np.ascontiguousarray(w, dtype=np.float64) for w in wl.walls]
        self.shape = tuple(len(w) - 1 for w in self.walls)
        self.rho = np.ascontiguousarray(wl.rho, dtype=np.float64).reshape(-1)
        self.nc = self.rho.size
        self.vol = T.cell_volumes(wl.grid_type, self.walls).reshape(-1)
        self.dust = T.DustTables(wl.nu, wl.chi, wl.albedo, wl.T_nodes)
        self.nu = np.ascontiguousarray(wl.nu, dtype=np.float64)
        self.chi = np.ascontiguousarray(wl.chi, dtype=np.float64)
        self.albedo = np.ascontiguousarray(wl.albedo, dtype=np.float64)
        self.T_nodes = np.ascontiguousarray(wl.T_nodes, dtype=np.float64)
        self.cdf_emit = np.ascontiguousarray(self.dust.cdf, dtype=np.float64)
        # sources: point sources, external isotropic sources, then an optional cell source
        ext = list(getattr(wl, "external_sources", []) or [])
        Ls = [float(s["L"]) for s in wl.sources] + [float(e["L"]) for e in ext]
        self.src_pos = np.ascontiguousarray([s["pos"] for s in wl.sources], dtype=np.float64).reshape(-1)
        # a point source's spectrum: a blackbody of Teff, or its own f_nu ("spectrum": (nu, f_nu))
        spectra = [("user", s["spectrum"]) if "spectrum" in s else ("bb", float(s["Teff"])) for s in wl.sources]
        spectra += [("bb", float(e["Teff"])) for e in ext]
        self.next = len(ext)
        self.ext_c = np.ascontiguousarray([e["center"] for e in ext], dtype=np.float64).reshape(-1)
        self.ext_R = np.ascontiguousarray([e["radius"] for e in ext], dtype=np.float64)
        # the grid scale L0: outer radius (spherical), largest |wall| of every axis (Cartesian) or
        # of R and z (cylindrical)
        axes = {0: (0, 1, 2), 1: (0,), 2: (0, 1)}[self.gtype]
        self.L0 = max(max(abs(float(self.walls[a][0])), abs(float(self.walls[a][-1]))) for a in axes)
        self.cell_cdf = None
        if wl.cell_source is not None:
            Lc = np.asarray(wl.cell_source["L"], dtype=np.float64).reshape(-1)
            Ls.append(float(Lc.sum()))
            spectra.append(("bb", float(wl.cell_source["Teff"])))
            cc = np.cumsum(Lc)
            self.cell_cdf = np.ascontiguousarray(cc / cc[-1])
            self.cell_cdf[-1] = 1.0
        self.L_tot = float(sum(Ls))
        cs = np.cumsum(Ls)
        self.src_cdf = np.ascontiguousarray(cs / cs[-1])
        self.src_cdf[-1] = 1.0
        specs = [T.source_spectrum(self.nu[0], self.nu[-1], v) if kind == "bb"
                 else T.user_source_spectrum(self.nu[0], self.nu[-1], *v) for kind, v in spectra]
        self.spec_nu = np.ascontiguousarray(specs[0][0])
        self.spec_cdf = np.ascontiguousarray(np.stack([s[1] for s in specs]))
        # observers
        n, ex, ey = T.observer_frames(wl.obs_incl, wl.obs_az)
        self.obs_n, self.obs_ex, self.obs_ey = (np.ascontiguousarray(a.reshape(-1)) for a in (n, ex, ey))
        self.nobs = len(wl.obs_incl)
        self.lam_min = wl.lam_min_um * 1e-4
        self.lam_max = wl.lam_max_um * 1e-4
        self.img_bin = np.ascontiguousarray(
            [T.sed_bin_of_lambda(l * 1e-4, wl.nsed, self.lam_min, self.lam_max) for l in wl.img_lam_um],
            dtype=np.int32)
        self.nimg = len(self.img_bin) if wl.img_nx > 0 else 0
        # state
        self.T = np.full(self.nc, float(t_init))
        self.adot = np.zeros(self.nc)
        self.iteration = 0
        self.Q_prev = None
        self.seed = int(wl.seed)
        self.model_key = 0
        self._emit_row = None
        self._struct = None

    # ---------------------------------------------------------------- struct
    def struct(self, emit_row):
        self._emit_row = np.ascontiguousarray(emit_row, dtype=np.int32)
        m = ORModel()
        m.gtype = self.gtype
        m.n = (C.c_int32 * 3)(*self.shape)
        m.w = (_dp * 3)(*[_ptr(w) for w in self.walls])
        m.rho = _ptr(self.rho)
        m.nnu = len(self.nu)
        m.nu, m.chi, m.albedo = _ptr(self.nu), _ptr(self.chi), _ptr(self.albedo)
        m.g = float(self.wl.g)
        m.nT = len(self.T_nodes)
        m.cdf_emit = _ptr(self.cdf_emit)
        m.emit_row = _ptr(self._emit_row, _ip)
        m.npoint = len(self.wl.sources)
        m.src_pos = _ptr(self.src_pos) if self.src_pos.size else None
        m.nsrc = len(self.src_cdf)
        m.src_cdf = _ptr(self.src_cdf)
        m.nspec = len(self.spec_nu)
        m.spec_nu = _ptr(self.spec_nu)
        m.spec_cdf = _ptr(self.spec_cdf)
        m.cell_cdf = _ptr(self.cell_cdf) if self.cell_cdf is not None else None
        m.nobs = self.nobs
        m.obs_n, m.obs_ex, m.obs_ey = _ptr(self.obs_n), _ptr(self.obs_ex), _ptr(self.obs_ey)
        m.nsed = self.wl.nsed
        m.lam_min, m.lam_max = self.lam_min, self.lam_max
        m.img_nx, m.img_ny, m.nimg = self.wl.img_nx, self.wl.img_ny, self.nimg
        m.img_half = float(self.wl.img_half_extent)
        m.img_bin = _ptr(self.img_bin, _ip)
        m.next = self.next
        m.ext_c = _ptr(self.ext_c) if self.next else None
        m.ext_R = _ptr(self.ext_R) if self.next else None
        m.L0 = self.L0
        m.mrw_k = _ptr(self._mrw_k) if getattr(self, "_mrw_k", None) is not None else None
        m.mrw_kp = _ptr(self._mrw_kp) if getattr(self, "_mrw_kp", None) is not None else None
        self._struct = m
        return m

    def mrw_tables(self):
        """Transport Rosseland mean extinction and Planck-mean absorption coefficient on the
        temperature nodes (the modified random walk, Sect. 2.2)."""
        if getattr(self, "_mrw_nodes", None) is None:
            self._mrw_nodes = (T.transport_rosseland_mean(self.nu, self.chi, self.albedo, self.wl.g, self.T_nodes),
                               T.planck_mean_kappa(self.nu, T.kappa_abs(self.chi, self.albedo), self.T_nodes))
        return self._mrw_nodes

    def set_mrw_cells(self, T_cells):
        """Per-cell rho chi_tR(T) and kappa_P(T) (log-log between the temperature nodes) at the
        temperatures a pass starts from."""
        chi_t, kp = self.mrw_tables()
        self._mrw_k = np.ascontiguousarray(self.rho * T.interp_loglog(T_cells, self.T_nodes, chi_t))
        self._mrw_kp = np.ascontiguousarray(T.interp_loglog(T_cells, self.T_nodes, kp))

    # ---------------------------------------------------------------- packets
    def run_packets(self, n_packets, iter_key, peel=False, max_interactions=1_000_000,
                    terminate_on_absorb=False, nthreads=1, first_packet=0, n_total=None, raytrace=False,
                    mrw_gamma=0.0):
        """Propagate packets first_packet .. first_packet+n_packets-1 with the temperatures held
        now; eps = L_tot / n_total (dt = 1 s).  With raytrace, point-source emission and dust
        re-emission are not peeled off (they reach the SEDs by raytracing, Sect. 2.6.3).
        mrw_gamma > 0 turns the modified random walk on (Sect. 2.2)."""
        n_total = n_packets if n_total is None else n_total
        emit_row = T.emission_row(self.T, self.T_nodes)
        if mrw_gamma > 0:
            self.set_mrw_cells(self.T)
        m = self.struct(emit_row)
        P = ORParams()
        P.n_packets = int(n_packets)
        P.first_packet = int(first_packet)
        P.key = (C.c_uint32 * 2)(self.seed & 0xFFFFFFFF, (self.seed >> 32) & 0xFFFFFFFF)
        P.iter_key = int(iter_key) & 0xFFFFFFFF
        P.model_key = int(self.model_key) & 0xFFFFFFFF
        P.eps = self.L_tot / float(n_total)
        P.max_interactions = int(max_interactions)
        P.peel = int(bool(peel))
        P.terminate_on_absorb = int(bool(terminate_on_absorb))
        P.nthreads = int(nthreads)
        P.raytrace = int(bool(raytrace))
        P.mrw_gamma = float(mrw_gamma)
        acc = np.zeros(self.nc)
        sed = np.zeros(max(1, self.nobs * self.wl.nsed))
        img = np.zeros(max(1, self.nobs * self.nimg * self.wl.img_nx * self.wl.img_ny))
        esc = np.zeros(N_ESC_MU * self.wl.nsed)
        visits = np.zeros(self.nc, np.int64)
        R = ORResult()
        R.acc, R.sed, R.img, R.esc = _ptr(acc), _ptr(sed), _ptr(img), _ptr(esc)
        R.visits = _ptr(visits, _lp)
        rc = lib().or_run_packets(C.byref(m), C.byref(P), C.byref(R))
        if rc != 0:
            raise RuntimeError("oracle packet loop failed")
        out = dict(acc=acc, visits=visits, sed=sed[: self.nobs * self.wl.nsed].reshape(self.nobs, self.wl.nsed),
                   esc=esc.reshape(N_ESC_MU, self.wl.nsed), eps=P.eps,
                   e_escaped=R.e_escaped, e_killed=R.e_killed, e_absorbed=R.e_absorbed,
                   n_interactions=R.n_interactions, n_scatter=R.n_scatter, n_absorb=R.n_absorb,
                   n_crossings=R.n_crossings, n_peel_crossings=R.n_peel_crossings, n_killed=R.n_killed,
                   n_mrw=R.n_mrw)
        if self.nimg:
            out["img"] = img.reshape(self.nobs, self.nimg, self.wl.img_ny, self.wl.img_nx)
        return out

    def chi_rosseland(self):
        """Rosseland mean extinction on the temperature nodes (App. A)."""
        if getattr(self, "_chi_r", None) is None:
            self._chi_r = T.rosseland_mean(self.nu, self.chi, self.T_nodes)
        return self._chi_r

    # ---------------------------------------------------------------- iteration
    def run_iteration(self, n_packets=None, p=0.99, quantity="T", peel=False, update=True,
                      max_interactions=1_000_000, terminate_on_absorb=False, nthreads=1, pda_min=0,
                      mrw_gamma=0.0):
        """One Lucy iteration (update=True) or one imaging pass (update=False).  pda_min > 0
        (spherical grids): cells with dust sampled by fewer than pda_min packet path segments
        take their temperature from the partial diffusion approximation (App. A).  mrw_gamma > 0:
        modified random walk in thick cells (Sect. 2.2)."""
        n = self.wl.n_packets if n_packets is None else int(n_packets)
        key = self.iteration if update else (IMAGING_KEY | self.iteration)
        out = self.run_packets(n, key, peel=peel, max_interactions=max_interactions,
                               terminate_on_absorb=terminate_on_absorb, nthreads=nthreads, mrw_gamma=mrw_gamma)
        if update:
            adot = out["acc"] / (self.vol * 1.0)                     # Eq. 2, dt = 1 s
            Tn, _, _ = T.temperature_from_adot(adot, self.T_nodes, self.dust.E)     # Eq. 3
            mask = self.rho > 0
            _, lo, hi = T.temperature_from_adot(adot[mask], self.T_nodes, self.dust.E)
            n_pda = 0
            if pda_min > 0 and self.gtype == 1:
                from . import pda
                Tn, pmask = pda.solve(self.walls, self.rho, Tn, self.T, out["visits"], pda_min, self.T_nodes,
                                      self.chi_rosseland())
                adot = adot.copy()
                adot[pmask] = T.interp_loglog(Tn[pmask], self.T_nodes, self.dust.E)
                n_pda = int(pmask.sum())
            prev = self.T if quantity == "T" else self.adot
            cur = Tn if quantity == "T" else adot
            if self.iteration == 0 and quantity != "T":
                Q, D = float("inf"), float("inf")
            else:
                Q, D = T.convergence(prev, cur, mask, p, self.Q_prev)
            self.Q_prev = Q
            self.T = Tn
            self.adot = adot
            self.iteration += 1
            out.update(adot=adot, T=Tn, Q=Q, Delta=D, clamp_low=lo, clamp_high=hi, n_pda=n_pda)
        return out
