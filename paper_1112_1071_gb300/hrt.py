"""Thin ctypes binding of libhrt (include/hrt.h).

Functions keep the C names (``hrt_create``, ``hrt_run_iteration``, ...) and only marshal
arguments: numpy arrays become host pointers, torch CUDA tensors become device pointers and
the current torch stream becomes the context stream.  Every step of the computation runs in
the library's CUDA kernels; there is no Python or CPU fallback, and ``load()`` raises when the
library has not been built.

``Model`` is a convenience wrapper that feeds a ``workloads.Workload`` through the same C calls.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhrt.so")

HRT_OK, HRT_EINVAL, HRT_ENOMEM, HRT_ESTATE, HRT_ECUDA, HRT_ETIMEDOUT, HRT_ERANGE = 0, -1, -2, -3, -4, -5, -6
HRT_KERNEL_EVENT, HRT_KERNEL_PLAIN, HRT_KERNEL_REGROUP = 0, 1, 2
_STATUS = {0: "HRT_OK", -1: "HRT_EINVAL", -2: "HRT_ENOMEM", -3: "HRT_ESTATE", -4: "HRT_ECUDA",
           -5: "HRT_ETIMEDOUT", -6: "HRT_ERANGE"}


class HrtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class hrt_run_params(C.Structure):
    _fields_ = [
        ("max_interactions", C.c_int64), ("peel", C.c_int32), ("update_temperature", C.c_int32),
        ("terminate_on_absorb", C.c_int32), ("quantity", C.c_int32), ("p", C.c_double),
        ("q_thres", C.c_double), ("delta_thres", C.c_double), ("kernel", C.c_int32),
        ("block_size", C.c_int32), ("blocks_per_sm", C.c_int32), ("regroup_threshold", C.c_int32),
        ("watchdog_ms", C.c_double), ("first_packet", C.c_int64), ("n_total", C.c_int64),
        ("pda_min_visits", C.c_int64), ("raytrace_rays", C.c_int64), ("mrw_gamma", C.c_double),
        ("peel_queue_events", C.c_int64),
    ]


class hrt_iter_stats(C.Structure):
    _fields_ = [
        ("iteration", C.c_int32), ("converged", C.c_int32), ("Q", C.c_double), ("Delta", C.c_double),
        ("e_emitted", C.c_double), ("e_escaped", C.c_double), ("e_killed", C.c_double),
        ("e_absorbed", C.c_double), ("n_packets", C.c_int64), ("n_interactions", C.c_int64),
        ("n_scatter", C.c_int64), ("n_absorb", C.c_int64), ("n_crossings", C.c_int64),
        ("n_peel_crossings", C.c_int64), ("n_killed", C.c_int64), ("clamp_low", C.c_int64),
        ("clamp_high", C.c_int64), ("ms_propagate", C.c_double), ("ms_total", C.c_double),
        ("kernel_launches", C.c_int64), ("n_pda", C.c_int64), ("pda_iterations", C.c_int64),
        ("pda_residual", C.c_double), ("n_mrw", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_i64 = C.c_int64

# name -> (restype, argtypes)
_SIGS = {
    "hrt_version": (C.c_char_p, []),
    "hrt_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_uint64, _vp]),
    "hrt_destroy": (C.c_int, [_vp]),
    "hrt_last_error": (C.c_char_p, [_vp]),
    "hrt_set_stream": (C.c_int, [_vp, _vp]),
    "hrt_set_grid_cartesian": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp]),
    "hrt_set_grid_spherical": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp]),
    "hrt_set_grid_cylindrical": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp]),
    "hrt_add_external_source": (C.c_int, [_vp, _vp, C.c_double, C.c_double, C.c_double]),
    "hrt_set_density": (C.c_int, [_vp, _vp, _i64]),
    "hrt_set_dust": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, C.c_double, C.c_int, _vp]),
    "hrt_add_point_source": (C.c_int, [_vp, _vp, C.c_double, C.c_double]),
    "hrt_add_point_source_spectrum": (C.c_int, [_vp, _vp, C.c_double, C.c_int, _vp, _vp]),
    "hrt_set_cell_source": (C.c_int, [_vp, _vp, _i64, C.c_double]),
    "hrt_clear_sources": (C.c_int, [_vp]),
    "hrt_set_peeloff": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                  C.c_double, C.c_int, _vp]),
    "hrt_default_params": (None, [C.POINTER(hrt_run_params)]),
    "hrt_run_iteration": (C.c_int, [_vp, _i64, C.POINTER(hrt_run_params), C.POINTER(hrt_iter_stats)]),
    "hrt_get_temperature": (C.c_int, [_vp, _vp, _i64]),
    "hrt_get_specific_energy": (C.c_int, [_vp, _vp, _i64]),
    "hrt_get_absorbed": (C.c_int, [_vp, _vp, _i64]),
    "hrt_get_sed": (C.c_int, [_vp, _vp, _i64]),
    "hrt_get_image": (C.c_int, [_vp, _vp, _i64]),
    "hrt_get_escape": (C.c_int, [_vp, _vp, _i64]),
    "hrt_get_temperature_device": (C.c_int, [_vp, _vp, _i64]),
    "hrt_get_sed_device": (C.c_int, [_vp, _vp, _i64]),
    "hrt_num_cells": (C.c_int64, [_vp]),
    "hrt_set_temperature": (C.c_int, [_vp, _vp, _i64]),
    "hrt_set_temperature_device": (C.c_int, [_vp, _vp, _i64]),
    "hrt_get_watchdog_report": (C.c_int, [_vp, _vp, _i64]),
    "hrt_set_iteration": (C.c_int, [_vp, C.c_int]),
    "hrt_set_specific_energy": (C.c_int, [_vp, _vp, _i64]),
    "hrt_set_convergence_state": (C.c_int, [_vp, C.c_int, C.c_double]),
    "hrt_get_convergence_state": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "hrt_set_model_id": (C.c_int, [_vp, C.c_uint32]),
    "hrt_step_philox": (C.c_int, [_i64, _vp, _vp, _vp, _vp]),
    "hrt_step_cell_exit": (C.c_int, [_vp, _i64, _vp, _vp, _vp, _vp, _vp]),
    "hrt_step_tau_to_edge": (C.c_int, [_vp, _i64, _vp, _vp, _vp, _vp]),
    "hrt_step_wall_distance": (C.c_int, [_vp, _i64, _vp, _vp, _vp]),
    "hrt_step_mrw_path": (C.c_int, [_i64, _vp, _vp, _vp, _vp]),
    "hrt_step_hg_scatter": (C.c_int, [_vp, _i64, _vp, _vp, _vp, _vp]),
    "hrt_step_sample_emission": (C.c_int, [_vp, _i64, _vp, _vp, _vp]),
    "hrt_step_sample_source": (C.c_int, [_vp, _i64, _vp, _vp, _vp]),
    "hrt_step_temperature": (C.c_int, [_vp, _i64, _vp, _vp]),
    "hrt_get_tables": (C.c_int, [_vp, _vp, _i64, _vp, _i64]),
    "hrt_get_rosseland": (C.c_int, [_vp, _vp, _i64]),
    "hrt_get_visits": (C.c_int, [_vp, _vp, _i64]),
    "hrt_quantile_ratio_noalloc": (C.c_int, [_i64, _vp, _vp, _vp, C.c_double, _vp, _vp]),
    "hrt_net_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_int, C.c_int, C.c_uint64, _vp]),
    "hrt_net_create_widths": (C.c_int, [C.POINTER(_vp), C.c_int, _vp, C.c_int, C.c_uint64, _vp]),
    "hrt_net_destroy": (C.c_int, [_vp]),
    "hrt_net_num_params": (C.c_int64, [_vp]),
    "hrt_net_get_params": (C.c_int, [_vp, _vp, _i64]),
    "hrt_net_set_params": (C.c_int, [_vp, _vp, _i64]),
    "hrt_net_forward": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp]),
    "hrt_net_gradients": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _i64,
                                    C.POINTER(C.c_double)]),
    "hrt_net_train_step": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, C.c_float,
                                     C.POINTER(C.c_double)]),
    "hrt_net_features": (C.c_int, [_vp, _vp, _i64]),
    "hrt_net_temperature_target": (C.c_int, [_vp, _vp, _i64]),
    "hrt_net_warm_start": (C.c_int, [_vp, _vp]),
    "hrt_nn_conv3d": (C.c_int, [C.c_int] * 6 + [_vp, _vp, _vp, C.c_int, _vp, _vp]),
    "hrt_nn_conv3d_mma": (C.c_int, [C.c_int] * 6 + [_vp, _vp, _vp, C.c_int, _vp, _vp]),
    "hrt_nn_conv3d_phased": (C.c_int, [C.c_int] * 6 + [_vp, _vp, _vp, C.c_int, _vp, _vp]),
    "hrt_nn_conv3d_backward": (C.c_int, [C.c_int] * 6 + [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "hrt_batch_create": (C.c_int, [C.POINTER(_vp), C.POINTER(_vp), C.c_int]),
    "hrt_batch_destroy": (C.c_int, [_vp]),
    "hrt_batch_run": (C.c_int, [_vp, _vp, C.c_int, C.POINTER(hrt_run_params), _vp, C.POINTER(C.c_int)]),
    "hrt_batch_tune": (C.c_int, [_vp, _vp]),
}

_lib = None


def load(path: str | None = None):
    """Load libhrt.so (built by ``paper_1112_1071_gb300.build``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libhrt.so not built at {p}: run `python -m paper_1112_1071_gb300.build` "
                          "(there is no CPU fallback)")
    lib = C.CDLL(p)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name, None)
        if f is None:
            continue
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def _ptr(a):
    """Host numpy array or torch tensor (CPU/CUDA) -> address."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def check(ctx, rc):
    if rc != HRT_OK:
        msg = load().hrt_last_error(ctx).decode() if ctx else ""
        raise HrtError(rc, msg)
    return rc


def default_params(**kw):
    p = hrt_run_params()
    load().hrt_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Model:
    """A workload held in one libhrt context (all setup through the C calls)."""

    def __init__(self, wl, device: int = 0, seed: int | None = None, stream=None):
        L = load()
        self.wl = wl
        self.ctx = C.c_void_p()
        rc = L.hrt_create(C.byref(self.ctx), device, int(wl.seed if seed is None else seed) & (2**64 - 1),
                          _stream_ptr(stream))
        if rc != HRT_OK:
            raise HrtError(rc, "hrt_create failed (no CUDA device?)")
        self._keep = []
        w = [_c64(x) for x in wl.walls]
        self._keep += w
        n1, n2, n3 = (len(x) - 1 for x in w)
        f = {"cartesian": L.hrt_set_grid_cartesian, "spherical": L.hrt_set_grid_spherical,
             "cylindrical": L.hrt_set_grid_cylindrical}[wl.grid_type]
        check(self.ctx, f(self.ctx, n1, n2, n3, _ptr(w[0]), _ptr(w[1]), _ptr(w[2])))
        rho = np.ascontiguousarray(wl.rho, dtype=np.float32).reshape(-1)
        check(self.ctx, L.hrt_set_density(self.ctx, _ptr(rho), rho.size))
        nu, chi, alb, Tn = _c64(wl.nu), _c64(wl.chi), _c64(wl.albedo), _c64(wl.T_nodes)
        check(self.ctx, L.hrt_set_dust(self.ctx, len(nu), _ptr(nu), _ptr(chi), _ptr(alb), float(wl.g), len(Tn), _ptr(Tn)))
        for s in wl.sources:
            x = _c64(s["pos"])
            if "spectrum" in s:                 # its own f_nu: (nu, f_nu)
                snu, sf = _c64(s["spectrum"][0]), _c64(s["spectrum"][1])
                check(self.ctx, L.hrt_add_point_source_spectrum(self.ctx, _ptr(x), float(s["L"]), len(snu), _ptr(snu),
                                                                _ptr(sf)))
            else:
                check(self.ctx, L.hrt_add_point_source(self.ctx, _ptr(x), float(s["L"]), float(s["Teff"])))
        for e in getattr(wl, "external_sources", []) or []:
            c = _c64(e["center"])
            check(self.ctx, L.hrt_add_external_source(self.ctx, _ptr(c), float(e["radius"]), float(e["L"]),
                                                      float(e["Teff"])))
        if wl.cell_source is not None:
            Lc = _c64(wl.cell_source["L"]).reshape(-1)
            check(self.ctx, L.hrt_set_cell_source(self.ctx, _ptr(Lc), Lc.size, float(wl.cell_source["Teff"])))
        inc, az, il = _c64(wl.obs_incl), _c64(wl.obs_az), _c64(wl.img_lam_um)
        self._keep += [inc, az, il]
        check(self.ctx, L.hrt_set_peeloff(self.ctx, len(inc), _ptr(inc), _ptr(az), int(wl.nsed), float(wl.lam_min_um),
                                          float(wl.lam_max_um), int(wl.img_nx), int(wl.img_ny),
                                          float(wl.img_half_extent), len(il), _ptr(il) if len(il) else None))
        self.ncells = int(L.hrt_num_cells(self.ctx))
        self.nobs = len(inc)

    def close(self):
        if self.ctx:
            load().hrt_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run_iteration(self, n_packets=None, params=None, **kw):
        n = int(self.wl.n_packets if n_packets is None else n_packets)
        p = params if params is not None else default_params(**kw)
        st = hrt_iter_stats()
        rc = load().hrt_run_iteration(self.ctx, n, C.byref(p), C.byref(st))
        check(self.ctx, rc)
        return st.as_dict()

    def _get(self, fname, n, dtype=np.float64):
        out = np.empty(n, dtype=dtype)
        check(self.ctx, getattr(load(), fname)(self.ctx, _ptr(out), n))
        return out

    def temperature(self):
        return self._get("hrt_get_temperature", self.ncells)

    def specific_energy(self):
        return self._get("hrt_get_specific_energy", self.ncells)

    def absorbed(self):
        return self._get("hrt_get_absorbed", self.ncells)

    def sed(self):
        return self._get("hrt_get_sed", self.nobs * self.wl.nsed).reshape(self.nobs, self.wl.nsed)

    def image(self):
        nimg = len(self.wl.img_lam_um) if self.wl.img_nx > 0 else 0
        n = self.nobs * nimg * self.wl.img_nx * self.wl.img_ny
        return self._get("hrt_get_image", max(n, 0)).reshape(self.nobs, nimg, self.wl.img_ny, self.wl.img_nx)

    def escape(self):
        return self._get("hrt_get_escape", 10 * self.wl.nsed).reshape(10, self.wl.nsed)

    def set_temperature(self, T):
        T = _c64(T).reshape(-1)
        check(self.ctx, load().hrt_set_temperature(self.ctx, _ptr(T), T.size))

    def set_iteration(self, i):
        check(self.ctx, load().hrt_set_iteration(self.ctx, int(i)))

    def set_specific_energy(self, adot):
        adot = _c64(adot).reshape(-1)
        check(self.ctx, load().hrt_set_specific_energy(self.ctx, _ptr(adot), adot.size))

    def convergence_state(self):
        have, q = C.c_int(), C.c_double()
        check(self.ctx, load().hrt_get_convergence_state(self.ctx, C.byref(have), C.byref(q)))
        return int(have.value), float(q.value)

    def set_convergence_state(self, have_Q, Q_prev):
        check(self.ctx, load().hrt_set_convergence_state(self.ctx, int(have_Q), float(Q_prev)))

    def tables(self):
        nT, nnu = len(self.wl.T_nodes), len(self.wl.nu)
        E = np.empty(nT)
        cdf = np.empty(nT * nnu, dtype=np.float32)
        check(self.ctx, load().hrt_get_tables(self.ctx, _ptr(E), nT, _ptr(cdf), cdf.size))
        return E, cdf.reshape(nT, nnu)

    def rosseland(self):
        out = np.empty(len(self.wl.T_nodes))
        check(self.ctx, load().hrt_get_rosseland(self.ctx, _ptr(out), out.size))
        return out

    def visits(self):
        return self._get("hrt_get_visits", self.ncells, np.uint32)

    # ---- single steps on torch CUDA tensors
    def step(self, name, *args):
        check(self.ctx, getattr(load(), name)(self.ctx, *args))
