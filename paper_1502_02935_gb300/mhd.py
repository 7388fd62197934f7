"""ctypes binding of libmhd.so (include/mhd.h).  Argument marshalling only.

Every step of the method runs in the library's CUDA kernels; if the library is
missing or cannot load, every entry point raises (there is no fallback).  PyTorch
is used only to hand device buffers and streams to the library.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .inputs import Geom, State

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmhd.so")

PREC_FP64 = 0
PREC_MIXED = 1
FLAG_GRAPH = 1
FLAG_PERSISTENT = 2
POT_NONE, POT_GAUSS_X, POT_LOG_DISC = 0, 1, 2

ERRORS = {0: "MHD_OK", -1: "MHD_ERR_ARG", -2: "MHD_ERR_CUDA", -3: "MHD_ERR_NONFINITE",
          -4: "MHD_ERR_NEGATIVE", -5: "MHD_ERR_TIMEOUT", -6: "MHD_ERR_STATE", -7: "MHD_ERR_NOMEM"}


class MHDError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class PatchDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("bc", C.c_int * 6), ("gamma", C.c_double)]


class GridDesc(C.Structure):
    _fields_ = [("n_patches", C.c_int), ("patches", C.POINTER(PatchDesc)), ("precision", C.c_int),
                ("cfl", C.c_double), ("flags", C.c_int), ("cuda_stream", C.c_void_p)]


class SourceDesc(C.Structure):
    _fields_ = [("potential", C.c_int), ("psi0", C.c_double), ("xc", C.c_double), ("xw", C.c_double),
                ("v0", C.c_double), ("rc", C.c_double), ("rho_floor", C.c_double), ("pr_floor", C.c_double),
                ("pr_ceil", C.c_double)]


class ThermalDesc(C.Structure):
    _fields_ = [("mode", C.c_int), ("gamma_heat", C.c_double), ("z", C.c_double), ("rate_unit", C.c_double),
                ("cap", C.c_double), ("nh_per_rho", C.c_double), ("t_per_pr", C.c_double)]


THERMAL_OFF, THERMAL_PLAIN, THERMAL_SURROGATE = 0, 1, 2


class Metrics(C.Structure):
    _fields_ = [("dt_last", C.c_double), ("sums", C.c_double * 5), ("max_divb", C.c_double),
                ("error_word", C.c_int), ("floored", C.c_ulonglong)]


_lib = None

EXPORTS = ["mhd_init_grid", "mhd_set_sources", "mhd_step", "mhd_cfl_dt", "mhd_cfl_dt_patches",
           "mhd_get_state", "mhd_set_state", "mhd_sync", "mhd_get_metrics", "mhd_launch_count",
           "mhd_last_error", "mhd_destroy", "mhd_riemann_hlld", "mhd_set_profiling", "mhd_get_profile",
           "mhd_cfl_dt_noalloc", "mhd_autotune", "mhd_set_wait_limit", "mhd_set_thermal",
           "mhd_thermal_stats", "mhd_thermal_cells", "mhd_surrogate_harvest", "mhd_surrogate_train",
           "mhd_surrogate_params", "mhd_surrogate_rows", "mhd_mlp_forward", "mhd_mlp_grad",
           "mhd_mlp_forward_tc", "mhd_mlp_grad_tc", "mhd_set_riemann", "mhd_riemann_flux", "mhd_set_reconstruction",
           "mhd_set_inflow", "mhd_set_scalars", "mhd_set_scalar_state", "mhd_get_scalar_state",
           "mhd_set_inflow_scalars", "mhd_surrogate_fallback_cells", "mhd_step_scheme",
           "mhd_set_step_scheme", "mhd_convert_fp", "mhd_set_flux_scheme"]

# Riemann solvers (Section 2.1): HLLD for MHD; HLLC and HLL for pure gas dynamics
RIEMANN = {"hlld": 0, "hllc": 1, "hll": 2}
# kernels of the y and z fluxes (mhd_set_flux_scheme)
FLUX_SCHEMES = {"auto": 0, "march": 1, "per_face": 2}
# corrector reconstructions of Eq. 12-14 (kappa = 1/3, 0, -1)
RECON = {"kappa_third": 0, "kappa_zero": 1, "kappa_upwind": 2}


def lib():
    """Load libmhd.so (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        from . import build
        build.build()
    L = C.CDLL(LIB_PATH)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
    L.mhd_init_grid.argtypes = [C.POINTER(vp), C.POINTER(GridDesc), C.POINTER(vp), C.POINTER(vp), ip]
    L.mhd_set_sources.argtypes = [vp, C.POINTER(SourceDesc)]
    L.mhd_step.argtypes = [vp, C.c_double]
    L.mhd_cfl_dt.argtypes = [vp, dp]
    L.mhd_cfl_dt_patches.argtypes = [vp, dp]
    L.mhd_get_state.argtypes = [vp, ip, vp, vp, ip]
    L.mhd_set_state.argtypes = [vp, ip, vp, vp, ip]
    L.mhd_sync.argtypes = [vp]
    L.mhd_get_metrics.argtypes = [vp, C.POINTER(Metrics)]
    L.mhd_launch_count.argtypes = [vp]
    L.mhd_launch_count.restype = C.c_longlong
    L.mhd_last_error.argtypes = [vp]
    L.mhd_last_error.restype = C.c_char_p
    L.mhd_destroy.argtypes = [vp]
    L.mhd_destroy.restype = None
    L.mhd_riemann_hlld.argtypes = [ip, vp, vp, vp, C.c_double, ip, vp, vp]
    L.mhd_riemann_flux.argtypes = [ip, ip, vp, vp, vp, C.c_double, ip, vp, vp]
    L.mhd_set_riemann.argtypes = [vp, ip]
    L.mhd_set_reconstruction.argtypes = [vp, ip]
    L.mhd_set_inflow.argtypes = [vp, ip, ip, dp]
    L.mhd_set_scalars.argtypes = [vp, ip]
    L.mhd_set_scalar_state.argtypes = [vp, ip, vp, ip]
    L.mhd_get_scalar_state.argtypes = [vp, ip, vp, ip]
    L.mhd_set_inflow_scalars.argtypes = [vp, ip, ip, dp]
    L.mhd_set_profiling.argtypes = [vp, ip]
    L.mhd_get_profile.argtypes = [vp, dp, C.POINTER(C.c_longlong), ip]
    L.mhd_cfl_dt_noalloc.argtypes = [C.POINTER(PatchDesc), C.c_double, vp, vp, vp, vp]
    L.mhd_autotune.argtypes = [vp, C.c_char_p, ip, C.POINTER(C.c_int)]
    L.mhd_step_scheme.argtypes = [vp, C.POINTER(C.c_int)]
    L.mhd_set_step_scheme.argtypes = [vp, ip]
    L.mhd_set_flux_scheme.argtypes = [vp, ip]
    L.mhd_convert_fp.argtypes = [C.c_longlong, vp, vp, vp, vp, vp]
    L.mhd_set_wait_limit.argtypes = [vp, C.c_double, ip]
    L.mhd_set_thermal.argtypes = [vp, C.POINTER(ThermalDesc)]
    L.mhd_thermal_stats.argtypes = [vp, C.POINTER(C.c_ulonglong)]
    L.mhd_thermal_cells.argtypes = [C.c_longlong, vp, vp, vp, vp, C.POINTER(ThermalDesc), vp, vp, vp]
    L.mhd_surrogate_harvest.argtypes = [vp, C.c_longlong, ip]
    L.mhd_surrogate_train.argtypes = [vp, ip, ip, C.c_double, C.c_ulonglong, C.c_double, dp,
                                      C.POINTER(C.c_longlong)]
    L.mhd_surrogate_params.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_float)]
    L.mhd_surrogate_rows.argtypes = [vp, vp, C.c_longlong, C.POINTER(C.c_longlong)]
    L.mhd_surrogate_fallback_cells.argtypes = [vp, vp, C.c_longlong, C.POINTER(C.c_longlong)]
    L.mhd_mlp_forward.argtypes = [C.c_longlong, vp, vp, vp, vp]
    L.mhd_mlp_grad.argtypes = [C.c_longlong, vp, vp, vp, vp, vp]
    L.mhd_mlp_forward_tc.argtypes = [C.c_longlong, vp, vp, vp, vp]
    L.mhd_mlp_grad_tc.argtypes = [C.c_longlong, vp, vp, vp, vp, vp]
    for name in EXPORTS:
        if name not in ("mhd_destroy", "mhd_last_error", "mhd_launch_count"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def patch_desc(g: Geom) -> PatchDesc:
    d = PatchDesc()
    d.nx, d.ny, d.nz = g.nx, g.ny, g.nz
    d.x0, d.y0, d.z0 = g.x0, g.y0, g.z0
    d.dx, d.dy, d.dz = g.dx, g.dy, g.dz
    for a in range(6):
        d.bc[a] = int(g.bc[a])
    d.gamma = g.gamma
    return d


def _prec(p) -> int:
    if p in (PREC_FP64, "fp64", "f64"):
        return PREC_FP64
    if p in (PREC_MIXED, "mixed", "fp32"):
        return PREC_MIXED
    raise ValueError(f"unknown precision {p!r}")


class Grid:
    """A set of independent patches advanced together on one GPU."""

    def __init__(self, states, precision="mixed", cfl: float = 0.4, flags: int = 0, stream=None):
        if isinstance(states, State):
            states = [states]
        self.L = lib()
        self.geoms = [s.geom for s in states]
        self.np = len(states)
        descs = (PatchDesc * self.np)(*[patch_desc(s.geom) for s in states])
        self._descs = descs
        gd = GridDesc(self.np, descs, _prec(precision), float(cfl), int(flags),
                      C.c_void_p(stream if isinstance(stream, int) else (stream or 0)))
        hostU = [np.ascontiguousarray(s.U, dtype=np.float64) for s in states]
        hostB = [np.ascontiguousarray(s.faces_flat(), dtype=np.float64) for s in states]
        Up = (C.c_void_p * self.np)(*[a.ctypes.data for a in hostU])
        Bp = (C.c_void_p * self.np)(*[a.ctypes.data for a in hostB])
        h = C.c_void_p()
        rc = self.L.mhd_init_grid(C.byref(h), C.byref(gd), Up, Bp, 0)
        if rc != 0:
            raise MHDError(rc, "mhd_init_grid")
        self.h = h

    # ---------------------------------------------------------------- calls --
    def _check(self, rc, what):
        if rc != 0:
            raise MHDError(rc, f"{what}: {self.L.mhd_last_error(self.h).decode()}")

    def set_sources(self, potential=POT_NONE, psi0=0.0, xc=0.0, xw=1.0, v0=0.0, rc=0.0, rho_floor=0.0,
                    pr_floor=0.0, pr_ceil=0.0):
        s = SourceDesc(int(potential), psi0, xc, xw, v0, rc, rho_floor, pr_floor, pr_ceil)
        self._check(self.L.mhd_set_sources(self.h, C.byref(s)), "mhd_set_sources")

    def set_riemann(self, solver: str):
        """"hlld" (default), "hllc" or "hll" for the following steps."""
        self._check(self.L.mhd_set_riemann(self.h, RIEMANN[solver]), "mhd_set_riemann")

    def set_inflow(self, patch: int, side: int, w):
        """Primitive state [rho, vx, vy, vz, p, Bx, By, Bz] beyond an inflow side (bc 2)."""
        arr = (C.c_double * 8)(*[float(v) for v in w])
        self._check(self.L.mhd_set_inflow(self.h, int(patch), int(side), arr), "mhd_set_inflow")

    def set_scalars(self, n: int):
        """n passive scalars (rho X, all zero) on every patch; 0 removes them."""
        self._check(self.L.mhd_set_scalars(self.h, int(n)), "mhd_set_scalars")
        self.n_scalars = int(n)

    def set_scalar_state(self, patch: int, S):
        """rho X of a patch, shape (n, nz, ny, nx)."""
        S = np.ascontiguousarray(S, dtype=np.float64)
        self._check(self.L.mhd_set_scalar_state(self.h, patch, S.ctypes.data, 0), "mhd_set_scalar_state")
        self.sync()

    def get_scalar_state(self, patch: int) -> np.ndarray:
        g = self.geoms[patch]
        out = np.empty((self.n_scalars, g.nz, g.ny, g.nx))
        self._check(self.L.mhd_get_scalar_state(self.h, patch, out.ctypes.data, 0), "mhd_get_scalar_state")
        return out

    def set_inflow_scalars(self, patch: int, side: int, xs):
        arr = (C.c_double * len(xs))(*[float(v) for v in xs])
        self._check(self.L.mhd_set_inflow_scalars(self.h, int(patch), int(side), arr), "mhd_set_inflow_scalars")

    def set_reconstruction(self, recon: str):
        """"kappa_third" (default), "kappa_zero" or "kappa_upwind" for the following steps."""
        self._check(self.L.mhd_set_reconstruction(self.h, RECON[recon]), "mhd_set_reconstruction")

    def step(self, dt: float = -1.0):
        self._check(self.L.mhd_step(self.h, float(dt)), "mhd_step")

    def cfl_dt(self) -> float:
        v = C.c_double()
        self._check(self.L.mhd_cfl_dt(self.h, C.byref(v)), "mhd_cfl_dt")
        return v.value

    def cfl_dt_patches(self) -> np.ndarray:
        out = np.zeros(self.np)
        self._check(self.L.mhd_cfl_dt_patches(self.h, out.ctypes.data_as(C.POINTER(C.c_double))),
                    "mhd_cfl_dt_patches")
        return out

    def get_state(self, patch: int = 0) -> State:
        g = self.geoms[patch]
        U = np.empty((5, g.nz, g.ny, g.nx))
        nb = (g.nx + 1) * g.ny * g.nz + g.nx * (g.ny + 1) * g.nz + g.nx * g.ny * (g.nz + 1)
        B = np.empty(nb)
        self._check(self.L.mhd_get_state(self.h, patch, U.ctypes.data, B.ctypes.data, 0), "mhd_get_state")
        n1 = (g.nx + 1) * g.ny * g.nz
        n2 = g.nx * (g.ny + 1) * g.nz
        return State(g, U, B[:n1].reshape(g.nz, g.ny, g.nx + 1).copy(),
                     B[n1:n1 + n2].reshape(g.nz, g.ny + 1, g.nx).copy(),
                     B[n1 + n2:].reshape(g.nz + 1, g.ny, g.nx).copy())

    def get_state_ptr(self, patch: int, U_ptr: int, B_ptr: int, on_device: bool):
        self._check(self.L.mhd_get_state(self.h, patch, U_ptr, B_ptr, int(on_device)), "mhd_get_state")

    def set_state(self, patch: int, st: State):
        U = np.ascontiguousarray(st.U, dtype=np.float64)
        B = np.ascontiguousarray(st.faces_flat(), dtype=np.float64)
        self._check(self.L.mhd_set_state(self.h, patch, U.ctypes.data, B.ctypes.data, 0), "mhd_set_state")

    def set_state_ptr(self, patch: int, U_ptr: int, B_ptr: int, on_device: bool):
        self._check(self.L.mhd_set_state(self.h, patch, U_ptr, B_ptr, int(on_device)), "mhd_set_state")

    def sync(self):
        self._check(self.L.mhd_sync(self.h), "mhd_sync")

    def sync_status(self) -> int:
        return int(self.L.mhd_sync(self.h))

    def metrics(self) -> dict:
        m = Metrics()
        self._check(self.L.mhd_get_metrics(self.h, C.byref(m)), "mhd_get_metrics")
        return {"dt_last": m.dt_last, "sums": list(m.sums), "max_divb": m.max_divb, "error_word": m.error_word,
                "floored": int(m.floored)}

    KERNEL_CLASSES = ["recovery", "flux1_x", "flux1_y", "flux1_z", "flux2_x", "flux2_y", "flux2_z",
                      "emf", "update", "cfl", "persistent", "thermal", "floor", "ghost", "emf_update", "scalars",
                      "flux1_xyz"]

    def set_thermal(self, mode, gamma_heat=2e-26, z=0.02, rate_unit=7.13e-31, cap=0.1, nh_per_rho=0.76,
                    t_per_pr=72.7):
        d = ThermalDesc(int(mode), gamma_heat, z, rate_unit, cap, nh_per_rho, t_per_pr)
        self._check(self.L.mhd_set_thermal(self.h, C.byref(d)), "mhd_set_thermal")

    def surrogate_harvest(self, capacity: int, stride: int = 1):
        self._check(self.L.mhd_surrogate_harvest(self.h, int(capacity), int(stride)), "mhd_surrogate_harvest")

    def surrogate_train(self, epochs=100, batch=8192, lr=3e-3, seed=1502, qmax=0.0):
        loss = C.c_double()
        rows = C.c_longlong()
        self._check(self.L.mhd_surrogate_train(self.h, int(epochs), int(batch), float(lr), int(seed), float(qmax),
                                               C.byref(loss), C.byref(rows)), "mhd_surrogate_train")
        return loss.value, rows.value

    def surrogate_params(self):
        p = (C.c_float * 4545)()
        r = (C.c_float * 10)()
        self._check(self.L.mhd_surrogate_params(self.h, p, r), "mhd_surrogate_params")
        return np.frombuffer(p, dtype=np.float32).copy(), np.frombuffer(r, dtype=np.float32).copy()

    def surrogate_rows(self, max_rows: int) -> np.ndarray:
        """Harvested rows (log10 n_H, log10 T, log10 dt, Z, q, change of log10 T), at most
        max_rows of them."""
        buf = np.zeros((max(int(max_rows), 0), 6), dtype=np.float32)
        held = C.c_longlong()
        self._check(self.L.mhd_surrogate_rows(self.h, buf.ctypes.data, buf.shape[0], C.byref(held)),
                    "mhd_surrogate_rows")
        return buf[:min(buf.shape[0], held.value)].copy()

    def surrogate_fallback_cells(self, max_cells: int) -> np.ndarray:
        """Interior cell indices i + nx (j + ny k) that the last surrogate thermal phase
        handed to the plain integrator (at most max_cells; unordered)."""
        buf = np.zeros(max(int(max_cells), 0), dtype=np.int32)
        held = C.c_longlong()
        self._check(self.L.mhd_surrogate_fallback_cells(self.h, buf.ctypes.data, buf.size, C.byref(held)),
                    "mhd_surrogate_fallback_cells")
        return buf[:min(buf.size, held.value)].copy()

    def thermal_stats(self) -> dict:
        out = (C.c_ulonglong * 4)()
        self._check(self.L.mhd_thermal_stats(self.h, out), "mhd_thermal_stats")
        return {"cells": out[0], "substeps": out[1], "capped": out[2], "fallback": out[3]}

    def autotune(self, cache_path=None, force: bool = False):
        tile = (C.c_int * 2)()
        path = cache_path.encode() if cache_path else None
        self._check(self.L.mhd_autotune(self.h, path, int(force), tile), "mhd_autotune")
        return int(tile[0]), int(tile[1])

    def step_scheme(self) -> str:
        """'persistent' (one launch per step) or 'per_phase' (the autotuner's choice on a
        context made with FLAG_PERSISTENT)."""
        v = C.c_int()
        self._check(self.L.mhd_step_scheme(self.h, C.byref(v)), "mhd_step_scheme")
        return "persistent" if v.value else "per_phase"

    def set_flux_scheme(self, scheme: str):
        """'auto', 'march' or 'per_face': the kernel of the y and z fluxes."""
        self._check(self.L.mhd_set_flux_scheme(self.h, FLUX_SCHEMES[scheme]), "mhd_set_flux_scheme")

    def set_step_scheme(self, scheme: str):
        self._check(self.L.mhd_set_step_scheme(self.h, 1 if scheme == "persistent" else 0), "mhd_set_step_scheme")

    def set_wait_limit(self, limit_ms: float, phantom_blocks: int = 0):
        self._check(self.L.mhd_set_wait_limit(self.h, float(limit_ms), int(phantom_blocks)), "mhd_set_wait_limit")

    def set_profiling(self, on: bool):
        self._check(self.L.mhd_set_profiling(self.h, int(on)), "mhd_set_profiling")

    def profile(self) -> dict:
        n = len(self.KERNEL_CLASSES)
        ms = (C.c_double * n)()
        cnt = (C.c_longlong * n)()
        self._check(self.L.mhd_get_profile(self.h, ms, cnt, n), "mhd_get_profile")
        return {k: (ms[i], int(cnt[i])) for i, k in enumerate(self.KERNEL_CLASSES)}

    def launch_count(self) -> int:
        return int(self.L.mhd_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.L.mhd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def riemann_hlld(wl, wr, bn, gamma: float, precision="fp64") -> np.ndarray:
    """HLLD fluxes of n interfaces computed on the GPU (see mhd_riemann_hlld)."""
    import torch
    wl = torch.as_tensor(np.ascontiguousarray(np.atleast_2d(wl), dtype=np.float64)).cuda()
    wr = torch.as_tensor(np.ascontiguousarray(np.atleast_2d(wr), dtype=np.float64)).cuda()
    bn = torch.as_tensor(np.ascontiguousarray(np.atleast_1d(bn), dtype=np.float64)).cuda()
    n = wl.shape[0]
    out = torch.zeros((n, 8), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib().mhd_riemann_hlld(n, wl.data_ptr(), wr.data_ptr(), bn.data_ptr(), float(gamma),
                                _prec(precision), out.data_ptr(), stream)
    if rc != 0:
        raise MHDError(rc, "mhd_riemann_hlld")
    return out.cpu().numpy()


def riemann_flux(solver: str, wl, wr, bn, gamma: float, precision="fp64") -> np.ndarray:
    """Fluxes of the solver "hlld", "hllc" or "hll" at n interfaces, on the GPU (see
    mhd_riemann_flux)."""
    import torch
    wl = torch.as_tensor(np.ascontiguousarray(np.atleast_2d(wl), dtype=np.float64)).cuda()
    wr = torch.as_tensor(np.ascontiguousarray(np.atleast_2d(wr), dtype=np.float64)).cuda()
    bn = torch.as_tensor(np.ascontiguousarray(np.atleast_1d(bn), dtype=np.float64)).cuda()
    n = wl.shape[0]
    out = torch.zeros((n, 8), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib().mhd_riemann_flux(RIEMANN[solver], n, wl.data_ptr(), wr.data_ptr(), bn.data_ptr(), float(gamma),
                                _prec(precision), out.data_ptr(), stream)
    if rc != 0:
        raise MHDError(rc, "mhd_riemann_flux")
    return out.cpu().numpy()


NOALLOC_MAX_CELLS = 8388608


def cfl_dt_noalloc(geom: Geom, cfl: float, U_ptr: int, B_ptr: int, dt_ptr: int, stream: int = 0) -> int:
    """Call mhd_cfl_dt_noalloc: device pointers in, device pointer out; returns the status."""
    d = patch_desc(geom)
    return int(lib().mhd_cfl_dt_noalloc(C.byref(d), float(cfl), U_ptr, B_ptr, dt_ptr, stream))


def thermal_cells(T0, nh, ce, dt, th: dict):
    """Plain FP64 thermal integrator on the GPU for independent cells; returns (T, status)."""
    import torch
    # (a broadcast view is read-only: copy it into a writable array first)
    arr = [torch.from_numpy(np.array(np.broadcast_to(np.asarray(a, dtype=np.float64), np.shape(T0)))).cuda()
           for a in (T0, nh, ce, dt)]
    out = torch.empty_like(arr[0])
    st = torch.zeros(arr[0].shape, dtype=torch.int32, device="cuda")
    d = ThermalDesc(THERMAL_PLAIN, th.get("gamma_heat", 2e-26), th.get("z", 0.02), th["rate_unit"], th.get("cap", 0.1),
                    th.get("nh_per_rho", 0.76), th.get("t_per_pr", 72.7))
    rc = lib().mhd_thermal_cells(out.numel(), *[a.data_ptr() for a in arr], C.byref(d), out.data_ptr(), st.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    if rc != 0:
        raise MHDError(rc, "mhd_thermal_cells")
    return out.cpu().numpy(), st.cpu().numpy()


MLP_NPARAM = 4545


def mlp_unpack(p):
    """FP32 parameter block -> dict of float64 arrays in the oracle's layout."""
    p = np.asarray(p, dtype=np.float64)
    H = 64
    o = 0
    out = {}
    for k, shape in (("W1", (H, 4)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))):
        n = int(np.prod(shape))
        out[k] = p[o:o + n].reshape(shape)
        o += n
    return out


def mlp_pack(d) -> np.ndarray:
    return np.concatenate([np.asarray(d[k], dtype=np.float32).ravel() for k in ("W1", "b1", "W2", "b2", "w3", "b3")])


def mlp_forward(xs, params, tcgen05: bool = False) -> np.ndarray:
    import torch
    x = torch.as_tensor(np.ascontiguousarray(xs, dtype=np.float32)).cuda()
    p = torch.as_tensor(np.ascontiguousarray(params, dtype=np.float32)).cuda()
    y = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
    fn = lib().mhd_mlp_forward_tc if tcgen05 else lib().mhd_mlp_forward
    rc = fn(x.shape[0], x.data_ptr(), p.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    if rc != 0:
        raise MHDError(rc, "mhd_mlp_forward")
    return y.cpu().numpy()


def mlp_grad(xs, targets, params, tcgen05: bool = False):
    import torch
    t = np.asarray(targets, dtype=np.float32)[:, None]
    rows = np.concatenate([np.asarray(xs, dtype=np.float32), t, np.zeros_like(t)], axis=1)  # harvested-row layout
    r = torch.as_tensor(np.ascontiguousarray(rows)).cuda()
    p = torch.as_tensor(np.ascontiguousarray(params, dtype=np.float32)).cuda()
    g = torch.empty(MLP_NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    fn = lib().mhd_mlp_grad_tc if tcgen05 else lib().mhd_mlp_grad
    rc = fn(rows.shape[0], r.data_ptr(), p.data_ptr(), g.data_ptr(), loss.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
    if rc != 0:
        raise MHDError(rc, "mhd_mlp_grad")
    return float(loss.item()), g.cpu().numpy()


def convert_fp(d, f):
    """The mixed path's FP64 -> FP32 and FP32 -> FP64 device conversions of d and f (numpy
    arrays of one length); returns (float32 array, float64 array)."""
    import torch
    d_t = torch.as_tensor(np.ascontiguousarray(d, dtype=np.float64)).cuda()
    f_t = torch.as_tensor(np.ascontiguousarray(f, dtype=np.float32)).cuda()
    o_f = torch.empty(d_t.numel(), dtype=torch.float32, device="cuda")
    o_d = torch.empty(f_t.numel(), dtype=torch.float64, device="cuda")
    if d_t.numel() != f_t.numel():
        raise ValueError("d and f must have the same length")
    rc = lib().mhd_convert_fp(d_t.numel(), d_t.data_ptr(), f_t.data_ptr(), o_f.data_ptr(), o_d.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    if rc != 0:
        raise MHDError(rc, "mhd_convert_fp")
    return o_f.cpu().numpy(), o_d.cpu().numpy()
