"""Plain FP64 CPU oracle of the MHD step of arXiv:1502.02935 (Section 2.1).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
``cpu_baseline`` / ``--impl reference`` legs may import this package; the product
library never does.  The C sources next to this file are compiled with gcc
(``-O2 -ffp-contract=off -fopenmp``) on first use, or by ``build()``.

State arrays use the library's host format: U is (5, nz, ny, nx) with fields
[rho, rho vx, rho vy, rho vz, E]; Bx is (nz, ny, nx+1), By (nz, ny+1, nx),
Bz (nz+1, ny, nx), each face array holding the face at the low side of its index.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["mhd_oracle.c", "thermal_oracle.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


class OrcPatch(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("bc", C.c_int * 6), ("gamma", C.c_double), ("riemann", C.c_int), ("recon", C.c_int),
                ("inflow", (C.c_double * 8) * 6), ("upwind_eps", C.c_double)]


# Width of Eq. 11's "no contact motion" band (|F_rho| <= eps rho_max max|S|): zero to the
# precision of FP64 data after the pressure recovery's cancellation (the default), and the
# same reading for data rounded to FP32 (the bulk arithmetic of the mixed path).
EQ11_EPS_FP64 = 2.0 ** -32
EQ11_EPS_FP32 = 64 * 2.0 ** -23


# Riemann solvers (Section 2.1): HLLD for MHD; HLLC and HLL for pure gas dynamics.  HLLC
# takes HLLD at faces that carry a field.
RIEMANN = {"hlld": 0, "hllc": 1, "hll": 2}
# Reconstructions of Eq. 12-14: kappa = 1/3 (default), 0, -1 in the standard arrangement, and
# kappa = 1/3 in the printed arrangement (oracle only: a cross-check of that reading).
RECON = {"kappa_third": 0, "kappa_zero": 1, "kappa_upwind": 2, "printed": 3}


class OrcSource(C.Structure):
    _fields_ = [("potential", C.c_int), ("psi0", C.c_double), ("xc", C.c_double),
                ("xw", C.c_double), ("v0", C.c_double), ("rc", C.c_double),
                ("rho_floor", C.c_double), ("pr_floor", C.c_double), ("pr_ceil", C.c_double)]


def build(force: bool = False) -> str:
    """Compile liboracle.so from the C sources beside this file."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS if os.path.exists(os.path.join(_HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "mhd_oracle.h")])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            dp = C.POINTER(C.c_double)
            L.orc_step.argtypes = [C.POINTER(OrcPatch), C.POINTER(OrcSource), dp, dp, dp, dp, C.c_double]
            L.orc_step.restype = C.c_int
            L.orc_cfl_dt.argtypes = [C.POINTER(OrcPatch), C.POINTER(OrcSource), dp, dp, dp, dp, C.c_double]
            L.orc_cfl_dt.restype = C.c_double
            L.orc_run.argtypes = [C.POINTER(OrcPatch), C.POINTER(OrcSource), dp, dp, dp, dp,
                                  C.c_double, C.c_double, C.c_int]
            L.orc_run.restype = C.c_int
            L.orc_step_scalars.argtypes = [C.POINTER(OrcPatch), C.POINTER(OrcSource), dp, dp, dp, dp, C.c_int, dp,
                                           dp, C.c_double]
            L.orc_step_scalars.restype = C.c_int
            L.orc_stage_emf.argtypes = [C.POINTER(OrcPatch), dp, dp, dp, dp, C.c_int, dp]
            L.orc_stage_emf.restype = C.c_int
            L.orc_hlld_batch.argtypes = [C.c_int, dp, dp, dp, C.c_double, dp]
            L.orc_riemann_batch.argtypes = [C.c_int, C.c_int, dp, dp, dp, C.c_double, dp]
            L.orc_reconstruct_1d.argtypes = [C.c_int, dp, dp, dp]
            L.orc_reconstruct_1d_ex.argtypes = [C.c_int, C.c_int, dp, dp, dp]
            L.orc_diagnostics.argtypes = [C.POINTER(OrcPatch), dp, dp, dp, dp, dp, dp]
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_set_threads.restype = C.c_int
            _bind_thermal(L)
            _lib = L
    return _lib


class OrcThermal(C.Structure):
    _fields_ = [("gamma_heat", C.c_double), ("z", C.c_double), ("rate_unit", C.c_double), ("cap", C.c_double),
                ("nh_per_rho", C.c_double), ("t_per_pr", C.c_double)]


def _bind_thermal(L):
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    L.orc_cooling.argtypes = [C.c_long, dp, C.c_double, dp, dp]
    L.orc_cooling.restype = None
    L.orc_thermal_cells.argtypes = [C.c_long, dp, dp, dp, dp, C.POINTER(OrcThermal), dp, ip]
    L.orc_thermal_cells.restype = C.c_int
    L.orc_thermal_apply.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(OrcThermal), dp, dp, dp, dp,
                                    C.c_double]
    L.orc_thermal_apply.restype = C.c_int
    L.orc_surrogate_apply.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(OrcThermal), dp, dp, dp, dp, dp,
                                      dp, C.c_double, ip, dp]
    L.orc_surrogate_apply.restype = C.c_int
    L.orc_bf16_round.argtypes = [C.c_long, dp, dp]
    L.orc_mlp_forward_bf16.argtypes = [C.c_long, dp, dp, dp]
    L.orc_mlp_forward_bf16.restype = None
    L.orc_bf16_round.restype = None
    L.orc_mlp_forward.argtypes = [C.c_long, dp, dp, dp, dp, dp, dp, dp, dp]
    L.orc_mlp_forward.restype = None
    L.orc_mlp_backward.argtypes = [C.c_long, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
    L.orc_mlp_backward.restype = C.c_double


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle wants C-contiguous float64"
    return a.ctypes.data_as(C.POINTER(C.c_double))


def patch_struct(g, riemann: str = "hlld", recon: str = "kappa_third", inflow=None,
                 eq11_eps: float | None = None) -> OrcPatch:
    """``inflow``: {side: [rho, vx, vy, vz, p, Bx, By, Bz]} for the sides whose bc is 2;
    ``eq11_eps``: width of Eq. 11's no-motion band (None: EQ11_EPS_FP64)."""
    p = OrcPatch()
    p.upwind_eps = float(EQ11_EPS_FP64 if eq11_eps is None else eq11_eps)
    p.riemann = RIEMANN[riemann]
    p.recon = RECON[recon]
    for side, w in (inflow or {}).items():
        for m in range(8):
            p.inflow[int(side)][m] = float(w[m])
    p.nx, p.ny, p.nz = g.nx, g.ny, g.nz
    p.x0, p.y0, p.z0 = g.x0, g.y0, g.z0
    p.dx, p.dy, p.dz = g.dx, g.dy, g.dz
    for a in range(6):
        p.bc[a] = int(g.bc[a])
    p.gamma = g.gamma
    return p


def source_struct(src) -> OrcSource:
    s = OrcSource()
    if src is None:
        return s
    s.potential = int(src.get("potential", 0))
    for k in ("psi0", "xc", "xw", "v0", "rc", "rho_floor", "pr_floor", "pr_ceil"):
        setattr(s, k, float(src.get(k, 0.0)))
    return s


def _copy_state(st):
    return (np.ascontiguousarray(st.U, dtype=np.float64).copy(),
            np.ascontiguousarray(st.Bx, dtype=np.float64).copy(),
            np.ascontiguousarray(st.By, dtype=np.float64).copy(),
            np.ascontiguousarray(st.Bz, dtype=np.float64).copy())


def step(st, dt: float, source=None, nsteps: int = 1, floored=None, riemann: str = "hlld",
         recon: str = "kappa_third", inflow=None, eq11_eps=None):
    """``nsteps`` van Leer steps of fixed size dt; returns a new State.  If ``floored``
    is a list, the per-step counts of cells changed by the end-of-step floors are
    appended to it.  ``riemann``: "hlld", "hllc" or "hll"; ``recon``: a key of RECON;
    ``inflow``: the states of the inflow sides (see patch_struct); ``eq11_eps``: width
    of Eq. 11's no-motion band (None: EQ11_EPS_FP64)."""
    L = lib()
    U, Bx, By, Bz = _copy_state(st)
    p, s = patch_struct(st.geom, riemann, recon, inflow, eq11_eps), source_struct(source)
    for _ in range(nsteps):
        n = L.orc_step(C.byref(p), C.byref(s), _p(U), _p(Bx), _p(By), _p(Bz), float(dt))
        if n < 0:
            raise ValueError("orc_step rejected its arguments")
        if floored is not None:
            floored.append(int(n))
    return st.replace(U=U, Bx=Bx, By=By, Bz=Bz)


def step_scalars(st, S, dt: float, source=None, riemann: str = "hlld", recon: str = "kappa_third", inflow=None,
                 inflow_x=None, eq11_eps=None):
    """One van Leer step that also advects passive scalars: S is rho X, shape
    (ns, nz, ny, nx); ``inflow_x`` = {side: [X_0, ..., X_ns-1]} beyond inflow sides.
    Returns (State, S)."""
    U, Bx, By, Bz = _copy_state(st)
    S = np.ascontiguousarray(S, dtype=np.float64).copy()
    ns = S.shape[0]
    p, s = patch_struct(st.geom, riemann, recon, inflow, eq11_eps), source_struct(source)
    ix = np.zeros(6 * max(ns, 1))
    for side, xs in (inflow_x or {}).items():
        ix[int(side) * ns:(int(side) + 1) * ns] = xs
    n = lib().orc_step_scalars(C.byref(p), C.byref(s), _p(U), _p(Bx), _p(By), _p(Bz), ns, _p(S), _p(ix), float(dt))
    if n < 0:
        raise ValueError("orc_step_scalars rejected its arguments")
    return st.replace(U=U, Bx=Bx, By=By, Bz=Bz), S


def cfl_dt(st, cfl: float, source=None, inflow=None) -> float:
    U, Bx, By, Bz = _copy_state(st)
    return float(lib().orc_cfl_dt(C.byref(patch_struct(st.geom, inflow=inflow)), C.byref(source_struct(source)),
                                  _p(U), _p(Bx), _p(By), _p(Bz), cfl))


def stage_emf(st, order: int = 1, eq11_eps=None) -> np.ndarray:
    """The corner EMFs (Eq. 9-11) of one stage for the state given: order 1 is the
    predictor's donor-cell stage, order 2 the corrector's.  Returns E of shape
    (3, nz, ny, nx); E[c][k, j, i] is the edge along axis c at cell (i, j, k)'s low corner."""
    U, Bx, By, Bz = _copy_state(st)
    nx, ny, nz = st.geom.nx, st.geom.ny, st.geom.nz
    E = np.zeros((3, nz, ny, nx))
    if lib().orc_stage_emf(C.byref(patch_struct(st.geom, eq11_eps=eq11_eps)), _p(U), _p(Bx), _p(By), _p(Bz), int(order), _p(E)) != 0:
        raise ValueError("orc_stage_emf rejected its arguments")
    return E


def run(st, cfl: float, t_end: float, max_steps: int = 10 ** 9, source=None, riemann: str = "hlld",
        recon: str = "kappa_third", inflow=None, eq11_eps=None):
    """Advance to t_end with CFL time steps; returns (State, steps)."""
    U, Bx, By, Bz = _copy_state(st)
    p, s = patch_struct(st.geom, riemann, recon, inflow, eq11_eps), source_struct(source)
    n = lib().orc_run(C.byref(p), C.byref(s), _p(U), _p(Bx), _p(By), _p(Bz), float(cfl),
                      float(t_end), int(max_steps))
    if n < 0:
        raise ValueError("orc_run rejected its arguments")
    return st.replace(U=U, Bx=Bx, By=By, Bz=Bz), n


def hlld(wl, wr, bn, gamma: float) -> np.ndarray:
    wl = np.ascontiguousarray(np.atleast_2d(wl), dtype=np.float64)
    wr = np.ascontiguousarray(np.atleast_2d(wr), dtype=np.float64)
    bn = np.ascontiguousarray(np.atleast_1d(bn), dtype=np.float64)
    n = wl.shape[0]
    out = np.zeros((n, 8))
    lib().orc_hlld_batch(n, _p(wl), _p(wr), _p(bn), float(gamma), _p(out))
    return out


def riemann_flux(solver: str, wl, wr, bn, gamma: float) -> np.ndarray:
    """Fluxes of the solver "hlld", "hllc" or "hll" at a batch of interfaces (same layout
    as hlld)."""
    wl = np.ascontiguousarray(np.atleast_2d(wl), dtype=np.float64)
    wr = np.ascontiguousarray(np.atleast_2d(wr), dtype=np.float64)
    bn = np.ascontiguousarray(np.atleast_1d(bn), dtype=np.float64)
    n = wl.shape[0]
    out = np.zeros((n, 8))
    lib().orc_riemann_batch(RIEMANN[solver], n, _p(wl), _p(wr), _p(bn), float(gamma), _p(out))
    return out


def reconstruct_1d(w, recon: str = "kappa_third"):
    w = np.ascontiguousarray(w, dtype=np.float64)
    wl = np.full_like(w, np.nan)
    wr = np.full_like(w, np.nan)
    lib().orc_reconstruct_1d_ex(RECON[recon], w.size, _p(w), _p(wl), _p(wr))
    return wl, wr


def diagnostics(st):
    """(sums of the 5 cell fields over the interior, max |div B| * min(d))."""
    U, Bx, By, Bz = _copy_state(st)
    sums = np.zeros(5)
    m = np.zeros(1)
    lib().orc_diagnostics(C.byref(patch_struct(st.geom)), _p(U), _p(Bx), _p(By), _p(Bz),
                          _p(sums), _p(m))
    return sums, float(m[0])


def set_threads(n: int) -> int:
    return int(lib().orc_set_threads(int(n)))


# ----------------------------------------------------------------- thermal ----

def thermal_struct(th: dict) -> OrcThermal:
    t = OrcThermal()
    t.gamma_heat = float(th.get("gamma_heat", 2e-26))
    t.z = float(th.get("z", 0.02))
    t.rate_unit = float(th["rate_unit"])
    t.cap = float(th.get("cap", 0.1))
    t.nh_per_rho = float(th["nh_per_rho"])
    t.t_per_pr = float(th["t_per_pr"])
    return t


def cooling(T, z: float = 0.02):
    T = np.ascontiguousarray(np.atleast_1d(T), dtype=np.float64)
    lam = np.empty_like(T)
    slope = np.empty_like(T)
    lib().orc_cooling(T.size, _p(T), float(z), _p(lam), _p(slope))
    return lam, slope


def thermal_cells(T0, nh, ce, dt, th: dict):
    """Backward-Euler thermal integration of independent cells; returns (T, status)."""
    arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), np.shape(T0))).copy()
            for a in (T0, nh, ce, dt)]
    out = np.empty_like(arrs[0])
    st = np.zeros(arrs[0].shape, dtype=np.int32)
    t = thermal_struct(th)
    lib().orc_thermal_cells(out.size, *[_p(a) for a in arrs], C.byref(t), _p(out),
                            st.ctypes.data_as(C.POINTER(C.c_int)))
    return out, st


def thermal_apply(st, dt: float, th: dict):
    """Operator-split thermal update of a State (returns a new State and the status bits)."""
    U, Bx, By, Bz = _copy_state(st)
    g = st.geom
    t = thermal_struct(th)
    rc = lib().orc_thermal_apply(g.nx, g.ny, g.nz, g.gamma, C.byref(t), _p(U), _p(Bx), _p(By), _p(Bz), float(dt))
    return st.replace(U=U), int(rc)


def bf16_round(v):
    """Round to the nearest BF16 value (8 significant bits, ties to even), in FP64."""
    v = np.ascontiguousarray(np.atleast_1d(v), dtype=np.float64)
    out = np.empty_like(v)
    lib().orc_bf16_round(v.size, _p(v), _p(out))
    return out


def mlp_forward_bf16(X, params):
    """The surrogate network as the step evaluates it (FP64, h1 and W2 rounded to BF16) on
    standardised rows X[n][4]; params: the 4545 values W1, b1, W2, b2, w3, b3."""
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 4)
    prm = np.ascontiguousarray(params, dtype=np.float64)
    assert prm.size == 4545
    Y = np.empty(X.shape[0])
    lib().orc_mlp_forward_bf16(X.shape[0], _p(X), _p(prm), _p(Y))
    return Y


def surrogate_apply(st, dt: float, th: dict, params, rng):
    """The surrogate thermal update of a State as the step applies it (see
    orc_surrogate_apply): ``params`` the 4545 network parameters (W1, b1, W2, b2, w3, b3),
    ``rng`` the 10 range values (lo[4], s[4], qmax, dmax).  Returns (State, fallback mask
    (nz, ny, nx), features (nz, ny, nx, 6) = standardised x[4], q, S, integrator status)."""
    U, Bx, By, Bz = _copy_state(st)
    g = st.geom
    prm = np.ascontiguousarray(params, dtype=np.float64)
    rg = np.ascontiguousarray(rng, dtype=np.float64)
    assert prm.size == 4545 and rg.size == 10
    fb = np.zeros((g.nz, g.ny, g.nx), dtype=np.int32)
    feat = np.zeros((g.nz, g.ny, g.nx, 6))
    t = thermal_struct(th)
    rc = lib().orc_surrogate_apply(g.nx, g.ny, g.nz, g.gamma, C.byref(t), _p(prm), _p(rg), _p(U), _p(Bx), _p(By),
                                   _p(Bz), float(dt), fb.ctypes.data_as(C.POINTER(C.c_int)), _p(feat))
    return st.replace(U=U), fb.astype(bool), feat, int(rc)


# --------------------------------------------------------------------- MLP ----
HIDDEN = 64


def mlp_forward(X, params):
    X = np.ascontiguousarray(X, dtype=np.float64)
    W1, b1, W2, b2, w3, b3 = [np.ascontiguousarray(params[k], dtype=np.float64) for k in ("W1", "b1", "W2", "b2", "w3", "b3")]
    Y = np.empty(X.shape[0])
    lib().orc_mlp_forward(X.shape[0], _p(X), _p(W1), _p(b1), _p(W2), _p(b2), _p(w3), _p(b3), _p(Y))
    return Y


def mlp_backward(X, T, params):
    """(loss, grads) with grads keyed like params."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    P = {k: np.ascontiguousarray(params[k], dtype=np.float64) for k in ("W1", "b1", "W2", "b2", "w3", "b3")}
    G = {k: np.zeros_like(v) for k, v in P.items()}
    loss = lib().orc_mlp_backward(X.shape[0], _p(X), _p(T), _p(P["W1"]), _p(P["b1"]), _p(P["W2"]), _p(P["b2"]),
                                  _p(P["w3"]), _p(P["b3"]), _p(G["W1"]), _p(G["b1"]), _p(G["W2"]), _p(G["b2"]),
                                  _p(G["w3"]), _p(G["b3"]))
    return float(loss), G
