"""Seeded synthetic initial states for the MHD step (shared by the CUDA path and the oracle).

This module only builds inputs: grid geometry, initial primitive fields and
their conserved form.  It contains none of the step's arithmetic.  All fields
are FP64 numpy arrays in the library's host format:

  U  : (5, nz, ny, nx)   [rho, rho vx, rho vy, rho vz, E]
  Bx : (nz, ny, nx+1)    Bx[k, j, i] on face x_{i-1/2}
  By : (nz, ny+1, nx)    on face y_{j-1/2}
  Bz : (nz+1, ny, nx)    on face z_{k-1/2}

Units are code units with Heaviside-Lorentz field (P* = P + B^2/2, the text
after Eq. 3 of arXiv:1502.02935); initial field values that the tests quote
with a 1/sqrt(4 pi) keep it.  Non-uniform fields are built from a vector
potential on cell edges, so that their discrete divergence is zero.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BC_PERIODIC = 0
BC_OUTFLOW = 1


@dataclasses.dataclass(frozen=True)
class Geom:
    nx: int
    ny: int
    nz: int
    x0: float = 0.0
    y0: float = 0.0
    z0: float = 0.0
    dx: float = 1.0
    dy: float = 1.0
    dz: float = 1.0
    bc: tuple = (0, 0, 0, 0, 0, 0)
    gamma: float = 5.0 / 3.0

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    def centres(self):
        x = self.x0 + (np.arange(self.nx) + 0.5) * self.dx
        y = self.y0 + (np.arange(self.ny) + 0.5) * self.dy
        z = self.z0 + (np.arange(self.nz) + 0.5) * self.dz
        return x, y, z

    def faces(self):
        x = self.x0 + np.arange(self.nx + 1) * self.dx
        y = self.y0 + np.arange(self.ny + 1) * self.dy
        z = self.z0 + np.arange(self.nz + 1) * self.dz
        return x, y, z


@dataclasses.dataclass
class State:
    geom: Geom
    U: np.ndarray
    Bx: np.ndarray
    By: np.ndarray
    Bz: np.ndarray

    def replace(self, **kw) -> "State":
        return dataclasses.replace(self, **kw)

    def copy(self) -> "State":
        return State(self.geom, self.U.copy(), self.Bx.copy(), self.By.copy(), self.Bz.copy())

    def faces_flat(self) -> np.ndarray:
        """Bx, By, Bz concatenated (the library's face block)."""
        return np.concatenate([self.Bx.ravel(), self.By.ravel(), self.Bz.ravel()])

    def bcc(self):
        """Cell-centred field as the mean of the two face values (Eq. 6 of the paper)."""
        return (0.5 * (self.Bx[:, :, :-1] + self.Bx[:, :, 1:]),
                0.5 * (self.By[:, :-1, :] + self.By[:, 1:, :]),
                0.5 * (self.Bz[:-1, :, :] + self.Bz[1:, :, :]))


def face_block_size(g: Geom) -> int:
    return ((g.nx + 1) * g.ny * g.nz + g.nx * (g.ny + 1) * g.nz + g.nx * g.ny * (g.nz + 1))


def state_from_prim(g: Geom, rho, vx, vy, vz, p, Bx, By, Bz) -> State:
    """Conserved state from primitive cell fields and face fields.

    E = p/(gamma-1) + rho v^2/2 + Bcc^2/2 with Bcc the mean of the face values, so
    that the closure recovers p exactly up to rounding (text after Eq. 3)."""
    shp = (g.nz, g.ny, g.nx)
    rho, vx, vy, vz, p = (np.broadcast_to(np.asarray(a, dtype=np.float64), shp) for a in (rho, vx, vy, vz, p))
    Bx = np.ascontiguousarray(np.broadcast_to(np.asarray(Bx, dtype=np.float64), (g.nz, g.ny, g.nx + 1)))
    By = np.ascontiguousarray(np.broadcast_to(np.asarray(By, dtype=np.float64), (g.nz, g.ny + 1, g.nx)))
    Bz = np.ascontiguousarray(np.broadcast_to(np.asarray(Bz, dtype=np.float64), (g.nz + 1, g.ny, g.nx)))
    st = State(g, np.zeros((5,) + shp), Bx, By, Bz)
    bx, by, bz = st.bcc()
    U = st.U
    U[0] = rho
    U[1] = rho * vx
    U[2] = rho * vy
    U[3] = rho * vz
    U[4] = p / (g.gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * (bx * bx + by * by + bz * bz)
    return st


def faces_from_Az(g: Geom, Az):
    """Face fields of B = curl(A_z z^) from A_z(x, y) sampled on z-edges (exact zero divergence)."""
    xf, yf, _ = g.faces()
    A = Az(xf[None, :], yf[:, None])  # (ny+1, nx+1) at edges (x_{i-1/2}, y_{j-1/2})
    bx = (A[1:, :] - A[:-1, :]) / g.dy          # (ny, nx+1)
    by = -(A[:, 1:] - A[:, :-1]) / g.dx         # (ny+1, nx)
    Bx = np.broadcast_to(bx, (g.nz, g.ny, g.nx + 1))
    By = np.broadcast_to(by, (g.nz, g.ny + 1, g.nx))
    Bz = np.zeros((g.nz + 1, g.ny, g.nx))
    return Bx, By, Bz


def faces_from_A(g: Geom, Ax, Ay, Az):
    """Face fields of B = curl A with A sampled on cell edges: A_x on (x_i, y_{j-1/2},
    z_{k-1/2}), A_y on (x_{i-1/2}, y_j, z_{k-1/2}), A_z on (x_{i-1/2}, y_{j-1/2}, z_k).
    Each callable takes broadcastable (x, y, z) arrays.  Exact zero discrete divergence."""
    xc, yc, zc = g.centres()
    xf, yf, zf = g.faces()
    # A_z on (nz, ny+1, nx+1), A_y on (nz+1, ny, nx+1), A_x on (nz+1, ny+1, nx)
    az = np.broadcast_to(Az(xf[None, None, :], yf[None, :, None], zc[:, None, None]), (g.nz, g.ny + 1, g.nx + 1))
    ay = np.broadcast_to(Ay(xf[None, None, :], yc[None, :, None], zf[:, None, None]), (g.nz + 1, g.ny, g.nx + 1))
    ax = np.broadcast_to(Ax(xc[None, None, :], yf[None, :, None], zf[:, None, None]), (g.nz + 1, g.ny + 1, g.nx))
    Bx = (az[:, 1:, :] - az[:, :-1, :]) / g.dy - (ay[1:, :, :] - ay[:-1, :, :]) / g.dz
    By = (ax[1:, :, :] - ax[:-1, :, :]) / g.dz - (az[:, :, 1:] - az[:, :, :-1]) / g.dx
    Bz = (ay[:, :, 1:] - ay[:, :, :-1]) / g.dx - (ax[:, 1:, :] - ax[:, :-1, :]) / g.dy
    return np.ascontiguousarray(Bx), np.ascontiguousarray(By), np.ascontiguousarray(Bz)


def smooth_random(g: Geom, seed: int, bamp: float = 0.5) -> State:
    """Smooth random positive state (a few low Fourier modes per field) with a field
    from a random smooth vector potential; used for parity on odd-sized boxes with any
    boundary conditions."""
    rng = np.random.default_rng(seed)
    L = (g.nx * g.dx, g.ny * g.dy, g.nz * g.dz)

    def fld(base, amp):
        c = rng.normal(size=(4, 3))
        ph = rng.uniform(0, 2 * np.pi, 4)

        def f(x, y, z):
            out = base
            for m in range(4):
                out = out + amp * c[m, 0] * np.sin(2 * np.pi * (x - g.x0) / L[0] * (1 + m % 2) + ph[m]) \
                    * np.cos(2 * np.pi * (y - g.y0) / L[1] * (m // 2) + c[m, 1]) \
                    * np.cos(2 * np.pi * (z - g.z0) / L[2] * (m % 3) + c[m, 2])
            return out
        return f

    x, y, z = g.centres()
    X, Y, Z = x[None, None, :], y[None, :, None], z[:, None, None]
    rho = fld(1.0, 0.08)(X, Y, Z)
    p = fld(0.8, 0.06)(X, Y, Z)
    vx, vy, vz = (fld(0.0, 0.2)(X, Y, Z) for _ in range(3))
    A = [fld(0.0, bamp * 0.1) for _ in range(3)]
    B0 = rng.normal(size=3) * bamp
    Ax = lambda xx, yy, zz: A[0](xx, yy, zz) + B0[1] * zz
    Ay = lambda xx, yy, zz: A[1](xx, yy, zz) + B0[2] * xx
    Az = lambda xx, yy, zz: A[2](xx, yy, zz) + B0[0] * yy
    Bx, By, Bz = faces_from_A(g, Ax, Ay, Az)
    return state_from_prim(g, rho, vx, vy, vz, p, Bx, By, Bz)


def slow_contact(n=(24, 16, 12), u: float = 3e-6, seed: int = 7) -> State:
    """Density contacts carried slowly along x on a periodic box: rho alternates between 1
    and 2 in x-blocks of seeded widths, vx = u everywhere, and vy, vz, p, By(z), Bz(y) and a
    uniform Bx vary only across x, so that every x-face of the initial state holds an
    isolated contact whose mass flux is about u / (2 c_f) of the face's scale."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    g = Geom(nx, ny, nz, 0.0, 0.0, 0.0, 1.0 / nx, 1.0 / ny, 1.0 / nz, (0,) * 6, 5.0 / 3.0)
    cuts = np.sort(rng.choice(np.arange(1, nx), size=3, replace=False))
    rho_x = np.ones(nx)
    for m, c in enumerate(cuts):
        if m % 2 == 0:
            rho_x[c:] = 2.0
        else:
            rho_x[c:] = 1.0
    x, y, z = g.centres()
    Y, Z = y[None, :, None], z[:, None, None]
    ph = rng.uniform(0, 2 * np.pi, 6)
    vy = 0.3 * np.sin(2 * np.pi * Y + ph[0]) * np.cos(2 * np.pi * Z + ph[1]) + 0 * x[None, None, :]
    vz = 0.2 * np.cos(2 * np.pi * Y + ph[2]) + 0.1 * np.sin(4 * np.pi * Z + ph[3]) + 0 * x[None, None, :]
    p = 1.0 + 0.1 * np.sin(2 * np.pi * Y + ph[4]) * np.sin(2 * np.pi * Z + ph[5]) + 0 * x[None, None, :]
    rho = rho_x[None, None, :] * np.ones((nz, ny, 1))
    By = (0.5 + 0.2 * np.sin(2 * np.pi * z))[:, None, None] * np.ones((1, ny + 1, nx))
    Bz = (-0.3 + 0.25 * np.cos(2 * np.pi * y))[None, :, None] * np.ones((nz + 1, 1, nx))
    return state_from_prim(g, rho, u, vy, vz, p, 0.6, By, Bz)


# ---------------------------------------------------------------- workloads --

def brio_wu(n: int = 800, axis: int = 0, transverse: int = 1) -> State:
    """Brio-Wu shock tube (Section 3.4): gamma = 2, Bn = 0.75; left rho = 1, p = 1,
    Bt = 1; right rho = 0.125, p = 0.1, Bt = -1; domain [0, 1], interface at 0.5,
    outflow ends.  The tube runs along ``axis``; ``transverse`` other cells pad the
    other axes (periodic) for plane-parallel checks."""
    dims = [transverse, transverse, transverse]
    dims[axis] = n
    d = [1.0 / n, 1.0 / n, 1.0 / n]
    bc = [BC_PERIODIC] * 6
    bc[2 * axis] = bc[2 * axis + 1] = BC_OUTFLOW
    g = Geom(dims[0], dims[1], dims[2], 0.0, 0.0, 0.0, d[0], d[1], d[2], tuple(bc), 2.0)
    t1 = (axis + 1) % 3
    xs = g.centres()[axis]
    left = xs < 0.5
    shp = (g.nz, g.ny, g.nx)

    def along(v):
        s = [1, 1, 1]
        s[2 - axis] = v.size
        return np.broadcast_to(v.reshape(s), shp)

    rho = along(np.where(left, 1.0, 0.125))
    p = along(np.where(left, 1.0, 0.1))
    bt = np.where(left, 1.0, -1.0)
    B = [None, None, None]
    fshape = [(g.nz, g.ny, g.nx + 1), (g.nz, g.ny + 1, g.nx), (g.nz + 1, g.ny, g.nx)]
    for a in range(3):
        if a == axis:
            B[a] = np.full(fshape[a], 0.75)
        elif a == t1:
            s = [1, 1, 1]
            s[2 - axis] = n
            B[a] = np.broadcast_to(bt.reshape(s), fshape[a]).copy()
        else:
            B[a] = np.zeros(fshape[a])
    return state_from_prim(g, rho, 0.0, 0.0, 0.0, p, *B)


def ryu_jones(n: int = 800) -> State:
    """Ryu-Jones 7-wave Riemann problem (Section 3.5), gamma = 5/3, on [0, 1] with the
    discontinuity at 0.5 and outflow ends.  Left: rho 1.08, p 0.95, v (1.2, 0.01, 0.5),
    B (Bx, 3.6, 2)/sqrt(4 pi); right: rho 1, p 1, v 0, B (Bx, 4, 2)/sqrt(4 pi), with
    Bx = 2/sqrt(4 pi) (the paper prints 4/sqrt(4 pi); its printed shock Mach numbers
    belong to Bx = 2/sqrt(4 pi))."""
    g = Geom(n, 1, 1, 0.0, 0.0, 0.0, 1.0 / n, 1.0, 1.0, (1, 1, 0, 0, 0, 0), 5.0 / 3.0)
    x = g.centres()[0]
    left = x < 0.5
    s4 = 1.0 / math.sqrt(4.0 * math.pi)
    sel = lambda a, b: np.where(left, a, b)[None, None, :]
    Bx = np.full((1, 1, n + 1), 2.0 * s4)
    By = np.broadcast_to(sel(3.6 * s4, 4.0 * s4), (1, 2, n)).copy()
    Bz = np.broadcast_to(sel(2.0 * s4, 2.0 * s4), (2, 1, n)).copy()
    return state_from_prim(g, sel(1.08, 1.0), sel(1.2, 0.0), sel(0.01, 0.0), sel(0.5, 0.0),
                           sel(0.95, 1.0), Bx, By, Bz)


def sod(n: int = 200) -> State:
    """Sod shock tube (Section 3.1) with B = 0, gamma = 1.4, on [-1, 1], interface at 0."""
    g = Geom(n, 1, 1, -1.0, 0.0, 0.0, 2.0 / n, 1.0, 1.0, (1, 1, 0, 0, 0, 0), 1.4)
    x = g.centres()[0]
    left = (x < 0.0)[None, None, :]
    return state_from_prim(g, np.where(left, 1.0, 0.125), 0.0, 0.0, 0.0, np.where(left, 1.0, 0.1),
                           0.0, 0.0, 0.0)


def shu_osher(n: int = 800, amp: float = 0.2) -> State:
    """Shu-Osher problem (Section 3.2) with B = 0, gamma = 1.4, on [0, 1], outflow: the printed
    state rho = 3.857143, p = 10.33333, u = 2.629369 for x < 0.125, and rho = 1 + amp sin(16 pi x),
    p = 1, u = 0 beyond.  amp = 0 leaves the shock alone."""
    g = Geom(n, 1, 1, 0.0, 0.0, 0.0, 1.0 / n, 1.0, 1.0, (1, 1, 0, 0, 0, 0), 1.4)
    x = g.centres()[0]
    left = (x < 0.125)[None, None, :]
    rho = np.where(left, 3.857143, 1.0 + amp * np.sin(16.0 * math.pi * x)[None, None, :])
    return state_from_prim(g, rho, np.where(left, 2.629369, 0.0), 0.0, 0.0, np.where(left, 10.33333, 1.0),
                           0.0, 0.0, 0.0)


def sedov(nx: int = 512, ny: int = 768, r0: float = 0.01, e0: float = 1.0, p0: float = 1e-5,
          gamma: float = 1.4) -> State:
    """2D Sedov-Taylor blast (Section 3.7) with B = 0 on [-0.5, 0.5] x [-0.75, 0.75] (cells
    of side 1/512 at the paper's 512 x 768), outflow boundaries: rho = 1, p = p0, and the
    energy e0 (per unit length) deposited as pressure in the cells whose centres lie within
    r0 of the centre: p = (gamma - 1) e0 / (their area), so that exactly e0 is added.
    (The printed in-sphere pressure is garbled; this is the standard point explosion.)"""
    d = 1.0 / 512.0 * (512.0 / nx)
    g = Geom(nx, ny, 1, -0.5 * nx * d, -0.5 * ny * d, 0.0, d, d, 1.0, (1, 1, 1, 1, 0, 0), gamma)
    x, y, _ = g.centres()
    X, Y = np.meshgrid(x, y, indexing="xy")
    inside = (X * X + Y * Y < r0 * r0)
    n_in = int(inside.sum())
    if n_in == 0:
        raise ValueError("r0 is smaller than a cell")
    p = np.where(inside, (gamma - 1.0) * e0 / (n_in * d * d), p0)[None]
    return state_from_prim(g, 1.0, 0.0, 0.0, 0.0, p, 0.0, 0.0, 0.0)


def rotor(n: int = 512, v0: float = 2.0, gamma: float = 1.4) -> State:
    """Magnetic rotor (Section 3.6) on [-0.5, 0.5]^2, outflow: rho = 10 and rigid rotation
    v = v0 (-y, x)/r0 for r < r0 = 0.1; rho = 1 + 9 f, v = v0 f (-y, x)/r0 with
    f = (r1 - r)/(r1 - r0) for r0 < r < r1 = 0.2 (as printed); rho = 1 at rest beyond;
    p = 1 and Bx = 5/sqrt(4 pi) everywhere.  v0, gamma, the domain and the end time are not
    given (v0 = 2, gamma = 1.4, t = 0.15 taken)."""
    g = Geom(n, n, 1, -0.5, -0.5, 0.0, 1.0 / n, 1.0 / n, 1.0, (1, 1, 1, 1, 0, 0), gamma)
    x, y, _ = g.centres()
    X, Y = np.meshgrid(x, y, indexing="xy")
    r = np.sqrt(X * X + Y * Y)
    r0, r1 = 0.1, 0.2
    f = np.where(r < r0, 1.0, np.where(r < r1, (r1 - r) / (r1 - r0), 0.0))
    rho = np.where(r < r0, 10.0, 1.0 + 9.0 * f)
    vx, vy = -v0 * f * Y / r0, v0 * f * X / r0
    return state_from_prim(g, rho[None], vx[None], vy[None], 0.0, 1.0, 5.0 / math.sqrt(4.0 * math.pi), 0.0, 0.0)


def bow_shock(n: int = 400, psi0: float = 5.0, x0: float = 0.1):
    """Flow through a potential well (Section 3.3): rho = 1, p = 1, vx = 1, gamma = 1.4 on
    [-0.5, 0.5] (the domain is not given), Psi = -psi0 exp(-(x/x0)^2); steady inflow of the
    initial state at the left, free (outflow) at the right.  Returns (state, source,
    inflow)."""
    g = Geom(n, 1, 1, -0.5, 0.0, 0.0, 1.0 / n, 1.0, 1.0, (2, 1, 0, 0, 0, 0), 1.4)
    st = state_from_prim(g, 1.0, 1.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0)
    src = dict(potential=1, psi0=psi0, xc=0.0, xw=x0)
    return st, src, {0: (1.0, 1.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0)}


def isothermal_well(n: int = 128, psi0: float = 1.0, x0: float = 0.1) -> tuple:
    """Hydrostatic isothermal gas (p = rho, at rest) in the Gaussian well of the bow-shock
    test: rho = exp(-Psi) = exp(psi0 exp(-(x/x0)^2)), outflow boundaries on [-0.5, 0.5],
    gamma = 1.4.  An exact steady state of the equations; the scheme holds it to its
    truncation error.  Returns (state, source)."""
    g = Geom(n, 1, 1, -0.5, 0.0, 0.0, 1.0 / n, 1.0, 1.0, (1, 1, 0, 0, 0, 0), 1.4)
    x = g.centres()[0]
    rho = np.exp(psi0 * np.exp(-(x / x0) ** 2))[None, None, :]
    return state_from_prim(g, rho, 0.0, 0.0, 0.0, rho, 0.0, 0.0, 0.0), dict(potential=1, psi0=psi0, xc=0.0, xw=x0)


# Floors for the Sedov blast at the paper's resolution: with its 1e8 pressure jump from a
# five-cell source the plain scheme drives ambient cells ahead of the shock to p < 0 within
# ten steps (the FP64 oracle too); p/rho >= 1e-6 (ambient 1e-5) keeps it positive.
SEDOV_FLOORS = dict(rho_floor=1e-8, pr_floor=1e-6, pr_ceil=0.0)


def orszag_tang(nx: int = 512, ny: int | None = None) -> State:
    """2D periodic MHD vortex on [0, 1]^2, gamma = 5/3, rho = 25/(36 pi), p = 5/(12 pi),
    v = (-sin 2 pi y, sin 2 pi x, 0), B = (-sin 2 pi y, sin 4 pi x, 0)/sqrt(4 pi)
    from A_z = (cos 4 pi x/(4 pi) + cos 2 pi y/(2 pi))/sqrt(4 pi)."""
    ny = nx if ny is None else ny
    g = Geom(nx, ny, 1, 0.0, 0.0, 0.0, 1.0 / nx, 1.0 / ny, 1.0, (0,) * 6, 5.0 / 3.0)
    s4 = 1.0 / math.sqrt(4.0 * math.pi)
    Az = lambda x, y: (np.cos(4 * np.pi * x) / (4 * np.pi) + np.cos(2 * np.pi * y) / (2 * np.pi)) * s4
    Bx, By, Bz = faces_from_Az(g, Az)
    x, y, _ = g.centres()
    X, Y = np.meshgrid(x, y, indexing="xy")
    vx = -np.sin(2 * np.pi * Y)[None]
    vy = np.sin(2 * np.pi * X)[None]
    return state_from_prim(g, 25.0 / (36.0 * np.pi), vx, vy, 0.0, 5.0 / (12.0 * np.pi), Bx, By, Bz)


def solenoidal_velocity(n: tuple, seed: int, kmin: float = 2.0, kmax: float = 8.0) -> np.ndarray:
    """Random-phase solenoidal field on a periodic (nz, ny, nx) box: Gaussian modes for
    integer wavevectors with kmin <= |k| <= kmax, amplitude |v(k)| ~ |k|^-2 (shell
    spectrum ~ k^-2), projected with v <- v - k (k.v)/k^2; unit rms.  Returns
    (3, nz, ny, nx)."""
    nz, ny, nx = n
    rng = np.random.default_rng(seed)
    kz = np.fft.fftfreq(nz, 1.0 / nz)[:, None, None]
    ky = np.fft.fftfreq(ny, 1.0 / ny)[None, :, None]
    kx = np.fft.rfftfreq(nx, 1.0 / nx)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    kk = np.sqrt(k2)
    mask = (kk >= kmin) & (kk <= kmax)
    shape = k2.shape
    amp = np.where(mask, np.maximum(kk, 1e-30) ** -2.0, 0.0)
    vh = []
    for _ in range(3):
        re = rng.standard_normal(shape)
        im = rng.standard_normal(shape)
        vh.append(amp * (re + 1j * im))
    kdotv = kx * vh[0] + ky * vh[1] + kz * vh[2]
    k2s = np.where(k2 > 0, k2, 1.0)
    vh = [vh[0] - kx * kdotv / k2s, vh[1] - ky * kdotv / k2s, vh[2] - kz * kdotv / k2s]
    v = np.stack([np.fft.irfftn(c, s=(nz, ny, nx), axes=(0, 1, 2)) for c in vh])
    rms = math.sqrt(float(np.mean(np.sum(v * v, axis=0))))
    return v / rms


def turbulence(n=256, seed: int = 1502, mach: float = 2.0, b0: float = 0.1) -> State:
    """Driven-free turbulent box: periodic [0, 1]^3, gamma = 5/3, rho = 1, p = 1,
    B = (b0, 0, 0) (0.1; 0 for pure gas dynamics), solenoidal random velocity
    (2 <= |k| <= 8, shell spectrum ~ k^-2) scaled to rms Mach ``mach``.  ``n`` is an int
    or (nx, ny, nz)."""
    nx, ny, nz = (n, n, n) if isinstance(n, int) else n
    g = Geom(nx, ny, nz, 0.0, 0.0, 0.0, 1.0 / nx, 1.0 / ny, 1.0 / nz, (0,) * 6, 5.0 / 3.0)
    v = solenoidal_velocity((nz, ny, nx), seed) * (mach * math.sqrt(5.0 / 3.0))
    return state_from_prim(g, 1.0, v[0], v[1], v[2], 1.0, b0, 0.0, 0.0)


def _splitmix64(state: int):
    state = (state + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return state, z ^ (z >> 31)


def blast_patch_specs(n_patches: int = 64, seed: int = 1502, sizes=(32, 48, 64, 96, 128)):
    """Per-patch (edge, centre, field direction) drawn with splitmix64 from ``seed``."""
    s = seed & 0xFFFFFFFFFFFFFFFF
    out = []

    def u01():
        nonlocal s
        s, z = _splitmix64(s)
        return (z >> 11) * (1.0 / 9007199254740992.0)

    for _ in range(n_patches):
        edge = sizes[min(int(u01() * len(sizes)), len(sizes) - 1)]
        centre = (u01(), u01(), u01())
        cz = 2.0 * u01() - 1.0
        ph = 2.0 * math.pi * u01()
        r = math.sqrt(max(0.0, 1.0 - cz * cz))
        out.append((edge, centre, (r * math.cos(ph), r * math.sin(ph), cz)))
    return out


def blast(edge: int, centre, direction, gamma: float = 5.0 / 3.0) -> State:
    """Periodic blast patch on [0, 1]^3 with edge^3 cells: rho = 1, p = 0.1, p = 10 within
    0.1 (minimum-image distance) of ``centre``, uniform B = (1/sqrt 2) * direction."""
    n = edge
    g = Geom(n, n, n, 0.0, 0.0, 0.0, 1.0 / n, 1.0 / n, 1.0 / n, (0,) * 6, gamma)
    x, y, z = g.centres()

    def mi(a, c):
        d = np.abs(a - c)
        return np.minimum(d, 1.0 - d)

    r2 = (mi(z, centre[2])[:, None, None] ** 2 + mi(y, centre[1])[None, :, None] ** 2
          + mi(x, centre[0])[None, None, :] ** 2)
    p = np.where(r2 < 0.01, 10.0, 0.1)
    b = [c / math.sqrt(2.0) for c in direction]
    return state_from_prim(g, 1.0, 0.0, 0.0, 0.0, p, b[0], b[1], b[2])


def blast_batch(n_patches: int = 64, seed: int = 1502, sizes=(32, 48, 64, 96, 128)):
    return [blast(e, c, d) for (e, c, d) in blast_patch_specs(n_patches, seed, sizes)]


def uniform(g: Geom, rho=1.0, v=(0.0, 0.0, 0.0), p=1.0, B=(0.0, 0.0, 0.0)) -> State:
    return state_from_prim(g, rho, v[0], v[1], v[2], p, B[0], B[1], B[2])


def alfven_wave(n: int, amp: float = 1e-6, gamma: float = 5.0 / 3.0, polarisation: str = "inplane") -> State:
    """Linear Alfven wave on the periodic box [0, 1]^2 (n x n cells): rho = 1, p = 1/gamma,
    B0 = khat (|B0| = 1 along k = 2 pi (1, 1), wavelength 1/sqrt 2, Alfven speed 1).
    dv = amp sin(k.x) e, dB = -sqrt(rho) dv (a wave moving along +k), with e either the
    in-plane unit vector perpendicular to k ("inplane", field from a vector potential)
    or z ("z")."""
    rho0, p0 = 1.0, 1.0 / gamma
    g = Geom(n, n, 1, 0.0, 0.0, 0.0, 1.0 / n, 1.0 / n, 1.0, (0,) * 6, gamma)
    kx = ky = 2.0 * np.pi
    kn = math.hypot(kx, ky)
    kh = (kx / kn, ky / kn)
    x, y, _ = g.centres()
    X, Y = np.meshgrid(x, y, indexing="xy")
    sph = np.sin(kx * X + ky * Y)[None]
    if polarisation == "inplane":
        e = (-kh[1], kh[0])
        c = -amp * math.sqrt(rho0) / kn
        # B = curl(A_z z) with A_z = y kh_x - x kh_y (uniform B0 = khat) + c cos(k.x)
        Az = lambda xx, yy: yy * kh[0] - xx * kh[1] + c * np.cos(kx * xx + ky * yy)
        Bx, By, Bz = faces_from_Az(g, Az)
        return state_from_prim(g, rho0, amp * e[0] * sph, amp * e[1] * sph, 0.0, p0, Bx, By, Bz)
    Az = lambda xx, yy: yy * kh[0] - xx * kh[1]
    Bx, By, _ = faces_from_Az(g, Az)
    Bz = np.broadcast_to(-math.sqrt(rho0) * amp * sph, (2, n, n)).copy()
    return state_from_prim(g, rho0, 0.0, 0.0, amp * sph, p0, Bx, By, Bz)


# Code units of the disc workload: length kpc, velocity km/s (time unit 0.978 Gyr),
# density unit = the gas mass per hydrogen atom (m_H/0.76) per cm^3.
#   T = 72.7 K * (p/rho) [mu = 0.6],  n_H = 0.76 rho,
#   energy-rate unit = 2.2e-14 erg cm^-3 / 3.086e16 s = 7.13e-31 erg cm^-3 s^-1.
DISC_THERMAL = dict(gamma_heat=2e-26, z=0.02, rate_unit=7.13e-31, cap=0.1, nh_per_rho=0.76, t_per_pr=72.7)
DISC_POTENTIAL = dict(potential=2, v0=220.0, rc=0.5)
# floors of the disc run: rho >= 1e-4 of the central density (the initial floor of
# disc() at its default n_H = 5 cm^-3) and 10 K <= T <= 1e8 K as bounds on p/rho
DISC_FLOORS = dict(rho_floor=1e-4 * (5.0 / DISC_THERMAL["nh_per_rho"]), pr_floor=10.0 / DISC_THERMAL["t_per_pr"],
                   pr_ceil=1e8 / DISC_THERMAL["t_per_pr"])


def disc(nx: int = 512, ny: int = 512, nz: int = 128, n_h0: float = 5.0, T0: float = 1e4, beta: float = 10.0,
         v0: float = 220.0, rc: float = 0.5, rd: float = 3.0, z0: float = 0.2, floor: float = 1e-4) -> State:
    """Isolated gas disc on [-20, 20]^2 x [-5, 5] kpc, outflow on all faces, gamma = 5/3:
    rho = rho0 exp(-R/rd) sech^2(z/z0) floored at floor*rho0 (rho0 from the central n_H),
    T = T0, circular velocity v0 R/sqrt(R^2 + rc^2) of Psi = v0^2/2 ln(R^2 + rc^2 + z^2),
    toroidal field with plasma beta = beta for the unfloored profile, from
    A_z = -2 rd sqrt(2 (p/rho) rho0/beta) sech(z/z0) (1 - exp(-R/(2 rd))) on z-edges."""
    L = (40.0, 40.0, 10.0)
    g = Geom(nx, ny, nz, -20.0, -20.0, -5.0, L[0] / nx, L[1] / ny, L[2] / nz, (1,) * 6, 5.0 / 3.0)
    u = DISC_THERMAL
    rho0 = n_h0 / u["nh_per_rho"]
    pr = T0 / u["t_per_pr"]  # p/rho
    x, y, z = g.centres()
    X, Y, Z = x[None, None, :], y[None, :, None], z[:, None, None]
    R = np.sqrt(X * X + Y * Y)
    rho = np.maximum(rho0 * np.exp(-R / rd) / np.cosh(Z / z0) ** 2, floor * rho0)
    vc = v0 * R / np.sqrt(R * R + rc * rc)
    Rs = np.where(R > 0, R, 1.0)
    vx = -vc * Y / Rs
    vy = vc * X / Rs
    C0 = math.sqrt(2.0 * pr * rho0 / beta)
    zero = lambda xx, yy, zz: np.zeros(np.broadcast_shapes(np.shape(xx), np.shape(yy), np.shape(zz)))
    Az = lambda xx, yy, zz: -2.0 * rd * C0 / np.cosh(zz / z0) * (1.0 - np.exp(-np.sqrt(xx * xx + yy * yy) / (2.0 * rd)))
    Bx, By, Bz = faces_from_A(g, zero, zero, Az)
    return state_from_prim(g, rho, vx, vy, 0.0, pr * rho, Bx, By, Bz)
