"""Independent textbook references used to pin the oracle (test helpers only).

* ``physical_flux``: the ideal-MHD flux of Eq. 3 in the frame of an interface.
* ``hllc``: Toro's HLLC flux for the Euler equations (B = 0) with the same outer
  speed estimates; Miyoshi & Kusano's HLLD reduces to it when B vanishes.
* ``hll``: the HLL flux (Toro, Sec. 10.3) for the ideal-MHD flux of Eq. 3 with the
  same outer speed estimates from the fast magnetosonic speed.
* ``exact_riemann_euler``: Toro's exact Riemann solver for an ideal gas (two-shock /
  two-rarefaction pressure function, Newton iteration on p*), sampled at x/t.

These are standard published methods written out here on their own; none of
them is shared with the oracle or the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np


def physical_flux(w, bn, gamma):
    """w = [rho, un, ut1, ut2, p, -, Bt1, Bt2] -> F in the same frame (8 components)."""
    rho, u, v, ww, p, _, b1, b2 = w
    b2sum = bn * bn + b1 * b1 + b2 * b2
    pt = p + 0.5 * b2sum
    e = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + ww * ww) + 0.5 * b2sum
    vb = u * bn + v * b1 + ww * b2
    return np.array([rho * u, rho * u * u + pt - bn * bn, rho * u * v - bn * b1, rho * u * ww - bn * b2,
                     (e + pt) * u - vb * bn, 0.0, b1 * u - bn * v, b2 * u - bn * ww])


def conserved(w, bn, gamma):
    rho, u, v, ww, p, _, b1, b2 = w
    e = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + ww * ww) + 0.5 * (bn * bn + b1 * b1 + b2 * b2)
    return np.array([rho, rho * u, rho * v, rho * ww, e, bn, b1, b2])


def hllc(wl, wr, gamma):
    """Toro's HLLC (Riemann Solvers and Numerical Methods for Fluid Dynamics, Sec. 10.4)
    with S_L = min(uL, uR) - max(cL, cR), S_R = max(uL, uR) + max(cL, cR)."""
    rl, ul, vl, wl_, pl = wl[0], wl[1], wl[2], wl[3], wl[4]
    rr, ur, vr, wr_, pr = wr[0], wr[1], wr[2], wr[3], wr[4]
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    sl = min(ul, ur) - max(cl, cr)
    sr = max(ul, ur) + max(cl, cr)
    FL = physical_flux(wl, 0.0, gamma)
    FR = physical_flux(wr, 0.0, gamma)
    if sl > 0:
        return FL
    if sr < 0:
        return FR
    ss = (pr - pl + rl * ul * (sl - ul) - rr * ur * (sr - ur)) / (rl * (sl - ul) - rr * (sr - ur))

    def ustar(r, u, v, w_, p, s):
        e = p / (gamma - 1.0) + 0.5 * r * (u * u + v * v + w_ * w_)
        f = r * (s - u) / (s - ss)
        return np.array([f, f * ss, f * v, f * w_, f * (e / r + (ss - u) * (ss + p / (r * (s - u)))), 0, 0, 0])

    if ss >= 0:
        return FL + sl * (ustar(rl, ul, vl, wl_, pl, sl) - conserved(wl, 0.0, gamma))
    return FR + sr * (ustar(rr, ur, vr, wr_, pr, sr) - conserved(wr, 0.0, gamma))


def fast_magnetosonic(rho, p, bn, bt1, bt2, gamma):
    """c_f^2 = (a^2 + b^2)/2 + sqrt((a^2 + b^2)^2 - 4 a^2 b_n^2)/2, a^2 = gamma p/rho,
    b^2 = |B|^2/rho, b_n^2 = B_n^2/rho."""
    a2 = gamma * p / rho
    b2 = (bn * bn + bt1 * bt1 + bt2 * bt2) / rho
    bn2 = bn * bn / rho
    return math.sqrt(0.5 * (a2 + b2 + math.sqrt(max((a2 + b2) ** 2 - 4.0 * a2 * bn2, 0.0))))


def hll(wl, wr, bn, gamma):
    """HLL: F_L if S_L >= 0, F_R if S_R <= 0, else the flux of the single intermediate
    state, (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L), with
    S_L = min(uL, uR) - max(cfL, cfR), S_R = max(uL, uR) + max(cfL, cfR)."""
    cl = fast_magnetosonic(wl[0], wl[4], bn, wl[6], wl[7], gamma)
    cr = fast_magnetosonic(wr[0], wr[4], bn, wr[6], wr[7], gamma)
    sl = min(wl[1], wr[1]) - max(cl, cr)
    sr = max(wl[1], wr[1]) + max(cl, cr)
    FL, FR = physical_flux(wl, bn, gamma), physical_flux(wr, bn, gamma)
    if sl >= 0:
        return FL
    if sr <= 0:
        return FR
    UL, UR = conserved(wl, bn, gamma), conserved(wr, bn, gamma)
    return (sr * FL - sl * FR + sl * sr * (UR - UL)) / (sr - sl)


def exact_riemann_euler(left, right, gamma, xi):
    """Exact solution (rho, u, p) of the 1D Euler Riemann problem at similarity
    coordinates xi = x/t.  left/right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    g1 = (gamma - 1) / (2 * gamma)
    g2 = (gamma + 1) / (2 * gamma)

    def fk(p, rk, pk, ck):
        if p > pk:
            A = 2 / ((gamma + 1) * rk)
            B = (gamma - 1) / (gamma + 1) * pk
            q = math.sqrt(A / (p + B))
            return (p - pk) * q, q * (1 - 0.5 * (p - pk) / (B + p))
        f = 2 * ck / (gamma - 1) * ((p / pk) ** g1 - 1)
        return f, 1 / (rk * ck) * (p / pk) ** (-g2)

    p = max(1e-8, 0.5 * (pl + pr))
    for _ in range(100):
        f1, d1 = fk(p, rl, pl, cl)
        f2, d2 = fk(p, rr, pr, cr)
        dp = (f1 + f2 + ur - ul) / (d1 + d2)
        pn = max(1e-12, p - dp)
        if abs(pn - p) < 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    f1, _ = fk(p, rl, pl, cl)
    f2, _ = fk(p, rr, pr, cr)
    us = 0.5 * (ul + ur) + 0.5 * (f2 - f1)

    out = np.zeros((3, len(xi)))
    for n, s in enumerate(xi):
        if s <= us:  # left of contact
            if p > pl:  # left shock
                sL = ul - cl * math.sqrt(g2 * p / pl + g1)
                if s <= sL:
                    out[:, n] = (rl, ul, pl)
                else:
                    r = rl * ((p / pl + (gamma - 1) / (gamma + 1)) / ((gamma - 1) / (gamma + 1) * p / pl + 1))
                    out[:, n] = (r, us, p)
            else:
                shl = ul - cl
                cs = cl * (p / pl) ** g1
                stl = us - cs
                if s <= shl:
                    out[:, n] = (rl, ul, pl)
                elif s >= stl:
                    out[:, n] = (rl * (p / pl) ** (1 / gamma), us, p)
                else:
                    u = 2 / (gamma + 1) * (cl + (gamma - 1) / 2 * ul + s)
                    c = 2 / (gamma + 1) * (cl + (gamma - 1) / 2 * (ul - s))
                    out[:, n] = (rl * (c / cl) ** (2 / (gamma - 1)), u, pl * (c / cl) ** (2 * gamma / (gamma - 1)))
        else:
            if p > pr:
                sR = ur + cr * math.sqrt(g2 * p / pr + g1)
                if s >= sR:
                    out[:, n] = (rr, ur, pr)
                else:
                    r = rr * ((p / pr + (gamma - 1) / (gamma + 1)) / ((gamma - 1) / (gamma + 1) * p / pr + 1))
                    out[:, n] = (r, us, p)
            else:
                shr = ur + cr
                cs = cr * (p / pr) ** g1
                str_ = us + cs
                if s >= shr:
                    out[:, n] = (rr, ur, pr)
                elif s <= str_:
                    out[:, n] = (rr * (p / pr) ** (1 / gamma), us, p)
                else:
                    u = 2 / (gamma + 1) * (-cr + (gamma - 1) / 2 * ur + s)
                    c = 2 / (gamma + 1) * (cr - (gamma - 1) / 2 * (ur - s))
                    out[:, n] = (rr * (c / cr) ** (2 / (gamma - 1)), u, pr * (c / cr) ** (2 * gamma / (gamma - 1)))
    return out
