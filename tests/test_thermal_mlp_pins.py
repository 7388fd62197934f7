"""Pins of the thermal-source oracle and of the MLP-surrogate oracle (CPU only).

Thermal module: Section 3.10 of arXiv:1502.02935 (heating/cooling in S of Eq. 2).  The
paper's rate tables are not available; the oracle uses a documented piecewise power-law
stand-in.  The pins below hold for any such table:
  * with heating off and T inside one power-law segment, Lambda = C T^a and the isochoric
    equation dT/dt = -K T^a has the closed form T^(1-a)(t) = T0^(1-a) - (1-a) K t; the
    sub-stepped backward Euler converges to it at first order in the sub-step cap;
  * a temperature where n Gamma = n^2 Lambda(T) is a fixed point, and cells relax onto the
    stable equilibrium from both sides;
  * the operator-split update changes only E, by exactly the internal energy c_e dT.
MLP oracle: the backward pass equals central finite differences of the loss, and equals
torch autograd on the same network (CPU, FP64).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1502_02935_gb300 import inputs

LT = [1.0, 2.0, 3.0, 3.8, 4.0, 4.2, 5.0, 5.4, 6.0, 7.0, 8.0]
TH = dict(rate_unit=5.4e-31, nh_per_rho=0.76, t_per_pr=72.7, cap=0.1, gamma_heat=2e-26, z=0.02)


# The stand-in cooling table as defined for this build (log10 T [K], log10 Lambda [erg cm^3/s])
# at Z = 0.02; Lambda is a power law in T between neighbouring knots, continued beyond the
# end knots with the end segments' slopes, and scales as (0.2 + 0.8 Z / 0.02).
LL = [-28.5, -27.0, -26.2, -25.9, -23.5, -21.8, -21.3, -21.2, -22.0, -22.7, -22.6]


@pytest.mark.parametrize("z", [0.02, 0.0, 0.04])
def test_cooling_table_knots_segments_and_metallicity(z):
    """The stand-in Lambda(T, Z) against its definition: the printed value at every knot;
    continuity across every interior knot (1e-12 relative); on each side of a knot the slope
    of the segment on that side (a segment search shifted by one index fails here); the
    midpoint of each segment on the straight line in log-log; the end segments continued
    below 10 K and above 1e8 K; the metallicity scale 0.2 + 0.8 Z / 0.02."""
    scale = 0.2 + 0.8 * z / 0.02
    lam, _ = oracle.cooling([10.0 ** t for t in LT], z)
    want = np.array([10.0 ** l for l in LL]) * scale
    assert np.max(np.abs(lam / want - 1.0)) <= 1e-12
    slopes = [(LL[k + 1] - LL[k]) / (LT[k + 1] - LT[k]) for k in range(len(LT) - 1)]
    for k in range(1, len(LT) - 1):
        t = 10.0 ** LT[k]
        lo, s_lo = oracle.cooling([t * (1 - 1e-13)], z)
        hi, s_hi = oracle.cooling([t * (1 + 1e-13)], z)
        # the two sides differ only by the 2e-13 step in T along slopes of up to 12
        assert abs(lo[0] / hi[0] - 1.0) <= 1e-12 + 1e-13 * (abs(s_lo[0]) + abs(s_hi[0])), (k, lo, hi)
        assert s_lo[0] == pytest.approx(slopes[k - 1], rel=1e-14), k
        assert s_hi[0] == pytest.approx(slopes[k], rel=1e-14), k
    mids = [0.5 * (LT[k] + LT[k + 1]) for k in range(len(LT) - 1)]
    lam, sl = oracle.cooling([10.0 ** t for t in mids], z)
    wmid = np.array([10.0 ** (0.5 * (LL[k] + LL[k + 1])) for k in range(len(LT) - 1)]) * scale
    assert np.max(np.abs(lam / wmid - 1.0)) <= 1e-12
    assert np.max(np.abs(sl - np.array(slopes))) <= 1e-14
    lam, sl = oracle.cooling([10.0 ** 0.5, 10.0 ** 8.5], z)
    wend = np.array([10.0 ** (LL[0] - 0.5 * slopes[0]), 10.0 ** (LL[-1] + 0.5 * slopes[-1])]) * scale
    assert np.max(np.abs(lam / wend - 1.0)) <= 1e-12
    assert sl[0] == pytest.approx(slopes[0], rel=1e-14) and sl[1] == pytest.approx(slopes[-1], rel=1e-14)


def test_power_law_cooling_closed_form_first_order():
    th = dict(TH, gamma_heat=0.0)
    T0 = 10 ** 5.95
    lam0, slope = oracle.cooling([T0], th["z"])
    a = float(slope[0])
    C = float(lam0[0]) / T0 ** a
    nh, ce = 1.0, 1.0 / (72.7 * (2.0 / 3.0))
    K = nh * nh * C / (th["rate_unit"] * ce)
    T_end = 10 ** 5.7  # inside the segment [10^5.4, 10^6], away from the finite-time collapse
    t_end = (T0 ** (1 - a) - T_end ** (1 - a)) / ((1 - a) * K)
    errs = []
    for cap in (0.1, 0.01, 0.001):
        T, st = oracle.thermal_cells([T0], [nh], [ce], [t_end], dict(th, cap=cap))
        assert st[0] == 0
        errs.append(abs(T[0] - T_end) / T_end)
    assert errs[0] / errs[1] > 6 and errs[1] / errs[2] > 6, errs
    assert errs[2] < 2e-3, errs


def _equilibrium(nh, th):
    f = lambda T: nh * th["gamma_heat"] - nh * nh * oracle.cooling([T], th["z"])[0][0]
    lo, hi = 10 ** 3.0, 10 ** 3.99  # heating wins at lo, cooling at hi (n_H = 1)
    assert f(lo) > 0 > f(hi)
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if f(mid) > 0:
            lo = mid
        else:
            hi = mid
    return math.sqrt(lo * hi)


def test_equilibrium_is_fixed_point_and_attracts():
    nh, ce = 1.0, 1.0 / (72.7 * (2.0 / 3.0))
    Teq = _equilibrium(nh, TH)
    T, st = oracle.thermal_cells([Teq], [nh], [ce], [1.0], TH)
    assert abs(T[0] - Teq) <= 1e-9 * Teq
    for T0 in (0.7 * Teq, 1.6 * Teq):
        T, st = oracle.thermal_cells([T0], [nh], [ce], [10.0], TH)
        assert abs(T[0] - Teq) <= 1e-6 * Teq, (T0, T[0], Teq)


def test_thermal_apply_changes_only_internal_energy():
    st0 = inputs.turbulence((6, 5, 4), seed=3)
    U = st0.U.copy()
    U[4] = U[4] * 0.2 + 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0] * 0.8  # cooler gas
    st0 = st0.replace(U=U)
    st1, status = oracle.thermal_apply(st0, 1e-3, TH)
    assert np.array_equal(st1.U[:4], st0.U[:4])
    g = st0.geom

    def temp(st):
        bx, by, bz = st.bcc()
        kin = 0.5 * (st.U[1] ** 2 + st.U[2] ** 2 + st.U[3] ** 2) / st.U[0]
        p = (g.gamma - 1) * (st.U[4] - kin - 0.5 * (bx * bx + by * by + bz * bz))
        return TH["t_per_pr"] * p / st.U[0]

    T0, T1 = temp(st0), temp(st1)
    ce = st0.U[0] / (TH["t_per_pr"] * (g.gamma - 1))
    Tref, _ = oracle.thermal_cells(T0.ravel(), (TH["nh_per_rho"] * st0.U[0]).ravel(), ce.ravel(),
                                   np.full(T0.size, 1e-3), TH)
    assert np.max(np.abs(T1.ravel() - Tref) / Tref) < 1e-9


def _params(seed, scale=0.4):
    rng = np.random.default_rng(seed)
    H = oracle.HIDDEN
    return {"W1": rng.normal(0, scale, (H, 4)), "b1": rng.normal(0, 0.1, H), "W2": rng.normal(0, scale / 4, (H, H)),
            "b2": rng.normal(0, 0.1, H), "w3": rng.normal(0, scale / 4, H), "b3": rng.normal(0, 0.1, 1)}


def test_mlp_backward_matches_finite_differences():
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (24, 4))
    T = rng.normal(0, 0.3, 24)
    P = _params(6)
    loss, G = oracle.mlp_backward(X, T, P)
    y = oracle.mlp_forward(X, P)
    assert abs(loss - np.mean((y - T) ** 2)) < 1e-14
    h = 1e-6
    for k in P:
        flat = P[k].ravel()
        idx = rng.choice(flat.size, size=min(flat.size, 12), replace=False)
        for q in idx:
            Pp = {kk: vv.copy() for kk, vv in P.items()}
            Pm = {kk: vv.copy() for kk, vv in P.items()}
            Pp[k].ravel()[q] += h
            Pm[k].ravel()[q] -= h
            fd = (oracle.mlp_backward(X, T, Pp)[0] - oracle.mlp_backward(X, T, Pm)[0]) / (2 * h)
            g = G[k].ravel()[q]
            assert abs(fd - g) <= 1e-7 * max(abs(g), 1e-3), (k, q, fd, g)


def test_mlp_backward_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    X = rng.uniform(-1, 1, (40, 4))
    T = rng.normal(0, 0.3, 40)
    P = _params(8)
    loss, G = oracle.mlp_backward(X, T, P)
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in P.items()}
    x = torch.tensor(X)
    h1 = torch.tanh(x @ tp["W1"].T + tp["b1"])
    h2 = torch.tanh(h1 @ tp["W2"].T + tp["b2"])
    y = h2 @ tp["w3"] + tp["b3"]
    L = torch.mean((y - torch.tensor(T)) ** 2)
    L.backward()
    assert abs(L.item() - loss) < 1e-14
    for k in P:
        assert np.max(np.abs(tp[k].grad.numpy() - G[k])) < 1e-13


# ------------------------------------------------------- surrogate thermal step ----

def test_bf16_rounding_matches_torch_and_ties_to_even():
    """The oracle's BF16 rounding (8 significant bits, nearest, ties to even) equals torch's
    float32 -> bfloat16 conversion on random FP32 values over 60 binades, and takes the even
    neighbour at exact ties."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    v = (rng.uniform(-1, 1, 200000) * 2.0 ** rng.integers(-30, 30, 200000)).astype(np.float32)
    want = torch.tensor(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.bf16_round(v.astype(np.float64)), want)
    ties = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.75 + 2 ** -9, 0.0])
    assert np.array_equal(oracle.bf16_round(ties), [1.0, 1 + 2 ** -6, -1.0, 0.75, 0.0])


def _unit_network(b3=1.0):
    """All weights zero and b3 = 1: the network returns q = 1 exactly."""
    p = np.zeros(4545)
    p[-1] = b3
    return p


def _cells(st, th):
    g = st.geom
    bx, by, bz = st.bcc()
    rho = st.U[0]
    p = (g.gamma - 1) * (st.U[4] - 0.5 * (st.U[1] ** 2 + st.U[2] ** 2 + st.U[3] ** 2) / rho
                         - 0.5 * (bx * bx + by * by + bz * bz))
    T = th["t_per_pr"] * p / rho
    nh = th["nh_per_rho"] * rho
    ce = rho / (th["t_per_pr"] * (g.gamma - 1))
    return T, nh, ce


def _wide_range(st, th, dt, qmax=10.0, dmax=10.0):
    T, nh, _ = _cells(st, th)
    raw = [np.log10(nh), np.log10(np.clip(T, 10.0, 1e8)), np.full(T.shape, np.log10(dt)), np.full(T.shape, th["z"])]
    lo = [float(r.min()) - 0.1 for r in raw]
    s = [2.0 / (float(r.max()) + 0.1 - l) for r, l in zip(raw, lo)]
    return np.array(lo + s + [qmax, dmax])


def test_surrogate_step_with_unit_network_is_the_explicit_change():
    """With a network that returns q = 1 the applied change of log10 T is S = D / (1 + |D|),
    D = rate(T) dt / (T ln 10): to first order in D the explicit Euler change rate(T) dt of
    the isochoric equation, with rate = (n_H Gamma - n_H^2 Lambda(T, Z)) / (rate_unit c_e).
    The remainder is second order, |dT - rate dt| <= 5 D^2 T (ln 10 D^2 from the saturation,
    (ln 10 D)^2 / 2 from the exponential)."""
    th = inputs.DISC_THERMAL
    st = inputs.disc(24, 24, 12)
    dt = 2e-7
    out, fb, feat, _ = oracle.surrogate_apply(st, dt, th, _unit_network(), _wide_range(st, th, dt))
    assert not fb.any()
    T, nh, ce = _cells(st, th)
    lam, _ = oracle.cooling(T.ravel(), th["z"])
    rate = (nh * th["gamma_heat"] - nh * nh * lam.reshape(T.shape)) / (th["rate_unit"] * ce)
    D = rate * dt / (T * math.log(10.0))
    assert np.max(np.abs(D)) < 0.05 and np.max(np.abs(D)) > 1e-4
    assert np.max(np.abs(feat[..., 5] - D / (1 + np.abs(D)))) <= 1e-12 * np.max(np.abs(D))
    dT = (out.U[4] - st.U[4]) / ce
    assert np.all(np.abs(dT - rate * dt) <= 5 * D * D * T + 1e-12 * T)
    assert np.all(feat[..., 4] == 1.0)


def test_surrogate_step_features_and_fallback_bounds():
    """The standardised features are (log10 n_H - lo) s - 1, (log10 T - lo) s - 1, ...; a cell
    whose feature leaves [-1, 1], whose |q| exceeds qmax, or whose change |q S| exceeds dmax,
    takes the plain integrator and ends bit for bit where the plain thermal update puts it;
    every other cell takes the network's change."""
    th = inputs.DISC_THERMAL
    st = inputs.disc(24, 24, 12)
    dt = 2e-7
    T, nh, _ = _cells(st, th)
    rng = _wide_range(st, th, dt)
    plain, _ = oracle.thermal_apply(st, dt, th)
    # feature definition
    _, fb, feat, _ = oracle.surrogate_apply(st, dt, th, _unit_network(), rng)
    assert np.allclose(feat[..., 0], (np.log10(nh) - rng[0]) * rng[4] - 1.0, rtol=0, atol=1e-13)
    # (T carries the rounding of the pressure recovery's cancellation, ~1e-13 on the floor gas)
    assert np.allclose(feat[..., 1], (np.log10(np.clip(T, 10, 1e8)) - rng[1]) * rng[5] - 1.0, rtol=0, atol=1e-11)
    assert np.allclose(feat[..., 2], (math.log10(dt) - rng[2]) * rng[6] - 1.0, rtol=0, atol=1e-13)
    # density range cut at its median: the denser half leaves [-1, 1] and falls back
    ln = np.log10(nh)
    med = float(np.median(ln))
    cut = rng.copy()
    cut[4] = 2.0 / (med - cut[0])
    out, fb, _, _ = oracle.surrogate_apply(st, dt, th, _unit_network(), cut)
    want_fb = (ln - cut[0]) * cut[4] - 1.0 > 1.0
    assert 0 < want_fb.sum() < want_fb.size and np.array_equal(fb, want_fb)
    assert np.array_equal(out.U[4][fb], plain.U[4][fb])
    assert not np.array_equal(out.U[4][~fb], plain.U[4][~fb])
    # |q| = 1 above qmax, and every change above dmax: all cells fall back
    for q_d in ((0.999, 10.0), (10.0, 1e-9)):
        lim = rng.copy()
        lim[8], lim[9] = q_d
        out, fb, _, _ = oracle.surrogate_apply(st, dt, th, _unit_network(), lim)
        assert fb.all() and np.array_equal(out.U, plain.U)


def test_surrogate_network_rounds_h1_and_w2_to_bf16():
    """The network of the surrogate step is the FP64 forward pass (pinned above) with the
    operands of the 64 x 64 layer, h1 and W2, rounded to BF16: against oracle.mlp_forward on
    BF16-rounded W2 it differs by the rounding of h1 alone, at most
    sum_j |w3_j| sum_k |W2b_jk| 2^-8 |h1_k| (tanh is 1-Lipschitz), and not by nothing."""
    th = inputs.DISC_THERMAL
    st = inputs.disc(16, 16, 8)
    dt = 2e-7
    P = _params(12, scale=0.8)
    flat = np.concatenate([P[k].ravel() for k in ("W1", "b1", "W2", "b2", "w3", "b3")])
    _, _, feat, _ = oracle.surrogate_apply(st, dt, th, flat, _wide_range(st, th, dt))
    X = feat[..., :4].reshape(-1, 4)
    Pb = dict(P, W2=oracle.bf16_round(P["W2"].ravel()).reshape(P["W2"].shape))
    y = oracle.mlp_forward(X, Pb)
    h1 = np.tanh(X @ P["W1"].T + P["b1"])
    bound = (np.abs(h1) * 2.0 ** -8) @ np.abs(Pb["W2"]).T @ np.abs(P["w3"])
    diff = np.abs(feat[..., 4].ravel() - y)
    assert np.all(diff <= bound + 1e-14) and diff.max() > 0
