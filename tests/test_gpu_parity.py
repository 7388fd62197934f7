"""GPU parity: the CUDA step (through the C ABI) against the FP64 CPU oracle.

Error scale.  For each field the magnitude M is the maximum of |oracle| over the box;
for the momentum and the face field, M is taken over all three components (a vector's
component is compared against the vector's size, not against itself: a component that
starts at zero would otherwise be judged against its own rounding noise).

  FP64 path : |gpu - oracle| <= 1e-12 * max(|oracle|, 1e-3 M) at every value, every step.
              The two evaluate the same formulas in a different operation order; each
              operation differs by ~1e-16.
  mixed path: max |gpu - oracle| <= MIXED_TOL * M per step.  FP32 bulk arithmetic: the
              increment h div F of one step is ~CFL |U| and carries ~1e-7 relative
              rounding; the FP64 recovery and accumulation keep it from growing in |U|.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_1502_02935_gb300 import inputs, mhd

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-6
# The oracle each path is held to at these tolerances: Eq. 11's no-motion band read for the
# precision of the path's data (FP64: 2^-32 of the mass-flux scale, the oracle's default;
# mixed: 64 * 2^-23, FP32 rounding).  What the mixed path's reading costs against the
# FP64 reading is measured separately (test_mixed_against_the_fp64_reading_of_eq11).
EQ11 = {"fp64": None, "mixed": oracle.EQ11_EPS_FP32}


def _fields(st):
    mmag = float(np.max(np.abs(st.U[1:4])))
    bmag = max(float(np.max(np.abs(st.Bx))), float(np.max(np.abs(st.By))), float(np.max(np.abs(st.Bz))))
    out = [("rho", st.U[0], float(np.max(np.abs(st.U[0])))), ("mx", st.U[1], mmag), ("my", st.U[2], mmag),
           ("mz", st.U[3], mmag), ("E", st.U[4], float(np.max(np.abs(st.U[4]))))]
    out += [(k, getattr(st, k), bmag) for k in ("Bx", "By", "Bz")]
    return out


def errors(got: inputs.State, ref: inputs.State):
    """{field: (pointwise scaled max error, max error / M)}"""
    res = {}
    for (name, a, _), (_, b, M) in zip(_fields(got), _fields(ref)):
        M = max(M, 1e-300)
        d = np.abs(a - b)
        res[name] = (float(np.max(d / np.maximum(np.abs(b), 1e-3 * M))), float(np.max(d)) / M)
    return res


def assert_close(got: inputs.State, ref: inputs.State, tol: float, what: str = "", normalized: bool = False):
    for name, (pw, nm) in errors(got, ref).items():
        err = nm if normalized else pw
        assert err <= tol, f"{what} {name}: {'normalized' if normalized else 'pointwise'} error {err:.3e} > {tol:.1e}"


def _geom(n, bc, d=(0.1, 0.11, 0.13), lo=(0.0, 0.0, 0.0), gamma=5.0 / 3.0):
    return inputs.Geom(n[0], n[1], n[2], lo[0], lo[1], lo[2], d[0], d[1], d[2], bc, gamma)


CASES = {
    "brio_wu_800": lambda: (inputs.brio_wu(800), None),
    "ryu_jones_400": lambda: (inputs.ryu_jones(400), None),
    "sod_300_hydro": lambda: (inputs.sod(300), None),
    "orszag_tang_64x48": lambda: (inputs.orszag_tang(64, 48), None),
    "turbulence_37x29x23": lambda: (inputs.turbulence((37, 29, 23), seed=5), None),
    "blast_24": lambda: (inputs.blast(24, (0.3, 0.6, 0.45), (0.6, 0.0, 0.8)), None),
    "slow_contact_24x16x12": lambda: (inputs.slow_contact((24, 16, 12)), None),
    "outflow_17x9x5": lambda: (inputs.smooth_random(_geom((17, 9, 5), (1,) * 6), 3), None),
    "mixed_bc_13x11x6": lambda: (inputs.smooth_random(_geom((13, 11, 6), (1, 1, 0, 0, 1, 1)), 4), None),
    "disc_gravity_20x18x8": lambda: (
        inputs.smooth_random(_geom((20, 18, 8), (1,) * 6, d=(0.5, 0.5, 0.25), lo=(-5.0, -4.5, -1.0)), 9),
        dict(potential=2, v0=1.3, rc=0.5)),
    "gauss_well_1d_200": lambda: (
        inputs.smooth_random(_geom((200, 1, 1), (1, 1, 0, 0, 0, 0), d=(0.005, 1.0, 1.0), lo=(-0.5, 0, 0)), 2, 0.0),
        dict(potential=1, psi0=5.0, xc=0.0, xw=0.1)),
    # degenerate shapes: planes and lines off the x-y orientation (the per-direction kernels,
    # the corner-EMF kernel and the update with periodic images of a trivial x or y axis),
    # the smallest active axes (2 cells: each ghost is an image of an interior cell) and a
    # slab two planes thick
    "yz_plane_1x20x14": lambda: (inputs.smooth_random(_geom((1, 20, 14), (0, 0, 1, 1, 0, 0)), 21), None),
    "xz_plane_18x1x12": lambda: (inputs.smooth_random(_geom((18, 1, 12), (1, 1, 0, 0, 0, 0)), 22), None),
    "brio_wu_z_200": lambda: (inputs.brio_wu(200, axis=2), None),
    "tiny_2x2x2": lambda: (inputs.smooth_random(_geom((2, 2, 2), (0,) * 6), 23), None),
    "tiny_3x2x2_outflow": lambda: (inputs.smooth_random(_geom((3, 2, 2), (1,) * 6), 24), None),
    "slab_33x9x2": lambda: (inputs.smooth_random(_geom((33, 9, 2), (0, 0, 1, 1, 0, 0)), 25), None),
}


def _run_pair(st, src, precision, nsteps, cfl=0.4, counts=None, flux=None):
    g = mhd.Grid(st, precision=precision, cfl=cfl)
    if src:
        g.set_sources(**src)
    if flux:
        g.set_flux_scheme(flux)
    ref = st
    dts, floored = [], []
    for _ in range(nsteps):
        dt = oracle.cfl_dt(ref, cfl, source=src)
        dts.append(dt)
        g.step(dt)
        ref = oracle.step(ref, dt, source=src, floored=floored, eq11_eps=EQ11[precision])
    got = g.get_state(0)
    if counts is not None:
        counts.extend([g.metrics()["floored"], sum(floored)])
    g.close()
    return got, ref, dts


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp64_one_step_parity(case):
    st, src = CASES[case]()
    got, ref, _ = _run_pair(st, src, "fp64", 1)
    assert_close(got, ref, FP64_TOL, case)


@pytest.mark.parametrize("case", ["turbulence_37x29x23", "orszag_tang_64x48", "outflow_17x9x5", "brio_wu_800"])
def test_fp64_multi_step_parity(case):
    st, src = CASES[case]()
    got, ref, _ = _run_pair(st, src, "fp64", 5)
    assert_close(got, ref, 5 * FP64_TOL, case)


@pytest.mark.parametrize("case", sorted(c for c in CASES if c != "slow_contact_24x16x12"))
def test_mixed_one_step_parity(case):
    st, src = CASES[case]()
    got, ref, _ = _run_pair(st, src, "mixed", 1)
    assert_close(got, ref, MIXED_TOL, case, normalized=True)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("flux", ["march", "per_face"])
@pytest.mark.parametrize("case", ["turbulence_37x29x23", "outflow_17x9x5", "mixed_bc_13x11x6", "blast_24",
                                  "disc_gravity_20x18x8", "orszag_tang_64x48"])
def test_flux_kernels_match_oracle(case, flux, precision):
    """Both kernels of the y and z fluxes against the oracle (the automatic choice takes the
    per-face kernel on boxes this small): the marching kernel over ragged segments (29 y-faces
    and 23 z-faces in segments of 16), outflow and mixed boundaries, a potential, and a 2D
    plane.  FP64 two steps, mixed one (from the second step on, faces whose mass flux sits at
    the edge of the mixed path's no-motion band appear behind the blast front, as on the
    slow contacts)."""
    st, src = CASES[case]()
    if precision == "fp64":
        got, ref, _ = _run_pair(st, src, precision, 2, flux=flux)
        assert_close(got, ref, 2 * FP64_TOL, f"{case} {flux}")
    else:
        got, ref, _ = _run_pair(st, src, precision, 1, flux=flux)
        assert_close(got, ref, MIXED_TOL, f"{case} {flux}", normalized=True)


def test_mixed_one_step_parity_slow_contact():
    """The slowly moving contacts put the corrector's x-face mass fluxes around 1e-6 to 1e-5
    of their scale, across the edge of the mixed path's no-motion band (64 * 2^-23 = 7.6e-6):
    there FP32 rounding of the flux decides between the mean and the upwind side, against the
    oracle's FP64 flux under the same band.  Measured 7.6e-6 of the field's scale (B); bound
    2e-5."""
    st, src = CASES["slow_contact_24x16x12"]()
    got, ref, _ = _run_pair(st, src, "mixed", 1)
    assert_close(got, ref, 2e-5, "slow_contact_24x16x12", normalized=True)


def _l1(a, b):
    return float(np.sum(np.abs(a - b)) / max(np.sum(np.abs(b)), 1e-300))


@pytest.mark.parametrize("case", sorted(CASES))
def test_mixed_against_the_fp64_reading_of_eq11(case):
    """The mixed path's per-field error against the FP64 oracle under its default reading of
    Eq. 11 (no-motion band 2^-32 of the mass-flux scale), one step.  Where a face's mass flux
    lies between 2^-32 and 64 * 2^-23 of its scale the mixed path takes the mean of the two
    one-sided EMF derivatives where the oracle upwinds: FP32 fluxes cannot tell such a motion
    from rounding.  The edges involved change the face field by up to a few 1e-4 of B's scale
    on the blast (measured 1.0e-3 of it after the flux and energy updates) and leave the
    L1 error of every field at rounding level (<= 4e-7), except on the slowly moving contacts,
    which put every x-face into that range (L1 2.4e-5 in the momentum).  Bounds: max 2e-3 of
    the scale; L1 1e-6, and 5e-5 on the slow contacts."""
    st, src = CASES[case]()
    dt = oracle.cfl_dt(st, 0.4, source=src)
    g = mhd.Grid(st, precision="mixed", cfl=0.4)
    if src:
        g.set_sources(**src)
    g.step(dt)
    got = g.get_state(0)
    g.close()
    ref = oracle.step(st, dt, source=src)
    for name, (_, nm) in errors(got, ref).items():
        assert nm <= 2e-3, (case, name, nm)
    l1_bound = 5e-5 if case.startswith("slow_contact") else 1e-6
    for name, a, b in (("rho", got.U[0], ref.U[0]), ("m", got.U[1:4], ref.U[1:4]), ("E", got.U[4], ref.U[4]),
                       ("B", got.faces_flat(), ref.faces_flat())):
        if np.any(b):
            assert _l1(a, b) <= l1_bound, (case, name, _l1(a, b))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-14), ("mixed", 1e-6)])
def test_cfl_dt_matches_oracle(precision, tol):
    for case in ("turbulence_37x29x23", "brio_wu_800", "outflow_17x9x5"):
        st, _ = CASES[case]()
        g = mhd.Grid(st, precision=precision, cfl=0.4)
        a = g.cfl_dt()
        g.close()
        b = oracle.cfl_dt(st, 0.4)
        assert abs(a - b) <= tol * b, (case, a, b)


def test_device_cfl_step_equals_host_dt_step():
    """mhd_step(dt <= 0) uses the device CFL limit; it must equal stepping with the
    dt that mhd_cfl_dt reports."""
    st = inputs.turbulence((24, 20, 16), seed=3)
    a = mhd.Grid(st, precision="fp64", cfl=0.4)
    b = mhd.Grid(st, precision="fp64", cfl=0.4)
    for _ in range(3):
        a.step(-1.0)
        b.step(b.cfl_dt())
    sa, sb = a.get_state(0), b.get_state(0)
    assert np.array_equal(sa.U, sb.U) and np.array_equal(sa.Bx, sb.Bx)
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_is_bitwise_equal(precision):
    """Graph replay, direct launches (both with the y and z flux kernels on side streams) and
    the profiled step (every kernel on one stream) give the same bits: the side streams join
    before the update reads the fluxes."""
    st = inputs.turbulence((64, 48, 40), seed=8)
    a = mhd.Grid(st, precision=precision, cfl=0.4, flags=mhd.FLAG_GRAPH)
    b = mhd.Grid(st, precision=precision, cfl=0.4)
    c = mhd.Grid(st, precision=precision, cfl=0.4)
    c.set_profiling(True)
    for _ in range(4):
        a.step(-1.0)
        b.step(-1.0)
        c.step(-1.0)
    sa, sb, sc = a.get_state(0), b.get_state(0), c.get_state(0)
    for f in ("U", "Bx", "By", "Bz"):
        assert np.array_equal(getattr(sa, f), getattr(sb, f))
        assert np.array_equal(getattr(sa, f), getattr(sc, f))
    assert a.launch_count() > 0
    for g in (a, b, c):
        g.close()


def test_conservation_and_divb_on_device():
    """Properties that hold at any size: on a periodic box the FP64 path conserves the
    totals to roundoff and keeps div B = 0 to roundoff (CT)."""
    st = inputs.turbulence((48, 40, 36), seed=12)
    g = mhd.Grid(st, precision="fp64", cfl=0.4)
    m0 = g.metrics()
    for _ in range(10):
        g.step(-1.0)
    m1 = g.metrics()
    absU = np.abs(st.U).reshape(5, -1).sum(axis=1)
    for f in range(5):
        assert abs(m1["sums"][f] - m0["sums"][f]) <= 2e-13 * absU[f]
    assert m1["max_divb"] <= 1e-13 * 0.1 * 10
    g.close()


def _subbox(st: inputs.State, c, h):
    """(2h+1)^3 window of a periodic state centred on cell c, as an outflow patch."""
    g = st.geom
    n = (g.nx, g.ny, g.nz)
    idx = [np.arange(c[a] - h, c[a] + h + 1) % n[a] for a in range(3)]
    fidx = [np.arange(c[a] - h, c[a] + h + 2) % n[a] for a in range(3)]
    U = st.U[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]
    Bx = st.Bx[idx[2]][:, idx[1]][:, :, fidx[0]]
    By = st.By[idx[2]][:, fidx[1]][:, :, idx[0]]
    Bz = st.Bz[fidx[2]][:, idx[1]][:, :, idx[0]]
    gs = inputs.Geom(2 * h + 1, 2 * h + 1, 2 * h + 1, 0.0, 0.0, 0.0, g.dx, g.dy, g.dz, (1,) * 6, g.gamma)
    return inputs.State(gs, np.ascontiguousarray(U), np.ascontiguousarray(Bx), np.ascontiguousarray(By),
                        np.ascontiguousarray(Bz))


@pytest.mark.parametrize("precision,tol", [("mixed", MIXED_TOL), ("fp64", FP64_TOL)])
def test_full_size_turbulence_sampled_parity(precision, tol):
    """The 256^3 turbulent box in the configuration bench.py times: one step on the GPU,
    compared at sampled cells with the oracle run on a 11^3 window around each sample
    (a cell after one step depends only on cells within 3 of it)."""
    st = inputs.turbulence(256, seed=1502)
    g = mhd.Grid(st, precision=precision, cfl=0.4, flags=mhd.FLAG_GRAPH)
    dt = g.cfl_dt()
    g.step(dt)
    got = g.get_state(0)
    g.close()
    rng = np.random.default_rng(99)
    h = 5
    samples = [tuple(int(v) for v in rng.integers(0, 256, 3)) for _ in range(12)] + [(0, 0, 0), (255, 255, 255)]
    M = {name: m for name, _, m in _fields(got)}
    floor = 1e-3 if precision == "fp64" else 1.0
    for c in samples:
        sub = _subbox(st, c, h)
        out = oracle.step(sub, dt, eq11_eps=EQ11[precision])
        for f, name in enumerate(("rho", "mx", "my", "mz", "E")):
            a = got.U[f, c[2], c[1], c[0]]
            b = out.U[f, h, h, h]
            assert abs(a - b) <= tol * max(abs(b) if precision == "fp64" else 0.0, floor * M[name]), (c, f, a, b)
        for name in ("Bx", "By", "Bz"):
            a = getattr(got, name)[c[2], c[1], c[0]]
            b = getattr(out, name)[h, h, h]
            assert abs(a - b) <= tol * max(abs(b) if precision == "fp64" else 0.0, floor * M[name]), (c, name, a, b)


def test_hlld_device_matches_oracle():
    rng = np.random.default_rng(4)
    n = 4000
    wl = np.zeros((n, 8))
    wr = np.zeros((n, 8))
    for w in (wl, wr):
        w[:, 0] = rng.uniform(0.1, 3.0, n)
        w[:, 1:4] = rng.normal(0, 1.5, (n, 3))
        w[:, 4] = rng.uniform(0.01, 3.0, n)
        w[:, 6:8] = rng.normal(0, 1.0, (n, 2))
    bn = rng.normal(0, 1.0, n)
    bn[:200] = 0.0                     # hydro limit
    wl[200:400, 6:8] = 0.0             # degenerate: Bt = 0 with strong Bn
    wr[200:400, 6:8] = 0.0
    bn[200:400] = 3.0
    wr[400:600] = wl[400:600]          # equal states
    wl[600:700, 1] = 20.0              # supersonic both ways
    wr[600:700, 1] = 20.0
    ref = oracle.hlld(wl, wr, bn, 5.0 / 3.0)
    got = mhd.riemann_hlld(wl, wr, bn, 5.0 / 3.0, "fp64")
    scale = np.max(np.abs(ref), axis=1, keepdims=True) + 1e-3
    assert np.max(np.abs(got - ref) / scale) <= 1e-13
    got32 = mhd.riemann_hlld(wl, wr, bn, 5.0 / 3.0, "mixed")
    assert np.max(np.abs(got32 - ref) / scale) <= 2e-5
    # the mass-flux scale sits in the normal-field slot only inside the step; here it is 0
    assert np.all(got[:, 5] == 0.0)


def test_nonfinite_and_negative_inputs_are_reported():
    """Fault paths on the host side: a NaN or a negative density in the input is flagged
    by the device error word and returned as a status (no trap, no hang)."""
    st = inputs.turbulence((16, 16, 16), seed=1)
    bad = st.copy()
    bad.U[0, 3, 4, 5] = float("nan")
    g = mhd.Grid(bad, precision="mixed")
    g.step(1e-4)
    assert g.sync_status() == -3
    g.close()
    bad = st.copy()
    bad.U[0, 3, 4, 5] = -1.0
    g = mhd.Grid(bad, precision="fp64")
    g.step(1e-4)
    assert g.sync_status() == -4
    g.close()
    with pytest.raises(mhd.MHDError):
        mhd.Grid(inputs.State(inputs.Geom(0, 4, 4), np.zeros((5, 4, 4, 0)), np.zeros((4, 4, 1)),
                              np.zeros((4, 5, 0)), np.zeros((5, 4, 0))))


# ----------------------------------------------------------------- floors ----

def _negative_pressure_case():
    """Smooth outflow box with one cell whose energy leaves p < 0."""
    st = inputs.smooth_random(_geom((10, 8, 6), (1,) * 6, d=(0.1, 0.1, 0.1)), 3)
    U = st.U.copy()
    U[4, 3, 4, 5] = 0.0
    return st.replace(U=U), {"rho_floor": 1e-3, "pr_floor": 1e-2}


def test_floors_parity_negative_pressure_cell_fp64():
    """Floors in the recovery and after each step, against the oracle's floors, over three
    steps: the FP64 bound and the same count of floored cells."""
    st, src = _negative_pressure_case()
    counts = []
    got, ref, _ = _run_pair(st, src, "fp64", 3, counts=counts)
    assert_close(got, ref, 3 * FP64_TOL, "floors")
    assert counts[0] == counts[1] and counts[1] >= 1, counts


def test_floors_parity_negative_pressure_cell_mixed():
    """The same case on the mixed path, per step: each of three steps starts the device
    from the oracle's state and is compared after one step.  The floored cell (E = 0, its
    pressure clamped about two decades below its neighbours') puts a strong jump into the
    FP32 fluxes, and the momentum next to it carries a larger share of rounding than on the
    smooth cases: 4.7e-7, 1.4e-6 and 2.5e-6 (normalized) in the three steps, the same with
    the update and the recovery in separate kernels.  The bound is 4x the mixed per-step
    bound."""
    st, src = _negative_pressure_case()
    ref = st
    for s in range(3):
        counts = []
        got, nxt, _ = _run_pair(ref, src, "mixed", 1, counts=counts)
        assert_close(got, nxt, 4 * MIXED_TOL, f"floors step {s}", normalized=True)
        assert abs(counts[0] - counts[1]) <= 1, counts
        ref = nxt


def test_floors_parity_negative_pressure_cell_plane_fp64():
    """The floors on an x-y plane (the single-plane EMF + update kernel): a 2D outflow box with
    a 3 x 3 block of cells whose energy leaves p < 0, three steps, the FP64 bound and the same
    floored cells (the oracle floors four of them in the first step)."""
    st = inputs.smooth_random(_geom((40, 20, 1), (1, 1, 1, 1, 0, 0), d=(0.1, 0.1, 1.0)), 5)
    U = st.U.copy()
    U[4, 0, 6:9, 12:15] = 0.0
    st, src = st.replace(U=U), {"rho_floor": 1e-3, "pr_floor": 1e-2}
    counts = []
    got, ref, _ = _run_pair(st, src, "fp64", 3, counts=counts)
    assert_close(got, ref, 3 * FP64_TOL, "plane floors")
    assert counts[0] == counts[1] and counts[1] >= 1, counts


def test_floors_parity_disc():
    """Small disc (24 x 24 x 12) with its potential and floors, FP64, three steps.  Cells
    sitting exactly at the density floor may land either side of it by rounding, so the
    counts agree to 5 %."""
    st = inputs.disc(24, 24, 12)
    src = dict(inputs.DISC_POTENTIAL, **inputs.DISC_FLOORS)
    counts = []
    got, ref, _ = _run_pair(st, src, "fp64", 3, counts=counts)
    assert_close(got, ref, 3 * FP64_TOL, "disc floors")
    assert counts[1] > 0 and abs(counts[0] - counts[1]) <= 0.05 * counts[1] + 2, counts


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_floors_off_leave_the_step_unchanged(precision):
    """Floors that no cell reaches leave the device step bit for bit as without them.  On the
    mixed path the update kernel with floors stages the edge EMFs' inputs in shared memory
    and the one without reads them from global memory: the same bits over ragged tiles
    (40 x 20 cells: x tiles of 32 and 8, y tiles of 8, 8 and 4) and several planes."""
    st = inputs.turbulence((40, 20, 12), seed=7)
    a = mhd.Grid(st, precision=precision, cfl=0.4)
    b = mhd.Grid(st, precision=precision, cfl=0.4)
    b.set_sources(rho_floor=1e-12, pr_floor=1e-12, pr_ceil=1e12)
    for _ in range(3):
        a.step(-1.0)
        b.step(-1.0)
    sa, sb = a.get_state(0), b.get_state(0)
    assert np.array_equal(sa.U, sb.U) and np.array_equal(sa.Bz, sb.Bz)
    assert b.metrics()["floored"] == 0
    a.close()
    b.close()


def test_disc_with_floors_runs_without_error():
    """The disc (64 x 64 x 24, mixed path, plain thermal source) reaches negative pressure
    within a few steps without floors; with them 40 CFL steps complete without a device
    error, the CFL step stays within a factor 4 of its start, and cells are floored."""
    st = inputs.disc(64, 64, 24)
    g = mhd.Grid(st, precision="mixed", cfl=0.4)
    g.set_sources(**inputs.DISC_POTENTIAL, **inputs.DISC_FLOORS)
    g.set_thermal(mhd.THERMAL_PLAIN, **inputs.DISC_THERMAL)
    dts = []
    for _ in range(40):
        g.step(-1.0)
        dts.append(g.metrics()["dt_last"])
    g.sync()
    m = g.metrics()
    g.close()
    assert m["error_word"] == 0 and m["floored"] > 0
    assert min(dts) >= 0.25 * dts[0], (dts[0], min(dts))


def test_orszag_tang_to_t05_against_oracle():
    """The 2D vortex (128^2, periodic) run to t = 0.5 (about 400 CFL steps), each side with
    its own CFL step sequence: the FP64 path stays within 1e-10 (L1, relative) of the oracle
    per field, and the mixed path within 1e-3, the bound stated for the vortex in L1 at
    t = 0.5 (measured on 512^2: 8.7e-7)."""
    st = inputs.orszag_tang(128, 128)
    ref, nref = oracle.run(st, 0.4, 0.5)
    for precision, bound in (("fp64", 1e-10), ("mixed", 1e-3)):
        g = mhd.Grid(st, precision=precision, cfl=0.4)
        t, n = 0.0, 0
        while t < 0.5 * (1 - 1e-14):
            dt = min(g.cfl_dt(), 0.5 - t)
            g.step(dt)
            t += dt
            n += 1
        got = g.get_state(0)
        g.close()
        if precision == "fp64":
            assert n == nref, (n, nref)
        for name, a, b in (("rho", got.U[0], ref.U[0]), ("mx", got.U[1], ref.U[1]), ("my", got.U[2], ref.U[2]),
                           ("E", got.U[4], ref.U[4]), ("Bx", got.Bx, ref.Bx), ("By", got.By, ref.By)):
            l1 = float(np.sum(np.abs(a - b)) / np.sum(np.abs(b)))
            assert l1 <= bound, (precision, name, l1)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_restart_is_bitwise(precision):
    """Six device-CFL steps in one run equal three steps, a read-out of the state, a new
    context from it and three more steps, bit for bit (the recovery that the new context
    starts with gives the same W and CFL step as the update fused with it), with and
    without graph replay."""
    st = inputs.turbulence((24, 20, 16), seed=11)
    for flags in (0, mhd.FLAG_GRAPH):
        a = mhd.Grid(st, precision=precision, cfl=0.4, flags=flags)
        for _ in range(6):
            a.step(-1.0)
        sa = a.get_state(0)
        a.close()
        b = mhd.Grid(st, precision=precision, cfl=0.4, flags=flags)
        for _ in range(3):
            b.step(-1.0)
        mid = b.get_state(0)
        b.close()
        c = mhd.Grid(mid, precision=precision, cfl=0.4, flags=flags)
        for _ in range(3):
            c.step(-1.0)
        sc = c.get_state(0)
        c.close()
        for f in ("U", "Bx", "By", "Bz"):
            assert np.array_equal(getattr(sa, f), getattr(sc, f)), (flags, f)


def _window(st: inputs.State, c, h):
    """(2h+1)^3 window of a non-periodic state around interior cell c (at least h + 1 cells
    from every boundary), as an outflow patch at the same coordinates."""
    g = st.geom
    sl = [slice(c[a] - h, c[a] + h + 1) for a in range(3)]
    fl = [slice(c[a] - h, c[a] + h + 2) for a in range(3)]
    U = st.U[:, sl[2], sl[1], sl[0]]
    Bx = st.Bx[sl[2], sl[1], fl[0]]
    By = st.By[sl[2], fl[1], sl[0]]
    Bz = st.Bz[fl[2], sl[1], sl[0]]
    lo = (g.x0 + (c[0] - h) * g.dx, g.y0 + (c[1] - h) * g.dy, g.z0 + (c[2] - h) * g.dz)
    gs = inputs.Geom(2 * h + 1, 2 * h + 1, 2 * h + 1, lo[0], lo[1], lo[2], g.dx, g.dy, g.dz, (1,) * 6, g.gamma)
    return inputs.State(gs, np.ascontiguousarray(U), np.ascontiguousarray(Bx), np.ascontiguousarray(By),
                        np.ascontiguousarray(Bz))


def _sampled_compare(got, out, c, h, tol, precision, M, what):
    floor = 1e-3 if precision == "fp64" else 1.0
    for f, name in enumerate(("rho", "mx", "my", "mz", "E")):
        a, b = got.U[f, c[2], c[1], c[0]], out.U[f, h, h, h]
        assert abs(a - b) <= tol * max(abs(b) if precision == "fp64" else 0.0, floor * M[name]), (what, c, f, a, b)
    for name in ("Bx", "By", "Bz"):
        a, b = getattr(got, name)[c[2], c[1], c[0]], getattr(out, name)[h, h, h]
        assert abs(a - b) <= tol * max(abs(b) if precision == "fp64" else 0.0, floor * M[name]), (what, c, name, a, b)


@pytest.mark.parametrize("precision,tol", [("mixed", MIXED_TOL), ("fp64", FP64_TOL)])
def test_full_size_disc_sampled_parity(precision, tol):
    """The 512 x 512 x 128 disc in the configuration the bench's disc leg runs (log
    potential, floors, plain thermal source, graph replay): one device-CFL step, compared at
    sampled cells with the oracle step + thermal update of an 11^3 window around each."""
    st = inputs.disc(512, 512, 128)
    src = dict(inputs.DISC_POTENTIAL, **inputs.DISC_FLOORS)
    th = inputs.DISC_THERMAL
    g = mhd.Grid(st, precision=precision, cfl=0.4, flags=mhd.FLAG_GRAPH)
    g.set_sources(**src)
    g.set_thermal(mhd.THERMAL_PLAIN, **th)
    dt = g.cfl_dt()
    g.step(dt)
    got = g.get_state(0)
    g.close()
    rng = np.random.default_rng(12)
    h = 5
    samples = [(int(rng.integers(8, 504)), int(rng.integers(8, 504)), int(rng.integers(8, 120))) for _ in range(8)]
    samples += [(256, 256, 64), (200, 300, 63), (300, 210, 66), (256, 100, 64)]  # disc plane and centre
    M = {name: m for name, _, m in _fields(got)}
    for c in samples:
        win = _window(st, c, h)
        out = oracle.step(win, dt, source=src, eq11_eps=EQ11[precision])
        out, _ = oracle.thermal_apply(out, dt, th)
        _sampled_compare(got, out, c, h, tol, precision, M, "disc")


@pytest.mark.parametrize("scheme", ["per_phase", "persistent"])
@pytest.mark.parametrize("precision,tol", [("mixed", MIXED_TOL), ("fp64", FP64_TOL)])
def test_full_size_blast_batch_sampled_parity(precision, tol, scheme):
    """The 64-patch blast batch the bench's batched leg runs, in both of its schemes
    (per-phase graphs with the patches on their streams; one persistent launch under a
    graph), each patch with its own CFL dt: one step, one sampled cell in each of 16
    patches against the oracle on a periodic 11^3 window with that patch's dt."""
    sts = inputs.blast_batch(64, seed=1502)
    flags = mhd.FLAG_GRAPH | (mhd.FLAG_PERSISTENT if scheme == "persistent" else 0)
    g = mhd.Grid(sts, precision=precision, cfl=0.4, flags=flags)
    dts = g.cfl_dt_patches()
    g.step(-1.0)
    rng = np.random.default_rng(13)
    h = 5
    for p in rng.choice(64, 16, replace=False):
        st = sts[p]
        got = g.get_state(int(p))
        M = {name: m for name, _, m in _fields(got)}
        n = (st.geom.nx, st.geom.ny, st.geom.nz)
        c = tuple(int(rng.integers(0, n[a])) for a in range(3))
        out = oracle.step(_subbox(st, c, h), dts[p], eq11_eps=EQ11[precision])
        _sampled_compare(got, out, c, h, tol, precision, M, f"patch {p}")
    g.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 4e-5)])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_blast_reflection_symmetry_on_gpu(precision, tol, axis):
    """The reflection symmetry of a centred blast in a field along x (as the oracle pin), kept by
    the GPU path over 20 steps on a 40^3 box: the tiles of the update kernel (32 x 8 cells) are
    not mirror symmetric, so an indexing error at a tile edge would show as an asymmetry.
    The FP64 path is symmetric to roundoff.  The mixed path rounds the mirrored FP32 sums in
    another order; each of its steps is within 1e-6 of the scale of the (symmetric) FP64 one,
    so after 20 steps a state and its mirror image differ by at most 2 x 20 x 1e-6 = 4e-5
    (measured 1.2e-5)."""
    st = inputs.blast(40, (0.5, 0.5, 0.5), (1.0, 0.0, 0.0))
    g = mhd.Grid(st, precision=precision, cfl=0.4)
    for _ in range(20):
        g.step(-1.0)
    out = g.get_state(0)
    g.close()
    sgn = np.ones(5)
    sgn[1 + axis] = -1.0
    mU = np.flip(out.U, axis=3 - axis) * sgn[:, None, None, None]
    assert np.max(np.abs(out.U - mU)) <= tol * np.max(np.abs(out.U))
    faces = [out.Bx, out.By, out.Bz]
    bmax = max(np.max(np.abs(b)) for b in faces)
    for c, b in enumerate(faces):
        s = (1.0 if c == axis else -1.0) if axis == 0 else (-1.0 if c == axis else 1.0)
        assert np.max(np.abs(b - s * np.flip(b, axis=2 - axis))) <= tol * bmax, c


def test_oversized_grids_are_refused_and_leave_the_device_usable():
    """Maximum sizes.  A 2048^3 patch (1.1 TB of FP64 state alone) is refused with
    MHD_ERR_NOMEM by its first allocation, before any host array is read; a patch above
    2^40 cells with MHD_ERR_ARG, before any allocation.  The failed allocation leaves no
    error behind: a small grid made afterwards steps and matches the oracle."""
    import ctypes as C
    L = mhd.lib()
    dummy = np.zeros(8)
    for n, want in (((2048, 2048, 2048), -7), ((1 << 14, 1 << 14, 1 << 13), -1)):
        d = (mhd.PatchDesc * 1)()
        d[0].nx, d[0].ny, d[0].nz = n
        d[0].dx = d[0].dy = d[0].dz = 1.0 / n[0]
        d[0].gamma = 5.0 / 3.0
        gd = mhd.GridDesc(1, d, 1, 0.4, 0, None)
        ptr = (C.c_void_p * 1)(dummy.ctypes.data)
        h = C.c_void_p()
        assert L.mhd_init_grid(C.byref(h), C.byref(gd), ptr, ptr, 0) == want, n
        assert not h.value
    st, src = CASES["outflow_17x9x5"]()
    got, ref, _ = _run_pair(st, src, "fp64", 1)
    assert_close(got, ref, FP64_TOL, "after the refused grids")
