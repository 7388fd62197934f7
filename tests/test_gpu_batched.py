"""Batched uneven patches in one persistent launch per step (GPU).

* The persistent step gives bit-for-bit the same state as the per-phase launches
  (same phase functions, deterministic CFL minimum), with and without graph replay.
* Every patch keeps its own CFL time step; each patch matches the oracle run with
  that patch's dt (FP64 path at 1e-12, mixed at the stated bound).
* The autotuner leaves the state unchanged and returns a tile shape.
* A barrier wait that cannot complete ends the launch with MHD_ERR_TIMEOUT.
"""
import numpy as np
import pytest

import oracle
from paper_1502_02935_gb300 import inputs, mhd
from tests.test_gpu_parity import EQ11, FP64_TOL, MIXED_TOL, assert_close

pytestmark = pytest.mark.gpu


def batch():
    g = lambda n, bc, d=(0.05, 0.06, 0.07): inputs.Geom(n[0], n[1], n[2], 0, 0, 0, d[0], d[1], d[2], bc, 5.0 / 3.0)
    return [inputs.blast(16, (0.3, 0.6, 0.45), (0.6, 0.0, 0.8)),
            inputs.turbulence((24, 20, 12), seed=31),
            inputs.blast(12, (0.5, 0.5, 0.5), (0.0, 0.6, 0.8)),
            inputs.smooth_random(g((19, 13, 7), (1,) * 6), 32),
            inputs.orszag_tang(40, 24),
            inputs.brio_wu(120)]


def _all_states(grid, n):
    return [grid.get_state(p) for p in range(n)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_persistent_matches_per_phase_launches(precision):
    """Same phase functions in two launch schemes: equal up to the rounding of differently
    contracted FMAs (the compiler may fuse multiply-adds differently in the two kernels)."""
    sts = batch()
    a = mhd.Grid(sts, precision=precision, cfl=0.4)
    b = mhd.Grid(sts, precision=precision, cfl=0.4, flags=mhd.FLAG_PERSISTENT | mhd.FLAG_GRAPH)
    for _ in range(3):
        a.step(-1.0)
        b.step(-1.0)
    tol = 3 * FP64_TOL if precision == "fp64" else 1e-6
    for p, (sa, sb) in enumerate(zip(_all_states(a, len(sts)), _all_states(b, len(sts)))):
        assert_close(sb, sa, tol, f"patch {p}", normalized=(precision == "mixed"))
    a.close()
    b.close()


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("mixed", MIXED_TOL)])
def test_persistent_per_patch_dt_matches_oracle(precision, tol):
    sts = batch()
    g = mhd.Grid(sts, precision=precision, cfl=0.4, flags=mhd.FLAG_PERSISTENT)
    dts = g.cfl_dt_patches()
    g.step(-1.0)
    for p, st in enumerate(sts):
        want_dt = oracle.cfl_dt(st, 0.4)
        assert abs(dts[p] - want_dt) <= (1e-14 if precision == "fp64" else 1e-6) * want_dt
        ref = oracle.step(st, dts[p], eq11_eps=EQ11[precision])
        assert_close(g.get_state(p), ref, tol, f"patch {p}", normalized=(precision == "mixed"))
    g.close()


def test_autotune_keeps_state_and_caches(tmp_path):
    sts = batch()
    g = mhd.Grid(sts, precision="mixed", cfl=0.4, flags=mhd.FLAG_PERSISTENT | mhd.FLAG_GRAPH)
    before = _all_states(g, len(sts))
    cache = str(tmp_path / "tune.json")
    tx, ty = g.autotune(cache)
    assert tx * ty in (128, 256, 512)
    scheme = g.step_scheme()
    assert scheme in ("persistent", "per_phase")
    after = _all_states(g, len(sts))
    for sa, sb in zip(before, after):
        assert np.array_equal(sa.U, sb.U)
    assert g.autotune(cache) == (tx, ty)  # served from the cache
    assert g.step_scheme() == scheme
    assert '"persistent": %d' % (scheme == "persistent") in open(cache).read()
    g.step(-1.0)
    g.sync()
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_switching_schemes_on_one_context(precision):
    """A context made with FLAG_PERSISTENT steps with either scheme: two steps per phase after
    two persistent steps equal the same four steps on a per-phase context (within the step's
    tolerance: the two schemes order some sums differently), and the persistent scheme is
    refused on a context made without the flag."""
    sts = batch()[:3]
    a = mhd.Grid(sts, precision=precision, cfl=0.4, flags=mhd.FLAG_PERSISTENT | mhd.FLAG_GRAPH)
    b = mhd.Grid(sts, precision=precision, cfl=0.4, flags=mhd.FLAG_GRAPH)
    for s in range(4):
        if s == 2:
            a.set_step_scheme("per_phase")
            assert a.step_scheme() == "per_phase"
        a.step(-1.0)
        b.step(-1.0)
    tol = 3 * FP64_TOL if precision == "fp64" else 1e-6
    for p in range(len(sts)):
        assert_close(a.get_state(p), b.get_state(p), 4 * tol, f"patch {p}", normalized=(precision == "mixed"))
    with pytest.raises(mhd.MHDError):
        b.set_step_scheme("persistent")
    a.close()
    b.close()


def test_barrier_timeout_is_reported():
    sts = batch()[:2]
    g = mhd.Grid(sts, precision="mixed", cfl=0.4, flags=mhd.FLAG_PERSISTENT)
    g.set_wait_limit(50.0, phantom_blocks=1)
    g.step(-1.0)
    assert g.sync_status() == -5
    g.close()


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("mixed", MIXED_TOL)])
def test_batch_with_inflow_solvers_and_scalars_matches_oracle(precision, tol):
    """Per-phase batch (each patch a chain on its own stream): a 3D periodic patch (fused
    EMF + update with periodic images), a 3D patch with an inflow side (fused, ghost fill), a
    2D patch (separate EMF kernel), all carrying two passive scalars, with the HLLC solver
    and kappa = 0.  Each patch equals the oracle run with its own CFL dt."""
    gm = lambda n, bc: inputs.Geom(n[0], n[1], n[2], 0, 0, 0, 0.05, 0.06, 0.07, bc, 1.4)
    sts = [inputs.turbulence((24, 20, 12), seed=31, b0=0.0),
           inputs.smooth_random(gm((19, 13, 9), (2, 1, 0, 0, 1, 1)), 33, 0.0),
           inputs.smooth_random(gm((30, 22, 1), (1, 1, 0, 0, 0, 0)), 34, 0.0)]
    inflow = {0: (1.2, 0.9, 0.1, 0.0, 1.1, 0.0, 0.0, 0.0)}
    xs = {0: [0.7, 0.2]}
    rng = np.random.default_rng(8)
    S = [np.stack([st.U[0] * rng.uniform(0.1, 0.9, st.U[0].shape) for _ in range(2)]) for st in sts]
    g = mhd.Grid(sts, precision=precision, cfl=0.4, flags=mhd.FLAG_GRAPH)
    g.set_riemann("hllc")
    g.set_reconstruction("kappa_zero")
    g.set_inflow(1, 0, inflow[0])
    g.set_scalars(2)
    for p in range(3):
        g.set_scalar_state(p, S[p])
    g.set_inflow_scalars(1, 0, xs[0])
    dts = g.cfl_dt_patches()
    g.step(-1.0)
    for p, st in enumerate(sts):
        infl = inflow if p == 1 else None
        want_dt = oracle.cfl_dt(st, 0.4, inflow=infl)
        assert abs(dts[p] - want_dt) <= (1e-14 if precision == "fp64" else 1e-6) * want_dt
        ref, Sref = oracle.step_scalars(st, S[p], dts[p], riemann="hllc", recon="kappa_zero", inflow=infl,
                                        eq11_eps=EQ11[precision],
                                        inflow_x=xs if p == 1 else None)
        assert_close(g.get_state(p), ref, tol, f"patch {p}", normalized=(precision == "mixed"))
        Sg = g.get_scalar_state(p)
        err = np.max(np.abs(Sg - Sref)) / np.max(np.abs(Sref))
        assert err <= (1e-12 if precision == "fp64" else 1e-6), (p, err)
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_persistent_carries_solver_and_reconstruction(precision):
    """The persistent step reads the Riemann solver and the kappa-scheme coefficients from its
    patch tables: with HLLC and kappa = 0 it matches the per-phase launches (to the rounding
    of differently compiled kernels)."""
    sts = [inputs.turbulence((24, 20, 12), seed=31, b0=0.0), inputs.blast(16, (0.3, 0.6, 0.45), (0.6, 0.0, 0.8))]
    a = mhd.Grid(sts, precision=precision, cfl=0.4)
    b = mhd.Grid(sts, precision=precision, cfl=0.4, flags=mhd.FLAG_PERSISTENT | mhd.FLAG_GRAPH)
    for g in (a, b):
        g.set_riemann("hllc")
        g.set_reconstruction("kappa_zero")
    for _ in range(3):
        a.step(-1.0)
        b.step(-1.0)
    tol = 3 * FP64_TOL if precision == "fp64" else 1e-6
    for p, (sa, sb) in enumerate(zip(_all_states(a, len(sts)), _all_states(b, len(sts)))):
        assert_close(sb, sa, tol, f"patch {p}", normalized=(precision == "mixed"))
    a.close()
    b.close()


def degenerate_batch():
    g = lambda n, bc: inputs.Geom(n[0], n[1], n[2], 0, 0, 0, 0.05, 0.06, 0.07, bc, 5.0 / 3.0)
    return [inputs.turbulence((13, 11, 6), seed=41),
            inputs.smooth_random(g((1, 20, 14), (0, 0, 1, 1, 0, 0)), 42),
            inputs.smooth_random(g((18, 1, 12), (1, 1, 0, 0, 0, 0)), 43),
            inputs.smooth_random(g((2, 2, 2), (0,) * 6), 44),
            inputs.smooth_random(g((3, 2, 2), (1,) * 6), 45),
            inputs.smooth_random(g((33, 9, 2), (0, 0, 1, 1, 0, 0)), 46),
            inputs.brio_wu(64, axis=2)]


@pytest.mark.parametrize("scheme", ["per_phase", "persistent"])
@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("mixed", MIXED_TOL)])
def test_degenerate_patches_match_oracle(precision, tol, scheme):
    """A batch of degenerate patches in both schemes: a y-z and an x-z plane, 2 x 2 x 2 and
    3 x 2 x 2 boxes (the per-phase chains run the fused donor-cell kernel on them, in
    segments of 2 planes), a slab two planes thick and a line along z, beside a small 3D box.
    Each patch equals the oracle run with its own CFL dt."""
    sts = degenerate_batch()
    flags = mhd.FLAG_PERSISTENT if scheme == "persistent" else mhd.FLAG_GRAPH
    g = mhd.Grid(sts, precision=precision, cfl=0.4, flags=flags)
    dts = g.cfl_dt_patches()
    g.step(-1.0)
    for p, st in enumerate(sts):
        want_dt = oracle.cfl_dt(st, 0.4)
        assert abs(dts[p] - want_dt) <= (1e-14 if precision == "fp64" else 1e-6) * want_dt, p
        ref = oracle.step(st, dts[p], eq11_eps=EQ11[precision])
        assert_close(g.get_state(p), ref, tol, f"patch {p}", normalized=(precision == "mixed"))
    g.close()
