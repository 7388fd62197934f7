"""GPU parity of the passive scalars (several gas components carried by the flow) against
the FP64 oracle, and their transfer paths.  The flow itself is unchanged by them."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1502_02935_gb300 import inputs, mhd
from tests.test_gpu_parity import EQ11, FP64_TOL, MIXED_TOL, assert_close

pytestmark = pytest.mark.gpu


def _scalars(st, seed, n=3):
    rng = np.random.default_rng(seed)
    x, y, z = st.geom.centres()
    X = [0.4 + 0.3 * np.sin(2 * np.pi * x)[None, None, :] * np.cos(2 * np.pi * y)[None, :, None],
         np.full(st.U[0].shape, 0.8), rng.uniform(0.0, 1.0, st.U[0].shape)]
    return np.stack([st.U[0] * X[m] for m in range(n)])


def _cases():
    g = inputs.Geom(16, 12, 8, 0.0, 0.0, 0.0, 0.1, 0.12, 0.09, (2, 1, 1, 1, 0, 0), 5.0 / 3.0)
    return {
        "turbulence_37x29x23": (inputs.turbulence((37, 29, 23), seed=5), None, None),
        "inflow_16x12x8": (inputs.smooth_random(g, 5), {0: (1.1, 0.6, 0.1, 0.0, 0.9, 0.2, 0.1, -0.1)},
                           {0: [0.9, 0.8, 0.1]}),
        "orszag_tang_64x48": (inputs.orszag_tang(64, 48), None, None),
        # a y-z plane (trivial x) with X entering through the z-lo inflow face
        "yz_inflow_1x20x14": (inputs.smooth_random(
            inputs.Geom(1, 20, 14, 0.0, 0.0, 0.0, 0.1, 0.12, 0.09, (0, 0, 1, 1, 2, 1), 5.0 / 3.0), 6),
            {4: (1.1, 0.1, -0.2, 0.7, 0.9, 0.15, 0.2, 0.3)}, {4: [0.2, 0.9, 0.5]}),
    }


@pytest.mark.parametrize("recon", ["kappa_third", "kappa_upwind"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["turbulence_37x29x23", "inflow_16x12x8", "orszag_tang_64x48", "yz_inflow_1x20x14"])
def test_scalars_match_oracle(case, precision, recon):
    st, inflow, inflow_x = _cases()[case]
    S = _scalars(st, 7)
    g = mhd.Grid(st, precision=precision, cfl=0.4)
    g.set_reconstruction(recon)
    for side, w in (inflow or {}).items():
        g.set_inflow(0, side, w)
    g.set_scalars(S.shape[0])
    g.set_scalar_state(0, S)
    for side, xs in (inflow_x or {}).items():
        g.set_inflow_scalars(0, side, xs)
    ref, Sref = st, S
    nsteps = 3 if precision == "fp64" else 1
    for _ in range(nsteps):
        dt = oracle.cfl_dt(ref, 0.4, inflow=inflow)
        g.step(dt)
        ref, Sref = oracle.step_scalars(ref, Sref, dt, recon=recon, inflow=inflow, inflow_x=inflow_x,
                                        eq11_eps=EQ11[precision])
    got, Sg = g.get_state(0), g.get_scalar_state(0)
    g.close()
    tol = FP64_TOL if precision == "fp64" else MIXED_TOL
    assert_close(got, ref, tol, case, normalized=(precision == "mixed"))
    for m in range(S.shape[0]):
        scale = np.max(np.abs(Sref[m]))
        if precision == "fp64":
            err = np.max(np.abs(Sg[m] - Sref[m]) / np.maximum(np.abs(Sref[m]), 1e-3 * scale))
        else:
            err = np.max(np.abs(Sg[m] - Sref[m])) / scale
        assert err <= tol, (case, m, err)


def test_scalars_leave_the_flow_bitwise_unchanged():
    st = inputs.turbulence((37, 29, 23), seed=5)
    a = mhd.Grid(st, precision="mixed", cfl=0.4, flags=mhd.FLAG_GRAPH)
    b = mhd.Grid(st, precision="mixed", cfl=0.4, flags=mhd.FLAG_GRAPH)
    b.set_scalars(2)
    b.set_scalar_state(0, _scalars(st, 3, 2))
    for _ in range(4):
        a.step(-1.0)
        b.step(-1.0)
    assert np.array_equal(a.get_state(0).U, b.get_state(0).U)
    a.close()
    b.close()


def test_scalar_state_round_trip_and_errors():
    st = inputs.turbulence((37, 29, 23), seed=5)
    g = mhd.Grid(st, precision="fp64", cfl=0.4)
    buf = np.empty(8)
    assert g.L.mhd_get_scalar_state(g.h, 0, buf.ctypes.data, 0) == -6  # MHD_ERR_STATE: no scalars yet
    g.set_scalars(3)
    S = _scalars(st, 9)
    g.set_scalar_state(0, S)
    assert np.array_equal(g.get_scalar_state(0), S)
    assert g.L.mhd_set_scalars(g.h, 9) == -1  # MHD_ERR_ARG: above MHD_MAX_SCALARS
    g.close()
