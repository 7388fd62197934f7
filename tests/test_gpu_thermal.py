"""GPU parity of the thermal source term (plain FP64 integrator) against the oracle.

The integrator is the same algorithm on both sides (sub-stepped backward Euler with
Newton and bisection safeguard, FP64).  The two differ only in the rounding of the math
library (log10/pow) and of operation order, so results agree to ~1e-12 relative except
where a sub-step boundary moves; the tolerance below is 1e-10 relative on T.
"""
import numpy as np
import pytest

import oracle
from paper_1502_02935_gb300 import inputs, mhd
from tests.test_gpu_parity import EQ11, FP64_TOL, MIXED_TOL, assert_close

pytestmark = pytest.mark.gpu

TH = inputs.DISC_THERMAL


def test_thermal_cells_match_oracle():
    rng = np.random.default_rng(13)
    n = 3000
    T0 = 10 ** rng.uniform(1.0, 8.0, n)
    nh = 10 ** rng.uniform(-3.0, 3.0, n)
    ce = nh / 0.76 / (72.7 * (2.0 / 3.0))
    dt = 10 ** rng.uniform(-6.0, -2.0, n)
    ref, sref = oracle.thermal_cells(T0, nh, ce, dt, TH)
    got, sgot = mhd.thermal_cells(T0, nh, ce, dt, TH)
    rel = np.abs(got - ref) / ref
    assert np.quantile(rel, 0.99) <= 1e-10 and np.max(rel) <= 1e-6, (np.max(rel), np.quantile(rel, 0.99))
    assert np.mean(sgot == sref) > 0.99


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", MIXED_TOL)])
def test_disc_step_with_plain_thermal_matches_oracle(precision, tol):
    st = inputs.disc(32, 32, 12)
    g = mhd.Grid(st, precision=precision, cfl=0.4)
    g.set_sources(**inputs.DISC_POTENTIAL)
    g.set_thermal(mhd.THERMAL_PLAIN, **TH)
    dt = oracle.cfl_dt(st, 0.4)
    g.step(dt)
    got = g.get_state(0)
    stats = g.thermal_stats()
    g.close()
    ref = oracle.step(st, dt, source=inputs.DISC_POTENTIAL, eq11_eps=EQ11[precision])
    ref, status = oracle.thermal_apply(ref, dt, TH)
    assert stats["cells"] == st.geom.ncell and stats["capped"] == 0
    assert_close(got, ref, tol, precision, normalized=(precision == "mixed"))
