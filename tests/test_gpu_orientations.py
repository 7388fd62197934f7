"""The device step under a cyclic relabelling of the axes (x -> y -> z -> x).

Each direction of the step runs in its own kernels (the fused donor-cell kernel marches in
z, the kappa-scheme x faces share reconstructions between lanes, the y and z faces march,
the EMF + update kernel tiles x and y and marches in z), so the same problem laid along
another axis goes through other code.  The scheme treats the directions by cyclic
permutation (text after Eq. 11; the oracle keeps the invariance to rounding, pinned in
tests/test_oracle_pins.py), so the relabelled problem must step to the relabelled result.
FP64 path, three steps at one fixed dt; the shapes are ragged in every orientation
(37 x 29 x 23 becomes 23 x 37 x 29 and 29 x 23 x 37), the 2D vortex turns into a y-z and a
z-x plane, the shock tube into a line along y and z.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1502_02935_gb300 import inputs, mhd
from tests.axes import rotate

pytestmark = pytest.mark.gpu

TOL = 1e-12  # of each field's scale, after three steps


def _geom(n, bc, d=(0.1, 0.11, 0.13)):
    return inputs.Geom(n[0], n[1], n[2], 0.0, 0.0, 0.0, d[0], d[1], d[2], bc, 5.0 / 3.0)


CASES = {
    "turbulence_37x29x23": lambda: inputs.turbulence((37, 29, 23), seed=5),
    "mixed_bc_13x11x6": lambda: inputs.smooth_random(_geom((13, 11, 6), (1, 1, 0, 0, 1, 1)), 4),
    "blast_24": lambda: inputs.blast(24, (0.3, 0.6, 0.45), (0.6, 0.0, 0.8)),
    "orszag_tang_64x48": lambda: inputs.orszag_tang(64, 48),
    "brio_wu_400": lambda: inputs.brio_wu(400),
}


def _scaled_max(a: inputs.State, b: inputs.State) -> float:
    e = 0.0
    for f in range(5):
        e = max(e, float(np.max(np.abs(a.U[f] - b.U[f]))) / max(float(np.max(np.abs(b.U[f]))), 1e-300))
    bmax = max(float(np.max(np.abs(getattr(b, k)))) for k in ("Bx", "By", "Bz"))
    for k in ("Bx", "By", "Bz"):
        e = max(e, float(np.max(np.abs(getattr(a, k) - getattr(b, k)))) / max(bmax, 1e-300))
    return e


@pytest.mark.parametrize("case", sorted(CASES))
def test_relabelled_axes_step_alike(case):
    st = CASES[case]()
    dt = oracle.cfl_dt(st, 0.4)
    outs = []
    for r in range(3):
        s = rotate(st, r)
        g = mhd.Grid(s, precision="fp64", cfl=0.4)
        for _ in range(3):
            g.step(dt)
        outs.append(rotate(g.get_state(0), 3 - r))
        g.close()
    for r in (1, 2):
        e = _scaled_max(outs[r], outs[0])
        assert e <= TOL, f"{case}: rotated {r} time(s), {e:.3e} of the scale"
