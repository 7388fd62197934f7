"""Cyclic rotation of a state's axes (x -> y -> z -> x), for invariance tests.

The scheme of Section 2 treats the three directions by cyclic permutation (text after
Eq. 11): the fluxes of each direction come from the same Riemann problem with the normal
component first, and the corner EMFs of Eq. 9-11 are built the same way about each axis.
A state whose x, y and z axes are relabelled cyclically (together with its vector
components, face arrays, spacings, origins and boundary conditions) must therefore step to
the relabelled result, up to rounding where the order of a sum over components changes.
A transposed operand, an axis index swapped in one direction, or a face array read with
another direction's strides breaks that.
"""
from __future__ import annotations

import numpy as np

from paper_1502_02935_gb300 import inputs


def rotate(st: inputs.State, times: int = 1) -> inputs.State:
    """The state with new axis (a + 1) mod 3 taking old axis a, applied ``times`` times
    (three times is the identity).  Arrays are (z, y, x); the new (z', y', x') are the old
    (y, x, z), so every cell or face array is transposed by (1, 2, 0)."""
    for _ in range(times % 3):
        g = st.geom
        ng = inputs.Geom(g.nz, g.nx, g.ny, g.z0, g.x0, g.y0, g.dz, g.dx, g.dy,
                         (g.bc[4], g.bc[5], g.bc[0], g.bc[1], g.bc[2], g.bc[3]), g.gamma)

        def t(a):
            return np.ascontiguousarray(np.transpose(a, (1, 2, 0)))

        U = np.stack([t(st.U[0]), t(st.U[3]), t(st.U[1]), t(st.U[2]), t(st.U[4])])
        # new x faces are the old z faces, new y the old x, new z the old y
        st = inputs.State(ng, U, t(st.Bz), t(st.Bx), t(st.By))
    return st
