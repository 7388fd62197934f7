"""Empty and out-of-range inputs of the unit entry points (GPU).

Each entry that takes a count n accepts n = 0 (nothing launched, null pointers allowed)
and refuses a negative n with MHD_ERR_ARG; the training gradient needs at least one row.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

from paper_1502_02935_gb300 import mhd

pytestmark = pytest.mark.gpu

ERR_ARG = -1


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_riemann_entries_accept_zero_faces(precision):
    w = np.zeros((0, 8))
    assert mhd.riemann_hlld(w, w, np.zeros(0), 5.0 / 3.0, precision).shape == (0, 8)
    for solver in ("hlld", "hllc", "hll"):
        assert mhd.riemann_flux(solver, w, w, np.zeros(0), 5.0 / 3.0, precision).shape == (0, 8)


def test_cell_entries_accept_zero_cells():
    f32, f64 = mhd.convert_fp(np.zeros(0), np.zeros(0, dtype=np.float32))
    assert f32.shape == (0,) and f64.shape == (0,)
    T, status = mhd.thermal_cells(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), {"rate_unit": 1.0})
    assert T.shape == (0,) and status.shape == (0,)
    params = np.zeros(mhd.MLP_NPARAM, dtype=np.float32)
    for tc in (False, True):
        assert mhd.mlp_forward(np.zeros((0, 4), dtype=np.float32), params, tcgen05=tc).shape == (0,)


def test_negative_counts_and_empty_training_are_refused():
    L = mhd.lib()
    null = None
    assert L.mhd_riemann_hlld(-1, null, null, null, 5.0 / 3.0, 0, null, null) == ERR_ARG
    assert L.mhd_riemann_flux(1, -1, null, null, null, 5.0 / 3.0, 0, null, null) == ERR_ARG
    assert L.mhd_convert_fp(-1, null, null, null, null, null) == ERR_ARG
    d = mhd.ThermalDesc(mhd.THERMAL_PLAIN, 2e-26, 0.02, 1.0, 0.1, 0.76, 72.7)
    assert L.mhd_thermal_cells(-1, null, null, null, null, C.byref(d), null, null, null) == ERR_ARG
    params = np.zeros(mhd.MLP_NPARAM, dtype=np.float32)
    for fn in (L.mhd_mlp_forward, L.mhd_mlp_forward_tc):
        assert fn(-1, null, params.ctypes.data, null, null) == ERR_ARG
    for tc in (False, True):
        with pytest.raises(mhd.MHDError) as e:
            mhd.mlp_grad(np.zeros((0, 4), dtype=np.float32), np.zeros(0), params, tcgen05=tc)
        assert e.value.code == ERR_ARG
