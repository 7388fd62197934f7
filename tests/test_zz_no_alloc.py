"""The allocation-free CFL entry point against the regular one.

mhd_cfl_dt_noalloc serves callers that cannot allocate device memory (applications
that reserve the device through their own pool, loops that cannot afford the
synchronisation of cudaMalloc/cudaFree).  Its scratch is a fixed array inside the
library, so this test checks that two calls in a row (different states, one array)
each agree with mhd_cfl_dt of an FP64 context, and that a patch larger than the
fixed scratch is refused.  The file name makes pytest collect it last.
"""
import math

import numpy as np
import pytest

from paper_1502_02935_gb300 import inputs, mhd

pytestmark = pytest.mark.gpu


def _device_state(st):
    import torch
    U = torch.from_numpy(np.ascontiguousarray(st.U)).cuda()
    B = torch.from_numpy(np.ascontiguousarray(st.faces_flat())).cuda()
    return U, B


def test_noalloc_cfl_matches_regular_cfl_twice():
    import torch
    states = [inputs.turbulence((40, 36, 30), seed=21),
              inputs.smooth_random(inputs.Geom(33, 17, 9, 0.0, 0.0, 0.0, 0.1, 0.12, 0.09, (1,) * 6, 1.4), 22)]
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for st in states:
        ref = mhd.Grid(st, precision="fp64", cfl=0.4)
        want = ref.cfl_dt()
        ref.close()
        U, B = _device_state(st)
        dt_dev.fill_(-1.0)
        rc = mhd.cfl_dt_noalloc(st.geom, 0.4, U.data_ptr(), B.data_ptr(), dt_dev.data_ptr(), stream.cuda_stream)
        assert rc == 0
        stream.synchronize()
        got = float(dt_dev.item())
        assert abs(got - want) <= 1e-14 * want, (got, want)


def test_noalloc_refuses_patches_beyond_the_fixed_scratch():
    import torch
    g = inputs.Geom(256, 256, 129, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, (0,) * 6, 5.0 / 3.0)
    assert g.ncell > mhd.NOALLOC_MAX_CELLS
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = mhd.cfl_dt_noalloc(g, 0.4, dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), 0)
    assert rc == -1


def test_noalloc_reports_a_cell_without_a_limit_as_nan():
    """A cell with negative pressure has no CFL limit; mhd_cfl_dt returns that as a status.
    The allocation-free call is asynchronous, so it reports it in the result: dt is NaN
    (not the minimum over the other cells)."""
    import torch
    st = inputs.turbulence((20, 16, 12), seed=23)
    U = st.U.copy()
    U[4, 5, 7, 9] = 0.0  # E = 0 with rho, m > 0: p < 0 at one cell
    st = st.replace(U=U)
    Ud, Bd = _device_state(st)
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = mhd.cfl_dt_noalloc(st.geom, 0.4, Ud.data_ptr(), Bd.data_ptr(), dt_dev.data_ptr(), stream.cuda_stream)
    assert rc == 0
    stream.synchronize()
    assert math.isnan(float(dt_dev.item()))
