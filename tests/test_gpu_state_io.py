"""State transfer paths of mhd_get_state / mhd_set_state: staged (pageable host arrays),
direct through mapped page-locked host memory, and direct on device pointers.  All three
must move exactly the same values (a pure copy: compared bit for bit), including the
high boundary faces of periodic and outflow axes and ragged extents."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_1502_02935_gb300 import inputs, mhd

pytestmark = pytest.mark.gpu


def _geom(n, bc):
    return inputs.Geom(n[0], n[1], n[2], 0.0, 0.0, 0.0, 0.1, 0.11, 0.13, bc, 5.0 / 3.0)


CASES = {
    "periodic_37x29x23": lambda: inputs.turbulence((37, 29, 23), seed=5),
    "outflow_17x9x5": lambda: inputs.smooth_random(_geom((17, 9, 5), (1,) * 6), 3),
    "orszag_tang_40x24": lambda: inputs.orszag_tang(40, 24),
    "yz_plane_1x20x14": lambda: inputs.smooth_random(_geom((1, 20, 14), (0, 0, 1, 1, 0, 0)), 21),
    "tiny_2x2x2": lambda: inputs.smooth_random(_geom((2, 2, 2), (0,) * 6), 23),
}


def _same(a: inputs.State, U: np.ndarray, B: np.ndarray):
    assert np.array_equal(U.view(np.uint64), np.ascontiguousarray(a.U).reshape(-1).view(np.uint64))
    assert np.array_equal(B.view(np.uint64), np.ascontiguousarray(a.faces_flat()).reshape(-1).view(np.uint64))


@pytest.mark.parametrize("case", sorted(CASES))
def test_get_state_paths_agree(case):
    st = CASES[case]()
    g = mhd.Grid(st, precision="mixed", cfl=0.4)
    g.step(-1.0)
    ref = g.get_state(0)  # pageable host arrays: staged
    nU, nB = ref.U.size, ref.faces_flat().size
    U_h = torch.full((nU,), np.nan, dtype=torch.float64).pin_memory()
    B_h = torch.full((nB,), np.nan, dtype=torch.float64).pin_memory()
    g.get_state_ptr(0, U_h.data_ptr(), B_h.data_ptr(), False)  # mapped host: direct
    _same(ref, U_h.numpy(), B_h.numpy())
    U_d = torch.full((nU,), np.nan, dtype=torch.float64, device="cuda")
    B_d = torch.full((nB,), np.nan, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    g.get_state_ptr(0, U_d.data_ptr(), B_d.data_ptr(), True)  # device pointers: direct
    _same(ref, U_d.cpu().numpy(), B_d.cpu().numpy())
    g.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_set_state_paths_agree(case):
    st = CASES[case]()
    src = mhd.Grid(st, precision="mixed", cfl=0.4)
    src.step(-1.0)
    ref = src.get_state(0)
    src.close()
    U = np.ascontiguousarray(ref.U).reshape(-1)
    B = np.ascontiguousarray(ref.faces_flat()).reshape(-1)
    U_h = torch.from_numpy(U.copy()).pin_memory()
    B_h = torch.from_numpy(B.copy()).pin_memory()
    U_d, B_d = U_h.cuda(), B_h.cuda()
    torch.cuda.synchronize()
    for ptrs, on_device in (((U_h.data_ptr(), B_h.data_ptr()), False), ((U_d.data_ptr(), B_d.data_ptr()), True)):
        g = mhd.Grid(st, precision="mixed", cfl=0.4)
        g.set_state_ptr(0, ptrs[0], ptrs[1], on_device)
        g.sync()
        got = g.get_state(0)
        _same(got, U, B)
        # and the step from it equals the step from the staged upload
        h = mhd.Grid(st, precision="mixed", cfl=0.4)
        h.set_state(0, ref)
        g.step(-1.0)
        h.step(-1.0)
        a, b = g.get_state(0), h.get_state(0)
        _same(a, np.ascontiguousarray(b.U).reshape(-1), np.ascontiguousarray(b.faces_flat()).reshape(-1))
        g.close()
        h.close()
