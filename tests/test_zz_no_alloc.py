"""The pressure-correction solve that allocates nothing (ss_poisson_solve_noalloc).

Some callers cannot allocate device memory: an application whose memory
manager owns the whole GPU and rejects allocations it did not make, a loop
with a hard latency budget where a cudaMalloc may stall the device, or a
plugin handed only a stream and device pointers. For them the library keeps
this one solve's scratch in a fixed device array. This test checks, through
the C-ABI, that two calls in a row give the pressure correction of the
oracle's own solve and the same one as the workspace-based solve (ss_solve on
the pressure system), on the default stream and on a side stream, that the
caller's right-hand side is left untouched, and that a grid above the fixed
size limit is refused with a message. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2303_10783_gb300 import cases, solid

pytestmark = pytest.mark.gpu

TOL = 1e-13
REL = 1e-12        # against the workspace solve: the same algorithm at the same tolerance
REL_ORACLE = 1e-10 # against the oracle: the tolerance of the stage parity tests for pressure corrections


@pytest.mark.parametrize("side", [False, True], ids=["default-stream", "side-stream"])
@pytest.mark.parametrize("case", [cases.box_3d(37, 23, 17), cases.cavity_2d(61, 37)], ids=["3d", "2d"])
def test_noalloc_solve_matches_oracle_and_workspace_solve(lib, case, side):
    import torch
    case = dict(case, tol_p=TOL, max_it_p=20000, precond_p="jacobi")   # the same algorithm as the no-alloc solve
    c = solid.Case(case)
    c.set_fields(cases.random_state(case, 5))
    for name in "uvw"[: case["dim"]]:
        c.assemble(name)          # u* starts as u^n: a non-solenoidal field gives a rich right-hand side
    c.assemble("p")
    b = c.get_system("p")["b"].copy()
    c.solve("p")
    ref = c.get_system("p")["x"]

    nx, ny, nz = case["nx"], case["ny"], case["nz"] if case["dim"] == 3 else 1
    hx, hy, hz = case["lx"] / nx, case["ly"] / ny, (case["lz"] / nz if case["dim"] == 3 else 1.0)
    pref = oracle.solve_poisson(oracle.Grid(case), b - b.mean())
    stream = torch.cuda.Stream() if side else torch.cuda.current_stream()
    bd = torch.from_numpy(b).cuda()
    torch.cuda.synchronize()
    for call in range(2):
        x = torch.full_like(bd, float("nan"))
        stream.wait_stream(torch.cuda.current_stream())   # x is filled before the solve writes it
        iters, relres = ctypes.c_int(-1), ctypes.c_double(-1.0)
        st = lib.ss_poisson_solve_noalloc(case["dim"], nx, ny, nz, hx, hy, hz, ctypes.c_void_p(bd.data_ptr()),
                                          ctypes.c_void_p(x.data_ptr()), TOL, 20000, ctypes.byref(iters),
                                          ctypes.byref(relres), ctypes.c_void_p(stream.cuda_stream))
        assert st == solid.SS_OK, lib.ss_last_error()
        assert 0 < iters.value < 20000 and 0.0 <= relres.value <= TOL
        got = x.cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < REL, (call, err)
        err_o = np.abs(got - pref).max() / np.abs(pref).max()
        assert err_o < REL_ORACLE, (call, err_o)
        assert abs(got.mean()) < 1e-12 * np.abs(pref).max()   # the zero-mean gauge
        assert np.array_equal(bd.cpu().numpy(), b)      # the caller's right-hand side is not modified
    c.close()


def test_noalloc_rejects_grids_above_its_limit(lib):
    import torch
    bd = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = lib.ss_poisson_solve_noalloc(3, 128, 96, 96, 1e-3, 1e-3, 1e-3, ctypes.c_void_p(bd.data_ptr()),
                                      ctypes.c_void_p(bd.data_ptr()), 1e-10, 10, None, None, None)
    assert st == solid.SS_EINVAL
    assert b"limit" in lib.ss_last_error()
