"""The allocation-free solve agrees with the regular solve.

cgp_poisson_solve_noalloc is for callers that cannot call cudaMalloc when
they solve (their device memory belongs to a pool or arena they do not
control, or allocating is forbidden in their time-critical loop).  It runs
the solver with the library's static scratch array instead of scratch held
by a mesh.  This file is collected last so that a failure here cannot hide
any other test in a run that stops at the first failure.
"""
import ctypes

import numpy as np
import pytest

from paper_2003_00082_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"


@pytest.fixture(scope="module")
def cgp():
    from paper_2003_00082_gb300 import build, cgp as c
    build.build()
    c.load()
    assert torch.cuda.is_available()
    return c


def rel(a, r):
    return float(torch.linalg.norm(a - r) / torch.linalg.norm(r))


def test_noalloc_solve_matches_the_regular_solve_twice_in_a_row(cgp):
    xy, tri = inputs.ogrid(64, 32)
    m = cgp.Mesh(xy, tri)
    xy_f, _, _ = m.fine_geometry()
    mats = m.matrices()
    rowptr = torch.as_tensor(mats["rowptr"], dtype=torch.int32, device=DEV)
    col = torch.as_tensor(mats["col"], dtype=torch.int32, device=DEV)
    K = torch.as_tensor(mats["K"], dtype=torch.float64, device=DEV)
    dinv = torch.as_tensor(mats["dinv"], dtype=torch.float64, device=DEV)

    # two different right-hand sides, solved back to back through the static scratch
    for step, kind in ((0, cgp.CGP_RHS_POTENTIAL), (5, cgp.CGP_RHS_PRESSURE)):
        u, v = inputs.velocity(xy_f, step, 0, vortices=True, noise_std=1e-3)
        uf = torch.as_tensor(u, device=DEV)
        vf = torch.as_tensor(v, device=DEV)
        b = torch.empty(m.n_c, dtype=torch.float64, device=DEV)
        cgp.cgp_restrict(m.handle, kind, (0.0, 1.0, 1.0), 20.0, uf, vf, b)
        x_ref = torch.zeros(m.n_c, dtype=torch.float64, device=DEV)
        ref = cgp.cgp_poisson_solve(m.handle, b, x_ref, tol=1e-12)
        x = torch.full((m.n_c,), 7.0, dtype=torch.float64, device=DEV)   # ignored: use_x0 is off
        info = cgp.cgp_poisson_solve_noalloc(m.n_c, rowptr, col, K, dinv, b, x, tol=1e-12)
        torch.cuda.synchronize()
        assert ref["status"] == cgp.CGP_OK and info["status"] == cgp.CGP_OK, (ref, info)
        assert abs(info["iterations"] - ref["iterations"]) <= 2
        assert rel(x, x_ref) <= 1e-10
        assert info["rel_res_true"] <= 1e-11
    m.close()


def test_noalloc_rejects_systems_larger_than_its_scratch(cgp):
    n = cgp.CGP_STATIC_MAX_ROWS + 1
    st = cgp.load().cgp_poisson_solve_noalloc(n, ctypes.c_void_p(1), ctypes.c_void_p(1), ctypes.c_void_p(1),
                                              ctypes.c_void_p(1), ctypes.c_void_p(1), ctypes.c_void_p(1),
                                              None, None, None)
    assert st == cgp.CGP_ERR_INVALID_ARG
    assert b"static scratch" in cgp.load().cgp_last_error()


def test_noalloc_solve_leaves_device_memory_untouched(cgp):
    """After a first call on the device, a call takes no device memory: the free bytes the driver
    reports are the same before and after it."""
    xy, tri = inputs.ogrid(32, 16)
    m = cgp.Mesh(xy, tri)
    mats = m.matrices()
    rowptr = torch.as_tensor(mats["rowptr"], dtype=torch.int32, device=DEV)
    col = torch.as_tensor(mats["col"], dtype=torch.int32, device=DEV)
    K = torch.as_tensor(mats["K"], dtype=torch.float64, device=DEV)
    dinv = torch.as_tensor(mats["dinv"], dtype=torch.float64, device=DEV)
    b = torch.randn(m.n_c, dtype=torch.float64, device=DEV, generator=torch.Generator(device=DEV).manual_seed(3))
    b -= b.mean()
    x = torch.zeros_like(b)
    first = cgp.cgp_poisson_solve_noalloc(m.n_c, rowptr, col, K, dinv, b, x, tol=1e-10)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    x.zero_()
    again = cgp.cgp_poisson_solve_noalloc(m.n_c, rowptr, col, K, dinv, b, x, tol=1e-10)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert first["status"] == again["status"] == cgp.CGP_OK
    assert first["iterations"] == again["iterations"]
    assert free_after == free_before
    m.close()
