"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(cgp_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_00082_gb300 import build, cgp
    build.build()
    return cgp.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cgp_assemble", "cgp_restrict", "cgp_poisson_solve", "cgp_prolong", "cgp_lorentz"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_binding_covers_the_header(lib):
    from paper_2003_00082_gb300 import cgp
    assert sorted(cgp.EXPORTS) == declared_functions()
    for name in cgp.EXPORTS:
        if name != "cgp_last_error":
            assert callable(getattr(cgp, name)), name


def test_host_side_argument_checks_need_no_gpu(lib):
    """Argument validation runs on the host and reports INVALID_ARG before any CUDA call."""
    from paper_2003_00082_gb300 import cgp
    import numpy as np
    with pytest.raises(cgp.CgpError) as e:
        cgp.cgp_assemble(np.zeros((2, 2)), np.zeros((1, 3), dtype=np.int32))
    assert e.value.status == cgp.CGP_ERR_INVALID_ARG
    # clockwise triangle
    xy = np.array([[0.0, 0.0], [0.0, 1.0], [1.0, 0.0]])
    with pytest.raises(cgp.CgpError) as e:
        cgp.cgp_assemble(xy, np.array([[0, 1, 2]], dtype=np.int32))
    assert e.value.status == cgp.CGP_ERR_INVALID_ARG and "clockwise" in str(e.value)
    # index out of range
    with pytest.raises(cgp.CgpError) as e:
        cgp.cgp_assemble(xy, np.array([[0, 2, 5]], dtype=np.int32))
    assert e.value.status == cgp.CGP_ERR_INVALID_ARG
    # the fine mesh of k levels must stay within 32-bit indexing (checked before any GPU work)
    big = np.zeros((6_000_000, 3), dtype=np.int32)
    with pytest.raises(cgp.CgpError) as e:
        cgp.cgp_assemble(xy, big, levels=3)
    assert e.value.status == cgp.CGP_ERR_INVALID_ARG and "too large" in str(e.value)
    del big
    # one to three coarsening levels (Eq. 18)
    for bad in (0, 4):
        with pytest.raises(cgp.CgpError) as e:
            cgp.cgp_assemble(xy, np.array([[0, 2, 1]], dtype=np.int32), levels=bad)
        assert e.value.status == cgp.CGP_ERR_INVALID_ARG and "levels" in str(e.value)
    # NULL handles
    assert lib.cgp_prolong(None, None, None, None) == cgp.CGP_ERR_INVALID_ARG
    assert lib.cgp_velocity_correct(None, None, None, None, 0.05, None, None, None) == cgp.CGP_ERR_INVALID_ARG
    assert lib.cgp_mesh_levels(None, None, None) == cgp.CGP_ERR_INVALID_ARG
    assert lib.cgp_set_far_field(None, 1) == cgp.CGP_ERR_INVALID_ARG
    assert lib.cgp_mesh_set_ogrid(None, 8, 4) == cgp.CGP_ERR_INVALID_ARG
    assert lib.cgp_far_field_nodes(None, None, None) == cgp.CGP_ERR_INVALID_ARG
    assert lib.cgp_set_tuning(None, 0, 0, 0, 0, 0) == cgp.CGP_ERR_INVALID_ARG
    assert lib.cgp_barrier_selftest(0, 0, 1, None) == cgp.CGP_ERR_INVALID_ARG
    assert b"nblk" in lib.cgp_last_error()


def test_product_path_does_not_import_the_oracle():
    """Only tests, smoke() and the benchmark's CPU leg may touch oracle/."""
    pkg = os.path.join(ROOT, "paper_2003_00082_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "cgp_oracle" not in text, fn
