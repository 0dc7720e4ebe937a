"""The C ABI library builds, loads and exports every entry point that
include/air.h declares; no GPU needed."""
import os
import re

import paper_2010_11130_gb300 as air
from paper_2010_11130_gb300.air import EXPORTED

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "air.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(air_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_binding_names():
    assert sorted(EXPORTED) == _declared()


def test_library_exports_every_declared_symbol():
    air.build()
    L = air.lib()
    for name in _declared():
        assert hasattr(L, name), name


def test_status_strings_and_defaults():
    assert air.status_string(0) == "ok"
    assert "iteration cap" in air.status_string(-6)
    o = air.default_options()
    assert abs(o.theta - 0.25) < 1e-15 and o.relax == b"FCF" and o.restart == 30


def test_entry_points_reject_missing_arguments_without_a_gpu():
    """Argument checks come before any CUDA call: NULL or out-of-range
    arguments return AIR_ERR_INVALID_ARG (-1) on a machine without a GPU."""
    import ctypes as C
    air.build()
    L = air.lib()
    null = C.c_void_p(0)
    assert L.air_setup_batch(-1, None, 0.25, 1, None, None, None, None) == -1
    assert L.air_gmres_solve_batch(-1, None, None, None, None, 1e-8, None, None, None) == -1
    assert L.air_vcycle_multi(null, 4, null, null, null) == -1
    assert L.air_vcycle_multi_f32(null, 4, null, null, null) == -1
    assert L.air_bicgstab_solve_multi(None, null, 4, null, null, 1e-8, null, None) == -1
    assert L.air_bicgstab_solve(None, null, null, null, 1e-8, null, None) == -1
    assert L.air_csr_transpose(None, null, null, null, null) == -1
    assert L.air_csr_outer(None, null, null, 1.0, null, null) == -1


def test_hdg_entry_points_reject_missing_arguments_without_a_gpu():
    import ctypes as C
    air.build()
    L = air.lib()
    null = C.c_void_p(0)
    n, nnz = C.c_int64(0), C.c_int64(0)
    assert L.air_hdg_points(None, None, null, null, null, null) == -1
    assert L.air_hdg_size(None, None, 1, C.byref(n), C.byref(nnz), null) == -1
    assert L.air_hdg_assemble(None, None, None, 1, null, null, null, null, null, null, null) == -1
    assert L.air_hdg_velocity_gradient(None, None, None, null, null, null, null, null, null) == -1
    # a mesh of the wrong dimension or tables of the wrong size
    from paper_2010_11130_gb300.air import air_hdg_mesh, air_hdg_ref
    m = air_hdg_mesh(4, 1, 1, 1, 1, 1, 1, 1, 1, 1)
    r = air_hdg_ref(2, 10, 6, 64, 16, 6)
    assert L.air_hdg_points(C.byref(m), C.byref(r), null, null, null, null) == -1
    m.D = 3
    r.nq = 63
    assert L.air_hdg_size(C.byref(m), C.byref(r), 1, C.byref(n), C.byref(nnz), null) == -1


def test_adjoint_block_entry_points_reject_bad_arguments_without_a_gpu():
    import ctypes as C
    air.build()
    L = air.lib()
    null = C.c_void_p(0)
    assert L.air_csr_transpose_scaled(None, 6, null, null, null, null, null) == -1
    assert L.air_block_diag_apply(4, 0, null, 0, null, null, null) == -1
    assert L.air_block_diag_apply(4, 6, null, 7, null, null, null) == -1
    assert L.air_block_diag_apply(0, 6, null, 0, null, null, null) == 0
