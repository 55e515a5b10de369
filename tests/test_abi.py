"""The C ABI library loads, exports every symbol of include/unfitted.h, and its host-side
entry points behave as documented (CPU only: no compute call needs a GPU here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads
from paper_2404_07911_gb300 import binding
from paper_2404_07911_gb300.binding import UnfittedError, UnfittedOperator

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "unfitted.h")


def _declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(uf_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = binding.load_library()
    declared = _declared_functions()
    assert "uf_create_unfitted_operator" in declared and "uf_vmult" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTED) == declared


def test_host_only_create_info_destroy():
    op = UnfittedOperator(workloads.cfg_2d_q1(), device=-1)
    info = op.info
    assert info["n_active"] == 165 and info["n_cut"] == 52 and info["n_dofs"] == 660
    assert info["n_faces"] == 302 and info["n_faces_cut"] == 52 and info["n_faces_gp"] == 100
    assert info["dofs_per_cell"] == 4 and info["bytes_fp64"] > info["bytes_fp32"] > 0
    op.close()
    op.close()  # idempotent


def test_destroy_null_is_ok():
    lib = binding.load_library()
    assert lib.uf_destroy(None) == binding.UF_OK


@pytest.mark.parametrize("change,status", [
    (dict(dim=4), binding.UF_EINVAL),
    (dict(degree=0), binding.UF_EINVAL),
    (dict(degree=9), binding.UF_EUNSUPPORTED),
    (dict(quad_order=0), binding.UF_EINVAL),
    (dict(gp_max_order=5), binding.UF_EINVAL),
    (dict(radius=-1.0), binding.UF_EINVAL),
    (dict(n_cells=(16, 8, 1)), binding.UF_EUNSUPPORTED),   # anisotropic cells
    (dict(center=(10.0, 10.0, 0.0)), binding.UF_EGEOMETRY),  # no active cell
    (dict(ls_kind="plane", normal=(0.0, 0.0, 0.0), offset=0.5), binding.UF_EINVAL),  # zero normal
    (dict(ls_kind="plane", normal=(0.0, 1.0, 0.0), offset=-5.0), binding.UF_EGEOMETRY),  # plane below the box
    (dict(gp_kind="volume", gp_tau=0.0), binding.UF_EINVAL),
    (dict(n_cells=(40000, 40000, 1)), binding.UF_EUNSUPPORTED),  # background grid > 2^30 cells
])
def test_invalid_parameters(change, status):
    cfg = workloads.cfg_2d_q1()
    cfg.update(change)
    with pytest.raises(UnfittedError) as err:
        UnfittedOperator(cfg, device=-1)
    assert err.value.status == status
    assert binding.load_library().uf_last_error().decode()


def test_vmult_on_host_only_operator_is_refused():
    op = UnfittedOperator(workloads.cfg_2d_q1(), device=-1)
    lib = binding.load_library()
    buf = np.zeros(op.n_dofs)
    st = lib.uf_vmult(op._h, binding.UF_FP64, buf.ctypes.data_as(ctypes.c_void_p),
                      buf.ctypes.data_as(ctypes.c_void_p), None)
    assert st == binding.UF_ENODEVICE
    st = lib.uf_vmult(None, binding.UF_FP64, None, None, None)
    assert st == binding.UF_EINVAL


def test_host_buffer_calls_on_host_only_operator_are_refused():
    op = UnfittedOperator(workloads.cfg_2d_q1(), device=-1)
    lib = binding.load_library()
    buf = np.zeros(op.n_dofs)
    p = buf.ctypes.data_as(ctypes.c_void_p)
    for fn in (lib.uf_vmult_host, lib.uf_vmult_adjoint_host, lib.uf_vmult_host_async,
               lib.uf_vmult_adjoint_host_async):
        assert fn(op._h, binding.UF_FP64, p, p, None) == binding.UF_ENODEVICE
    assert lib.uf_host_wait(op._h, None) == binding.UF_ENODEVICE
    assert lib.uf_host_wait(None, None) == binding.UF_EINVAL
    op.close()


def test_kappa_validation():
    cfg = workloads.cfg_2d_q1()
    with pytest.raises(UnfittedError):
        UnfittedOperator(cfg, device=-1, kappa=-np.ones(165))
    op = UnfittedOperator(cfg, device=-1, kappa=np.ones(165))
    with pytest.raises(UnfittedError):
        op.set_kappa(np.zeros(165))
    op.set_kappa(np.full(165, 2.0))
