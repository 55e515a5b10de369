"""uf_kappa_gradient_noalloc: the kappa gradient for callers that cannot allocate device memory
(their device memory is held by another allocator, or allocation's device-wide synchronisation is
not acceptable in their loop).  Its partial buffer is a fixed array inside the library, so it
must give the same gradients as the allocating entry point, call after call.  Kept in a file that
pytest collects last."""
import ctypes

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _call_noalloc(lib, op, dk, r, x):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.uf_kappa_gradient_noalloc(op._h, ctypes.c_void_p(dk.data_ptr()),
                                         ctypes.c_void_p(r.data_ptr()),
                                         ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(stream))


# A 3D DG operator (one partial slot per cell and face, 1 + 6 per cell), a 2D DG operator
# (1 + 4 slots per cell) and a 3D continuous operator (gathers into the operator's cell-local
# work vectors first), each with a log-normal kappa.
NOALLOC_CASES = {
    "3d_dg_q3_24": workloads.cfg_kappa(N=24),
    "2d_dg_q2_12": workloads.small(p=2, N=12, dim=2),
    "3d_cg_q2_8": dict(workloads.small(p=2, N=8), discretization="cg"),
}


def test_noalloc_matches_allocating_entry_point_twice():
    """Two rounds over three operators: between the two calls on one operator the others have
    left their own partials in the shared array, so stale contents would show."""
    from paper_2404_07911_gb300 import UnfittedOperator, binding

    lib = binding.load_library()
    ops = []
    for name, cfg in NOALLOC_CASES.items():
        probe = UnfittedOperator(cfg, device=-1)
        n_active = probe.info["n_active"]
        probe.close()
        kappa = workloads.kappa_vector(n_active, seed=4)
        op = UnfittedOperator(cfg, device=0, kappa=kappa)
        xh, rh = workloads.x_and_b(op.n_dofs, seed=5)
        x = torch.from_numpy(xh).cuda()
        r = torch.from_numpy(rh).cuda()
        ref = op.kappa_gradient(r, x)
        torch.cuda.synchronize()
        ops.append((name, op, n_active, x, r, ref))
    for _ in range(2):
        for name, op, n_active, x, r, ref in ops:
            dk = torch.full((n_active,), float("nan"), dtype=torch.float64, device="cuda")
            assert _call_noalloc(lib, op, dk, r, x) == binding.UF_OK
            torch.cuda.synchronize()
            err = ((dk - ref).abs().max() / ref.abs().max()).item()
            assert err <= 1e-12, (name, err)
    for _, op, *_ in ops:
        op.close()


def test_noalloc_rejects_operators_beyond_its_buffer():
    from paper_2404_07911_gb300 import UnfittedOperator, binding

    lib = binding.load_library()
    cfg = workloads.small(p=1, N=100)  # about 2.9e5 active cells > 149,796
    op = UnfittedOperator(cfg, device=0, precisions=binding.UF_FP64)
    assert op.info["n_active"] * 7 > (1 << 20)
    dk = torch.zeros(op.info["n_active"], dtype=torch.float64, device="cuda")
    v = torch.zeros(op.n_dofs, dtype=torch.float64, device="cuda")
    assert _call_noalloc(lib, op, dk, v, v) == binding.UF_EINVAL
    assert b"fixed partial buffer" in lib.uf_last_error()
    op.close()
