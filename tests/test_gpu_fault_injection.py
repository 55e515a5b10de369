"""Fault injection on the host around device allocations: every device and pinned allocation of
operator creation, of the first discontinuous solve (work vectors), of the split operator's cell
lists and of the CSR assembly is made to fail once.  Each failing call returns UF_ENOMEM with
nothing left allocated, and the operator keeps working afterwards.  No GPU fault is involved: the
failing allocation is never handed to CUDA."""
import numpy as np
import pytest

import workloads
from paper_2404_07911_gb300 import (UnfittedError, UnfittedOperator, debug_fail_allocation,
                                    debug_live_allocations)
from paper_2404_07911_gb300.binding import UF_ENOMEM, UF_FP64

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {"3d_dg_q2_6": workloads.small(p=2, N=6),
         "3d_cg_q2_6": dict(workloads.small(p=2, N=6), discretization="cg")}


@pytest.fixture(autouse=True)
def _disarm():
    yield
    debug_fail_allocation(-1)


def _fails_cleanly(call):
    live = debug_live_allocations()
    debug_fail_allocation(0)
    with pytest.raises(UnfittedError) as ei:
        call()
    assert ei.value.status == UF_ENOMEM
    assert debug_live_allocations() == live
    debug_fail_allocation(-1)


@pytest.mark.parametrize("key", list(CASES))
def test_every_allocation_failure_is_clean(key):
    cfg = CASES[key]
    base = debug_live_allocations()
    k = 0
    while True:
        debug_fail_allocation(k)
        try:
            op = UnfittedOperator(cfg, device=0)
        except UnfittedError as e:
            assert e.status == UF_ENOMEM
            assert debug_live_allocations() == base, k
            k += 1
            assert k < 100
            continue
        break
    debug_fail_allocation(-1)
    # creation makes exactly k allocations: each of them was made to fail once
    assert debug_live_allocations() - base == k
    assert k >= 4
    x = torch.from_numpy(workloads.uniform_vector(op.n_dofs, 5)).cuda()
    ref = UnfittedOperator(cfg, device=0)
    assert torch.equal(op.vmult(x), ref.vmult(x))
    ref.close()

    b = op.vmult(x)
    dg = cfg.get("discretization") != "cg"

    def residual(xs):
        return float(torch.linalg.norm(op.vmult(xs) - b) / torch.linalg.norm(b))

    if dg:
        # the first solve of a discontinuous operator allocates the work vectors
        _fails_cleanly(lambda: op.solve(b, mode="fp64", tol=1e-8))
        xs, st = op.solve(b, mode="fp64", tol=1e-8)
        assert st["converged"] == 1 and residual(xs) <= 2e-8
    # the split operator's cell lists
    _fails_cleanly(lambda: op.solve(b, mode="ir_split", tol=1e-8))
    xs, st = op.solve(b, mode="ir_split", tol=1e-8)
    assert st["converged"] == 1 and residual(xs) <= 2e-8
    if dg:
        _fails_cleanly(lambda: op.assemble_csr(UF_FP64))
        op.assemble_csr(UF_FP64)
        y = op.csr_spmv(x).cpu().numpy()
        yb = b.cpu().numpy()
        assert np.max(np.abs(y - yb)) <= 1e-12 * np.max(np.abs(yb))
    op.close()
    assert debug_live_allocations() == base
