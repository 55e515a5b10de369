"""The assembled-matrix baseline: the CSR matrix built on the device from the matrix-free
operator equals the oracle's brute-force assembly entry by entry, and its SpMV agrees with the
oracle and with the matrix-free product."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import forms, mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _op(cfg):
    from paper_2404_07911_gb300 import UnfittedOperator

    return UnfittedOperator(cfg, device=0)


@pytest.mark.parametrize("cfg", [workloads.cfg_2d_q1(), workloads.small(p=2, N=6),
                                 workloads.small(p=3, N=5, center=(0.0, 0.0, 0.0))],
                         ids=["2d_q1", "3d_q2_6", "3d_q3_5_center_on_grid"])
def test_csr_matches_oracle_assembly(cfg):
    from paper_2404_07911_gb300 import UF_FP32, UF_FP64

    A_ref = forms.Oracle(mesh.problem_from_dict(cfg)).assemble()
    op = _op(cfg)
    op.assemble_csr(UF_FP64)
    rp, col, val = op.export_csr(UF_FP64)
    n = op.n_dofs
    assert rp[0] == 0 and rp[-1] == len(col)
    for r in range(0, n, max(1, n // 50)):
        assert np.all(np.diff(col[rp[r]:rp[r + 1]]) > 0)  # ascending, unique
    A = sp.csr_matrix((val, col, rp), shape=(n, n))
    diff = abs(A - A_ref).max()
    assert diff <= 1e-12 * abs(A_ref).max()
    # every nonzero of the oracle's matrix lies in the CSR pattern
    pattern = sp.csr_matrix((np.ones_like(val), col, rp), shape=(n, n))
    outside = abs(A_ref) - abs(A_ref).multiply(pattern)
    assert outside.max() <= 1e-14 * abs(A_ref).max()
    x = workloads.uniform_vector(n, 3)
    y = op.csr_spmv(torch.from_numpy(x).cuda()).cpu().numpy()
    y_ref = A_ref @ x
    assert np.max(np.abs(y - y_ref)) <= 1e-12 * np.max(np.abs(y_ref))
    op.assemble_csr(UF_FP32)
    x32 = x.astype(np.float32)
    y32 = op.csr_spmv(torch.from_numpy(x32).cuda()).double().cpu().numpy()
    y32_ref = A_ref @ x32.astype(np.float64)
    assert np.max(np.abs(y32 - y32_ref)) <= 1e-5 * np.max(np.abs(y32_ref))
    op.release_csr()
    op.release_csr()


def test_csr_full_size_matches_matrix_free():
    from paper_2404_07911_gb300 import UF_FP64

    cfg = workloads.cfg_3d_q3()
    op = _op(cfg)
    op.assemble_csr(UF_FP64)
    nnz, byts = op.csr_info(UF_FP64)
    # interior rows couple to the cell and its 6 face neighbours: 7 n^3 = 448 nonzeros
    assert 0.9 * op.n_dofs * 448 < nnz <= op.n_dofs * 448
    x = torch.from_numpy(workloads.uniform_vector(op.n_dofs, cfg["seed"])).cuda()
    y_csr = op.csr_spmv(x)
    y_mf = op.vmult(x)
    err = (y_csr - y_mf).abs().max().item() / y_mf.abs().max().item()
    assert err <= 1e-12
    op.release_csr()
