"""The library's manufactured load vector and L2 error (host, FP64) against the oracle's (CPU)."""
import math

import numpy as np
import pytest

import workloads
from oracle import forms, manufactured as mf, mesh
from paper_2404_07911_gb300.binding import UnfittedOperator

OMEGA = 2.0 * math.pi


@pytest.mark.parametrize("disc", ["dg", "cg"])
@pytest.mark.parametrize("dim,p,N", [(2, 2, 8), (3, 1, 6), (3, 3, 5)])
def test_rhs_and_l2_error_match_oracle(disc, dim, p, N):
    cfg = dict(workloads.accuracy(p, N, dim=dim), discretization=disc)
    op = UnfittedOperator(cfg, device=-1)
    o = forms.Oracle(mesh.problem_from_dict(cfg), disc)
    c = np.zeros(dim)
    b_ref = o.load_vector(lambda X: mf.rhs(X, c, 1.0, OMEGA))
    if disc == "cg":
        b_ref = o.cg_prolongation().T @ b_ref
    b = op.manufactured_rhs(OMEGA)
    assert np.max(np.abs(b - b_ref)) <= 1e-13 * np.max(np.abs(b_ref))
    x = workloads.uniform_vector(op.n_dofs, 3)
    err, nrm = op.l2_error(OMEGA, x)
    err_ref, nrm_ref = o.l2_error(x, lambda X: mf.solution(X, c, 1.0, OMEGA))
    assert abs(err - err_ref) <= 1e-13 * err_ref and abs(nrm - nrm_ref) <= 1e-13 * nrm_ref
    op.close()


def test_plane_operator_rejects_the_sphere_benchmark():
    from paper_2404_07911_gb300.binding import UnfittedError

    op = UnfittedOperator(workloads.plane(p=1, N=4, dim=2), device=-1)
    with pytest.raises(UnfittedError):
        op.manufactured_rhs(OMEGA)
    op.close()
