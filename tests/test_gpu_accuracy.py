"""Sphere accuracy benchmark on the GPU: the manufactured problem solved with the library's
Jacobi-PCG (continuous and discontinuous operators) converges at the optimal L2 rate p + 1, and
the solution equals the oracle's direct solve of the same system."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads
from oracle import forms, mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OMEGA = 2.0 * math.pi


def _solve(cfg, mode="fp64"):
    from paper_2404_07911_gb300 import UnfittedOperator

    op = UnfittedOperator(cfg, device=0)
    b = op.manufactured_rhs(OMEGA)
    x, st = op.solve(torch.from_numpy(b).cuda(), mode=mode, tol=1e-12, max_iter=200000)
    assert st["converged"] == 1
    xh = x.cpu().numpy()
    err, nrm = op.l2_error(OMEGA, xh)
    op.close()
    return xh, b, err / nrm


@pytest.mark.parametrize("disc", ["cg", "dg"])
@pytest.mark.parametrize("dim,p,Ns", [(2, 2, (8, 16)), (3, 1, (6, 12)), (3, 2, (6, 12))])
def test_optimal_rate(disc, dim, p, Ns):
    errs = [_solve(dict(workloads.accuracy(p, N, dim=dim), discretization=disc))[2] for N in Ns]
    rate = math.log(errs[0] / errs[1], 2)
    assert rate > p + 1 - 0.35, (errs, rate)


@pytest.mark.parametrize("disc", ["cg", "dg"])
def test_solution_matches_direct_solve(disc):
    cfg = dict(workloads.accuracy(2, 6, dim=3), discretization=disc)
    x, b, _ = _solve(cfg, mode="ir")
    o = forms.Oracle(mesh.problem_from_dict(cfg), disc)
    A = o.cg_matrix() if disc == "cg" else o.assemble()
    x_ref = spla.spsolve(A.tocsc(), b)
    assert np.max(np.abs(x - x_ref)) <= 1e-8 * np.max(np.abs(x_ref))
