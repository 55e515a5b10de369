"""Pins of the oracle's continuous Q_p operator (CPU).

* numbering: the CG DoF count the paper prints in Sec. 6.2 (CG, p = 3, 48^3: 1,597,645);
* the exact solution of -Lap u = 1 in the ball with u = 0 on the sphere is the quadratic
  u = (R^2 - |x - c|^2) / (2 d); it lies in Q_p for p >= 2, and the Nitsche / ghost-penalty form
  is consistent, so the discrete solution reproduces it up to the quadrature error (this pins the
  operator, the load vector and the numbering together) - for CG and for DG;
* the load vector sums to |Omega| (partition of unity) and A_cg is symmetric positive definite.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads
from oracle import forms, mesh


def test_cg_numbering_reproduces_paper_count():
    prob = mesh.Problem(3, 3, (48,) * 3, (-1.035,) * 3, (1.035,) * 3, (0.0,) * 3, 1.0, 4, 1, 1, 3, 0.5)
    o = forms.Oracle(prob, "cg")
    n_cg, l2g = o.cg_numbering()
    assert n_cg == 1597645
    assert l2g.shape == (o.mesh.n_active, 64) and l2g.max() == n_cg - 1


def _exact(X, c, dim):
    return (1.0 - np.sum((X - np.asarray(c)[:dim]) ** 2, axis=1)) / (2 * dim)


def _node_coordinates(o):
    """Physical coordinates of every (cell, local DoF) Lobatto node."""
    from oracle import basis
    z = basis.gauss_lobatto_nodes(o.n)
    X = np.zeros((o.mesh.n_active, o.ndof, o.prob.dim))
    for e in range(o.mesh.n_active):
        lo, _ = mesh.cell_box(o.prob, o.mesh.index_of(e))
        for a in range(o.prob.dim):
            X[e, :, a] = lo[a] + o.prob.h * z[o.lidx[:, a]]
    return X


# (discretisation, dim, p, N, q, tolerance): the error left is the quadrature error of the cut
# cells, tiny in 2D at high q and larger on the very coarse 3D grids (h = 0.4)
@pytest.mark.parametrize("disc,dim,p,N,q,tol", [("cg", 2, 3, 10, 10, 1e-10), ("cg", 2, 2, 8, 8, 1e-9),
                                                ("dg", 2, 2, 8, 10, 1e-11), ("cg", 3, 2, 6, 8, 1e-6)])
def test_quadratic_solution_is_reproduced(disc, dim, p, N, q, tol):
    cfg = workloads.small(p=p, N=N, dim=dim)
    cfg["quad_order"] = q
    o = forms.Oracle(mesh.problem_from_dict(cfg), disc)
    X = _node_coordinates(o)
    if disc == "cg":
        A, b = o.cg_matrix(), o.cg_load_vector()
        n_cg, l2g = o.cg_numbering()
        u_ex = np.zeros(n_cg)
        u_ex[l2g.reshape(-1)] = _exact(X.reshape(-1, dim), cfg["center"], dim)
        assert abs(b.sum() - (math.pi if dim == 2 else 4 * math.pi / 3)) < 1e-8
    else:
        A, b = o.assemble(), o.load_vector()
        u_ex = _exact(X.reshape(-1, dim), cfg["center"], dim)
    assert abs(A - A.T).max() <= 1e-13 * abs(A).max()
    u = spla.spsolve(A.tocsc(), b)
    assert np.max(np.abs(u - u_ex)) < tol * np.max(np.abs(u_ex))
    # the residual of the exact nodal solution is at the level of the quadrature error
    assert np.max(np.abs(A @ u_ex - b)) < 20 * tol * np.max(np.abs(b))
