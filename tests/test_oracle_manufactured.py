"""Pins of the manufactured solution and of the oracle's load vector and L2 error (CPU).

  * -Lap u = f by central differences and u = 0 on the sphere (independent of the formula for f);
  * the discrete solution of A u_h = b converges to u at the optimal rate p + 1 in L2 for the
    continuous and the discontinuous space (2D disc and 3D ball, two grid levels): a wrong load
    vector, Nitsche sign or L2 error stalls the rate.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads
from oracle import forms, manufactured as mf, mesh

OMEGA = 2.0 * math.pi


@pytest.mark.parametrize("d", [2, 3])
def test_manufactured_pair(d):
    rng = np.random.default_rng(0)
    X = rng.uniform(-0.7, 0.7, (30, d))
    c = np.zeros(d)
    h = 1e-4
    lap = np.zeros(len(X))
    for a in range(d):
        e = np.zeros(d)
        e[a] = h
        lap += (mf.solution(X + e, c, 1.0, OMEGA) - 2 * mf.solution(X, c, 1.0, OMEGA)
                + mf.solution(X - e, c, 1.0, OMEGA)) / h ** 2
    f = mf.rhs(X, c, 1.0, OMEGA)
    assert np.max(np.abs(-lap - f)) < 1e-6 * np.max(np.abs(f))
    # zero on the sphere, finite at the centre
    Y = rng.normal(size=(10, d))
    Y /= np.linalg.norm(Y, axis=1)[:, None]
    assert np.max(np.abs(mf.solution(Y, c, 1.0, OMEGA))) < 1e-14
    assert np.isfinite(mf.rhs(np.zeros((1, d)), c, 1.0, OMEGA)).all()


def _error(cfg, disc):
    o = forms.Oracle(mesh.problem_from_dict(cfg), disc)
    c = np.asarray(cfg["center"][:cfg["dim"]])

    def f(X):
        return mf.rhs(X, c, cfg["radius"], OMEGA)

    def u(X):
        return mf.solution(X, c, cfg["radius"], OMEGA)

    if disc == "cg":
        A = o.cg_matrix()
        b = o.cg_prolongation().T @ o.load_vector(f)
    else:
        A = o.assemble()
        b = o.load_vector(f)
    uh = spla.spsolve(A.tocsc(), b)
    err, nrm = o.l2_error(uh, u)
    return err / nrm


@pytest.mark.parametrize("disc", ["cg", "dg"])
@pytest.mark.parametrize("dim,p,Ns", [(2, 1, (16, 32)), (2, 2, (8, 16)), (3, 1, (6, 12))])
def test_optimal_l2_rate(disc, dim, p, Ns):
    errs = [_error(workloads.accuracy(p, N, dim=dim), disc) for N in Ns]
    rate = math.log(errs[0] / errs[1], 2)
    assert rate > p + 1 - 0.35, (errs, rate)
