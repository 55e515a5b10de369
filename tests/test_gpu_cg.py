"""Continuous Q_p operator on the GPU: A = P^T A_loc P against the oracle's assembly, its kappa
gradient, and the two solvers (FP64 PCG; FP32 PCG inside FP64 iterative refinement) against a
direct solve of the oracle's matrix and against the exact quadratic solution of -Lap u = 1."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads
from oracle import forms, mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "3d_q2_6": workloads.small(p=2, N=6),
    "3d_q4_5": workloads.small(p=4, N=5),
    "2d_q3_10": workloads.small(p=3, N=10, dim=2),
    "3d_plane_q3_4": workloads.plane(p=3, N=4, dim=3),
    "3d_q3_5_volume_gp": dict(workloads.small(p=3, N=5), gp_kind="volume", gp_tau=0.7),
    "3d_spheres_q2_8": workloads.spheres(p=2, N=8, m=2, R=0.2),
    "3d_random_spheres_q2_8": workloads.spheres_random(p=2, N=8, n=8, R=0.22, seed=5,
                                                       discretization="cg"),
}


def _cg(cfg):
    return dict(cfg, discretization="cg")


def _op(cfg, kappa=None):
    from paper_2404_07911_gb300 import UnfittedOperator

    return UnfittedOperator(_cg(cfg), device=0, kappa=kappa)


def _apply(op, x, dtype=torch.float64, adjoint=False):
    xt = torch.from_numpy(np.asarray(x)).to(device="cuda", dtype=dtype)
    y = op.vmult_adjoint(xt) if adjoint else op.vmult(xt)
    return y.double().cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("key", list(CASES))
def test_cg_operator_matches_oracle(key):
    cfg = _cg(CASES[key])
    o = forms.Oracle(mesh.problem_from_dict(cfg), "cg")
    A = o.cg_matrix()
    op = _op(CASES[key])
    assert op.n_dofs == A.shape[0]
    x = workloads.uniform_vector(op.n_dofs, 3)
    assert _rel(_apply(op, x), A @ x) <= 1e-12
    assert _rel(_apply(op, x, adjoint=True), A.T @ x) <= 1e-12
    x32 = x.astype(np.float32).astype(np.float64)
    assert _rel(_apply(op, x32, torch.float32), A @ x32) <= 1e-5


def test_cg_kappa_operator_and_gradient():
    cfg = _cg(CASES["3d_q2_6"])
    o0 = forms.Oracle(mesh.problem_from_dict(cfg), "cg")
    kappa = workloads.kappa_vector(o0.mesh.n_active, seed=4)
    o = forms.Oracle(mesh.problem_from_dict(cfg, kappa), "cg")
    op = _op(CASES["3d_q2_6"], kappa)
    x, r = workloads.x_and_b(op.n_dofs, seed=5)
    assert _rel(_apply(op, x), o.cg_matrix() @ x) <= 1e-12
    P = o.cg_prolongation()
    ref = o.kappa_gradient(P @ x, P @ r)
    dk = op.kappa_gradient(torch.from_numpy(r).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    assert _rel(dk, ref) <= 1e-12


def _node_coords(o):
    from oracle import basis

    z = basis.gauss_lobatto_nodes(o.n)
    n_cg, l2g = o.cg_numbering()
    X = np.zeros((n_cg, o.prob.dim))
    for e in range(o.mesh.n_active):
        lo, _ = mesh.cell_box(o.prob, o.mesh.index_of(e))
        for a in range(o.prob.dim):
            X[l2g[e], a] = lo[a] + o.prob.h * z[o.lidx[:, a]]
    return X


@pytest.mark.parametrize("mode", ["ir", "fp64", "ir_split"])
@pytest.mark.parametrize("key,q,tol_exact", [("2d_q3_10", 10, 1e-9), ("3d_q2_6", 8, 1e-6)])
def test_cg_solvers(mode, key, q, tol_exact):
    cfg = _cg(dict(CASES[key], quad_order=q))
    o = forms.Oracle(mesh.problem_from_dict(cfg), "cg")
    A = o.cg_matrix()
    b = o.cg_load_vector()
    from paper_2404_07911_gb300 import UnfittedOperator

    op = UnfittedOperator(cfg, device=0)
    _, rhs, _ = op.export_cg()
    assert np.max(np.abs(rhs - b)) <= 1e-13 * np.max(np.abs(b))
    bt = torch.from_numpy(rhs).cuda()
    x, stats = op.solve(bt, mode=mode, tol=1e-10)
    assert stats["converged"] == 1 and stats["rel_residual"] <= 1e-10
    u = x.cpu().numpy()
    # residual checked with the oracle's matrix
    assert np.linalg.norm(b - A @ u) <= 2e-10 * np.linalg.norm(b)
    u_ref = spla.spsolve(A.tocsc(), b)
    assert np.max(np.abs(u - u_ref)) <= 1e-7 * np.max(np.abs(u_ref))
    X = _node_coords(o)
    dim = cfg["dim"]
    u_ex = (1.0 - np.sum((X - np.asarray(cfg["center"][:dim])) ** 2, axis=1)) / (2 * dim)
    assert np.max(np.abs(u - u_ex)) <= tol_exact * np.max(np.abs(u_ex))
    if mode != "fp64":
        assert stats["outer"] >= 2  # the FP32 inner solves alone cannot reach 1e-10


def test_split_operator_rows():
    """The split FP32 operator (inner operator of mode ir_split): on a discontinuous problem the
    rows of cut cells and of cells with a ghost-penalty face (the active face neighbours of cut
    cells) equal the FP64 operator applied to the FP32 input, rounded once, bit for bit, and every
    other row equals the FP32 operator; on a continuous problem (node sums in FP32) the result
    stays within FP32 accuracy of the FP64 operator."""
    from paper_2404_07911_gb300 import UnfittedOperator

    cfg = workloads.small(p=2, N=6)
    op = UnfittedOperator(cfg, device=0)
    nd = op.info["dofs_per_cell"]
    m = mesh.Mesh(mesh.problem_from_dict(cfg))
    o = forms.Oracle(mesh.problem_from_dict(cfg))
    cut = set(int(e) for e in np.nonzero(m.active_type == mesh.CUT)[0])
    split = set(cut)
    for e in cut:
        split.update(nb for _, _, nb in o.faces_of(e))
    split = np.array(sorted(split))
    other = np.setdiff1d(np.arange(m.n_active), split)
    assert len(split) > 0 and len(other) > 0
    x32 = torch.from_numpy(workloads.uniform_vector(op.n_dofs, 3).astype(np.float32)).cuda()
    ys = op.vmult_split(x32).cpu().numpy().reshape(-1, nd)
    y32 = op.vmult(x32).cpu().numpy().reshape(-1, nd)
    y64 = op.vmult(x32.double()).cpu().numpy().reshape(-1, nd)
    assert np.array_equal(ys[split], y64[split].astype(np.float32))
    assert np.array_equal(ys[other], y32[other])
    # only the cut cells below a volume fraction of 0.25, with their face neighbours
    h3 = op.info["h"] ** 3
    cut_sorted = sorted(cut)
    frac = np.array([op.export_cut_cell_rule(c, 0)[1].sum() / h3 for c in range(len(cut_sorted))])
    tiny = [cut_sorted[c] for c in np.nonzero(frac < 0.25)[0]]
    sub = set(tiny)
    for e in tiny:
        sub.update(nb for _, _, nb in o.faces_of(e))
    sub = np.array(sorted(sub))
    assert 0 < len(sub) < len(split)
    op.set_split_fraction(0.25)
    ys = op.vmult_split(x32).cpu().numpy().reshape(-1, nd)
    rest = np.setdiff1d(np.arange(m.n_active), sub)
    assert np.array_equal(ys[sub], y64[sub].astype(np.float32))
    assert np.array_equal(ys[rest], y32[rest])
    op.close()

    cfg = _cg(workloads.small(p=2, N=6))
    op = UnfittedOperator(cfg, device=0)
    x32 = torch.from_numpy(workloads.uniform_vector(op.n_dofs, 4).astype(np.float32)).cuda()
    ys = op.vmult_split(x32).double().cpu().numpy()
    y32 = op.vmult(x32).double().cpu().numpy()
    y64 = op.vmult(x32.double()).cpu().numpy()
    assert np.max(np.abs(ys - y64)) <= 1e-5 * np.max(np.abs(y64))
    assert not np.array_equal(ys, y32)
    op.close()
