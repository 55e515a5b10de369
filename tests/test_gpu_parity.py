"""Parity of the CUDA operator (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative infinity norm over the compared rows):
  FP64  1e-12   (the accuracy target of the method's FP64 evaluation)
  FP32  1e-5    against the oracle applied to the FP32-rounded input (FP32 rounding of x, the
                geometry data and every partial sum; the penalty terms make ||A|| ~ 1e4 / h)
"""
import functools

import numpy as np
import pytest

import workloads
from oracle import forms, mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@functools.lru_cache(maxsize=None)
def _oracle(key):
    cfg = SMALL[key]
    o = forms.Oracle(mesh.problem_from_dict(cfg))
    return o, o.assemble()


def _gpu_op(cfg, kappa=None):
    from paper_2404_07911_gb300 import UnfittedOperator

    return UnfittedOperator(cfg, device=0, kappa=kappa)


def _apply(op, x, dtype=torch.float64, adjoint=False):
    xt = torch.from_numpy(np.asarray(x)).to(device="cuda", dtype=dtype)
    y = op.vmult_adjoint(xt) if adjoint else op.vmult(xt)
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


SMALL = {
    "2d_q1_16x16_disc": workloads.cfg_2d_q1(),
    "2d_q2_10": workloads.small(p=2, N=10, dim=2),
    "2d_q5_8": workloads.small(p=5, N=8, dim=2),
    "2d_q8_6": workloads.small(p=8, N=6, dim=2),
    "3d_q1_10": workloads.small(p=1, N=10),
    "3d_q2_8": workloads.small(p=2, N=8),
    "3d_q3_8": workloads.small(p=3, N=8),
    "3d_q4_6": workloads.small(p=4, N=6),
    "3d_q3_center_on_grid": workloads.small(p=3, N=6, center=(0.0, 0.0, 0.0)),
    "3d_q6_4": workloads.small(p=6, N=4),
    # every structured-kernel block shape: n = 6, 7 take 4 and 3 cells per CTA (160 threads),
    # n = 9 one cell (FP32: 3 cells, 256 threads); 2D n = 6, 7 take 16 and 9 cells
    "3d_q5_4": workloads.small(p=5, N=4),
    "3d_q7_3": workloads.small(p=7, N=3),
    "3d_q8_3": workloads.small(p=8, N=3),
    "2d_q6_8": workloads.small(p=6, N=8, dim=2),
    # volume-based ghost penalty on stable-neighbour patches
    "3d_q3_6_volume_gp": dict(workloads.small(p=3, N=6), gp_kind="volume", gp_tau=0.7),
    "2d_q2_10_volume_gp": dict(workloads.small(p=2, N=10, dim=2), gp_kind="volume"),
    # unions of separated balls
    "3d_spheres_q2_10": workloads.spheres(p=2, N=10, m=2, R=0.2),
    "2d_spheres_q3_16": workloads.spheres(p=3, N=16, m=3, R=0.12, dim=2),
    # unions of intersecting balls (cells met by two and three spheres, covered cut cells)
    "3d_random_spheres_q2_10": workloads.spheres_random(p=2, N=10, n=8, R=0.22, seed=5),
    "3d_random_spheres_q1_14": workloads.spheres_random(p=1, N=14, n=14, R=(0.08, 0.22), seed=6),
    "2d_random_spheres_q3_16": workloads.spheres_random(p=3, N=16, n=9, R=0.19, seed=2, dim=2),
    # half-spaces below tilted planes (the plane benchmark's geometry)
    "2d_plane_q2_7": workloads.plane(p=2, N=7, dim=2),
    "3d_plane_q1_6": workloads.plane(p=1, N=6, dim=3),
    "3d_plane_q3_5_steep": workloads.plane(p=3, N=5, dim=3, normal=(0.2, -0.3, 0.9), offset_cells=1.55),
    "3d_plane_q2_4_one_layer": workloads.plane(p=2, N=4, dim=3, layers=1, offset_cells=0.25,
                                               normal=(-0.075, -0.05, 1.0)),
}


@pytest.mark.parametrize("key", list(SMALL))
def test_parity_fp64_fp32_adjoint(key):
    cfg = SMALL[key]
    o, A = _oracle(key)
    op = _gpu_op(cfg)
    assert op.n_dofs == A.shape[0]
    x = workloads.uniform_vector(op.n_dofs, cfg["seed"])
    y_ref = A @ x
    y64 = _apply(op, x)
    assert _rel(y64, y_ref) <= TOL64
    # adjoint: A^T x from the assembled matrix
    ya = _apply(op, x, adjoint=True)
    assert _rel(ya, A.T @ x) <= TOL64
    # FP32 against the oracle on the FP32-rounded input
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = _apply(op, x32, dtype=torch.float32)
    assert _rel(y32, A @ x32) <= TOL32


def test_parity_kappa_lognormal():
    cfg = workloads.small(p=3, N=6)
    o0 = forms.Oracle(mesh.problem_from_dict(cfg))
    kappa = workloads.kappa_vector(o0.mesh.n_active, seed=4)
    o = forms.Oracle(mesh.problem_from_dict(cfg, kappa))
    A = o.assemble()
    op = _gpu_op(cfg, kappa=kappa)
    x = workloads.uniform_vector(op.n_dofs, 5)
    assert _rel(_apply(op, x), A @ x) <= TOL64
    assert _rel(_apply(op, x, adjoint=True), A.T @ x) <= TOL64
    # set_kappa replaces the coefficient in place
    kappa2 = workloads.kappa_vector(o0.mesh.n_active, seed=6)
    op.set_kappa(kappa2)
    A2 = forms.Oracle(mesh.problem_from_dict(cfg, kappa2)).assemble()
    assert _rel(_apply(op, x), A2 @ x) <= TOL64


def test_uniform_kappa_scales_the_operator():
    """kappa = 2.5 everywhere: A(kappa) = 2.5 A(1) (the uniform-coefficient path)."""
    cfg = workloads.small(p=3, N=6)
    o = forms.Oracle(mesh.problem_from_dict(cfg))
    A = o.assemble()
    op = _gpu_op(cfg, kappa=np.full(o.mesh.n_active, 2.5))
    x = workloads.uniform_vector(op.n_dofs, 12)
    assert _rel(_apply(op, x), 2.5 * (A @ x)) <= TOL64
    assert _rel(_apply(op, x, adjoint=True), 2.5 * (A.T @ x)) <= TOL64


def test_all_cells_inside_no_cut_cells():
    cfg = workloads.small(p=3, N=5)
    cfg.update(radius=50.0)
    o = forms.Oracle(mesh.problem_from_dict(cfg))
    A = o.assemble()
    op = _gpu_op(cfg)
    assert op.info["n_cut"] == 0
    x = workloads.uniform_vector(op.n_dofs, 3)
    assert _rel(_apply(op, x), A @ x) <= TOL64


def test_single_cut_cell_with_subdivision():
    """A sphere inside one background cell: one active (cut) cell, no faces, subdivided rule."""
    cfg = workloads.small(p=2, N=4)
    cfg.update(center=(0.31, 0.29, 0.33), radius=0.1, lo=(-1.0,) * 3, hi=(1.0,) * 3)
    o = forms.Oracle(mesh.problem_from_dict(cfg))
    A = o.assemble()
    op = _gpu_op(cfg)
    assert op.info["n_active"] == 1 and op.info["n_faces"] == 0
    x = workloads.uniform_vector(op.n_dofs, 3)
    assert _rel(_apply(op, x), A @ x) <= TOL64


def test_ghost_penalty_off():
    cfg = workloads.small(p=2, N=6)
    cfg.update(gp_max_order=0)
    o = forms.Oracle(mesh.problem_from_dict(cfg))
    A = o.assemble()
    op = _gpu_op(cfg)
    x = workloads.uniform_vector(op.n_dofs, 8)
    assert _rel(_apply(op, x), A @ x) <= TOL64


# ------------------------------------------------------------------ full-size workload
@pytest.fixture(scope="module")
def full():
    cfg = workloads.cfg_3d_q3()
    op = _gpu_op(cfg)
    o = forms.Oracle(mesh.problem_from_dict(cfg))
    x = workloads.uniform_vector(op.n_dofs, cfg["seed"])
    return cfg, op, o, x


def _sample_cells(o, count=36, seed=0):
    m = o.mesh
    rng = np.random.default_rng(seed)
    cut = np.nonzero(m.active_type == mesh.CUT)[0]
    inside = np.nonzero(m.active_type == mesh.INSIDE)[0]
    # inside cells next to cut cells carry ghost-penalty faces
    gp_inside = [e for e in inside[rng.permutation(len(inside))[:2000]]
                 if any(m.active_type[nb] == mesh.CUT for _, _, nb in o.faces_of(e))]
    cells = list(rng.choice(cut, count // 2, replace=False))
    cells += list(rng.choice(inside, count // 4, replace=False))
    cells += gp_inside[: count // 4]
    cells += [0, m.n_active - 1]
    return sorted(set(int(c) for c in cells))


def test_full_size_sampled_rows_fp64_fp32(full):
    cfg, op, o, x = full
    nd = op.info["dofs_per_cell"]
    cells = _sample_cells(o)
    y64 = _apply(op, x).reshape(-1, nd)[cells]
    ref = o.apply_rows(x, cells)
    assert _rel(y64, ref) <= TOL64
    ya = _apply(op, x, adjoint=True).reshape(-1, nd)[cells]
    assert _rel(ya, ref) <= TOL64
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = _apply(op, x32, dtype=torch.float32).reshape(-1, nd)[cells]
    assert _rel(y32, o.apply_rows(x32, cells)) <= TOL32


def test_full_size_symmetry_and_determinism(full):
    cfg, op, o, x = full
    v = workloads.uniform_vector(op.n_dofs, 99)
    xt = torch.from_numpy(x).cuda()
    vt = torch.from_numpy(v).cuda()
    Ax = op.vmult(xt)
    Av = op.vmult(vt)
    lhs = float(torch.dot(vt, Ax))
    rhs = float(torch.dot(xt, Av))
    assert abs(lhs - rhs) <= 1e-12 * (torch.abs(vt) @ torch.abs(Ax)).item()
    Ax2 = op.vmult(xt)
    assert torch.equal(Ax, Ax2)


def test_host_buffer_path_matches_device(full):
    cfg, op, o, x = full
    y_host = op.vmult_host(x)
    y_dev = _apply(op, x)
    assert np.array_equal(y_host, y_dev)
    y_host32 = op.vmult_host(x.astype(np.float32))
    y_dev32 = _apply(op, x, dtype=torch.float32)
    assert np.array_equal(y_host32.astype(np.float64), y_dev32)


@pytest.mark.parametrize("cfg", [workloads.small(p=2, N=128, dim=2), workloads.small(p=1, N=32)],
                         ids=["2d_q2_128", "3d_q1_32"])
def test_host_pipeline_matches_device(cfg):
    """Operators with at least 8192 cells take the pipelined host path (parts of consecutive
    cells, copies overlapping the kernels): bit for bit the device path, vmult and adjoint, FP64
    and FP32, with a log-normal coefficient."""
    from paper_2404_07911_gb300 import UnfittedOperator
    from paper_2404_07911_gb300.binding import UF_FP32, UF_FP64

    n_active = mesh.Mesh(mesh.problem_from_dict(cfg)).n_active
    assert n_active >= 8192
    op = UnfittedOperator(cfg, device=0, kappa=workloads.kappa_vector(n_active, seed=4))
    x = workloads.uniform_vector(op.n_dofs, 3)
    for dt, prec in ((np.float64, UF_FP64), (np.float32, UF_FP32)):
        xh = x.astype(dt)
        for adjoint in (False, True):
            yh = np.empty_like(xh)
            op.vmult_host_ptr(prec, yh.ctypes.data, xh.ctypes.data, 0, adjoint=adjoint)
            xt = torch.from_numpy(xh).cuda()
            yd = (op.vmult_adjoint(xt) if adjoint else op.vmult(xt)).cpu().numpy()
            assert np.array_equal(yh, yd), (dt, adjoint)
    # asynchronous calls on pinned buffers: four chained products (both staging sets twice)
    # before one synchronisation, each equal to its device result
    s = torch.cuda.Stream()
    xs = [torch.from_numpy(workloads.uniform_vector(op.n_dofs, 10 + i)).pin_memory() for i in range(4)]
    ys = [torch.empty_like(v).pin_memory() for v in xs]
    for i in range(4):
        op.vmult_host_ptr(UF_FP64, ys[i].data_ptr(), xs[i].data_ptr(), s.cuda_stream,
                          adjoint=(i % 2 == 1), wait=False)
    op.host_wait(s.cuda_stream)
    for i in range(4):
        xt = xs[i].cuda()
        yd = (op.vmult_adjoint(xt) if i % 2 == 1 else op.vmult(xt)).cpu()
        assert torch.equal(ys[i], yd), i
    op.close()


def test_parity_volume_gp_with_kappa():
    """Volume ghost penalty with a log-normal coefficient: {kappa} on the patches, the general
    per-cell path of the structured kernel, vmult and adjoint."""
    cfg = dict(workloads.small(p=2, N=7), gp_kind="volume", gp_tau=0.7)
    o0 = forms.Oracle(mesh.problem_from_dict(cfg))
    kappa = workloads.kappa_vector(o0.mesh.n_active, seed=4)
    A = forms.Oracle(mesh.problem_from_dict(cfg, kappa)).assemble()
    op = _gpu_op(cfg, kappa=kappa)
    x = workloads.uniform_vector(op.n_dofs, 5)
    assert _rel(_apply(op, x), A @ x) <= TOL64
    assert _rel(_apply(op, x, adjoint=True), A.T @ x) <= TOL64
