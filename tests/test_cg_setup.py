"""Host setup of the continuous Q_p operator against the oracle (CPU): global numbering, load
vector (f = 1) and the diagonal of A = P^T A_loc P."""
import numpy as np
import pytest

import workloads
from oracle import forms, mesh
from paper_2404_07911_gb300.binding import UnfittedOperator


@pytest.mark.parametrize("cfg", [workloads.small(p=2, N=6), workloads.small(p=4, N=5),
                                 workloads.small(p=3, N=10, dim=2),
                                 dict(workloads.small(p=3, N=6), gp_kind="volume", gp_tau=0.7),
                                 dict(workloads.small(p=2, N=10, dim=2), gp_kind="volume", gp_tau=1.3)],
                         ids=["3d_q2", "3d_q4", "2d_q3", "3d_q3_volume_gp", "2d_q2_volume_gp"])
def test_cg_numbering_rhs_diag_match_oracle(cfg):
    cfg = dict(cfg, discretization="cg")
    op = UnfittedOperator(cfg, device=-1)
    o = forms.Oracle(mesh.problem_from_dict(cfg), "cg")
    n_cg, l2g_ref = o.cg_numbering()
    l2g, rhs, diag = op.export_cg()
    assert op.n_dofs == n_cg
    assert np.array_equal(l2g, l2g_ref)
    b_ref = o.cg_load_vector()
    assert np.max(np.abs(rhs - b_ref)) <= 1e-13 * np.max(np.abs(b_ref))
    A = o.cg_matrix()
    d_ref = A.diagonal()
    assert np.max(np.abs(diag - d_ref)) <= 1e-12 * np.max(np.abs(d_ref))


def test_cg_with_kappa():
    cfg = dict(workloads.small(p=2, N=6), discretization="cg")
    o0 = forms.Oracle(mesh.problem_from_dict(cfg), "cg")
    kappa = workloads.kappa_vector(o0.mesh.n_active, seed=4)
    op = UnfittedOperator(cfg, device=-1, kappa=kappa)
    d_ref = forms.Oracle(mesh.problem_from_dict(cfg, kappa), "cg").cg_matrix().diagonal()
    _, _, diag = op.export_cg()
    assert np.max(np.abs(diag - d_ref)) <= 1e-12 * np.max(np.abs(d_ref))


@pytest.mark.parametrize("cfg", [dict(workloads.small(p=3, N=6), gp_kind="volume"),
                                 dict(workloads.plane(p=2, N=5, dim=3), gp_kind="volume")],
                         ids=["ball", "plane"])
def test_volume_gp_patch_count(cfg):
    """The library's stable-neighbour patches of the volume ghost penalty against the oracle's."""
    op = UnfittedOperator(cfg, device=-1)
    o = forms.Oracle(mesh.problem_from_dict(cfg))
    assert op.info["n_faces_gp"] == len(o.volume_gp_patches())
    op.close()
