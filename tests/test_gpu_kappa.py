"""kappa-gradient and the differentiable operator: against the oracle's gradient by its
definition (dk_K = r^T A(e_K) x) on small grids, and against central differences of
J = 1/2 ||A(kappa) x - b||^2 (quadratic in kappa and x, so exact up to rounding) on the 48^3
workload."""
import numpy as np
import pytest

import workloads
from oracle import forms, mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _op(cfg, kappa):
    from paper_2404_07911_gb300 import UnfittedOperator

    return UnfittedOperator(cfg, device=0, kappa=kappa)


@pytest.mark.parametrize("cfg", [workloads.cfg_kappa(N=6), workloads.small(p=2, N=8),
                                 workloads.small(p=2, N=10, dim=2),
                                 dict(workloads.small(p=3, N=6), gp_kind="volume", gp_tau=0.7),
                                 workloads.plane(p=2, N=5, dim=3),
                                 workloads.spheres_random(p=2, N=8, n=8, R=0.22, seed=5)],
                         ids=["3d_q3_6_check_grid", "3d_q2_8", "2d_q2_10", "3d_q3_6_volume_gp",
                              "3d_plane_q2_5", "3d_random_spheres_q2_8"])
def test_kappa_gradient_matches_oracle(cfg):
    o = forms.Oracle(mesh.problem_from_dict(cfg))
    kappa = workloads.kappa_vector(o.mesh.n_active, seed=4)
    o = forms.Oracle(mesh.problem_from_dict(cfg, kappa))
    x, r = workloads.x_and_b(o.mesh.n_dofs, seed=5)
    ref = o.kappa_gradient(x, r)
    op = _op(cfg, kappa)
    dk = op.kappa_gradient(torch.from_numpy(r).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.max(np.abs(dk - ref)) <= 1e-12 * np.max(np.abs(ref))
    # the coefficient does not enter the gradient (A is linear in kappa)
    op.set_kappa(np.ones(o.mesh.n_active))
    dk1 = op.kappa_gradient(torch.from_numpy(r).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.max(np.abs(dk1 - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_autograd_matches_central_differences():
    from paper_2404_07911_gb300.autograd import unfitted_poisson

    cfg = workloads.cfg_kappa(N=48)
    from paper_2404_07911_gb300 import UnfittedOperator

    op0 = UnfittedOperator(cfg, device=-1)
    n_act, n = op0.info["n_active"], op0.info["n_dofs"]
    op0.close()
    kappa0 = torch.from_numpy(workloads.kappa_vector(n_act, seed=4)).cuda()
    xh, bh = workloads.x_and_b(n, seed=5)
    x0 = torch.from_numpy(xh).cuda()
    b = torch.from_numpy(bh).cuda()
    op = _op(cfg, None)

    def J(x, kappa):
        y = unfitted_poisson(x, kappa, op)
        return 0.5 * torch.sum((y - b) ** 2)

    x = x0.clone().requires_grad_(True)
    kappa = kappa0.clone().requires_grad_(True)
    loss = J(x, kappa)
    loss.backward()
    gk, gx = kappa.grad.clone(), x.grad.clone()
    rng = np.random.default_rng(7)
    eps = 1e-6
    with torch.no_grad():
        for _ in range(20):
            d = torch.from_numpy(rng.standard_normal(n_act)).cuda()
            fd = (J(x0, kappa0 + eps * d) - J(x0, kappa0 - eps * d)).item() / (2 * eps)
            assert abs(fd - torch.dot(gk, d).item()) <= 1e-6 * abs(fd)
        for _ in range(3):
            d = torch.from_numpy(rng.standard_normal(n)).cuda()
            fd = (J(x0 + eps * d, kappa0) - J(x0 - eps * d, kappa0)).item() / (2 * eps)
            assert abs(fd - torch.dot(gx, d).item()) <= 1e-6 * abs(fd)
