"""Pin of the oracle's kappa-gradient: J(kappa) = 1/2 ||A(kappa) x - b||^2 is quadratic in kappa,
so central differences of J (with matrices assembled independently for each kappa) equal the
directional derivative g . d up to rounding, with g_K = r^T A_K x, r = A(kappa) x - b."""
import numpy as np

import workloads
from oracle import forms, mesh


def test_kappa_gradient_matches_central_differences():
    cfg = workloads.small(p=2, N=4)
    o = forms.Oracle(mesh.problem_from_dict(cfg))
    n_act = o.mesh.n_active
    k0 = workloads.kappa_vector(n_act, seed=4)
    x, b = workloads.x_and_b(o.mesh.n_dofs, seed=5)

    def J(kappa):
        A = forms.Oracle(mesh.problem_from_dict(cfg, kappa)).assemble()
        res = A @ x - b
        return 0.5 * res @ res

    ok = forms.Oracle(mesh.problem_from_dict(cfg, k0))
    r = ok.assemble() @ x - b
    g = ok.kappa_gradient(x, r)
    rng = np.random.default_rng(0)
    eps = 1e-3
    for _ in range(3):
        d = rng.standard_normal(n_act)
        fd = (J(k0 + eps * d) - J(k0 - eps * d)) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-9 * abs(fd)


def test_kappa_gradient_of_linear_functional():
    """With r fixed, r^T A(kappa) x is linear in kappa: sum_K kappa_K g_K reproduces it."""
    cfg = workloads.small(p=1, N=5)
    o = forms.Oracle(mesh.problem_from_dict(cfg))
    k = workloads.kappa_vector(o.mesh.n_active, seed=1)
    x = workloads.uniform_vector(o.mesh.n_dofs, 2)
    r = workloads.uniform_vector(o.mesh.n_dofs, 3)
    A = forms.Oracle(mesh.problem_from_dict(cfg, k)).assemble()
    g = o.kappa_gradient(x, r)
    assert abs(k @ g - r @ (A @ x)) <= 1e-12 * abs(r @ (A @ x))
