"""Pins of the oracle's classification and numbering (CPU).

The paper prints four DoF counts of its single-sphere benchmark (unit ball at the origin,
background [-1.035, 1.035]^3 refined from 12^3 cells); the exact box-distance classification and
the DG / CG numbering must reproduce all four.
"""
import json
import os

import numpy as np
import pytest

from oracle import mesh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_dof_counts.json")


def _sphere_problem(p, N, dim=3):
    return mesh.Problem(dim, p, (N,) * dim, (-1.035,) * dim, (1.035,) * dim, (0.0,) * dim, 1.0,
                        p + 1, 1.0, 1.0, p, 0.5)


def _cg_dof_count(m, p):
    """Unique lattice nodes of the active cells of a continuous Q_p space."""
    d = m.prob.dim
    shape = tuple(p * N + 1 for N in m.prob.n_cells[::-1])
    mark = np.zeros(shape, dtype=bool)
    base = [m.active_idx[:, a] * p for a in range(d)]
    for off in np.ndindex(*(p + 1,) * d):
        idx = tuple(base[a] + off[a] for a in range(d))
        mark[idx[::-1]] = True
    return int(mark.sum())


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"],
                         ids=lambda c: f"{c['disc']}_p{c['degree']}_{c['cells_per_dir']}")
def test_paper_dof_counts(case):
    p = case["degree"]
    m = mesh.Mesh(_sphere_problem(p, case["cells_per_dir"]))
    if case["disc"] == "DG":
        assert m.n_active * (p + 1) ** 3 == case["dofs"]
    else:
        assert _cg_dof_count(m, p) == case["dofs"]


def test_classification_against_sampling():
    """Brute force: dense point sampling of random boxes never contradicts the classification."""
    rng = np.random.default_rng(3)
    c = np.array([0.1, -0.2, 0.05])
    R = 0.7
    grid = np.stack(np.meshgrid(*[np.linspace(0, 1, 9)] * 3, indexing="ij"), -1).reshape(-1, 3)
    for _ in range(400):
        lo = rng.uniform(-1, 1, 3)
        hi = lo + rng.uniform(0.01, 0.4, 3)
        t = mesh.classify_box(c, R, lo, hi)
        r = np.linalg.norm(lo + grid * (hi - lo) - c, axis=1)
        if t == mesh.INSIDE:
            assert np.all(r <= R + 1e-15)
        elif t == mesh.OUTSIDE:
            assert np.all(r >= R - 1e-15)
        else:
            # a cut box has points on both sides (sampling may miss thin slivers: check the
            # exact nearest / farthest points instead)
            near = np.clip(c, lo, hi)
            far = np.where(np.abs(lo - c) > np.abs(hi - c), lo, hi)
            assert np.linalg.norm(near - c) < R < np.linalg.norm(far - c)


def test_numbering_and_faces_small():
    prob = mesh.Problem(3, 2, (6, 5, 7), (-1.2, -1.0, -1.4), (1.2, 1.0, 1.4), (0.01, 0.02, 0.03),
                        1.0, 3, 1, 1, 2, 0.5)
    m = mesh.Mesh(prob)
    act = m.active
    # lexicographic, x fastest
    keys = [a[2] * 35 + a[1] * 6 + a[0] for a in act]
    assert keys == sorted(keys)
    for e in range(m.n_active):
        for axis in range(3):
            for side in range(2):
                nb = m.neighbor(e, axis, side)
                if nb >= 0:
                    assert m.neighbor(nb, axis, 1 - side) == e
        if m.active_type[e] == mesh.INSIDE:
            # an inside cell has all 2d neighbours active and all its faces full
            for axis in range(3):
                for side in range(2):
                    nb = m.neighbor(e, axis, side)
                    assert nb >= 0
                    em = e if side == 1 else nb
                    assert m.face_type(em, axis) == mesh.FACE_FULL


def test_benchmark_config_counts():
    """Regression of the cell counts of the 3D Q3 64^3 ball workload."""
    prob = mesh.Problem(3, 3, (64,) * 3, (-1.21,) * 3, (1.21,) * 3, (0.01, 0.02, 0.03), 1.0, 4,
                        40.0, 160.0, 3, 0.5)
    m = mesh.Mesh(prob)
    assert m.n_active == 84218
    assert int(np.sum(m.active_type == mesh.CUT)) == 13180
    assert m.n_dofs == 5389952
