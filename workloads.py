"""Seeded synthetic workloads: problem presets and input vectors.

This module holds no arithmetic of the method.  It is the one place both sides of a parity test
draw from: the CPU oracle (``oracle/``) and the CUDA library (``paper_2404_07911_gb300``) receive
the same problem description and the same seeded vectors from here.

Problem presets follow the workloads of arXiv 2404.07911 (unit-radius ball embedded in a
Cartesian background grid, Sec. 4 and Sec. 5.1) with the sizes, penalties and seeds of the
benchmark configurations:

  * ``cfg_2d_q1``      2D, DG Q1, 16^2 background cells on [-1.21, 1.21]^2, disc |x-(0.03,0.02)| < 1,
                       quadrature order q = 2, SIPG 8/h, Nitsche 20/h, ghost penalty order 1,
                       gamma_1 = 0.5 h; x ~ U[-1, 1] seed 0.
  * ``cfg_3d_q3``      3D, DG Q3 (64 DoF/cell), 64^3 cells on [-1.21, 1.21]^3, ball
                       |x-(0.01,0.02,0.03)| < 1, q = 4, SIPG 2.5 (p+1)^2 / h, Nitsche 10 (p+1)^2 / h,
                       ghost penalty orders 1..3 with gamma_j = 0.5 h^(2j-1) / (j!)^2; x ~ U[-1, 1]
                       seed 1.
  * ``cfg_sweep(p)``   3D, DG Q_p, p = 1..8, same ball and penalties, background cells per direction
                       chosen so that the DoF count is about 2e7; q = p + 1; seed 2.
  * ``cfg_kappa``      3D, DG Q3 on a 48^3 background, same ball and penalties; per-cell
                       kappa ~ LogNormal(0, 0.5) seed 4; x then b ~ U[-1, 1] seed 5.
  * ``cfg_cg_q4``      3D continuous Q4 on an 80^3 background, ball of radius 1 at the origin,
                       Nitsche u = 0, ghost penalty orders 1..4, f = 1 (the solve workload).
  * ``small(...)``     reduced grids of the same geometry for tests the oracle finishes in seconds.
  * ``plane(...)``     half-space below a slightly tilted plane in a box of cubes (the paper's plane
                       benchmark, Sec. 5.2, positions the plane to set the ratio of cut cells);
                       ``cfg_plane(kind, ratio)`` sizes the box so that the cut layer is a fraction
                       ``ratio`` of the active cells.

Vectors are drawn with ``numpy.random.default_rng(seed)`` in DoF order (active cells
lexicographic with x fastest, local index i + n j + n^2 k).
"""
import numpy as np

SWEEP_N = {1: 202, 2: 134, 3: 100, 4: 80, 5: 66, 6: 56, 7: 49, 8: 43}


def _penalties(p):
    n = p + 1
    return dict(sipg_gamma=2.5 * n * n, nitsche_gamma=10.0 * n * n, gp_max_order=p, gp_gamma=0.5)


def cfg_2d_q1():
    return dict(name="2d_dg_q1_16x16_disc", dim=2, degree=1, n_cells=(16, 16, 1),
                lo=(-1.21, -1.21, 0.0), hi=(1.21, 1.21, 0.0), center=(0.03, 0.02, 0.0), radius=1.0,
                quad_order=2, sipg_gamma=8.0, nitsche_gamma=20.0, gp_max_order=1, gp_gamma=0.5,
                seed=0)


def cfg_3d(p=3, N=64, center=(0.01, 0.02, 0.03), name=None, seed=1, quad_order=None):
    return dict(name=name or f"3d_dg_q{p}_{N}^3_ball", dim=3, degree=p, n_cells=(N, N, N),
                lo=(-1.21, -1.21, -1.21), hi=(1.21, 1.21, 1.21), center=center, radius=1.0,
                quad_order=quad_order if quad_order is not None else 4 if p == 3 else p + 1,
                seed=seed, **_penalties(p))


def cfg_3d_q3():
    return cfg_3d(3, 64, name="3d_dg_q3_64^3_ball", seed=1)


def cfg_sweep(p):
    return cfg_3d(p, SWEEP_N[p], name=f"3d_dg_q{p}_{SWEEP_N[p]}^3_ball_sweep", seed=2,
                  quad_order=p + 1)


def cfg_kappa(N=48):
    return cfg_3d(3, N, name=f"3d_dg_q3_{N}^3_ball_kappa", seed=5)


def cfg_cg_q4(N=80):
    """Continuous Q4 solve: ball of radius 1 at the origin, 80^3 background cells on
    [-1.21, 1.21]^3, Nitsche u = 0 on the sphere (10 (p+1)^2 / h), face ghost penalty orders
    1..4, f = 1, quadrature order p + 1."""
    c = cfg_3d(4, N, center=(0.0, 0.0, 0.0), name=f"3d_cg_q4_{N}^3_ball_solve", seed=0, quad_order=5)
    c["discretization"] = "cg"
    return c


def small(p=3, N=8, dim=3, center=None, seed=7):
    """A reduced grid of the same geometry (tests)."""
    if dim == 2:
        c = cfg_2d_q1()
        c.update(name=f"2d_dg_q{p}_{N}^2", degree=p, n_cells=(N, N, 1), seed=seed)
        if p != 1:
            c.update(quad_order=p + 1, **_penalties(p))
        if center is not None:
            c["center"] = tuple(center) + (0.0,)
        return c
    return cfg_3d(p, N, center=center or (0.01, 0.02, 0.03), name=f"3d_dg_q{p}_{N}^3", seed=seed)


def uniform_vector(n, seed):
    """x ~ U[-1, 1], float64, length n."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


def kappa_vector(n_active, seed=4):
    """kappa ~ LogNormal(0, 0.5) per active cell."""
    return np.random.default_rng(seed).lognormal(0.0, 0.5, n_active)


def x_and_b(n, seed=5):
    """x then b ~ U[-1, 1] from one generator."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, n), rng.uniform(-1.0, 1.0, n)


def accuracy(p, N, dim=3):
    """Sphere accuracy benchmark (paper Sec. 4): unit ball at the origin in the background box
    [-1.035, 1.035]^d with N cells per direction, q = p + 1, penalties as for the ball workloads;
    the right-hand side and exact solution are the manufactured pair of that section."""
    pad = (0.0,) * (3 - dim)
    return dict(name=f"{dim}d_q{p}_{N}_accuracy", dim=dim, degree=p, n_cells=(N,) * dim + (1,) * (3 - dim),
                lo=(-1.035,) * dim + pad, hi=(1.035,) * dim + pad, center=(0.0, 0.0, 0.0), radius=1.0,
                quad_order=p + 1, seed=0, **_penalties(p))


PLANE_NORMAL = (-0.04, -0.03, 1.0)


def plane(p=2, N=5, dim=3, layers=None, offset_cells=None, discretization="dg", quad_order=None,
          seed=9, normal=None):
    """Half-space normal . x < offset in the box [0, 1]^(d-1) x [0, layers h], h = 1 / N: the
    plane is tilted by a few per cent against the last axis and crosses the box at about
    offset_cells cells above the bottom.  Penalties as for the ball workloads."""
    layers = N if layers is None else layers
    nrm = tuple((normal or PLANE_NORMAL)[3 - dim:]) if dim == 2 else tuple(normal or PLANE_NORMAL)
    h = 1.0 / N
    oc = (layers - 0.45) if offset_cells is None else offset_cells
    n_cells = (N,) * (dim - 1) + (layers,)
    lo = (0.0,) * dim
    hi = (1.0,) * (dim - 1) + (layers * h,)
    pad = (0.0,) * (3 - dim)
    c = dict(name=f"{dim}d_{discretization}_q{p}_plane_{N}x{layers}", dim=dim, degree=p,
             n_cells=n_cells + (1,) * (3 - dim), lo=lo + pad, hi=hi + pad, center=(0.0, 0.0, 0.0),
             radius=1.0, ls_kind="plane", normal=nrm + pad, offset=oc * h,
             quad_order=quad_order if quad_order is not None else p + 1, seed=seed,
             discretization=discretization, **_penalties(p))
    return c


def cfg_plane(discretization, p, ratio, n_dofs=2.0e7):
    """Plane benchmark: the active cells are `layers` cell layers of an N x N footprint with the
    plane in the top one, so that about 1 / layers of the active cells are cut; `ratio` = 0
    puts the plane above the box (no cut cell).  N is chosen for about n_dofs unknowns."""
    layers = 1 if ratio >= 1.0 else (100 if ratio <= 0.0 else int(round(1.0 / ratio)))
    per_cell = (p + 1) ** 3 if discretization == "dg" else p ** 3
    N = max(4, int(round((n_dofs / per_cell / layers) ** 0.5)))
    # the plane rises by h / 2 across the box, so it stays inside the top cell layer
    oc = layers + 10.0 if ratio <= 0.0 else layers - 0.75
    c = plane(p=p, N=N, dim=3, layers=layers, offset_cells=oc, discretization=discretization,
              seed=10, normal=(-0.3 / N, -0.2 / N, 1.0))
    c["name"] = f"3d_{discretization}_q{p}_plane_ratio_{ratio:g}"
    return c


def sphere_lattice(m, R, dim=3):
    """m^d balls of radius R centred on the lattice (i + 1/2) / m of the unit box."""
    out = []
    for k in range(m if dim == 3 else 1):
        for j in range(m):
            for i in range(m):
                out.append(((i + 0.5) / m, (j + 0.5) / m, (k + 0.5) / m if dim == 3 else 0.0, R))
    return out


def spheres(p=2, N=12, m=2, R=0.2, dim=3, discretization="dg", quad_order=None, seed=11):
    """Union of m^d balls of radius R on a lattice in [0, 1]^d, N cells per direction;
    penalties as for the ball workloads."""
    pad = (0.0,) * (3 - dim)
    return dict(name=f"{dim}d_{discretization}_q{p}_{m}^{dim}_spheres_{N}", dim=dim, degree=p,
                n_cells=(N,) * dim + (1,) * (3 - dim), lo=(0.0,) * dim + pad, hi=(1.0,) * dim + pad,
                center=(0.0, 0.0, 0.0), radius=1.0, ls_kind="spheres",
                spheres=sphere_lattice(m, R, dim), quad_order=quad_order if quad_order else p + 1,
                seed=seed, discretization=discretization, **_penalties(p))


def random_spheres(n, R, seed, dim=3):
    """n balls of radius R (a number, or a (min, max) range drawn uniformly) with centres drawn
    uniformly in the unit box: numpy default_rng(seed), all centres first (x, y, z per ball),
    then the radii.  The balls intersect freely."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, 1.0, size=(n, dim))
    r = np.full(n, float(R)) if np.isscalar(R) else rng.uniform(R[0], R[1], size=n)
    out = []
    for i in range(n):
        xyz = [float(v) for v in c[i]] + [0.0] * (3 - dim)
        out.append((xyz[0], xyz[1], xyz[2], float(r[i])))
    return out


def spheres_random(p=2, N=12, n=6, R=0.2, seed=5, dim=3, discretization="dg", quad_order=None):
    """Union of n intersecting balls (random_spheres) in [0, 1]^d, N cells per direction."""
    c = spheres(p=p, N=N, m=1, R=R if np.isscalar(R) else R[1], dim=dim,
                discretization=discretization, quad_order=quad_order)
    c["spheres"] = random_spheres(n, R, seed, dim)
    c["name"] = f"{dim}d_{discretization}_q{p}_{n}_random_spheres_{N}"
    return c


def cfg_spheres_random(p=1, discretization="dg"):
    """The paper's random-spheres benchmark (Sec. 6): 100 randomly placed, intersecting balls;
    their placement and radii are not given, so: random_spheres(100, (0.02, 0.131), seed 4),
    radius range and seed fitted to the printed DoF count and cut-cell ratio of the DG Q1 case,
    12^3 background cells refined four times (192^3); p = 1 and p = 3 on the same mesh."""
    c = spheres_random(p=p, N=192, n=100, R=(0.02, 0.131), seed=4, discretization=discretization)
    c["name"] = f"3d_{discretization}_q{p}_100_random_spheres_192^3"
    c["seed"] = 13
    return c


def cfg_spheres_regular(p=1, discretization="dg"):
    """The paper's regular-spheres benchmark (Sec. 6): 1000 balls on a regular pattern; their
    radius and placement are not given, so: the 10^3 lattice of the unit cube, radius 0.0362
    (fitted to the printed DoF count and cut-cell ratio), 12^3 background cells refined four
    times (192^3), DG Q1."""
    c = spheres(p=p, N=192, m=10, R=0.0362, discretization=discretization, seed=12)
    c["name"] = f"3d_{discretization}_q{p}_1000_spheres_192^3"
    return c

