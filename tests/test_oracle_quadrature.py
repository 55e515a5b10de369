"""Pins of the oracle's dimension-reduction quadrature against closed forms (CPU).

The rule itself has no printed reference; its integrals do: ball volume and sphere area, monomial
moments of ball and sphere (closed form through Gamma functions), plane sections of the ball, and
the divergence theorem on every cut cell (volume rule, surface rule and face rules together).
"""
import math

import numpy as np
import pytest

from oracle import mesh, saye


def _ball_moment(alpha, R, surface=False):
    """int over the ball (or sphere) of radius R centred at 0 of prod_i y_i^alpha_i."""
    if any(a % 2 for a in alpha):
        return 0.0
    d = len(alpha)
    s = sum(alpha)
    g = 2.0 * np.prod([math.gamma((a + 1) / 2.0) for a in alpha]) / math.gamma((s + d) / 2.0)
    return g * R ** (s + d - 1) if surface else g * R ** (s + d) / (s + d)


def _all_rules(prob):
    m = mesh.Mesh(prob)
    vol = []
    surf = []
    for e in range(m.n_active):
        lo, hi = mesh.cell_box(prob, m.index_of(e))
        if m.active_type[e] == mesh.INSIDE:
            vol += saye.tensor_gauss(lo, hi, prob.quad_order)
        else:
            v, s = saye.cell_rules(prob, lo, hi)
            vol += v
            surf += s
    vx = np.array([p for p, _ in vol])
    vw = np.array([w for _, w in vol])
    sx = np.array([p for p, _, _ in surf])
    sw = np.array([w for _, w, _ in surf])
    sn = np.array([nn for _, _, nn in surf])
    return vx, vw, sx, sw, sn


def _prob(dim, N, q, center, R=1.0):
    return mesh.Problem(dim, 3, (N,) * dim, (-1.21,) * dim, (1.21,) * dim, center, R, q, 1, 1, 1, 0.5)


@pytest.mark.parametrize("dim,center", [(2, (0.03, 0.02)), (3, (0.01, 0.02, 0.03))])
def test_volume_and_area_converge(dim, center):
    errs = []
    for N in (6, 12, 24):
        vx, vw, sx, sw, sn = _all_rules(_prob(dim, N, 4, center))
        V = math.pi if dim == 2 else 4.0 / 3.0 * math.pi
        S = 2.0 * math.pi if dim == 2 else 4.0 * math.pi
        errs.append((abs(vw.sum() - V), abs(sw.sum() - S)))
        # the surface normals integrate to zero (closed surface)
        assert np.max(np.abs(sw @ sn)) < 10 * errs[-1][1] + 1e-13
    # high order: two halvings of h gain at least 2^10 (order >= 5; q = 4 Gauss points)
    assert errs[2][0] < errs[0][0] / 1024 and errs[2][1] < errs[0][1] / 1024
    assert errs[-1][0] < 1e-10 and errs[-1][1] < 1e-9


def test_monomial_moments_3d():
    c = np.array([0.01, 0.02, 0.03])
    vx, vw, sx, sw, sn = _all_rules(_prob(3, 16, 4, tuple(c)))
    yv = vx - c
    ys = sx - c
    for alpha in [(0, 0, 0), (2, 0, 0), (0, 2, 2), (1, 0, 0), (2, 2, 0), (4, 0, 0), (1, 1, 2), (2, 1, 0)]:
        fv = np.prod([yv[:, i] ** alpha[i] for i in range(3)], axis=0)
        fs = np.prod([ys[:, i] ** alpha[i] for i in range(3)], axis=0)
        assert abs(vw @ fv - _ball_moment(alpha, 1.0)) < 2e-9
        assert abs(sw @ fs - _ball_moment(alpha, 1.0, surface=True)) < 2e-8


def test_plane_sections_3d():
    """The face rules of all faces in one grid plane integrate the disc section of the ball."""
    prob = _prob(3, 20, 4, (0.01, 0.02, 0.03))
    m = mesh.Mesh(prob)
    for axis in range(3):
        for plane in (6, 10, 13):
            xa = prob.lo[axis] + plane * prob.h
            total = 0.0
            for e in range(m.n_active):
                if m.index_of(e)[axis] != plane - 1:
                    continue
                ep = m.neighbor(e, axis, 1)
                if ep < 0:
                    continue
                lo, hi = m.face_box(e, axis)
                ft = m.face_type(e, axis)
                if ft == mesh.FACE_FULL:
                    total += prob.h ** 2
                elif ft == mesh.FACE_CUT:
                    total += sum(w for _, w in saye.face_rule(prob, lo, hi, axis))
            dist = xa - prob.center[axis]
            assert abs(total - math.pi * (1.0 - dist * dist)) < 1e-9


def test_divergence_theorem_per_cut_cell():
    """int_{K cap Omega} div F = int_{Gamma cap K} F.n + sum_faces int_{F cap Omega} F.n_K."""
    prob = _prob(3, 8, 5, (0.01, 0.02, 0.03))
    m = mesh.Mesh(prob)

    def F(x):
        return np.array([x[0] ** 2 * x[1], x[1] * x[2] ** 3 + x[0], x[0] * x[1] * x[2]])

    def divF(x):
        return 2 * x[0] * x[1] + x[2] ** 3 + x[0] * x[1]

    worst = 0.0
    for e in range(m.n_active):
        if m.active_type[e] != mesh.CUT:
            continue
        lo, hi = mesh.cell_box(prob, m.index_of(e))
        vol, surf = saye.cell_rules(prob, lo, hi)
        lhs = sum(w * divF(x) for x, w in vol)
        rhs = sum(w * F(x) @ np.array(nn) for x, w, nn in surf)
        for axis in range(3):
            for side, sign in ((0, -1.0), (1, 1.0)):
                flo = list(lo)
                fhi = list(hi)
                if side == 0:
                    fhi[axis] = lo[axis]
                else:
                    flo[axis] = hi[axis]
                for x, w in saye.face_rule(prob, tuple(flo), tuple(fhi), axis):
                    rhs += sign * w * F(x)[axis]
        worst = max(worst, abs(lhs - rhs))
    # quadrature error at h = 0.3 (q = 5) is ~1e-8; a dropped or mis-signed term gives O(h^2)
    assert worst < 5e-8


def test_brute_force_single_cell():
    """One cut cell: Saye volume vs a 2^7-per-direction midpoint sampling of the indicator."""
    lo, hi = (0.55, 0.52, 0.4), (0.85, 0.82, 0.7)
    c, R = (0.0, 0.0, 0.0), 1.0
    vol, surf = saye.sphere_rules(lo, hi, c, R * R, 4)
    V = sum(w for _, w in vol)
    k = 128
    t = (np.arange(k) + 0.5) / k
    X, Y, Z = np.meshgrid(*[lo[a] + (hi[a] - lo[a]) * t for a in range(3)], indexing="ij")
    inside = (X ** 2 + Y ** 2 + Z ** 2) < 1.0
    Vb = inside.mean() * np.prod(np.subtract(hi, lo))
    assert 0 < V < np.prod(np.subtract(hi, lo))
    assert abs(V - Vb) < 2e-3 * np.prod(np.subtract(hi, lo))


def test_inside_box_is_tensor_gauss_and_exact():
    lo, hi = (-0.2, -0.1, 0.0), (0.1, 0.2, 0.3)
    vol, surf = saye.sphere_rules(lo, hi, (0.0, 0.0, 0.0), 1.0, 3)
    assert not surf and len(vol) == 27
    # exact for x^5 y^4 z^3
    got = sum(w * x[0] ** 5 * x[1] ** 4 * x[2] ** 3 for x, w in vol)
    want = ((hi[0] ** 6 - lo[0] ** 6) / 6) * ((hi[1] ** 5 - lo[1] ** 5) / 5) * ((hi[2] ** 4 - lo[2] ** 4) / 4)
    assert abs(got - want) < 1e-17


def test_subdivision_path():
    """A box containing the centre of a small sphere needs bisection.  The children have height
    functions that are steep near the bisection planes, so the integrals converge algebraically in
    q there; check that they converge."""
    lo, hi = (-0.3, -0.2, -0.25), (0.3, 0.4, 0.35)
    c = (0.02, 0.01, -0.01)
    R = 0.15
    errs = []
    for q in (4, 8, 12):
        vol, surf = saye.sphere_rules(lo, hi, c, R * R, q)
        errs.append((abs(sum(w for _, w in vol) / (4.0 / 3.0 * math.pi * R ** 3) - 1.0),
                     abs(sum(w for _, w, _ in surf) / (4.0 * math.pi * R ** 2) - 1.0)))
    assert errs[0][0] < 1e-5 and errs[0][1] < 5e-3
    assert errs[2][0] < errs[0][0] / 10 and errs[2][1] < errs[0][1] / 100


# ------------------------------------------------------------------------------------------
# Plane level sets: the region below a plane in a box is a polytope, and every dimension-
# reduction piece is split exactly at the plane, so the rules integrate polynomials of degree
# <= 2q - 1 per direction exactly: closed forms hold to rounding.
# ------------------------------------------------------------------------------------------

def _plane_prob(dim, N, q, normal, offset):
    return mesh.Problem(dim, 2, (N,) * dim, (0.0,) * dim, (1.0,) * dim, (0.0,) * dim, 1.0, q, 1, 1,
                        1, 0.5, ls_kind="plane", normal=normal, offset=offset)


def _height(normal, offset):
    """The plane as a graph over the first d-1 coordinates: x_d = offset - sum a_i x_i."""
    nd = normal[-1]
    return lambda xs: (offset - sum(normal[i] * xs[i] for i in range(len(xs)))) / nd


@pytest.mark.parametrize("dim,normal,offset", [
    (2, (-0.1, 1.0), 0.43),
    (3, (-0.1, -0.05, 1.0), 0.43),
    (3, (0.2, -0.3, 0.9), 0.31),     # tilted enough that cut cells stack along the last axis
    (3, (0.0, 0.0, 1.0), 0.5),       # on a grid plane: the cut is a layer of full faces
])
def test_plane_rules_closed_forms(dim, normal, offset):
    import scipy.integrate as si

    prob = _plane_prob(dim, 5, 3, normal, offset)
    vx, vw, sx, sw, sn = _all_rules(prob)
    f = _height(normal, offset)
    nrm = math.sqrt(sum(v * v for v in normal))
    # the plane stays inside the box over the whole footprint for these cases
    if dim == 2:
        vol = si.quad(lambda x: f((x,)), 0, 1, epsabs=1e-15)[0]
        mom = si.quad(lambda x: x * f((x,)) ** 2 / 2, 0, 1, epsabs=1e-15)[0]
    else:
        vol = si.dblquad(lambda y, x: f((x, y)), 0, 1, 0, 1, epsabs=1e-15)[0]
        mom = si.dblquad(lambda y, x: x * f((x, y)) ** 2 / 2, 0, 1, 0, 1, epsabs=1e-15)[0]
    area = nrm / abs(normal[-1])  # the plane over the unit footprint
    assert abs(vw.sum() - vol) < 1e-14
    assert abs(sw.sum() - area) < 1e-14
    # int_Gamma n = projected area along every axis = normal / |normal_d|
    assert np.abs((sw[:, None] * sn).sum(axis=0) - np.array(normal) / abs(normal[-1])).max() < 1e-14
    # int x_0 x_d (degree 2, exact for q = 3)
    assert abs(vw @ (vx[:, 0] * vx[:, -1]) - mom) < 1e-14
    # every surface point lies on the plane, with the unit normal
    assert np.abs(sx @ np.array(normal) - offset).max() < 1e-14
    assert np.abs(sn - np.array(normal) / nrm).max() < 1e-15


def test_plane_divergence_theorem_per_cut_cell_exact():
    """Per cut cell, divergence theorem with the face rules; exact for a cubic field (q = 4)."""
    prob = _plane_prob(3, 4, 4, (0.2, -0.3, 0.9), 0.31)
    m = mesh.Mesh(prob)

    def F(x):
        return np.array([x[0] ** 2 * x[1], x[1] * x[2] ** 2 + x[0], x[0] * x[1] * x[2]])

    def divF(x):
        return 2 * x[0] * x[1] + x[2] ** 2 + x[0] * x[1]

    worst = 0.0
    n_cut = 0
    for e in range(m.n_active):
        if m.active_type[e] != mesh.CUT:
            continue
        n_cut += 1
        lo, hi = mesh.cell_box(prob, m.index_of(e))
        vol, surf = saye.cell_rules(prob, lo, hi)
        lhs = sum(w * divF(x) for x, w in vol)
        rhs = sum(w * F(x) @ np.array(nn) for x, w, nn in surf)
        for axis in range(3):
            for side, sign in ((0, -1.0), (1, 1.0)):
                flo = list(lo)
                fhi = list(hi)
                if side == 0:
                    fhi[axis] = lo[axis]
                else:
                    flo[axis] = hi[axis]
                for x, w in saye.face_rule(prob, tuple(flo), tuple(fhi), axis):
                    rhs += sign * w * F(x)[axis]
        worst = max(worst, abs(lhs - rhs))
    assert n_cut > 10
    assert worst < 1e-14


def test_plane_classification_against_sampling():
    """Inside / cut / outside of every cell against a dense sampling of the plane's sign."""
    normal, offset = (0.2, -0.3, 0.9), 0.31
    prob = _plane_prob(3, 6, 2, normal, offset)
    m = mesh.Mesh(prob)
    t = np.linspace(0.0, 1.0, 9)
    for flat in range(6 ** 3):
        idx = (flat % 6, (flat // 6) % 6, flat // 36)
        lo, hi = mesh.cell_box(prob, idx)
        g = np.stack(np.meshgrid(*[lo[a] + t * (hi[a] - lo[a]) for a in range(3)]), -1).reshape(-1, 3)
        phi = g @ np.array(normal) - offset
        want = mesh.INSIDE if phi.max() <= 0 else (mesh.OUTSIDE if phi.min() >= 0 else mesh.CUT)
        e = m.id_map[idx[::-1]]
        got = mesh.OUTSIDE if e < 0 else m.active_type[e]
        assert got == want


# ------------------------------------------------------------------------------------------
# Union of separated balls: each cut cell meets one sphere, whose rule it uses
# ------------------------------------------------------------------------------------------

_EIGHT = [(0.25 + 0.5 * i, 0.26 + 0.5 * j, 0.24 + 0.5 * k, 0.2 - 0.01 * (i + j + k))
          for k in range(2) for j in range(2) for i in range(2)]


def _spheres_prob(N, q, spheres=_EIGHT):
    return mesh.Problem(3, 2, (N,) * 3, (0.0,) * 3, (1.0,) * 3, (0.0,) * 3, 1.0, q, 1, 1, 1, 0.5,
                        ls_kind="spheres", spheres=spheres)


def test_union_of_separated_balls_converges():
    vol = sum(4.0 / 3.0 * math.pi * R ** 3 for *_, R in _EIGHT)
    area = sum(4.0 * math.pi * R ** 2 for *_, R in _EIGHT)
    errs = []
    for N in (10, 20, 40):
        _, vw, sx, sw, sn = _all_rules(_spheres_prob(N, 4))
        errs.append((abs(vw.sum() - vol) / vol, abs(sw.sum() - area) / area))
        assert np.abs(np.linalg.norm(sn, axis=1) - 1.0).max() < 1e-14
    assert errs[-1][0] < 1e-8 and errs[-1][1] < 1e-7
    # high order: at least h^4 per halving over two halvings
    assert errs[0][0] / errs[2][0] > 16 ** 2 and errs[0][1] / errs[2][1] > 16 ** 2


def test_union_classification_against_sampling():
    prob = _spheres_prob(12, 2)
    m = mesh.Mesh(prob)
    t = np.linspace(0.0, 1.0, 7)
    for flat in range(0, 12 ** 3, 5):
        idx = (flat % 12, (flat // 12) % 12, flat // 144)
        lo, hi = mesh.cell_box(prob, idx)
        g = np.stack(np.meshgrid(*[lo[a] + t * (hi[a] - lo[a]) for a in range(3)]), -1).reshape(-1, 3)
        phi = np.min([np.linalg.norm(g - np.array(c[:3]), axis=1) - R for *c, R in _EIGHT], axis=0)
        e = m.id_map[idx[::-1]]
        got = mesh.OUTSIDE if e < 0 else m.active_type[e]
        if phi.max() < 0:
            assert got == mesh.INSIDE
        elif phi.min() > 0:
            assert got == mesh.OUTSIDE
        else:
            assert got == mesh.CUT


# Intersecting balls: two with a lens, three meeting at triple points (generic positions)
_TWO = [(0.43, 0.47, 0.52, 0.26), (0.71, 0.58, 0.46, 0.19)]
_THREE = [(0.41, 0.45, 0.5, 0.24), (0.66, 0.52, 0.47, 0.21), (0.52, 0.71, 0.55, 0.205)]


def _union_two_closed_forms(balls):
    """Volume and area of the union of two intersecting balls (lens by two spherical caps)."""
    (x1, y1, z1, R1), (x2, y2, z2, R2) = balls
    D = math.sqrt((x2 - x1) ** 2 + (y2 - y1) ** 2 + (z2 - z1) ** 2)
    a1 = (D * D + R1 * R1 - R2 * R2) / (2 * D)
    h1 = R1 - a1
    h2 = R2 - (D - a1)
    cap = lambda R, h: math.pi * h * h * (3 * R - h) / 3.0
    vol = 4.0 / 3.0 * math.pi * (R1 ** 3 + R2 ** 3) - cap(R1, h1) - cap(R2, h2)
    area = 4.0 * math.pi * (R1 * R1 + R2 * R2) - 2.0 * math.pi * (R1 * h1 + R2 * h2)
    return vol, area


def test_union_of_two_intersecting_balls_converges():
    vol, area = _union_two_closed_forms(_TWO)
    errs = []
    for N in (8, 16, 32):
        _, vw, sx, sw, sn = _all_rules(_spheres_prob(N, 4, _TWO))
        errs.append((abs(vw.sum() - vol) / vol, abs(sw.sum() - area) / area))
        assert np.abs(np.linalg.norm(sn, axis=1) - 1.0).max() < 1e-14
    assert errs[-1][0] < 1e-9 and errs[-1][1] < 5e-8
    assert errs[0][0] / errs[2][0] > 16 ** 2 and errs[0][1] / errs[2][1] > 16 ** 2


def test_union_with_intersection_circle_in_a_grid_plane_converges():
    """Centres on one grid axis: the intersection circle lies in a plane x = const, seen along
    y or z as a segment; the rule still converges at high order."""
    balls = [(0.35, 0.5, 0.5, 0.2), (0.6, 0.5, 0.5, 0.2)]
    vol, area = _union_two_closed_forms(balls)
    errs = []
    for N in (8, 16, 32):
        _, vw, sx, sw, sn = _all_rules(_spheres_prob(N, 4, balls))
        errs.append((abs(vw.sum() - vol) / vol, abs(sw.sum() - area) / area))
    assert errs[-1][0] < 1e-9 and errs[-1][1] < 1e-8
    assert errs[0][0] / errs[2][0] > 16 ** 2 and errs[0][1] / errs[2][1] > 16 ** 2


def test_union_of_two_intersecting_discs():
    (x1, y1, _, R1), (x2, y2, _, R2) = _TWO
    D = math.hypot(x2 - x1, y2 - y1)
    lens = (R1 * R1 * math.acos((D * D + R1 * R1 - R2 * R2) / (2 * D * R1))
            + R2 * R2 * math.acos((D * D + R2 * R2 - R1 * R1) / (2 * D * R2))
            - 0.5 * math.sqrt((-D + R1 + R2) * (D + R1 - R2) * (D - R1 + R2) * (D + R1 + R2)))
    area = math.pi * (R1 * R1 + R2 * R2) - lens
    # perimeter: each circle minus its arc inside the other disc
    t1 = math.acos((D * D + R1 * R1 - R2 * R2) / (2 * D * R1))
    t2 = math.acos((D * D + R2 * R2 - R1 * R1) / (2 * D * R2))
    per = 2 * R1 * (math.pi - t1) + 2 * R2 * (math.pi - t2)
    prob = mesh.Problem(2, 2, (24, 24), (0.0, 0.0), (1.0, 1.0), (0.0, 0.0), 1.0, 8, 1, 1, 1, 0.5,
                        ls_kind="spheres", spheres=_TWO)
    _, vw, sx, sw, sn = _all_rules(prob)
    assert abs(vw.sum() - area) < 1e-13 and abs(sw.sum() - per) < 1e-12


def _divergence_residuals(prob, F, divF):
    m = mesh.Mesh(prob)
    d = prob.dim
    res = []
    for e in range(m.n_active):
        if m.active_type[e] != mesh.CUT:
            continue
        lo, hi = mesh.cell_box(prob, m.index_of(e))
        vol, surf = saye.cell_rules(prob, lo, hi)
        lhs = sum(w * divF(x) for x, w in vol)
        rhs = sum(w * F(x) @ np.array(nn) for x, w, nn in surf)
        for axis in range(d):
            for side, sign in ((0, -1.0), (1, 1.0)):
                flo = list(lo)
                fhi = list(hi)
                if side == 0:
                    fhi[axis] = lo[axis]
                else:
                    flo[axis] = hi[axis]
                for x, w in saye.face_rule(prob, tuple(flo), tuple(fhi), axis):
                    rhs += sign * w * F(x)[axis]
        res.append(abs(lhs - rhs))
    return np.array(res)


def test_union_of_three_balls_divergence_theorem_per_cell():
    """Cells that hold intersection circles and triple points, q = 8: every cell's residual
    stays at the level of the single-sphere cells (<= 5e-9 here; dropping the intersection
    circles as break curves gives 6e-5, dropping the break points on the cell faces and the
    triple points 2e-6)."""
    prob = _spheres_prob(16, 8, _THREE)

    def F(x):
        return np.array([x[0] ** 2 * x[1], x[1] * x[2] ** 2 + x[0], x[0] * x[1] * x[2]])

    def divF(x):
        return 2 * x[0] * x[1] + x[2] ** 2 + x[0] * x[1]

    res = _divergence_residuals(prob, F, divF)
    assert len(res) > 300 and res.max() < 3e-8


def test_union_of_three_discs_divergence_theorem_per_cell():
    """Dropping the circles' intersection points as break points gives 3e-3."""
    prob = mesh.Problem(2, 2, (16, 16), (0.0, 0.0), (1.0, 1.0), (0.0, 0.0), 1.0, 8, 1, 1, 1, 0.5,
                        ls_kind="spheres", spheres=_THREE)
    res = _divergence_residuals(prob, lambda x: np.array([x[0] ** 3 * x[1], x[1] ** 2 + x[0]]),
                                lambda x: 3 * x[0] ** 2 * x[1] + 2 * x[1])
    assert len(res) > 40 and res.max() < 1e-11


def test_union_intersecting_classification_against_sampling():
    prob = _spheres_prob(10, 2, _THREE)
    m = mesh.Mesh(prob)
    t = np.linspace(0.0, 1.0, 9)
    for flat in range(10 ** 3):
        idx = (flat % 10, (flat // 10) % 10, flat // 100)
        lo, hi = mesh.cell_box(prob, idx)
        g = np.stack(np.meshgrid(*[lo[a] + t * (hi[a] - lo[a]) for a in range(3)]), -1).reshape(-1, 3)
        phis = [np.linalg.norm(g - np.array(c[:3]), axis=1) - R for *c, R in _THREE]
        e = m.id_map[idx[::-1]]
        got = mesh.OUTSIDE if e < 0 else m.active_type[e]
        if any(p.max() < 0 for p in phis):
            assert got == mesh.INSIDE
        elif np.min(phis) > 0:
            assert got == mesh.OUTSIDE
        elif any(p.min() < 0 < p.max() for p in phis):
            assert got == mesh.CUT


def test_box_covered_by_two_balls_but_by_neither():
    """A cell inside the union but inside no single ball is cut, with the full volume and no
    surface points."""
    balls = [(0.2, 0.5, 0.5, 0.33), (0.8, 0.5, 0.5, 0.33)]
    lo, hi = (0.45, 0.45, 0.45), (0.55, 0.55, 0.55)
    prob = _spheres_prob(10, 3, balls)
    assert mesh.classify(prob, lo, hi) == mesh.CUT
    vol, surf = saye.cell_rules(prob, lo, hi)
    assert surf == [] and abs(sum(w for _, w in vol) - 1e-3) < 1e-17


_GL4 = np.polynomial.legendre.leggauss(4)


def _composite_gauss(lo, hi, panels):
    """Points and weights of a composite 4-point Gauss rule with `panels` equal panels."""
    g, w = 0.5 * (_GL4[0] + 1.0), 0.5 * _GL4[1]
    t = ((np.arange(panels)[:, None] + g[None, :]) / panels).ravel()
    return lo + (hi - lo) * t, np.tile(w, panels) * (hi - lo) / panels


def _union_of_intervals_length(intervals, lo, hi):
    """Length of the union of the intervals (a_i, b_i) (arrays over the evaluation points; empty
    ones given as a = b = hi) clipped to [lo, hi]: sort by start, merge, add up."""
    A = np.stack([np.clip(a, lo, hi) for a, _ in intervals])
    B = np.stack([np.clip(b, lo, hi) for _, b in intervals])
    order = np.argsort(A, axis=0)
    A = np.take_along_axis(A, order, 0)
    B = np.take_along_axis(B, order, 0)
    total = np.zeros(A.shape[1:])
    ca, cb = A[0].copy(), B[0].copy()
    for i in range(1, A.shape[0]):
        apart = A[i] > cb
        total += np.where(apart, cb - ca, 0.0)
        ca = np.where(apart, A[i], ca)
        cb = np.where(apart, B[i], np.maximum(cb, B[i]))
    return total + (cb - ca)


def _chords(balls, pts, axis, lo, hi):
    """Per ball, the chord of the ball along `axis` through each point of `pts` (the other
    coordinates), as an interval; empty chords collapse to [hi, hi]."""
    out = []
    for *c, R in balls:
        r2 = sum((pts[a] - c[a]) ** 2 for a in pts)
        h = np.sqrt(np.maximum(R * R - r2, 0.0))
        hit = r2 < R * R
        out.append((np.where(hit, c[axis] - h, hi), np.where(hit, c[axis] + h, hi)))
    return out


def test_union_of_three_balls_cell_volumes_from_chords():
    """A pin of the union rule that shares nothing with its construction: the volume of the
    union of three intersecting balls inside a cell is the integral, over the cell's (x, y)
    square, of the length of the union of the balls' chords along z (merged exactly and clipped
    to the cell).  A composite Gauss rule of 128 x 128 panels takes that integral to about
    3e-6 of the cell volume (the chord lengths have square-root edges on the balls'
    silhouettes: 1e-4 at 32 panels).  Checked on every cut cell met by two or three spheres
    (where the union's intersection circles and triple points act) and on every fourth other
    cut cell."""
    prob = _spheres_prob(16, 8, _THREE)
    m = mesh.Mesh(prob)
    checked = multi = 0
    for e in range(m.n_active):
        if m.active_type[e] != mesh.CUT:
            continue
        lo, hi = mesh.cell_box(prob, m.index_of(e))
        _, crossing = mesh.crossing_spheres(prob, lo, hi)
        if len(crossing) < 2 and e % 4:
            continue
        multi += len(crossing) >= 2
        x, wx = _composite_gauss(lo[0], hi[0], 128)
        y, wy = _composite_gauss(lo[1], hi[1], 128)
        X, Y = np.meshgrid(x, y, indexing="ij")
        length = _union_of_intervals_length(_chords(_THREE, {0: X, 1: Y}, 2, lo[2], hi[2]),
                                            lo[2], hi[2])
        exact = float(np.sum(np.outer(wx, wy) * length))
        rule = sum(w for _, w in saye.cell_rules(prob, lo, hi)[0])
        assert abs(rule - exact) <= 1e-5 * (hi[0] - lo[0]) ** 3, (e, rule, exact)
        checked += 1
    assert multi >= 20 and checked >= 100


def test_union_of_three_discs_cell_areas_from_chords():
    """The 2D counterpart: the area of the union of three discs inside a cell is the integral
    over x of the length of the union of the discs' chords along y, here with 4096 composite
    Gauss panels (7e-7 of the cell area; 2e-5 at 256 panels).  Every cut cell."""
    prob = mesh.Problem(2, 2, (16, 16), (0.0, 0.0), (1.0, 1.0), (0.0, 0.0), 1.0, 8, 1, 1, 1, 0.5,
                        ls_kind="spheres", spheres=_THREE)
    m = mesh.Mesh(prob)
    discs = [(cx, cy, R) for cx, cy, _, R in _THREE]
    checked = 0
    for e in range(m.n_active):
        if m.active_type[e] != mesh.CUT:
            continue
        lo, hi = mesh.cell_box(prob, m.index_of(e))
        x, wx = _composite_gauss(lo[0], hi[0], 4096)
        length = _union_of_intervals_length(_chords(discs, {0: x}, 1, lo[1], hi[1]), lo[1], hi[1])
        exact = float(np.sum(wx * length))
        rule = sum(w for _, w in saye.cell_rules(prob, lo, hi)[0])
        assert abs(rule - exact) <= 2e-6 * (hi[0] - lo[0]) ** 2, (e, rule, exact)
        checked += 1
    assert checked >= 40


def test_union_of_three_balls_cut_face_areas_from_chords():
    """The cut faces' rules, pinned the same way: on each face of a cut cell, the area of the
    union of the balls' sections by the face's plane is the integral, along one in-face axis, of
    the merged chords along the other (4096 composite Gauss panels, about 1e-7 of the face area).
    At the operator's q = 8 the rules agree to 2e-5 of the face area: on a face where a small
    section's vertical-tangent point lies just outside a sub-box, the height function is smooth
    but close to singular and Gauss converges slowly.  At q = 16 they agree to 4e-7, so the rules
    converge to the chord integral."""
    prob = _spheres_prob(16, 8, _THREE)
    m = mesh.Mesh(prob)
    checked = 0
    for e in range(m.n_active):
        if m.active_type[e] != mesh.CUT:
            continue
        lo, hi = mesh.cell_box(prob, m.index_of(e))
        for axis in range(3):
            a, b = [x for x in range(3) if x != axis]
            for v in (lo[axis], hi[axis]):
                flo, fhi = list(lo), list(hi)
                flo[axis] = fhi[axis] = v
                # the balls' sections by the plane x_axis = v, as discs in the (a, b) plane
                discs = [(c[a], c[b], math.sqrt(R * R - (v - c[axis]) ** 2))
                         for *c, R in _THREE if R * R > (v - c[axis]) ** 2]
                area = 0.0
                if discs:
                    x, wx = _composite_gauss(lo[a], hi[a], 4096)
                    length = _union_of_intervals_length(_chords(discs, {0: x}, 1, lo[b], hi[b]),
                                                        lo[b], hi[b])
                    area = float(np.sum(wx * length))
                fa = (hi[a] - lo[a]) * (hi[b] - lo[b])
                for q, tol in ((8, 5e-5), (16, 1e-6)):
                    rule = sum(w for _, w in saye.face_rule(prob, tuple(flo), tuple(fhi), axis, q=q))
                    assert abs(rule - area) <= tol * fa, (e, axis, v, q)
                checked += 1
    assert checked >= 1000
