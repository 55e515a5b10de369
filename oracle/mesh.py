"""Background grid, cell classification and face typing (oracle; test infrastructure only).

Sec. 1 / Sec. 2.1 of the paper: the geometry is embedded into a Cartesian background mesh by a
level set phi; the physical domain is Omega = {phi < 0}.  Sec. 2.3 classifies cells as inside
(structured quadrature), cut (unstructured quadrature) or outside (dropped), and interior faces as
inside faces (structured) or cut faces (unstructured).

Level sets: the sphere phi(x) = |x - c| - R, classified exactly through the squared minimum /
maximum distance from c to the closed box:
    inside  <=>  dmax^2 <= R^2,     outside  <=>  dmin^2 >= R^2,     cut otherwise;
and the plane phi(x) = n . x - off, classified exactly through its minimum / maximum over the box
(the corner chosen per direction by the sign of n_a):
    inside  <=>  max phi <= 0,      outside  <=>  min phi >= 0,      cut otherwise.
Sums are taken over the coordinate directions in increasing index order.

Active cells (inside + cut) are numbered lexicographically with the x index fastest; the DoFs of
active cell e are e * n^d + l with l = i + n j + n^2 k (Sec. 3.2).

Interior faces: a face between two active cells K- (lower index along the axis) and K+ is
  full  if the closed face lies in the closed ball   (structured SIPG),
  empty if it lies outside the open ball             (no SIPG, measure zero),
  cut   otherwise                                     (SIPG on F cap Omega, unstructured rule).
A face carries the face-based ghost penalty iff at least one of its two cells is cut.
"""
import math
from dataclasses import dataclass, field

import numpy as np

from . import saye

INSIDE, CUT, OUTSIDE = 0, 1, 2
FACE_FULL, FACE_CUT, FACE_EMPTY = 0, 1, 2


def box_dist2(c, lo, hi):
    """(dmin^2, dmax^2) from point c to the closed box [lo, hi] (any dimension)."""
    dmin2 = 0.0
    dmax2 = 0.0
    for a in range(len(c)):
        dl = lo[a] - c[a]
        dh = hi[a] - c[a]
        e = max(max(dl, 0.0), -dh)
        dmin2 += e * e
        dmax2 += max(dl * dl, dh * dh)
    return dmin2, dmax2


def classify_box(c, R, lo, hi):
    dmin2, dmax2 = box_dist2(c, lo, hi)
    r2 = R * R
    if dmax2 <= r2:
        return INSIDE
    if dmin2 >= r2:
        return OUTSIDE
    return CUT


def classify_plane_box(n, off, lo, hi):
    mn, mx = saye.lin_range(n, off, lo, hi)
    if mx <= 0.0:
        return INSIDE
    if mn >= 0.0:
        return OUTSIDE
    return CUT


def crossing_spheres(prob, lo, hi):
    """Union of balls: (inside, crossing) for the closed box: inside if one ball contains it,
    crossing = indices of the spheres whose surface meets it."""
    inside = False
    crossing = []
    for i, (c, R) in enumerate(prob.spheres):
        t = classify_box(c, R, lo, hi)
        if t == INSIDE:
            inside = True
        elif t == CUT:
            crossing.append(i)
    return inside, crossing


def classify(prob, lo, hi):
    """Type of the closed box [lo, hi] against the level set of `prob`.  A union of balls is
    classified box by box: inside if one ball contains it, cut if a sphere meets it, outside
    otherwise (a box covered by several balls but by none alone is cut, with a full volume
    rule and no surface points)."""
    if prob.ls_kind == "plane":
        return classify_plane_box(prob.normal, prob.offset, lo, hi)
    if prob.ls_kind == "spheres":
        inside, crossing = crossing_spheres(prob, lo, hi)
        if inside:
            return INSIDE
        return CUT if crossing else OUTSIDE
    return classify_box(prob.center, prob.radius, lo, hi)


@dataclass
class Problem:
    """One unfitted Poisson problem (sphere or half-space domain, uniform Cartesian background
    grid).  ls_kind "sphere": |x - center| < radius; "plane": normal . x < offset."""

    dim: int
    degree: int
    n_cells: tuple
    lo: tuple
    hi: tuple
    center: tuple
    radius: float
    quad_order: int
    sipg_gamma: float      # SIPG penalty  = sipg_gamma / h
    nitsche_gamma: float   # Nitsche penalty = nitsche_gamma / h
    gp_max_order: int      # J: ghost penalty on jumps of d^j/dn^j, j = 1..J
    gp_gamma: float        # gamma_j = gp_gamma * h^(2j-1) / (j!)^2
    kappa: np.ndarray = None  # per active cell diffusion coefficient (None = 1)
    ls_kind: str = "sphere"
    normal: tuple = None      # plane: phi(x) = normal . x - offset
    offset: float = 0.0
    gp_kind: str = "face"     # "face": jumps of normal derivatives on faces; "volume": patch jumps
    gp_tau: float = 1.0       # volume ghost penalty parameter tau_v
    spheres: tuple = None     # "spheres": ((cx, cy, cz, R), ...), the union of these balls
    # derived
    h: float = field(init=False)

    def __post_init__(self):
        d = self.dim
        self.n_cells = tuple(int(v) for v in self.n_cells[:d])
        self.lo = tuple(float(v) for v in self.lo[:d])
        self.hi = tuple(float(v) for v in self.hi[:d])
        self.center = tuple(float(v) for v in self.center[:d])
        if self.gp_kind not in ("face", "volume"):
            raise ValueError("gp_kind must be 'face' or 'volume'")
        if self.ls_kind not in ("sphere", "plane", "spheres"):
            raise ValueError("ls_kind must be 'sphere', 'plane' or 'spheres'")
        if self.ls_kind == "spheres":
            self.spheres = tuple((tuple(float(v) for v in sp[:d]), float(sp[3])) for sp in self.spheres)
        if self.ls_kind == "plane":
            self.normal = tuple(float(v) for v in self.normal[:d])
            self.offset = float(self.offset)
            if not any(v != 0.0 for v in self.normal):
                raise ValueError("the plane normal must not vanish")
        hs = [(self.hi[a] - self.lo[a]) / self.n_cells[a] for a in range(d)]
        if max(hs) - min(hs) > 1e-14 * max(hs):
            raise ValueError("the oracle needs a uniform (isotropic) background grid")
        self.hvec = tuple(hs)
        self.h = hs[0]

    @property
    def n(self):
        return self.degree + 1

    @property
    def dofs_per_cell(self):
        return self.n ** self.dim


def problem_from_dict(cfg, kappa=None):
    keys = ["dim", "degree", "n_cells", "lo", "hi", "center", "radius", "quad_order",
            "sipg_gamma", "nitsche_gamma", "gp_max_order", "gp_gamma"]
    extra = {k: cfg[k] for k in ("ls_kind", "normal", "offset", "gp_kind", "gp_tau", "spheres")
             if k in cfg}
    return Problem(**{k: cfg[k] for k in keys}, kappa=kappa, **extra)


def cell_box(prob, idx):
    lo = tuple(prob.lo[a] + idx[a] * prob.hvec[a] for a in range(prob.dim))
    hi = tuple(prob.lo[a] + (idx[a] + 1) * prob.hvec[a] for a in range(prob.dim))
    return lo, hi


class Mesh:
    """Classification and numbering of the background grid of `prob`."""

    def __init__(self, prob):
        self.prob = prob
        d = prob.dim
        N = prob.n_cells
        # Elementwise the same arithmetic as `classify_box`, vectorised over all background cells.
        # Arrays are indexed [k][j][i] (x index fastest in C order).
        shape = tuple(N[::-1])
        dmin2 = np.zeros(shape)
        dmax2 = np.zeros(shape)
        for a in range(d):
            idx = np.arange(N[a], dtype=np.float64)
            lo = prob.lo[a] + idx * prob.hvec[a]
            hi = prob.lo[a] + (idx + 1) * prob.hvec[a]
            bshape = [1] * d
            bshape[d - 1 - a] = N[a]
            if prob.ls_kind == "plane":
                # (min, max) of n . x over the cell, as in saye.lin_range
                na = prob.normal[a]
                lo_t, hi_t = (na * lo, na * hi) if na >= 0.0 else (na * hi, na * lo)
                dmin2 = dmin2 + lo_t.reshape(bshape)
                dmax2 = dmax2 + hi_t.reshape(bshape)
                continue
            dl = lo - prob.center[a]
            dh = hi - prob.center[a]
            e = np.maximum(np.maximum(dl, 0.0), -dh)
            dmin2 = dmin2 + (e * e).reshape(bshape)
            dmax2 = dmax2 + np.maximum(dl * dl, dh * dh).reshape(bshape)
        if prob.ls_kind == "spheres":
            t = self._classify_spheres(prob)
        else:
            t = np.full(shape, CUT, dtype=np.int8)
        if prob.ls_kind == "spheres":
            pass
        elif prob.ls_kind == "plane":
            t[dmin2 - prob.offset >= 0.0] = OUTSIDE
            t[dmax2 - prob.offset <= 0.0] = INSIDE
        else:
            r2 = prob.radius * prob.radius
            t[dmin2 >= r2] = OUTSIDE
            t[dmax2 <= r2] = INSIDE
        self.cell_type = t
        act = np.nonzero(t.reshape(-1) != OUTSIDE)[0]
        self.id_map = np.full(t.size, -1, dtype=np.int64)
        self.id_map[act] = np.arange(len(act))
        self.id_map = self.id_map.reshape(shape)
        multi = np.unravel_index(act, shape)          # (k, j, i) order
        self.active_idx = np.stack(multi[::-1], axis=1)  # columns i, j, k
        self.active_type = t.reshape(-1)[act]
        self.n_active = len(act)
        self.n_dofs = self.n_active * prob.dofs_per_cell
        if prob.kappa is None:
            self.kappa = np.ones(self.n_active)
        else:
            self.kappa = np.asarray(prob.kappa, dtype=np.float64)
            assert self.kappa.shape == (self.n_active,)

    @staticmethod
    def _classify_spheres(prob):
        """Cell types of a union of balls: each ball updates the cells of its bounding box with
        the arithmetic of classify_box (inside if one ball contains the cell, cut if a sphere
        meets it)."""
        d = prob.dim
        N = prob.n_cells
        shape = tuple(N[::-1])
        inside = np.zeros(shape, dtype=bool)
        count = np.zeros(shape, dtype=np.int32)
        for (c, R) in prob.spheres:
            rng = []
            for a in range(d):
                i0 = max(0, int(math.floor((c[a] - R - prob.lo[a]) / prob.hvec[a])) - 1)
                i1 = min(N[a], int(math.floor((c[a] + R - prob.lo[a]) / prob.hvec[a])) + 2)
                rng.append((i0, i1))
            if any(i1 <= i0 for i0, i1 in rng):
                continue
            sub = tuple(i1 - i0 for i0, i1 in rng)[::-1]
            dmin2 = np.zeros(sub)
            dmax2 = np.zeros(sub)
            for a in range(d):
                idx = np.arange(rng[a][0], rng[a][1], dtype=np.float64)
                lo = prob.lo[a] + idx * prob.hvec[a]
                hi = prob.lo[a] + (idx + 1) * prob.hvec[a]
                dl = lo - c[a]
                dh = hi - c[a]
                e = np.maximum(np.maximum(dl, 0.0), -dh)
                bshape = [1] * d
                bshape[d - 1 - a] = len(idx)
                dmin2 = dmin2 + (e * e).reshape(bshape)
                dmax2 = dmax2 + np.maximum(dl * dl, dh * dh).reshape(bshape)
            sl = tuple(slice(i0, i1) for i0, i1 in rng)[::-1]
            r2 = R * R
            inside[sl] |= dmax2 <= r2
            count[sl] += ((dmin2 < r2) & (dmax2 > r2)).astype(np.int32)
        t = np.full(shape, OUTSIDE, dtype=np.int8)
        t[count >= 1] = CUT
        t[inside] = INSIDE
        return t

    @property
    def active(self):
        return [tuple(int(v) for v in row) for row in self.active_idx]

    def index_of(self, e):
        return tuple(int(v) for v in self.active_idx[e])

    def neighbor(self, e, axis, side):
        """Active id of the face neighbour of active cell e across (axis, side), or -1.

        side = 0: lower face (neighbour at index - 1); side = 1: upper face.
        """
        idx = list(self.index_of(e))
        idx[axis] += 1 if side == 1 else -1
        if idx[axis] < 0 or idx[axis] >= self.prob.n_cells[axis]:
            return -1
        return int(self.id_map[tuple(idx[::-1])])

    def face_box(self, e_minus, axis):
        """The shared face between e_minus and its upper neighbour along `axis` (a degenerate
        d-dimensional box with lo[axis] == hi[axis])."""
        lo, hi = cell_box(self.prob, self.index_of(e_minus))
        lo = list(lo)
        hi = list(hi)
        lo[axis] = hi[axis]
        return tuple(lo), tuple(hi)

    def face_type(self, e_minus, axis):
        lo, hi = self.face_box(e_minus, axis)
        t = classify(self.prob, lo, hi)
        return {INSIDE: FACE_FULL, CUT: FACE_CUT, OUTSIDE: FACE_EMPTY}[t]

    def interior_faces(self):
        """All faces between two active cells: list of (e_minus, e_plus, axis, face_type, gp)."""
        faces = []
        for e in range(self.n_active):
            for axis in range(self.prob.dim):
                ep = self.neighbor(e, axis, 1)
                if ep < 0:
                    continue
                gp = bool(self.active_type[e] == CUT or self.active_type[ep] == CUT)
                faces.append((e, ep, axis, self.face_type(e, axis), gp))
        return faces

    def counts(self):
        faces = self.interior_faces()
        return {
            "n_active": self.n_active,
            "n_inside": int(np.sum(self.active_type == INSIDE)),
            "n_cut": int(np.sum(self.active_type == CUT)),
            "n_faces": len(faces),
            "n_faces_full": sum(1 for f in faces if f[3] == FACE_FULL),
            "n_faces_cut": sum(1 for f in faces if f[3] == FACE_CUT),
            "n_faces_empty": sum(1 for f in faces if f[3] == FACE_EMPTY),
            "n_faces_gp": sum(1 for f in faces if f[4]),
        }
