"""Dimension-reduction quadrature for sphere, plane and union-of-balls level sets (oracle; test
infrastructure only).

The paper generates the cut-cell (volume, surface) and cut-face rules with the dimension
reduction method of Saye (2015) (Sec. 1, Sec. 2.3) and adds uniform subdivision when needed
(Sec. 5.1, arithmetic-complexity paragraph on refined cut cells).  The paper states no details, so
this module restates the method for level sets of the form psi(x) = |x - c|^2 - rho, for which
every root along a coordinate line has a closed form.  This fixes one deterministic rule (the
CUDA library's host setup implements the same reading independently):

  volume / surface rule on a box U (dimension m) for {psi < 0} / {psi = 0}:
    1. U inside (dmax^2 <= rho): tensor Gauss rule with q points per direction (volume only);
       U outside (dmin^2 >= rho): nothing.
    2. height direction k = argmax_i |mid_i - c_i| (lowest index on ties), mid = (lo + hi) / 2.
       psi is strictly monotone along k on U unless lo_k < c_k < hi_k; in that case U is bisected
       in every direction and each child is treated from step 1 (depth <= MAX_DEPTH).
    3. the outer rule is the full-box rule (below) on U' = U without direction k, for the two
       restrictions psi(., lo_k), psi(., hi_k) (same centre, rho - (lo_k - c_k)^2 and
       rho - (hi_k - c_k)^2): the line integrals along k are smooth in x' away from their zero
       sets, which the full-box rule uses as break points.
    4. for each outer point (x', w'): the root t of psi(x', t) = 0 in the open interval
       (lo_k, hi_k) (t = c_k + s if c_k <= lo_k, else c_k - s, s = sqrt(rho - |x' - c'|^2)) splits
       [lo_k, hi_k]; every piece whose midpoint has psi < 0 gets q Gauss points (volume weight
       w' * len * w_i); the root itself is a surface point with weight w' * R / |t - c_k|
       (= w' |grad phi| / |d_k phi| with R = sqrt(rho)) and unit normal (x - c) / |x - c|.
  full-box rule on B (dimension m) with break functions {psi_f}:
    drop every psi_f that is one-signed on B; if none is left, tensor Gauss q^m.  If m = 1, split B
    at all roots c +- sqrt(rho) in (lo, hi) and put q Gauss points on each piece.  Otherwise choose
    k as in step 2 (bisect B in all directions if lo_k < c_k < hi_k), recurse on B' = B without k
    with the restrictions of every kept psi_f to x_k = lo_k and x_k = hi_k, and along each outer
    line split [lo_k, hi_k] at the roots of the kept psi_f and put q Gauss points on every piece.

Conventions that make the rule reproducible bit for bit: sums of squares run over coordinate
directions in increasing index order; children of a bisection are ordered with direction 0
fastest; tensor rules are ordered with direction 0 fastest; pieces and roots ascend; a point's
weight is w' * ((b - a) * w_i) and a tensor weight is the running product of (hi_a - lo_a) * w_a
over a = 0, 1, ...; pieces of zero length are dropped.
"""
import math

from . import basis

MAX_DEPTH = 8


class QuadratureError(RuntimeError):
    pass


_GAUSS_CACHE = {}


def gauss01(q):
    if q not in _GAUSS_CACHE:
        g, w = basis.gauss_legendre(q)
        _GAUSS_CACHE[q] = ([float(v) for v in g], [float(v) for v in w])
    return _GAUSS_CACHE[q]


def _box_dist2(c, lo, hi):
    dmin2 = 0.0
    dmax2 = 0.0
    for a in range(len(c)):
        dl = lo[a] - c[a]
        dh = hi[a] - c[a]
        e = max(max(dl, 0.0), -dh)
        dmin2 += e * e
        dmax2 += max(dl * dl, dh * dh)
    return dmin2, dmax2


def tensor_gauss(lo, hi, q):
    g, w = gauss01(q)
    m = len(lo)
    out = []
    for flat in range(q ** m):
        x = []
        wt = 1.0
        rem = flat
        for a in range(m):
            i = rem % q
            rem //= q
            x.append(lo[a] + (hi[a] - lo[a]) * g[i])
            wt *= (hi[a] - lo[a]) * w[i]
        out.append((tuple(x), wt))
    return out


def _children(lo, hi):
    m = len(lo)
    mid = [0.5 * (lo[a] + hi[a]) for a in range(m)]
    for bits in range(2 ** m):
        clo = []
        chi = []
        for a in range(m):
            if (bits >> a) & 1:
                clo.append(mid[a])
                chi.append(hi[a])
            else:
                clo.append(lo[a])
                chi.append(mid[a])
        yield tuple(clo), tuple(chi)


def _height_direction(c, lo, hi):
    k = 0
    best = -1.0
    for i in range(len(lo)):
        v = abs(0.5 * (lo[i] + hi[i]) - c[i])
        if v > best:
            best = v
            k = i
    return k


def _drop(t, k):
    return tuple(t[i] for i in range(len(t)) if i != k)


def _insert(t, k, v):
    return tuple(t[:k]) + (v,) + tuple(t[k:])


def _dist2_excl(x, c):
    r = 0.0
    for i in range(len(x)):
        d = x[i] - c[i]
        r += d * d
    return r


def _pieces(a, b, roots):
    brk = [a] + sorted(roots) + [b]
    return [(brk[i], brk[i + 1]) for i in range(len(brk) - 1) if brk[i + 1] > brk[i]]


def full_rule(lo, hi, fns, q, depth=0):
    """Rule for the whole box [lo, hi] whose pieces break at the zero sets of `fns`.

    fns: list of (c, rho), all with the same centre c, psi = |x - c|^2 - rho.
    """
    m = len(lo)
    keep = []
    for (c, rho) in fns:
        dmin2, dmax2 = _box_dist2(c, lo, hi)
        if not (dmin2 >= rho or dmax2 <= rho):
            keep.append((c, rho))
    if not keep:
        return tensor_gauss(lo, hi, q)
    g, w = gauss01(q)
    c = keep[0][0]
    if m == 1:
        roots = []
        for (cf, rho) in keep:
            s = math.sqrt(rho)
            for t in (cf[0] - s, cf[0] + s):
                if lo[0] < t < hi[0]:
                    roots.append(t)
        out = []
        for (a, b) in _pieces(lo[0], hi[0], roots):
            for i in range(q):
                out.append(((a + (b - a) * g[i],), (b - a) * w[i]))
        return out
    k = _height_direction(c, lo, hi)
    if lo[k] < c[k] < hi[k]:
        if depth >= MAX_DEPTH:
            raise QuadratureError("subdivision depth exceeded")
        out = []
        for clo, chi in _children(lo, hi):
            out += full_rule(clo, chi, keep, q, depth + 1)
        return out
    csub = _drop(c, k)
    dl = lo[k] - c[k]
    dh = hi[k] - c[k]
    fns2 = []
    for (cf, rho) in keep:
        fns2.append((csub, rho - dl * dl))
        fns2.append((csub, rho - dh * dh))
    outer = full_rule(_drop(lo, k), _drop(hi, k), fns2, q, depth)
    up = c[k] <= lo[k]
    out = []
    for (xp, wp) in outer:
        r = _dist2_excl(xp, csub)
        roots = []
        for (cf, rho) in keep:
            r2 = rho - r
            if r2 > 0.0:
                s = math.sqrt(r2)
                t = c[k] + s if up else c[k] - s
                if lo[k] < t < hi[k]:
                    roots.append(t)
        for (a, b) in _pieces(lo[k], hi[k], roots):
            for i in range(q):
                out.append((_insert(xp, k, a + (b - a) * g[i]), wp * ((b - a) * w[i])))
    return out


def sphere_rules(lo, hi, c, rho, q, depth=0, surface=True):
    """Volume rule for {psi < 0} cap [lo, hi] and (if `surface`) the surface rule for {psi = 0}.

    Returns (volume, surface): volume = list of (x, w); surface = list of (x, w, normal).
    """
    m = len(lo)
    dmin2, dmax2 = _box_dist2(c, lo, hi)
    if dmax2 <= rho:
        return tensor_gauss(lo, hi, q), []
    if dmin2 >= rho:
        return [], []
    g, w = gauss01(q)
    if m == 1:
        s = math.sqrt(rho)
        roots = [t for t in (c[0] - s, c[0] + s) if lo[0] < t < hi[0]]
        vol = []
        for (a, b) in _pieces(lo[0], hi[0], roots):
            mid = 0.5 * (a + b)
            if (mid - c[0]) * (mid - c[0]) - rho < 0.0:
                for i in range(q):
                    vol.append(((a + (b - a) * g[i],), (b - a) * w[i]))
        surf = [((t,), 1.0, (1.0 if t > c[0] else -1.0,)) for t in roots] if surface else []
        return vol, surf
    k = _height_direction(c, lo, hi)
    if lo[k] < c[k] < hi[k]:
        if depth >= MAX_DEPTH:
            raise QuadratureError("subdivision depth exceeded")
        vol = []
        surf = []
        for clo, chi in _children(lo, hi):
            v, s = sphere_rules(clo, chi, c, rho, q, depth + 1, surface)
            vol += v
            surf += s
        return vol, surf
    csub = _drop(c, k)
    dl = lo[k] - c[k]
    dh = hi[k] - c[k]
    outer = full_rule(_drop(lo, k), _drop(hi, k), [(csub, rho - dl * dl), (csub, rho - dh * dh)], q)
    up = c[k] <= lo[k]
    R = math.sqrt(rho)
    vol = []
    surf = []
    for (xp, wp) in outer:
        r = _dist2_excl(xp, csub)
        r2 = rho - r
        t = None
        if r2 > 0.0:
            s = math.sqrt(r2)
            tt = c[k] + s if up else c[k] - s
            if lo[k] < tt < hi[k]:
                t = tt
        for (a, b) in _pieces(lo[k], hi[k], [] if t is None else [t]):
            mid = 0.5 * (a + b)
            dm = mid - c[k]
            if (r + dm * dm) - rho < 0.0:
                for i in range(q):
                    vol.append((_insert(xp, k, a + (b - a) * g[i]), wp * ((b - a) * w[i])))
        if surface and t is not None:
            x = _insert(xp, k, t)
            nrm = math.sqrt(_dist2_excl(x, c))
            normal = tuple((x[i] - c[i]) / nrm for i in range(m))
            surf.append((x, wp * (R / abs(t - c[k])), normal))
    return vol, surf


# ------------------------------------------------------------------------------------------
# Plane level sets psi(x) = sum_a n_a x_a - off (n != 0; Omega = {psi < 0})
# ------------------------------------------------------------------------------------------
#
# The same method for a linear level set: psi is monotone along every direction with n_k != 0,
# so no bisection is needed.  Height direction k = argmax |n_i| (lowest index on ties); the
# restriction of psi to x_k = v is linear again, (n without k, off - n_k v); the root on the
# line through x' is t = (off - s) / n_k with s = sum_{a != k} n_a x'_a (increasing a); a
# surface point has weight w' |n| / |n_k| (= w' |grad phi| / |d_k phi|) and normal n / |n|.
# Sums run over coordinate directions in increasing index order.


def lin_range(n, off, lo, hi):
    """(min, max) of sum_a n_a x_a - off over the closed box [lo, hi]."""
    mn = 0.0
    mx = 0.0
    for a in range(len(n)):
        if n[a] >= 0.0:
            mn += n[a] * lo[a]
            mx += n[a] * hi[a]
        else:
            mn += n[a] * hi[a]
            mx += n[a] * lo[a]
    return mn - off, mx - off


def _lin_height(n):
    k = 0
    best = -1.0
    for i in range(len(n)):
        v = abs(n[i])
        if v > best:
            best = v
            k = i
    return k


def _lin_sum_excl(n, k, xp):
    """sum_{a != k} n_a x'_a, x' = the coordinates without direction k, increasing a."""
    s = 0.0
    j = 0
    for a in range(len(n)):
        if a == k:
            continue
        s += n[a] * xp[j]
        j += 1
    return s


def full_rule_linear(lo, hi, fns, q):
    """Rule for the whole box [lo, hi] whose pieces break at the zero sets of the linear
    functions `fns` (list of (n, off), all with the same n)."""
    m = len(lo)
    keep = []
    for (n, off) in fns:
        mn, mx = lin_range(n, off, lo, hi)
        if not (mn >= 0.0 or mx <= 0.0):
            keep.append((n, off))
    if not keep:
        return tensor_gauss(lo, hi, q)
    g, w = gauss01(q)
    n = keep[0][0]
    if m == 1:
        roots = []
        for (nf, off) in keep:
            t = off / nf[0]
            if lo[0] < t < hi[0]:
                roots.append(t)
        out = []
        for (a, b) in _pieces(lo[0], hi[0], roots):
            for i in range(q):
                out.append(((a + (b - a) * g[i],), (b - a) * w[i]))
        return out
    k = _lin_height(n)
    nsub = _drop(n, k)
    fns2 = []
    for (nf, off) in keep:
        fns2.append((nsub, off - n[k] * lo[k]))
        fns2.append((nsub, off - n[k] * hi[k]))
    outer = full_rule_linear(_drop(lo, k), _drop(hi, k), fns2, q)
    out = []
    for (xp, wp) in outer:
        s = _lin_sum_excl(n, k, xp)
        roots = []
        for (nf, off) in keep:
            t = (off - s) / n[k]
            if lo[k] < t < hi[k]:
                roots.append(t)
        for (a, b) in _pieces(lo[k], hi[k], roots):
            for i in range(q):
                out.append((_insert(xp, k, a + (b - a) * g[i]), wp * ((b - a) * w[i])))
    return out


def plane_rules(lo, hi, n, off, q, surface=True):
    """Volume rule for {psi < 0} cap [lo, hi] and (if `surface`) the surface rule for {psi = 0},
    psi(x) = sum_a n_a x_a - off.  Returns (volume, surface) as sphere_rules does."""
    m = len(lo)
    mn, mx = lin_range(n, off, lo, hi)
    if mx <= 0.0:
        return tensor_gauss(lo, hi, q), []
    if mn >= 0.0:
        return [], []
    g, w = gauss01(q)
    nn = 0.0
    for a in range(m):
        nn += n[a] * n[a]
    nn = math.sqrt(nn)
    if m == 1:
        t = off / n[0]
        roots = [t] if lo[0] < t < hi[0] else []
        vol = []
        for (a, b) in _pieces(lo[0], hi[0], roots):
            mid = 0.5 * (a + b)
            if n[0] * mid - off < 0.0:
                for i in range(q):
                    vol.append(((a + (b - a) * g[i],), (b - a) * w[i]))
        surf = [((t,), 1.0, (1.0 if n[0] > 0.0 else -1.0,)) for t in roots] if surface else []
        return vol, surf
    k = _lin_height(n)
    nsub = _drop(n, k)
    outer = full_rule_linear(_drop(lo, k), _drop(hi, k),
                             [(nsub, off - n[k] * lo[k]), (nsub, off - n[k] * hi[k])], q)
    vol = []
    surf = []
    for (xp, wp) in outer:
        s = _lin_sum_excl(n, k, xp)
        tt = (off - s) / n[k]
        t = tt if lo[k] < tt < hi[k] else None
        for (a, b) in _pieces(lo[k], hi[k], [] if t is None else [t]):
            mid = 0.5 * (a + b)
            if (s + n[k] * mid) - off < 0.0:
                for i in range(q):
                    vol.append((_insert(xp, k, a + (b - a) * g[i]), wp * ((b - a) * w[i])))
        if surface and t is not None:
            x = _insert(xp, k, t)
            normal = tuple(n[i] / nn for i in range(m))
            surf.append((x, wp * (nn / abs(n[k])), normal))
    return vol, surf


# ------------------------------------------------------------------------------------------
# Unions of balls: psi(x) = min_i psi_i(x), psi_i = |x - c_i|^2 - rho_i (Sec. 6: the union of
# spheres is the minimum of their level sets)
# ------------------------------------------------------------------------------------------
#
# Balls may intersect.  Along a coordinate line the union is the union of the balls' intervals,
# so the inner integrals stay exact; the outer integrand is smooth except where an interval
# starts or ends at the box, where two spheres' endpoints meet (the intersection circle of the
# two spheres, seen along the height direction) or where three such events meet at one point.
# The rule splits the outer integration at all of them, all in closed form:
#
#   box U (dimension m) with the balls S whose sphere meets the closed box (none contains U):
#     |S| = 0: empty; one ball contains U: tensor Gauss; |S| = 1: sphere_rules (unchanged).
#     m = 1: split [lo, hi] at every root c_i +- sqrt(rho_i) in (lo, hi); pieces whose midpoint
#       lies in a ball get q Gauss points (no surface rule: 1D boxes are faces here).
#     m >= 2: height direction k valid if no centre has lo_k < c_ik < hi_k; among the valid k the
#       one maximising min_i |mid_k - c_ik| (first on ties).  None valid: bisect in every
#       direction (children from the top, depth <= MAX_DEPTH); at MAX_DEPTH, the k maximising
#       the same quantity without the validity test.
#     outer rule on U' = U without k:
#       m = 2 (U' an interval): break points = roots of psi_i(., lo_k), psi_i(., hi_k), the
#         intersection points of every pair of circles, and (invalid k only) the silhouettes
#         c_i' +- R_i; pieces get q Gauss points.
#       m = 3 (U' a rectangle): break curves = the circles psi_i(., lo_k) = 0, psi_i(., hi_k) = 0
#         (and, invalid k only, the silhouettes |x' - c_i'| = R_i), and the intersection circle
#         of every pair of spheres whose bounding box overlaps the open U, projected along k;
#         break points = the intersection circles' points on the planes x_k = lo_k, hi_k and the
#         triple points of three spheres.  Rule of the rectangle B with these: keep the
#         2D circles that cross B and the 3D circles whose bounding box overlaps the open B (no
#         curve: tensor Gauss); line direction a: the points of a curve with tangent along a
#         (2D circle: (C_o +- r, C_a); 3D circle: its two points of extremal x_o) must lie
#         outside the open B (a 3D circle whose plane is normal to o within 1e-12 fails); among
#         the directions where all do, the one whose nearest such point (squared distance to
#         B, minimum over the kept curves) is farthest, a = 0 on ties; if none, bisect B in both
#         directions (depth <= MAX_DEPTH; at MAX_DEPTH a = 0).
#         o = the other direction; split (lo_o, hi_o) at the kept curves' points on the edges
#         x_a = lo_a, hi_a and at the break points' o-coordinates; q Gauss points per piece; on
#         each line x_o split (lo_a, hi_a) at the kept curves' points; q Gauss points per piece.
#     line through each outer point (x', w'): the intervals (c_ik - s_i, c_ik + s_i) cut to
#       [lo_k, hi_k] (s_i = sqrt(rho_i - |x' - c_i'|^2) where positive), sorted by start (ball
#       order on ties) and merged when they overlap or touch; every merged interval gets q Gauss
#       points; its start (end) is a surface point of the ball that starts (first reaches) it,
#       unless it lies on the box, with weight w' R_i / |t - c_ik| and normal (x - c_i) / |x - c_i|.
#       Surface points of a line ascend.
#
# Helpers on circles in 3D: the intersection circle of spheres i, j has centre q = c_i + a nu,
# nu = (c_j - c_i) / D, a = (D^2 + rho_i - rho_j) / (2 D), radius^2 rc2 = rho_i - a^2 (no
# circle if rc2 <= 0 or D = 0).  A plane mu . x = h meets it where the line of the two planes
# does: with mn = mu . nu, den = |mu|^2 - mn^2 (none if den <= 1e-24 |mu|^2),
# lam = (h - mu . q) / den, p0 = q + lam (mu - mn nu), s^2 = rc2 - lam^2 den (none if < 0), the
# points p0 -+ s (nu x mu) / sqrt(den).  Triple points of spheres i < j < l: the circle (i, j)
# on the radical plane 2 (c_l - c_i) . x = |c_l|^2 - |c_i|^2 - rho_l + rho_i.  Sums over
# coordinates run in increasing index order.


def _ball_status(balls, lo, hi):
    """(contained, S) of the closed box: contained if one ball contains it; S = indices of the
    balls whose sphere meets it (dmin^2 < rho < dmax^2), ascending."""
    contained = False
    S = []
    for i, (c, rho) in enumerate(balls):
        dmin2, dmax2 = _box_dist2(c, lo, hi)
        if dmax2 <= rho:
            contained = True
        elif dmin2 < rho:
            S.append(i)
    return contained, S


def _dot(u, v):
    r = 0.0
    for a in range(len(u)):
        r += u[a] * v[a]
    return r


def _pair_circle(ci, rhoi, cj, rhoj):
    """Intersection circle (q, nu, rc2) of two spheres (3D), or None."""
    dv = tuple(cj[a] - ci[a] for a in range(3))
    D2 = _dot(dv, dv)
    if D2 == 0.0:
        return None
    D = math.sqrt(D2)
    nu = tuple(dv[a] / D for a in range(3))
    a0 = (D2 + rhoi - rhoj) / (2.0 * D)
    rc2 = rhoi - a0 * a0
    if rc2 <= 0.0:
        return None
    return tuple(ci[a] + a0 * nu[a] for a in range(3)), nu, rc2


def _circle_plane(circ, mu, h):
    """Points of the circle (q, nu, rc2) on the plane mu . x = h (0 or 2 points)."""
    q, nu, rc2 = circ
    mn = _dot(mu, nu)
    mm = _dot(mu, mu)
    den = mm - mn * mn
    if den <= 1e-24 * mm:
        return []
    lam = (h - _dot(mu, q)) / den
    p0 = tuple(q[a] + lam * (mu[a] - mn * nu[a]) for a in range(3))
    s2 = rc2 - lam * lam * den
    if s2 < 0.0:
        return []
    ell = (nu[1] * mu[2] - nu[2] * mu[1], nu[2] * mu[0] - nu[0] * mu[2], nu[0] * mu[1] - nu[1] * mu[0])
    f = math.sqrt(s2) / math.sqrt(den)
    return [tuple(p0[a] - f * ell[a] for a in range(3)), tuple(p0[a] + f * ell[a] for a in range(3))]


def _axis_plane(A):
    return tuple(1.0 if a == A else 0.0 for a in range(3))


def _circle_halfwidth(circ, A):
    q, nu, rc2 = circ
    return math.sqrt(rc2) * math.sqrt(max(0.0, 1.0 - nu[A] * nu[A]))


def _circle_overlaps(circ, axes, lo, hi):
    """Bounding box of the circle overlaps the open box (lo, hi) in the listed 3D axes."""
    q = circ[0]
    for j, A in enumerate(axes):
        hw = _circle_halfwidth(circ, A)
        if not (q[A] - hw < hi[j] and q[A] + hw > lo[j]):
            return False
    return True


def _in_open(x, lo, hi):
    for a in range(len(lo)):
        if not (lo[a] < x[a] < hi[a]):
            return False
    return True


def _tangent_clearance(curve, a, axes, lo, hi):
    """Squared distance from the rectangle to the curve's points with tangent along direction a
    (the smaller of the two); 0 if one lies inside the open rectangle."""
    o = 1 - a
    pts = []
    if curve[0] == "c2":
        _, C, r2 = curve
        r = math.sqrt(r2)
        for t in (C[o] - r, C[o] + r):
            x = [0.0, 0.0]
            x[a] = C[a]
            x[o] = t
            pts.append(tuple(x))
    else:
        q, nu, rc2 = curve[1]
        O = axes[o]
        den = 1.0 - nu[O] * nu[O]
        if den <= 1e-12:
            return 0.0
        rc = math.sqrt(rc2)
        sd = math.sqrt(den)
        for sgn in (-1.0, 1.0):
            p = tuple(q[b] + sgn * rc * (((1.0 if b == O else 0.0) - nu[O] * nu[b]) / sd)
                      for b in range(3))
            pts.append((p[axes[0]], p[axes[1]]))
    best = math.inf
    for x in pts:
        if _in_open(x, lo, hi):
            return 0.0
        best = min(best, _box_dist2(x, lo, hi)[0])
    return best


def _curve_points_at(curve, along, v, axes):
    """Coordinates, in direction 1 - along of the rectangle, of the curve's points with
    coordinate `along` equal to v."""
    other = 1 - along
    if curve[0] == "c2":
        _, C, r2 = curve
        rr = r2 - (v - C[along]) * (v - C[along])
        if rr <= 0.0:
            return []
        s = math.sqrt(rr)
        return [C[other] - s, C[other] + s]
    pts = _circle_plane(curve[1], _axis_plane(axes[along]), v)
    return [p[axes[other]] for p in pts]


def _curve_rule_2d(lo, hi, curves, points, axes, q, depth=0):
    """Rule on the rectangle [lo, hi] whose pieces break at `curves` (("c2", centre, r^2) circles
    in the rectangle's coordinates, ("c3", circle) circles in 3D seen along the dropped axis)
    and at the 2D `points`; axes = the 3D axes of the rectangle's two directions."""
    keep = []
    for cv in curves:
        if cv[0] == "c2":
            dmin2, dmax2 = _box_dist2(cv[1], lo, hi)
            if dmin2 < cv[2] < dmax2:
                keep.append(cv)
        elif _circle_overlaps(cv[1], axes, lo, hi):
            keep.append(cv)
    if not keep:
        return tensor_gauss(lo, hi, q)
    a = None
    best = 0.0
    for cand in (0, 1):
        v = min(_tangent_clearance(cv, cand, axes, lo, hi) for cv in keep)
        if v > best:
            best = v
            a = cand
    if a is None:
        if depth < MAX_DEPTH:
            out = []
            for clo, chi in _children(lo, hi):
                out += _curve_rule_2d(clo, chi, keep, points, axes, q, depth + 1)
            return out
        a = 0
    o = 1 - a
    g, w = gauss01(q)
    splits = []
    for cv in keep:
        for v in (lo[a], hi[a]):
            for t in _curve_points_at(cv, a, v, axes):
                if lo[o] < t < hi[o]:
                    splits.append(t)
    for p in points:
        if lo[o] < p[o] < hi[o]:
            splits.append(p[o])
    out = []
    for (ao, bo) in _pieces(lo[o], hi[o], splits):
        for io in range(q):
            xo = ao + (bo - ao) * g[io]
            wo = (bo - ao) * w[io]
            roots = []
            for cv in keep:
                for t in _curve_points_at(cv, o, xo, axes):
                    if lo[a] < t < hi[a]:
                        roots.append(t)
            for (aa, ba) in _pieces(lo[a], hi[a], roots):
                for i in range(q):
                    x = [0.0, 0.0]
                    x[o] = xo
                    x[a] = aa + (ba - aa) * g[i]
                    out.append((tuple(x), wo * ((ba - aa) * w[i])))
    return out


def _union_height(act, lo, hi, check):
    k = None
    best = -1.0
    for kk in range(len(lo)):
        if check and any(lo[kk] < c[kk] < hi[kk] for c, _ in act):
            continue
        v = min(abs(0.5 * (lo[kk] + hi[kk]) - c[kk]) for c, _ in act)
        if v > best:
            best = v
            k = kk
    return k


def _union_outer(lo, hi, act, k, valid, q):
    m = len(lo)
    g, w = gauss01(q)
    if m == 2:
        a = 1 - k
        splits = []
        for (c, rho) in act:
            for v in (lo[k], hi[k]):
                r2 = rho - (v - c[k]) * (v - c[k])
                if r2 > 0.0:
                    s = math.sqrt(r2)
                    for t in (c[a] - s, c[a] + s):
                        if lo[a] < t < hi[a]:
                            splits.append(t)
            if not valid and lo[k] < c[k] < hi[k]:
                R = math.sqrt(rho)
                for t in (c[a] - R, c[a] + R):
                    if lo[a] < t < hi[a]:
                        splits.append(t)
        for i in range(len(act)):
            for j in range(i + 1, len(act)):
                ci, rhoi = act[i]
                cj, rhoj = act[j]
                dv = (cj[0] - ci[0], cj[1] - ci[1])
                D2 = dv[0] * dv[0] + dv[1] * dv[1]
                if D2 == 0.0:
                    continue
                D = math.sqrt(D2)
                nu = (dv[0] / D, dv[1] / D)
                a0 = (D2 + rhoi - rhoj) / (2.0 * D)
                rc2 = rhoi - a0 * a0
                if rc2 <= 0.0:
                    continue
                rc = math.sqrt(rc2)
                qc = (ci[0] + a0 * nu[0], ci[1] + a0 * nu[1])
                for sgn in (-1.0, 1.0):
                    p = (qc[0] - sgn * rc * nu[1], qc[1] + sgn * rc * nu[0])
                    if lo[a] < p[a] < hi[a]:
                        splits.append(p[a])
        out = []
        for (pa, pb) in _pieces(lo[a], hi[a], splits):
            for i in range(q):
                out.append(((pa + (pb - pa) * g[i],), (pb - pa) * w[i]))
        return out
    axes = tuple(b for b in range(3) if b != k)
    curves = []
    for (c, rho) in act:
        cp = _drop(c, k)
        for v in (lo[k], hi[k]):
            r2 = rho - (v - c[k]) * (v - c[k])
            if r2 > 0.0:
                curves.append(("c2", cp, r2))
        if not valid and lo[k] < c[k] < hi[k]:
            curves.append(("c2", cp, rho))
    circles = {}
    for i in range(len(act)):
        for j in range(i + 1, len(act)):
            circ = _pair_circle(act[i][0], act[i][1], act[j][0], act[j][1])
            if circ is not None and _circle_overlaps(circ, (0, 1, 2), lo, hi):
                circles[(i, j)] = circ
                curves.append(("c3", circ))
    pts3 = []
    for (i, j), circ in circles.items():
        for v in (lo[k], hi[k]):
            pts3 += _circle_plane(circ, _axis_plane(k), v)
        for l in range(j + 1, len(act)):
            ci, rhoi = act[i]
            cl, rhol = act[l]
            mu = tuple(cl[b] - ci[b] for b in range(3))
            hpl = 0.5 * ((_dot(cl, cl) - _dot(ci, ci)) - rhol + rhoi)
            pts3 += _circle_plane(circ, mu, hpl)
    points = [(p[axes[0]], p[axes[1]]) for p in pts3]
    return _curve_rule_2d(_drop(lo, k), _drop(hi, k), curves, points, axes, q)


def union_rules(lo, hi, balls, q, surface=True, depth=0):
    """Volume rule for the union of the balls `balls` ((c, rho) pairs, psi_i = |x - c|^2 - rho)
    cap [lo, hi] and (if `surface`) the rule on its boundary; returns (volume, surface) as
    sphere_rules does."""
    contained, S = _ball_status(balls, lo, hi)
    if contained:
        return tensor_gauss(lo, hi, q), []
    if not S:
        return [], []
    if len(S) == 1:
        c, rho = balls[S[0]]
        return sphere_rules(lo, hi, c, rho, q, depth, surface)
    act = [balls[i] for i in S]
    m = len(lo)
    g, w = gauss01(q)
    if m == 1:
        roots = []
        for (c, rho) in act:
            s = math.sqrt(rho)
            for t in (c[0] - s, c[0] + s):
                if lo[0] < t < hi[0]:
                    roots.append(t)
        vol = []
        for (a, b) in _pieces(lo[0], hi[0], roots):
            mid = 0.5 * (a + b)
            if any((mid - c[0]) * (mid - c[0]) - rho < 0.0 for c, rho in act):
                for i in range(q):
                    vol.append(((a + (b - a) * g[i],), (b - a) * w[i]))
        if surface:
            raise QuadratureError("no surface rule for a 1D union box")
        return vol, []
    k = _union_height(act, lo, hi, True)
    valid = k is not None
    if not valid:
        if depth < MAX_DEPTH:
            vol = []
            surf = []
            for clo, chi in _children(lo, hi):
                v, s = union_rules(clo, chi, act, q, surface, depth + 1)
                vol += v
                surf += s
            return vol, surf
        k = _union_height(act, lo, hi, False)
    outer = _union_outer(lo, hi, act, k, valid, q)
    vol = []
    surf = []
    for (xp, wp) in outer:
        ivs = []
        for idx, (c, rho) in enumerate(act):
            r2 = rho - _dist2_excl(xp, _drop(c, k))
            if r2 > 0.0:
                s = math.sqrt(r2)
                a = c[k] - s
                b = c[k] + s
                if a < lo[k]:
                    a = lo[k]
                if b > hi[k]:
                    b = hi[k]
                if a < b:
                    ivs.append((a, idx, b))
        ivs.sort()
        merged = []
        for (a, idx, b) in ivs:
            if merged and a <= merged[-1][1]:
                if b > merged[-1][1]:
                    merged[-1][1] = b
                    merged[-1][3] = idx
            else:
                merged.append([a, b, idx, idx])
        for (a, b, _, _) in merged:
            for i in range(q):
                vol.append((_insert(xp, k, a + (b - a) * g[i]), wp * ((b - a) * w[i])))
        if surface:
            for (a, b, ia, ib) in merged:
                for t, idx, on in ((a, ia, a > lo[k]), (b, ib, b < hi[k])):
                    if not on:
                        continue
                    c, rho = act[idx]
                    x = _insert(xp, k, t)
                    nrm = math.sqrt(_dist2_excl(x, c))
                    normal = tuple((x[b2] - c[b2]) / nrm for b2 in range(m))
                    surf.append((x, wp * (math.sqrt(rho) / abs(t - c[k])), normal))
    return vol, surf


def _balls(prob):
    return [(c, R * R) for (c, R) in prob.spheres]


def cell_rules(prob, lo, hi, q=None):
    """Volume and surface rule of the cell [lo, hi] cut by the level set of `prob`."""
    q = prob.quad_order if q is None else q
    if prob.ls_kind == "plane":
        return plane_rules(lo, hi, prob.normal, prob.offset, q)
    if prob.ls_kind == "spheres":
        return union_rules(lo, hi, _balls(prob), q)
    R = prob.radius
    return sphere_rules(lo, hi, prob.center, R * R, q)


def face_rule(prob, face_lo, face_hi, axis, q=None):
    """Rule for F cap Omega on the face x_axis = face_lo[axis] (a (d-1)-dimensional box)."""
    q = prob.quad_order if q is None else q
    xa = face_lo[axis]
    flo = _drop(face_lo, axis)
    fhi = _drop(face_hi, axis)
    if prob.ls_kind == "plane":
        vol, _ = plane_rules(flo, fhi, _drop(prob.normal, axis),
                             prob.offset - prob.normal[axis] * xa, q, surface=False)
    elif prob.ls_kind == "spheres":
        # the balls whose sphere meets the face, cut by the face's plane
        contained, S = _ball_status(_balls(prob), face_lo, face_hi)
        discs = []
        for i in S:
            c, R = prob.spheres[i]
            da = xa - c[axis]
            discs.append((_drop(c, axis), R * R - da * da))
        vol = tensor_gauss(flo, fhi, q) if contained else union_rules(flo, fhi, discs, q, surface=False)[0]
    else:
        c, R = prob.center, prob.radius
        da = xa - c[axis]
        rho = R * R - da * da
        vol, _ = sphere_rules(flo, fhi, _drop(c, axis), rho, q, surface=False)
    return [(_insert(x, axis, xa), wt) for (x, wt) in vol]
