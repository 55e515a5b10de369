"""Dimension-reduction quadrature for sphere and plane level sets (oracle; test infrastructure
only).

The paper generates the cut-cell (volume, surface) and cut-face rules with the dimension
reduction method of Saye (2015) (Sec. 1, Sec. 2.3) and adds uniform subdivision when needed
(Sec. 4.1, arithmetic-complexity paragraph on refined cut cells).  The paper states no details, so
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


def _crossing_sphere(prob, lo, hi):
    """Union of separated balls: the one sphere whose surface meets the closed box."""
    hits = []
    for (c, R) in prob.spheres:
        dmin2, dmax2 = _box_dist2(c, lo, hi)
        if dmin2 < R * R < dmax2:
            hits.append((c, R))
    if len(hits) != 1:
        raise QuadratureError("a cut box must meet exactly one sphere of the union")
    return hits[0]


def cell_rules(prob, lo, hi, q=None):
    """Volume and surface rule of the cell [lo, hi] cut by the level set of `prob` (for a union
    of separated balls: by the one sphere that meets the cell)."""
    q = prob.quad_order if q is None else q
    if prob.ls_kind == "plane":
        return plane_rules(lo, hi, prob.normal, prob.offset, q)
    if prob.ls_kind == "spheres":
        c, R = _crossing_sphere(prob, lo, hi)
        return sphere_rules(lo, hi, c, R * R, q)
    R = prob.radius
    return sphere_rules(lo, hi, prob.center, R * R, q)


def face_rule(prob, face_lo, face_hi, axis, q=None):
    """Rule for F cap Omega on the face x_axis = face_lo[axis] (a (d-1)-dimensional box)."""
    q = prob.quad_order if q is None else q
    xa = face_lo[axis]
    if prob.ls_kind == "plane":
        vol, _ = plane_rules(_drop(face_lo, axis), _drop(face_hi, axis), _drop(prob.normal, axis),
                             prob.offset - prob.normal[axis] * xa, q, surface=False)
    else:
        c, R = _crossing_sphere(prob, face_lo, face_hi) if prob.ls_kind == "spheres" else \
            (prob.center, prob.radius)
        da = xa - c[axis]
        rho = R * R - da * da
        vol, _ = sphere_rules(_drop(face_lo, axis), _drop(face_hi, axis), _drop(c, axis),
                              rho, q, surface=False)
    return [(_insert(x, axis, xa), wt) for (x, wt) in vol]
