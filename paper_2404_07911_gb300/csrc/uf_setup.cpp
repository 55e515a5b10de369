// Host setup of the unfitted DG operator: 1D tables, classification, numbering, face typing and
// dimension-reduction quadrature (arXiv 2404.07911, Sec. 2.3; Saye's method as cited in Sec. 1).
//
// Compiled with -ffp-contract=off so that every floating-point decision of the quadrature
// generator (classification, one-signedness, root brackets, sign of a piece) is taken with the
// same correctly rounded operations on every host architecture.
//
// Reading of the quadrature method (the paper gives no details; restated for level sets
// psi(x) = |x - c|^2 - rho, whose roots along coordinate lines have closed forms):
//  * volume / surface rule on a box U: inside -> tensor Gauss q^m, outside -> nothing; else the
//    height direction k maximises |mid_k - c_k| (first index on ties); if lo_k < c_k < hi_k the
//    box is bisected in all directions (children ordered with direction 0 fastest, depth <= 8);
//    otherwise the outer rule is the full-box rule on U without direction k for the restrictions
//    of psi to x_k = lo_k and x_k = hi_k, and each outer line is split at its root: pieces with
//    psi(mid) < 0 get q Gauss points, the root is a surface point of weight w' R / |t - c_k|.
//  * full-box rule: drop one-signed functions; none left -> tensor Gauss; m = 1 -> split at
//    every root; else recurse on the lower-dimensional box with the restrictions of the kept
//    functions to both k-faces and split each line at the roots of the kept functions.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "uf_host.h"

namespace uf {
namespace {

constexpr int kMaxDepth = 8;

// ------------------------------------------------------------------------------------------
// 1D polynomials
// ------------------------------------------------------------------------------------------

// Legendre P_m and its first two derivatives at t in (-1, 1), by the three-term recurrence.
void legendre(int m, double t, double &P, double &dP, double &d2P) {
  double pm1 = 1.0, pcur = t;
  if (m == 0) {
    P = 1.0;
    dP = 0.0;
    d2P = 0.0;
    return;
  }
  for (int k = 2; k <= m; ++k) {
    double pn = ((2.0 * k - 1.0) * t * pcur - (k - 1.0) * pm1) / k;
    pm1 = pcur;
    pcur = pn;
  }
  P = pcur;
  dP = m * (pm1 - t * pcur) / (1.0 - t * t);
  d2P = (2.0 * t * dP - m * (m + 1.0) * pcur) / (1.0 - t * t);
}

void gauss_rule(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    // i-th root counted from the right end of [-1, 1]
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP, d2P;
      legendre(n, t, P, dP, d2P);
      double dt = P / dP;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double P, dP, d2P;
    legendre(n, t, P, dP, d2P);
    x[n - 1 - i] = 0.5 * (1.0 + t);
    w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dP * dP);  // half of 2 / ((1 - t^2) P'^2)
  }
}

void lobatto_nodes(int n, double *z) {
  z[0] = 0.0;
  z[n - 1] = 1.0;
  const int m = n - 1;
  for (int i = 1; i < m; ++i) {
    double t = -std::cos(M_PI * i / m);
    for (int it = 0; it < 100; ++it) {
      double P, dP, d2P;
      legendre(m, t, P, dP, d2P);
      double dt = dP / d2P;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    z[i] = 0.5 * (1.0 + t);
  }
  std::sort(z + 1, z + n - 1);
}

// Derivatives 0..J of the i-th Lagrange polynomial at x: the product of linear factors is
// accumulated factor by factor with D^j[P (x - z)] = (x - z) D^j P + j D^{j-1} P.
void lagrange_derivs(const Tables1D &t, int i, double x, int J, double *out) {
  double d[kMaxN + 1];
  for (int j = 0; j <= J; ++j) d[j] = (j == 0) ? 1.0 : 0.0;
  for (int m = 0; m < t.n; ++m) {
    if (m == i) continue;
    const double f = x - t.z[m];
    for (int j = J; j >= 1; --j) d[j] = f * d[j] + j * d[j - 1];
    d[0] = f * d[0];
  }
  for (int j = 0; j <= J; ++j) out[j] = d[j] * t.den_inv[i];
}

// ------------------------------------------------------------------------------------------
// Dimension-reduction quadrature for psi = |x - c|^2 - rho
// ------------------------------------------------------------------------------------------

struct Box {
  int m;
  double lo[kMaxDim], hi[kMaxDim];
};

struct Gauss1 {
  int q;
  double x[32], w[32];
};

void box_dist2(const double *c, const Box &b, double &dmin2, double &dmax2) {
  dmin2 = 0.0;
  dmax2 = 0.0;
  for (int a = 0; a < b.m; ++a) {
    const double dl = b.lo[a] - c[a];
    const double dh = b.hi[a] - c[a];
    const double e = std::fmax(std::fmax(dl, 0.0), -dh);
    dmin2 += e * e;
    dmax2 += std::fmax(dl * dl, dh * dh);
  }
}

double dist2(const double *x, const double *c, int m) {
  double r = 0.0;
  for (int i = 0; i < m; ++i) {
    const double d = x[i] - c[i];
    r += d * d;
  }
  return r;
}

void tensor_rule(const Box &b, const Gauss1 &g, std::vector<QPoint> &out,
                 std::vector<QLine> *lines = nullptr) {
  if (lines) {
    // lines along axis 0: consecutive runs of q points in the direction-0-fastest order
    int64_t nl = 1;
    for (int a = 1; a < b.m; ++a) nl *= g.q;
    for (int64_t l = 0; l < nl; ++l)
      lines->push_back(QLine{0, (int64_t)out.size() + l * g.q, g.q, -1});
  }
  int total = 1;
  for (int a = 0; a < b.m; ++a) total *= g.q;
  for (int flat = 0; flat < total; ++flat) {
    QPoint p{};
    double wt = 1.0;
    int rem = flat;
    for (int a = 0; a < b.m; ++a) {
      const int i = rem % g.q;
      rem /= g.q;
      p.x[a] = b.lo[a] + (b.hi[a] - b.lo[a]) * g.x[i];
      wt *= (b.hi[a] - b.lo[a]) * g.w[i];
    }
    p.w = wt;
    out.push_back(p);
  }
}

int height_dir(const double *c, const Box &b) {
  int k = 0;
  double best = -1.0;
  for (int i = 0; i < b.m; ++i) {
    const double v = std::fabs(0.5 * (b.lo[i] + b.hi[i]) - c[i]);
    if (v > best) {
      best = v;
      k = i;
    }
  }
  return k;
}

Box child(const Box &b, int bits) {
  Box c = b;
  for (int a = 0; a < b.m; ++a) {
    const double mid = 0.5 * (b.lo[a] + b.hi[a]);
    if ((bits >> a) & 1)
      c.lo[a] = mid;
    else
      c.hi[a] = mid;
  }
  return c;
}

Box drop_dim(const Box &b, int k) {
  Box r;
  r.m = b.m - 1;
  for (int a = 0, j = 0; a < b.m; ++a)
    if (a != k) {
      r.lo[j] = b.lo[a];
      r.hi[j] = b.hi[a];
      ++j;
    }
  return r;
}

void drop_vec(const double *v, int m, int k, double *out) {
  for (int a = 0, j = 0; a < m; ++a)
    if (a != k) out[j++] = v[a];
}

// x (m - 1 coordinates) with value t inserted at position k
void insert_coord(const double *x, int m, int k, double t, double *out) {
  for (int a = 0, j = 0; a < m; ++a) out[a] = (a == k) ? t : x[j++];
}

// Break points of [a, b] at the sorted roots, zero-length pieces dropped.
int make_pieces(double a, double b, double *roots, int nr, double *pa, double *pb) {
  std::sort(roots, roots + nr);
  double brk[16];
  int nb = 0;
  brk[nb++] = a;
  for (int i = 0; i < nr; ++i) brk[nb++] = roots[i];
  brk[nb++] = b;
  int np = 0;
  for (int i = 0; i + 1 < nb; ++i)
    if (brk[i + 1] > brk[i]) {
      pa[np] = brk[i];
      pb[np] = brk[i + 1];
      ++np;
    }
  return np;
}

struct QuadError {};

void full_box_rule(const Box &b, const std::vector<Fn> &fns, const Gauss1 &g, int depth,
                   std::vector<QPoint> &out) {
  std::vector<Fn> keep;
  for (const Fn &f : fns) {
    double dmin2, dmax2;
    box_dist2(f.c, b, dmin2, dmax2);
    if (!(dmin2 >= f.rho || dmax2 <= f.rho)) keep.push_back(f);
  }
  if (keep.empty()) {
    tensor_rule(b, g, out);
    return;
  }
  const double *c = keep[0].c;
  if (b.m == 1) {
    double roots[16];
    int nr = 0;
    for (const Fn &f : keep) {
      const double s = std::sqrt(f.rho);
      const double cand[2] = {f.c[0] - s, f.c[0] + s};
      for (double t : cand)
        if (b.lo[0] < t && t < b.hi[0]) roots[nr++] = t;
    }
    double pa[16], pb[16];
    const int np = make_pieces(b.lo[0], b.hi[0], roots, nr, pa, pb);
    for (int ip = 0; ip < np; ++ip)
      for (int i = 0; i < g.q; ++i) {
        QPoint p{};
        p.x[0] = pa[ip] + (pb[ip] - pa[ip]) * g.x[i];
        p.w = (pb[ip] - pa[ip]) * g.w[i];
        out.push_back(p);
      }
    return;
  }
  const int k = height_dir(c, b);
  if (b.lo[k] < c[k] && c[k] < b.hi[k]) {
    if (depth >= kMaxDepth) throw QuadError{};
    for (int bits = 0; bits < (1 << b.m); ++bits) full_box_rule(child(b, bits), keep, g, depth + 1, out);
    return;
  }
  double csub[kMaxDim];
  drop_vec(c, b.m, k, csub);
  const double dl = b.lo[k] - c[k];
  const double dh = b.hi[k] - c[k];
  std::vector<Fn> fns2;
  for (const Fn &f : keep) {
    Fn a{}, bb{};
    std::memcpy(a.c, csub, sizeof(csub));
    std::memcpy(bb.c, csub, sizeof(csub));
    a.rho = f.rho - dl * dl;
    bb.rho = f.rho - dh * dh;
    fns2.push_back(a);
    fns2.push_back(bb);
  }
  std::vector<QPoint> outer;
  full_box_rule(drop_dim(b, k), fns2, g, depth, outer);
  const bool up = c[k] <= b.lo[k];
  for (const QPoint &op : outer) {
    const double r = dist2(op.x, csub, b.m - 1);
    double roots[16];
    int nr = 0;
    for (const Fn &f : keep) {
      const double r2 = f.rho - r;
      if (r2 > 0.0) {
        const double s = std::sqrt(r2);
        const double t = up ? c[k] + s : c[k] - s;
        if (b.lo[k] < t && t < b.hi[k]) roots[nr++] = t;
      }
    }
    double pa[16], pb[16];
    const int np = make_pieces(b.lo[k], b.hi[k], roots, nr, pa, pb);
    for (int ip = 0; ip < np; ++ip)
      for (int i = 0; i < g.q; ++i) {
        QPoint p{};
        insert_coord(op.x, b.m, k, pa[ip] + (pb[ip] - pa[ip]) * g.x[i], p.x);
        p.w = op.w * ((pb[ip] - pa[ip]) * g.w[i]);
        out.push_back(p);
      }
  }
}

void sphere_box_rules(const Box &b, const double *c, double rho, const Gauss1 &g, int depth,
                      bool surface, std::vector<QPoint> &vol, std::vector<QPoint> &surf,
                      std::vector<QLine> *lines = nullptr) {
  double dmin2, dmax2;
  box_dist2(c, b, dmin2, dmax2);
  if (dmax2 <= rho) {
    tensor_rule(b, g, vol, lines);
    return;
  }
  if (dmin2 >= rho) return;
  if (b.m == 1) {
    const double s = std::sqrt(rho);
    double roots[2];
    int nr = 0;
    const double cand[2] = {c[0] - s, c[0] + s};
    for (double t : cand)
      if (b.lo[0] < t && t < b.hi[0]) roots[nr++] = t;
    double surf_t[2] = {roots[0], roots[1]};
    const int ns = nr;
    double pa[16], pb[16];
    const int np = make_pieces(b.lo[0], b.hi[0], roots, nr, pa, pb);
    const int64_t vbeg = (int64_t)vol.size();
    for (int ip = 0; ip < np; ++ip) {
      const double mid = 0.5 * (pa[ip] + pb[ip]);
      if ((mid - c[0]) * (mid - c[0]) - rho < 0.0)
        for (int i = 0; i < g.q; ++i) {
          QPoint p{};
          p.x[0] = pa[ip] + (pb[ip] - pa[ip]) * g.x[i];
          p.w = (pb[ip] - pa[ip]) * g.w[i];
          vol.push_back(p);
        }
    }
    if (lines && (int64_t)vol.size() > vbeg)
      lines->push_back(QLine{0, vbeg, (int64_t)vol.size() - vbeg, -1});
    if (surface)
      for (int i = 0; i < ns; ++i) {
        QPoint p{};
        p.x[0] = surf_t[i];
        p.w = 1.0;
        p.nrm[0] = surf_t[i] > c[0] ? 1.0 : -1.0;
        surf.push_back(p);
      }
    return;
  }
  const int k = height_dir(c, b);
  if (b.lo[k] < c[k] && c[k] < b.hi[k]) {
    if (depth >= kMaxDepth) throw QuadError{};
    for (int bits = 0; bits < (1 << b.m); ++bits)
      sphere_box_rules(child(b, bits), c, rho, g, depth + 1, surface, vol, surf, lines);
    return;
  }
  double csub[kMaxDim];
  drop_vec(c, b.m, k, csub);
  const double dl = b.lo[k] - c[k];
  const double dh = b.hi[k] - c[k];
  std::vector<Fn> fns(2);
  std::memcpy(fns[0].c, csub, sizeof(csub));
  std::memcpy(fns[1].c, csub, sizeof(csub));
  fns[0].rho = rho - dl * dl;
  fns[1].rho = rho - dh * dh;
  std::vector<QPoint> outer;
  full_box_rule(drop_dim(b, k), fns, g, 0, outer);
  const bool up = c[k] <= b.lo[k];
  const double R = std::sqrt(rho);
  for (const QPoint &op : outer) {
    const double r = dist2(op.x, csub, b.m - 1);
    const double r2 = rho - r;
    bool has_root = false;
    double t = 0.0;
    if (r2 > 0.0) {
      const double s = std::sqrt(r2);
      const double tt = up ? c[k] + s : c[k] - s;
      if (b.lo[k] < tt && tt < b.hi[k]) {
        has_root = true;
        t = tt;
      }
    }
    double roots[1] = {t};
    double pa[4], pb[4];
    const int np = make_pieces(b.lo[k], b.hi[k], roots, has_root ? 1 : 0, pa, pb);
    const int64_t vbeg = (int64_t)vol.size();
    const int64_t sidx = (surface && has_root) ? (int64_t)surf.size() : -1;
    for (int ip = 0; ip < np; ++ip) {
      const double mid = 0.5 * (pa[ip] + pb[ip]);
      const double dm = mid - c[k];
      if ((r + dm * dm) - rho < 0.0)
        for (int i = 0; i < g.q; ++i) {
          QPoint p{};
          insert_coord(op.x, b.m, k, pa[ip] + (pb[ip] - pa[ip]) * g.x[i], p.x);
          p.w = op.w * ((pb[ip] - pa[ip]) * g.w[i]);
          vol.push_back(p);
        }
    }
    if (surface && has_root) {
      QPoint p{};
      insert_coord(op.x, b.m, k, t, p.x);
      const double nrm = std::sqrt(dist2(p.x, c, b.m));
      for (int a = 0; a < b.m; ++a) p.nrm[a] = (p.x[a] - c[a]) / nrm;
      p.w = op.w * (R / std::fabs(t - c[k]));
      surf.push_back(p);
    }
    if (lines && ((int64_t)vol.size() > vbeg || sidx >= 0))
      lines->push_back(QLine{k, vbeg, (int64_t)vol.size() - vbeg, sidx});
  }
}

// ------------------------------------------------------------------------------------------
// Unions of balls: psi = min_i (|x - c_i|^2 - rho_i) (Sec. 6), balls may intersect
// ------------------------------------------------------------------------------------------
// Along a coordinate line the union is the merged union of the balls' intervals (exact inner
// integrals).  The outer integration splits where an interval meets the box (the circles
// psi_i(., lo_k) = 0, psi_i(., hi_k) = 0), where two spheres' endpoints meet (their intersection
// circle seen along k) and at the 3D points where such events coincide (intersection circles on
// the planes x_k = lo_k, hi_k; triple points of three spheres), all in closed form.  Decisions:
//  * box status: contained in one ball -> tensor Gauss; S = balls whose sphere meets the closed
//    box; |S| = 0 -> nothing; |S| = 1 -> sphere_box_rules; m = 1 -> split at all roots, pieces
//    whose midpoint lies in a ball get Gauss points.
//  * height direction k: no centre with lo_k < c_ik < hi_k; among those the one maximising
//    min_i |mid_k - c_ik| (first on ties); none -> bisect (depth <= 8), at depth 8 the same
//    maximum without the test.
//  * outer rule, m = 2: split at the roots of psi_i(., lo_k), psi_i(., hi_k), at the pair
//    intersection points and (invalid k) at the silhouettes c_i' +- R_i.  m = 3: rectangle
//    rule with circles in 2D and intersection circles in 3D as break curves and the coincidence
//    points as break points; its line direction is the one whose curves' points with tangent
//    along it lie outside the open rectangle, farthest from it (squared distance, first on
//    ties); none -> bisect the rectangle (depth <= 8, then direction 0).
//  * each outer line: intervals sorted by start (ball order on ties), merged when they touch;
//    merged ends inside (lo_k, hi_k) are surface points of the ball that starts / first reaches
//    them, weight w' R_i / |t - c_ik|.  A line with two surface points is stored as two lines
//    (the second one without volume points).

using Pieces = std::vector<std::pair<double, double>>;

Pieces pieces_of(double a, double b, std::vector<double> &roots) {
  std::sort(roots.begin(), roots.end());
  Pieces out;
  double prev = a;
  for (double r : roots) {
    if (r > prev) out.emplace_back(prev, r);
    prev = std::max(prev, r);
  }
  if (b > prev) out.emplace_back(prev, b);
  return out;
}

double dot3(const double *u, const double *v) {
  double r = 0.0;
  for (int a = 0; a < 3; ++a) r += u[a] * v[a];
  return r;
}

struct Circle3 {  // circle of centre q, unit normal nu, radius^2 rc2 (3D)
  double q[3], nu[3], rc2;
};

bool pair_circle(const Fn &bi, const Fn &bj, Circle3 &out) {
  double dv[3];
  for (int a = 0; a < 3; ++a) dv[a] = bj.c[a] - bi.c[a];
  const double D2 = dot3(dv, dv);
  if (D2 == 0.0) return false;
  const double D = std::sqrt(D2);
  for (int a = 0; a < 3; ++a) out.nu[a] = dv[a] / D;
  const double a0 = (D2 + bi.rho - bj.rho) / (2.0 * D);
  out.rc2 = bi.rho - a0 * a0;
  if (out.rc2 <= 0.0) return false;
  for (int a = 0; a < 3; ++a) out.q[a] = bi.c[a] + a0 * out.nu[a];
  return true;
}

// Points of the circle on the plane mu . x = h (0 or 2), appended to pts (3 doubles each).
int circle_plane(const Circle3 &cc, const double *mu, double h, std::vector<double> &pts) {
  const double mn = dot3(mu, cc.nu);
  const double mm = dot3(mu, mu);
  const double den = mm - mn * mn;
  if (den <= 1e-24 * mm) return 0;
  const double lam = (h - dot3(mu, cc.q)) / den;
  double p0[3];
  for (int a = 0; a < 3; ++a) p0[a] = cc.q[a] + lam * (mu[a] - mn * cc.nu[a]);
  const double s2 = cc.rc2 - lam * lam * den;
  if (s2 < 0.0) return 0;
  const double ell[3] = {cc.nu[1] * mu[2] - cc.nu[2] * mu[1], cc.nu[2] * mu[0] - cc.nu[0] * mu[2],
                         cc.nu[0] * mu[1] - cc.nu[1] * mu[0]};
  const double f = std::sqrt(s2) / std::sqrt(den);
  for (int a = 0; a < 3; ++a) pts.push_back(p0[a] - f * ell[a]);
  for (int a = 0; a < 3; ++a) pts.push_back(p0[a] + f * ell[a]);
  return 2;
}

int axis_plane_points(const Circle3 &cc, int A, double v, std::vector<double> &pts) {
  const double mu[3] = {A == 0 ? 1.0 : 0.0, A == 1 ? 1.0 : 0.0, A == 2 ? 1.0 : 0.0};
  return circle_plane(cc, mu, v, pts);
}

// Bounding box of the circle overlaps the open box in the listed 3D axes (b.m of them).
bool circle_overlaps(const Circle3 &cc, const int *axes, const Box &b) {
  for (int j = 0; j < b.m; ++j) {
    const int A = axes[j];
    const double hw = std::sqrt(cc.rc2) * std::sqrt(std::fmax(0.0, 1.0 - cc.nu[A] * cc.nu[A]));
    if (!(cc.q[A] - hw < b.hi[j] && cc.q[A] + hw > b.lo[j])) return false;
  }
  return true;
}

bool in_open(const double *x, const Box &b) {
  for (int a = 0; a < b.m; ++a)
    if (!(b.lo[a] < x[a] && x[a] < b.hi[a])) return false;
  return true;
}

// A break curve of the rectangle rule: a circle in the rectangle's coordinates (c3 = false) or
// an intersection circle in 3D seen along the dropped axis.
struct Curve {
  bool c3;
  double C[2], r2;
  Circle3 circ;
};

// Squared distance from the rectangle to the curve's points with tangent along direction a
// (the nearer one); 0 if one lies inside the open rectangle.
double tangent_clearance(const Curve &cv, int a, const int *axes, const Box &b) {
  const int o = 1 - a;
  double pts[2][2];
  if (!cv.c3) {
    const double r = std::sqrt(cv.r2);
    const double t[2] = {cv.C[o] - r, cv.C[o] + r};
    for (int i = 0; i < 2; ++i) {
      pts[i][a] = cv.C[a];
      pts[i][o] = t[i];
    }
  } else {
    const Circle3 &cc = cv.circ;
    const int O = axes[o];
    const double den = 1.0 - cc.nu[O] * cc.nu[O];
    if (den <= 1e-12) return 0.0;
    const double rc = std::sqrt(cc.rc2);
    const double sd = std::sqrt(den);
    const double sg[2] = {-1.0, 1.0};
    for (int i = 0; i < 2; ++i) {
      double p[3];
      for (int bb = 0; bb < 3; ++bb)
        p[bb] = cc.q[bb] + sg[i] * rc * (((bb == O ? 1.0 : 0.0) - cc.nu[O] * cc.nu[bb]) / sd);
      pts[i][0] = p[axes[0]];
      pts[i][1] = p[axes[1]];
    }
  }
  double best = INFINITY;
  for (int i = 0; i < 2; ++i) {
    if (in_open(pts[i], b)) return 0.0;
    double dmin2, dmax2;
    box_dist2(pts[i], b, dmin2, dmax2);
    best = std::fmin(best, dmin2);
  }
  return best;
}

// Coordinates (direction 1 - along of the rectangle) of the curve's points with coordinate
// `along` equal to v.
void curve_points_at(const Curve &cv, int along, double v, const int *axes, std::vector<double> &out) {
  const int other = 1 - along;
  if (!cv.c3) {
    const double rr = cv.r2 - (v - cv.C[along]) * (v - cv.C[along]);
    if (rr <= 0.0) return;
    const double s = std::sqrt(rr);
    out.push_back(cv.C[other] - s);
    out.push_back(cv.C[other] + s);
    return;
  }
  std::vector<double> pts;
  const int n = axis_plane_points(cv.circ, axes[along], v, pts);
  for (int i = 0; i < n; ++i) out.push_back(pts[3 * i + axes[other]]);
}

void curve_rule_2d(const Box &b, const std::vector<Curve> &curves, const std::vector<double> &points,
                   const int *axes, const Gauss1 &g, int depth, std::vector<QPoint> &out) {
  std::vector<Curve> keep;
  for (const Curve &cv : curves) {
    if (!cv.c3) {
      double dmin2, dmax2;
      box_dist2(cv.C, b, dmin2, dmax2);
      if (dmin2 < cv.r2 && cv.r2 < dmax2) keep.push_back(cv);
    } else if (circle_overlaps(cv.circ, axes, b)) {
      keep.push_back(cv);
    }
  }
  if (keep.empty()) {
    tensor_rule(b, g, out);
    return;
  }
  int a = -1;
  double best = 0.0;
  for (int cand = 0; cand < 2; ++cand) {
    double v = INFINITY;
    for (const Curve &cv : keep) v = std::fmin(v, tangent_clearance(cv, cand, axes, b));
    if (v > best) {
      best = v;
      a = cand;
    }
  }
  if (a < 0) {
    if (depth < kMaxDepth) {
      for (int bits = 0; bits < 4; ++bits) curve_rule_2d(child(b, bits), keep, points, axes, g, depth + 1, out);
      return;
    }
    a = 0;
  }
  const int o = 1 - a;
  std::vector<double> splits, cand;
  for (const Curve &cv : keep) {
    const double vs[2] = {b.lo[a], b.hi[a]};
    for (double v : vs) {
      cand.clear();
      curve_points_at(cv, a, v, axes, cand);
      for (double t : cand)
        if (b.lo[o] < t && t < b.hi[o]) splits.push_back(t);
    }
  }
  for (size_t i = 0; i < points.size() / 2; ++i) {
    const double t = points[2 * i + o];
    if (b.lo[o] < t && t < b.hi[o]) splits.push_back(t);
  }
  std::vector<double> roots;
  for (const auto &po : pieces_of(b.lo[o], b.hi[o], splits))
    for (int io = 0; io < g.q; ++io) {
      const double xo = po.first + (po.second - po.first) * g.x[io];
      const double wo = (po.second - po.first) * g.w[io];
      roots.clear();
      for (const Curve &cv : keep) {
        cand.clear();
        curve_points_at(cv, o, xo, axes, cand);
        for (double t : cand)
          if (b.lo[a] < t && t < b.hi[a]) roots.push_back(t);
      }
      for (const auto &pa : pieces_of(b.lo[a], b.hi[a], roots))
        for (int i = 0; i < g.q; ++i) {
          QPoint p{};
          p.x[o] = xo;
          p.x[a] = pa.first + (pa.second - pa.first) * g.x[i];
          p.w = wo * ((pa.second - pa.first) * g.w[i]);
          out.push_back(p);
        }
    }
}

// Height direction of a union box (-1 if none is valid with `check`).
int union_height(const std::vector<Fn> &act, const Box &b, bool check) {
  int k = -1;
  double best = -1.0;
  for (int kk = 0; kk < b.m; ++kk) {
    bool ok = true;
    double v = INFINITY;
    for (const Fn &f : act) {
      if (check && b.lo[kk] < f.c[kk] && f.c[kk] < b.hi[kk]) ok = false;
      v = std::fmin(v, std::fabs(0.5 * (b.lo[kk] + b.hi[kk]) - f.c[kk]));
    }
    if (!ok) continue;
    if (v > best) {
      best = v;
      k = kk;
    }
  }
  return k;
}

void union_outer(const Box &b, const std::vector<Fn> &act, int k, bool valid, const Gauss1 &g,
                 std::vector<QPoint> &out) {
  const int na = (int)act.size();
  if (b.m == 2) {
    const int a = 1 - k;
    std::vector<double> splits;
    for (const Fn &f : act) {
      const double vs[2] = {b.lo[k], b.hi[k]};
      for (double v : vs) {
        const double r2 = f.rho - (v - f.c[k]) * (v - f.c[k]);
        if (r2 > 0.0) {
          const double s = std::sqrt(r2);
          const double t[2] = {f.c[a] - s, f.c[a] + s};
          for (double tt : t)
            if (b.lo[a] < tt && tt < b.hi[a]) splits.push_back(tt);
        }
      }
      if (!valid && b.lo[k] < f.c[k] && f.c[k] < b.hi[k]) {
        const double R = std::sqrt(f.rho);
        const double t[2] = {f.c[a] - R, f.c[a] + R};
        for (double tt : t)
          if (b.lo[a] < tt && tt < b.hi[a]) splits.push_back(tt);
      }
    }
    for (int i = 0; i < na; ++i)
      for (int j = i + 1; j < na; ++j) {
        const Fn &ci = act[i], &cj = act[j];
        const double dv[2] = {cj.c[0] - ci.c[0], cj.c[1] - ci.c[1]};
        const double D2 = dv[0] * dv[0] + dv[1] * dv[1];
        if (D2 == 0.0) continue;
        const double D = std::sqrt(D2);
        const double nu[2] = {dv[0] / D, dv[1] / D};
        const double a0 = (D2 + ci.rho - cj.rho) / (2.0 * D);
        const double rc2 = ci.rho - a0 * a0;
        if (rc2 <= 0.0) continue;
        const double rc = std::sqrt(rc2);
        const double qc[2] = {ci.c[0] + a0 * nu[0], ci.c[1] + a0 * nu[1]};
        const double sg[2] = {-1.0, 1.0};
        for (double sgn : sg) {
          const double p[2] = {qc[0] - sgn * rc * nu[1], qc[1] + sgn * rc * nu[0]};
          if (b.lo[a] < p[a] && p[a] < b.hi[a]) splits.push_back(p[a]);
        }
      }
    for (const auto &pc : pieces_of(b.lo[a], b.hi[a], splits))
      for (int i = 0; i < g.q; ++i) {
        QPoint p{};
        p.x[0] = pc.first + (pc.second - pc.first) * g.x[i];
        p.w = (pc.second - pc.first) * g.w[i];
        out.push_back(p);
      }
    return;
  }
  int axes[2], j = 0;
  for (int bb = 0; bb < 3; ++bb)
    if (bb != k) axes[j++] = bb;
  std::vector<Curve> curves;
  for (const Fn &f : act) {
    const double vs[2] = {b.lo[k], b.hi[k]};
    for (double v : vs) {
      const double r2 = f.rho - (v - f.c[k]) * (v - f.c[k]);
      if (r2 > 0.0) {
        Curve cv{};
        cv.C[0] = f.c[axes[0]];
        cv.C[1] = f.c[axes[1]];
        cv.r2 = r2;
        curves.push_back(cv);
      }
    }
    if (!valid && b.lo[k] < f.c[k] && f.c[k] < b.hi[k]) {
      Curve cv{};
      cv.C[0] = f.c[axes[0]];
      cv.C[1] = f.c[axes[1]];
      cv.r2 = f.rho;
      curves.push_back(cv);
    }
  }
  const int all3[3] = {0, 1, 2};
  std::vector<double> pts3;
  for (int i = 0; i < na; ++i)
    for (int jj = i + 1; jj < na; ++jj) {
      Curve cv{};
      cv.c3 = true;
      if (!pair_circle(act[i], act[jj], cv.circ) || !circle_overlaps(cv.circ, all3, b)) continue;
      curves.push_back(cv);
      axis_plane_points(cv.circ, k, b.lo[k], pts3);
      axis_plane_points(cv.circ, k, b.hi[k], pts3);
      for (int l = jj + 1; l < na; ++l) {
        const Fn &fi = act[i], &fl = act[l];
        double mu[3];
        for (int bb = 0; bb < 3; ++bb) mu[bb] = fl.c[bb] - fi.c[bb];
        const double hpl = 0.5 * ((dot3(fl.c, fl.c) - dot3(fi.c, fi.c)) - fl.rho + fi.rho);
        circle_plane(cv.circ, mu, hpl, pts3);
      }
    }
  std::vector<double> points;
  for (size_t i = 0; i < pts3.size() / 3; ++i) {
    points.push_back(pts3[3 * i + axes[0]]);
    points.push_back(pts3[3 * i + axes[1]]);
  }
  curve_rule_2d(drop_dim(b, k), curves, points, axes, g, 0, out);
}

void union_box_rules(const Box &b, const std::vector<Fn> &balls, const Gauss1 &g, int depth,
                     bool surface, std::vector<QPoint> &vol, std::vector<QPoint> &surf,
                     std::vector<QLine> *lines) {
  bool contained = false;
  std::vector<Fn> act;
  for (const Fn &f : balls) {
    double dmin2, dmax2;
    box_dist2(f.c, b, dmin2, dmax2);
    if (dmax2 <= f.rho)
      contained = true;
    else if (dmin2 < f.rho)
      act.push_back(f);
  }
  if (contained) {
    tensor_rule(b, g, vol, lines);
    return;
  }
  if (act.empty()) return;
  if (act.size() == 1) {
    sphere_box_rules(b, act[0].c, act[0].rho, g, depth, surface, vol, surf, lines);
    return;
  }
  if (b.m == 1) {
    if (surface) throw QuadError{};
    std::vector<double> roots;
    for (const Fn &f : act) {
      const double s = std::sqrt(f.rho);
      const double t[2] = {f.c[0] - s, f.c[0] + s};
      for (double tt : t)
        if (b.lo[0] < tt && tt < b.hi[0]) roots.push_back(tt);
    }
    const int64_t vbeg = (int64_t)vol.size();
    for (const auto &pc : pieces_of(b.lo[0], b.hi[0], roots)) {
      const double mid = 0.5 * (pc.first + pc.second);
      bool in = false;
      for (const Fn &f : act) in = in || ((mid - f.c[0]) * (mid - f.c[0]) - f.rho < 0.0);
      if (in)
        for (int i = 0; i < g.q; ++i) {
          QPoint p{};
          p.x[0] = pc.first + (pc.second - pc.first) * g.x[i];
          p.w = (pc.second - pc.first) * g.w[i];
          vol.push_back(p);
        }
    }
    if (lines && (int64_t)vol.size() > vbeg) lines->push_back(QLine{0, vbeg, (int64_t)vol.size() - vbeg, -1});
    return;
  }
  int k = union_height(act, b, true);
  const bool valid = k >= 0;
  if (!valid) {
    if (depth < kMaxDepth) {
      for (int bits = 0; bits < (1 << b.m); ++bits)
        union_box_rules(child(b, bits), act, g, depth + 1, surface, vol, surf, lines);
      return;
    }
    k = union_height(act, b, false);
  }
  std::vector<QPoint> outer;
  union_outer(b, act, k, valid, g, outer);
  struct Iv {
    double a, b;
    int idx;
  };
  struct Merged {
    double a, b;
    int ia, ib;
  };
  std::vector<Iv> ivs;
  std::vector<Merged> merged;
  for (const QPoint &op : outer) {
    ivs.clear();
    for (int idx = 0; idx < (int)act.size(); ++idx) {
      const Fn &f = act[idx];
      double csub[kMaxDim];
      drop_vec(f.c, b.m, k, csub);
      const double r2 = f.rho - dist2(op.x, csub, b.m - 1);
      if (r2 > 0.0) {
        const double s = std::sqrt(r2);
        double a = f.c[k] - s, bb = f.c[k] + s;
        if (a < b.lo[k]) a = b.lo[k];
        if (bb > b.hi[k]) bb = b.hi[k];
        if (a < bb) ivs.push_back(Iv{a, bb, idx});
      }
    }
    std::sort(ivs.begin(), ivs.end(), [](const Iv &x, const Iv &y) {
      return x.a < y.a || (x.a == y.a && x.idx < y.idx);
    });
    merged.clear();
    for (const Iv &iv : ivs) {
      if (!merged.empty() && iv.a <= merged.back().b) {
        if (iv.b > merged.back().b) {
          merged.back().b = iv.b;
          merged.back().ib = iv.idx;
        }
      } else {
        merged.push_back(Merged{iv.a, iv.b, iv.idx, iv.idx});
      }
    }
    const int64_t vbeg = (int64_t)vol.size();
    for (const Merged &mg : merged)
      for (int i = 0; i < g.q; ++i) {
        QPoint p{};
        insert_coord(op.x, b.m, k, mg.a + (mg.b - mg.a) * g.x[i], p.x);
        p.w = op.w * ((mg.b - mg.a) * g.w[i]);
        vol.push_back(p);
      }
    const int64_t vcnt = (int64_t)vol.size() - vbeg;
    int nsurf = 0;
    if (surface)
      for (const Merged &mg : merged) {
        const double ts[2] = {mg.a, mg.b};
        const int own[2] = {mg.ia, mg.ib};
        const bool on[2] = {mg.a > b.lo[k], mg.b < b.hi[k]};
        for (int e = 0; e < 2; ++e) {
          if (!on[e]) continue;
          const Fn &f = act[own[e]];
          QPoint p{};
          insert_coord(op.x, b.m, k, ts[e], p.x);
          const double nrm = std::sqrt(dist2(p.x, f.c, b.m));
          for (int a = 0; a < b.m; ++a) p.nrm[a] = (p.x[a] - f.c[a]) / nrm;
          p.w = op.w * (std::sqrt(f.rho) / std::fabs(ts[e] - f.c[k]));
          if (lines) {
            if (nsurf == 0)
              lines->push_back(QLine{k, vbeg, vcnt, (int64_t)surf.size()});
            else
              lines->push_back(QLine{k, vbeg + vcnt, 0, (int64_t)surf.size()});
          }
          surf.push_back(p);
          ++nsurf;
        }
      }
    if (lines && nsurf == 0 && vcnt > 0) lines->push_back(QLine{k, vbeg, vcnt, -1});
  }
}

// ------------------------------------------------------------------------------------------
// Dimension-reduction quadrature for a plane psi = n . x - off
// ------------------------------------------------------------------------------------------
// psi is monotone along every direction with n_k != 0, so no bisection is needed: the height
// direction maximises |n_k| (first index on ties), the restriction of psi to x_k = v is linear
// again (n without k, off - n_k v), the root on the line through x' is (off - s) / n_k with
// s = sum_{a != k} n_a x'_a, and a surface point has weight w' |n| / |n_k| and normal n / |n|.

struct LinFn {
  double n[kMaxDim];
  double off;
};

// minimum and maximum of n . x - off over the closed box
void lin_range(const double *n, double off, const Box &b, double &mn, double &mx) {
  mn = 0.0;
  mx = 0.0;
  for (int a = 0; a < b.m; ++a) {
    if (n[a] >= 0.0) {
      mn += n[a] * b.lo[a];
      mx += n[a] * b.hi[a];
    } else {
      mn += n[a] * b.hi[a];
      mx += n[a] * b.lo[a];
    }
  }
  mn -= off;
  mx -= off;
}

int lin_height(const double *n, int m) {
  int k = 0;
  double best = -1.0;
  for (int i = 0; i < m; ++i)
    if (std::fabs(n[i]) > best) {
      best = std::fabs(n[i]);
      k = i;
    }
  return k;
}

// sum over a != k of n_a x'_a, with x' the m - 1 coordinates other than k
double lin_sum_excl(const double *n, int m, int k, const double *xp) {
  double s = 0.0;
  for (int a = 0, j = 0; a < m; ++a)
    if (a != k) s += n[a] * xp[j++];
  return s;
}

void full_box_rule_lin(const Box &b, const std::vector<LinFn> &fns, const Gauss1 &g,
                       std::vector<QPoint> &out) {
  std::vector<LinFn> keep;
  for (const LinFn &f : fns) {
    double mn, mx;
    lin_range(f.n, f.off, b, mn, mx);
    if (!(mn >= 0.0 || mx <= 0.0)) keep.push_back(f);
  }
  if (keep.empty()) {
    tensor_rule(b, g, out);
    return;
  }
  const double *n = keep[0].n;  // kept functions are restrictions of one plane: same n
  if (b.m == 1) {
    double roots[16];
    int nr = 0;
    for (const LinFn &f : keep) {
      const double t = f.off / f.n[0];
      if (b.lo[0] < t && t < b.hi[0]) roots[nr++] = t;
    }
    double pa[16], pb[16];
    const int np = make_pieces(b.lo[0], b.hi[0], roots, nr, pa, pb);
    for (int ip = 0; ip < np; ++ip)
      for (int i = 0; i < g.q; ++i) {
        QPoint p{};
        p.x[0] = pa[ip] + (pb[ip] - pa[ip]) * g.x[i];
        p.w = (pb[ip] - pa[ip]) * g.w[i];
        out.push_back(p);
      }
    return;
  }
  const int k = lin_height(n, b.m);
  std::vector<LinFn> fns2;
  for (const LinFn &f : keep) {
    LinFn lo_f{}, hi_f{};
    drop_vec(n, b.m, k, lo_f.n);
    drop_vec(n, b.m, k, hi_f.n);
    lo_f.off = f.off - n[k] * b.lo[k];
    hi_f.off = f.off - n[k] * b.hi[k];
    fns2.push_back(lo_f);
    fns2.push_back(hi_f);
  }
  std::vector<QPoint> outer;
  full_box_rule_lin(drop_dim(b, k), fns2, g, outer);
  for (const QPoint &op : outer) {
    const double s = lin_sum_excl(n, b.m, k, op.x);
    double roots[16];
    int nr = 0;
    for (const LinFn &f : keep) {
      const double t = (f.off - s) / n[k];
      if (b.lo[k] < t && t < b.hi[k]) roots[nr++] = t;
    }
    double pa[16], pb[16];
    const int np = make_pieces(b.lo[k], b.hi[k], roots, nr, pa, pb);
    for (int ip = 0; ip < np; ++ip)
      for (int i = 0; i < g.q; ++i) {
        QPoint p{};
        insert_coord(op.x, b.m, k, pa[ip] + (pb[ip] - pa[ip]) * g.x[i], p.x);
        p.w = op.w * ((pb[ip] - pa[ip]) * g.w[i]);
        out.push_back(p);
      }
  }
}

void plane_box_rules(const Box &b, const double *n, double off, const Gauss1 &g, bool surface,
                     std::vector<QPoint> &vol, std::vector<QPoint> &surf,
                     std::vector<QLine> *lines = nullptr) {
  double mn, mx;
  lin_range(n, off, b, mn, mx);
  if (mx <= 0.0) {
    tensor_rule(b, g, vol, lines);
    return;
  }
  if (mn >= 0.0) return;
  double nn = 0.0;
  for (int a = 0; a < b.m; ++a) nn += n[a] * n[a];
  nn = std::sqrt(nn);
  if (b.m == 1) {
    const double t = off / n[0];
    double roots[1] = {t};
    const bool has_root = b.lo[0] < t && t < b.hi[0];
    double pa[4], pb[4];
    const int np = make_pieces(b.lo[0], b.hi[0], roots, has_root ? 1 : 0, pa, pb);
    const int64_t vbeg = (int64_t)vol.size();
    for (int ip = 0; ip < np; ++ip) {
      const double mid = 0.5 * (pa[ip] + pb[ip]);
      if (n[0] * mid - off < 0.0)
        for (int i = 0; i < g.q; ++i) {
          QPoint p{};
          p.x[0] = pa[ip] + (pb[ip] - pa[ip]) * g.x[i];
          p.w = (pb[ip] - pa[ip]) * g.w[i];
          vol.push_back(p);
        }
    }
    if (lines && (int64_t)vol.size() > vbeg)
      lines->push_back(QLine{0, vbeg, (int64_t)vol.size() - vbeg, -1});
    if (surface && has_root) {
      QPoint p{};
      p.x[0] = t;
      p.w = 1.0;
      p.nrm[0] = n[0] > 0.0 ? 1.0 : -1.0;
      surf.push_back(p);
    }
    return;
  }
  const int k = lin_height(n, b.m);
  std::vector<LinFn> fns(2);
  drop_vec(n, b.m, k, fns[0].n);
  drop_vec(n, b.m, k, fns[1].n);
  fns[0].off = off - n[k] * b.lo[k];
  fns[1].off = off - n[k] * b.hi[k];
  std::vector<QPoint> outer;
  full_box_rule_lin(drop_dim(b, k), fns, g, outer);
  for (const QPoint &op : outer) {
    const double s = lin_sum_excl(n, b.m, k, op.x);
    const double t = (off - s) / n[k];
    const bool has_root = b.lo[k] < t && t < b.hi[k];
    double roots[1] = {t};
    double pa[4], pb[4];
    const int np = make_pieces(b.lo[k], b.hi[k], roots, has_root ? 1 : 0, pa, pb);
    const int64_t vbeg = (int64_t)vol.size();
    const int64_t sidx = (surface && has_root) ? (int64_t)surf.size() : -1;
    for (int ip = 0; ip < np; ++ip) {
      const double mid = 0.5 * (pa[ip] + pb[ip]);
      if ((s + n[k] * mid) - off < 0.0)
        for (int i = 0; i < g.q; ++i) {
          QPoint p{};
          insert_coord(op.x, b.m, k, pa[ip] + (pb[ip] - pa[ip]) * g.x[i], p.x);
          p.w = op.w * ((pb[ip] - pa[ip]) * g.w[i]);
          vol.push_back(p);
        }
    }
    if (surface && has_root) {
      QPoint p{};
      insert_coord(op.x, b.m, k, t, p.x);
      for (int a = 0; a < b.m; ++a) p.nrm[a] = n[a] / nn;
      p.w = op.w * (nn / std::fabs(n[k]));
      surf.push_back(p);
    }
    if (lines && ((int64_t)vol.size() > vbeg || sidx >= 0))
      lines->push_back(QLine{k, vbeg, (int64_t)vol.size() - vbeg, sidx});
  }
}

}  // namespace

void lagrange_values(const Tables1D &t, double x, double *val, double *der) {
  for (int i = 0; i < t.n; ++i) {
    double dd[kMaxN + 1];
    lagrange_derivs(t, i, x, 1, dd);
    val[i] = dd[0];
    der[i] = dd[1];
  }
}

void build_tables_1d(int p, Tables1D &t) {
  std::memset(&t, 0, sizeof(t));
  t.p = p;
  t.n = p + 1;
  const int n = t.n;
  lobatto_nodes(n, t.z);
  for (int i = 0; i < n; ++i) {
    double den = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != i) den *= t.z[i] - t.z[m];
    t.den_inv[i] = 1.0 / den;
  }
  gauss_rule(n, t.gauss_x, t.gauss_w);
  double val[kMaxN][kMaxN], der[kMaxN][kMaxN];  // [q][i]
  for (int qp = 0; qp < n; ++qp)
    for (int i = 0; i < n; ++i) {
      double d[kMaxN + 1];
      lagrange_derivs(t, i, t.gauss_x[qp], 1, d);
      val[qp][i] = d[0];
      der[qp][i] = d[1];
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double m = 0.0, k = 0.0;
      for (int qp = 0; qp < n; ++qp) {
        m += t.gauss_w[qp] * val[qp][i] * val[qp][j];
        k += t.gauss_w[qp] * der[qp][i] * der[qp][j];
      }
      t.mass[i * n + j] = m;
      t.stiff[i * n + j] = k;
    }
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < n; ++i) {
      double d[kMaxN + 1];
      lagrange_derivs(t, i, (double)s, p, d);
      for (int j = 0; j <= p; ++j) t.deriv_end[s][j][i] = d[j];
    }
}

namespace {

// Union of balls: the spheres that meet a cut cell or one of the two cells of a face
// (ascending, without repeats).
void union_face_candidates(const HostOperator &op, int64_t e, int64_t nb, std::vector<int32_t> &cand) {
  cand.clear();
  for (int64_t c : {e, nb}) {
    if (c < 0 || op.act_type[c] != 1) continue;
    const int32_t ci = op.cut_of[c];
    for (int64_t i = op.cut_sph_off[ci]; i < op.cut_sph_off[ci + 1]; ++i) cand.push_back(op.cut_sph[i]);
  }
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
}

// Type of a face of a union of balls: 0 full (in one ball), 1 cut (a sphere meets it), 2 empty.
// A face of an inside cell lies in that cell's ball; otherwise every ball that contains or meets
// the face meets both (cut) cells, so their spheres are the only candidates.
int union_face_type(const HostOperator &op, const Box &fb, int64_t e, int64_t nb) {
  if (op.act_type[e] == 0 || op.act_type[nb] == 0) return 0;
  std::vector<int32_t> cand;
  union_face_candidates(op, e, nb, cand);
  int crossing = 0;
  for (int32_t i : cand) {
    const double *sp = &op.spheres[4 * (size_t)i];
    double dmin2, dmax2;
    box_dist2(sp, fb, dmin2, dmax2);
    const double r2 = sp[3] * sp[3];
    if (dmax2 <= r2) return 0;
    if (dmin2 < r2) ++crossing;
  }
  return crossing == 0 ? 2 : 1;
}

}  // namespace

uf_status build_host_operator(const uf_params &prm, HostOperator &op, std::string &msg) {
  op.params = prm;
  op.params.kappa = nullptr;
  const int d = prm.dim;
  if (d != 2 && d != 3) {
    msg = "dim must be 2 or 3";
    return UF_EINVAL;
  }
  if (prm.degree < 1 || prm.degree > 8) {
    msg = "degree must be in 1..8";
    return prm.degree < 1 ? UF_EINVAL : UF_EUNSUPPORTED;
  }
  if (prm.quad_order < 1 || prm.quad_order > 32) {
    msg = "quad_order must be in 1..32";
    return UF_EINVAL;
  }
  if (prm.gp_max_order < 0 || prm.gp_max_order > prm.degree) {
    msg = "gp_max_order must be in 0..degree";
    return UF_EINVAL;
  }
  if (prm.ls_kind != UF_LS_SPHERE && prm.ls_kind != UF_LS_PLANE && prm.ls_kind != UF_LS_SPHERES) {
    msg = "ls_kind must be UF_LS_SPHERE, UF_LS_PLANE or UF_LS_SPHERES";
    return UF_EUNSUPPORTED;
  }
  if (prm.ls_kind == UF_LS_SPHERES) {
    if (!prm.ls_spheres || prm.ls_n_spheres < 1) {
      msg = "UF_LS_SPHERES needs ls_spheres and ls_n_spheres >= 1";
      return UF_EINVAL;
    }
    for (int i = 0; i < prm.ls_n_spheres; ++i) {
      bool ok = prm.ls_spheres[4 * i + 3] > 0.0 && std::isfinite(prm.ls_spheres[4 * i + 3]);
      for (int a = 0; a < 3; ++a) ok = ok && std::isfinite(prm.ls_spheres[4 * i + a]);
      if (!ok) {
        msg = "every sphere needs a finite centre and a positive radius";
        return UF_EINVAL;
      }
    }
  }
  if (prm.ls_kind == UF_LS_SPHERE && !(prm.ls_radius > 0.0)) {
    msg = "ls_radius must be positive";
    return UF_EINVAL;
  }
  if (prm.ls_kind == UF_LS_PLANE) {
    bool nonzero = false, finite = std::isfinite(prm.ls_offset);
    for (int a = 0; a < d; ++a) {
      finite = finite && std::isfinite(prm.ls_normal[a]);
      if (prm.ls_normal[a] != 0.0) nonzero = true;
    }
    if (!nonzero || !finite) {
      msg = "the plane needs a finite, non-zero ls_normal and a finite ls_offset";
      return UF_EINVAL;
    }
  }
  if (prm.gp_kind != UF_GP_FACE && prm.gp_kind != UF_GP_VOLUME) {
    msg = "gp_kind must be UF_GP_FACE or UF_GP_VOLUME";
    return UF_EINVAL;
  }
  if (prm.gp_kind == UF_GP_VOLUME && prm.gp_max_order > 0 && !(prm.gp_tau > 0.0)) {
    msg = "gp_tau must be positive";
    return UF_EINVAL;
  }
  if (prm.discretization != UF_DG && prm.discretization != UF_CG) {
    msg = "discretization must be UF_DG or UF_CG";
    return UF_EINVAL;
  }
  op.cg = prm.discretization == UF_CG;
  op.dim = d;
  op.p = prm.degree;
  op.n = prm.degree + 1;
  op.q = prm.quad_order;
  op.ndof = 1;
  for (int a = 0; a < d; ++a) op.ndof *= op.n;
  double hv[kMaxDim];
  int64_t total = 1;
  for (int a = 0; a < d; ++a) {
    if (prm.n_cells[a] < 1 || !(prm.hi[a] > prm.lo[a])) {
      msg = "n_cells must be >= 1 and hi > lo";
      return UF_EINVAL;
    }
    op.N[a] = prm.n_cells[a];
    op.lo[a] = prm.lo[a];
    op.center[a] = prm.ls_center[a];
    op.normal[a] = prm.ls_normal[a];
    hv[a] = (prm.hi[a] - prm.lo[a]) / (double)prm.n_cells[a];
    total *= op.N[a];
  }
  if (total > (int64_t)1 << 30) {
    msg = "background grid too large";
    return UF_EUNSUPPORTED;
  }
  double hmin = hv[0], hmax = hv[0];
  for (int a = 1; a < d; ++a) {
    hmin = std::min(hmin, hv[a]);
    hmax = std::max(hmax, hv[a]);
  }
  if (hmax - hmin > 1e-14 * hmax) {
    msg = "cells must be cubes (isotropic h)";
    return UF_EUNSUPPORTED;
  }
  op.h = hv[0];
  op.radius = prm.ls_radius;
  op.ls_kind = prm.ls_kind;
  op.offset = prm.ls_offset;
  if (op.ls_kind == UF_LS_SPHERES) {
    op.spheres.assign(prm.ls_spheres, prm.ls_spheres + 4 * (size_t)prm.ls_n_spheres);
    op.params.ls_spheres = nullptr;  // the caller's array is not kept
  }
  // type of a closed box (d-dimensional, possibly a face): 0 inside, 1 cut, 2 outside
  auto classify = [&](const Box &b) {
    double lo_v, hi_v;
    if (op.ls_kind == UF_LS_PLANE) {
      lin_range(op.normal, op.offset, b, lo_v, hi_v);
      return hi_v <= 0.0 ? 0 : (lo_v >= 0.0 ? 2 : 1);
    }
    box_dist2(op.center, b, lo_v, hi_v);
    const double r2 = op.radius * op.radius;
    return hi_v <= r2 ? 0 : (lo_v >= r2 ? 2 : 1);
  };
  build_tables_1d(op.p, op.t);

  // ---- classification and numbering (x index fastest)
  op.n_background = total;
  op.id_map.assign(total, -1);
  std::vector<int8_t> bg_type(total);
  std::vector<std::pair<int64_t, int32_t>> bg_cross;  // union of balls: (cell, sphere meeting it)
  if (op.ls_kind == UF_LS_SPHERES) {
    // every ball updates the cells of its bounding box (cells beyond it lie outside the ball)
    std::vector<uint8_t> inside(total, 0), crossings(total, 0);
    const int ns = (int)(op.spheres.size() / 4);
    for (int i = 0; i < ns; ++i) {
      const double *c = &op.spheres[4 * i];
      const double R = c[3], r2 = R * R;
      int64_t i0[kMaxDim] = {0, 0, 0}, i1[kMaxDim] = {1, 1, 1};
      bool empty = false;
      for (int a = 0; a < d; ++a) {
        i0[a] = std::max<int64_t>(0, (int64_t)std::floor((c[a] - R - op.lo[a]) / hv[a]) - 1);
        i1[a] = std::min<int64_t>(op.N[a], (int64_t)std::floor((c[a] + R - op.lo[a]) / hv[a]) + 2);
        empty = empty || i1[a] <= i0[a];
      }
      if (empty) continue;
      for (int64_t k = i0[2]; k < i1[2]; ++k)
        for (int64_t j = i0[1]; j < i1[1]; ++j)
          for (int64_t ii = i0[0]; ii < i1[0]; ++ii) {
            const int64_t I[3] = {ii, j, k};
            Box b;
            b.m = d;
            int64_t flat = 0, stride = 1;
            for (int a = 0; a < d; ++a) {
              b.lo[a] = op.lo[a] + (double)I[a] * hv[a];
              b.hi[a] = op.lo[a] + (double)(I[a] + 1) * hv[a];
              flat += I[a] * stride;
              stride *= op.N[a];
            }
            double dmin2, dmax2;
            box_dist2(c, b, dmin2, dmax2);
            if (dmax2 <= r2) {
              inside[flat] = 1;
            } else if (dmin2 < r2 && dmax2 > r2) {
              crossings[flat] = 1;
              bg_cross.emplace_back(flat, i);
            }
          }
    }
    for (int64_t flat = 0; flat < total; ++flat)
      bg_type[flat] = inside[flat] ? 0 : (crossings[flat] ? 1 : 2);
    std::stable_sort(bg_cross.begin(), bg_cross.end(),
                     [](const std::pair<int64_t, int32_t> &a, const std::pair<int64_t, int32_t> &b) {
                       return a.first < b.first;
                     });
  } else {
    for (int64_t flat = 0; flat < total; ++flat) {
      Box b;
      b.m = d;
      int64_t rem = flat;
      for (int a = 0; a < d; ++a) {
        const int64_t I = rem % op.N[a];
        rem /= op.N[a];
        b.lo[a] = op.lo[a] + (double)I * hv[a];
        b.hi[a] = op.lo[a] + (double)(I + 1) * hv[a];
      }
      bg_type[flat] = (int8_t)classify(b);
    }
  }
  for (int64_t flat = 0; flat < total; ++flat) {
    if (bg_type[flat] == 2) continue;
    op.id_map[flat] = (int32_t)op.n_active;
    int64_t rem = flat;
    for (int a = 0; a < kMaxDim; ++a) {
      int64_t I = 0;
      if (a < d) {
        I = rem % op.N[a];
        rem /= op.N[a];
      }
      op.act_index.push_back((int32_t)I);
    }
    op.act_type.push_back(bg_type[flat]);
    ++op.n_active;
  }
  if (op.n_active == 0) {
    msg = "no active cell: the level set does not meet the background grid";
    return UF_EGEOMETRY;
  }
  if (op.n_active * (int64_t)op.ndof > ((int64_t)1 << 31) - 1) {
    msg = "too many DoFs for 32-bit cell offsets";
    return UF_EUNSUPPORTED;
  }
  op.kappa.assign(op.n_active, 1.0);

  // ---- neighbours, face typing
  const int nf = 2 * d;
  op.nbr.assign(op.n_active * nf, -1);
  op.flags.assign(op.n_active, 0u);
  op.cut_of.assign(op.n_active, -1);
  size_t cross_pos = 0;  // cut cells ascend in background order, as bg_cross does
  if (op.ls_kind == UF_LS_SPHERES) op.cut_sph_off.assign(1, 0);
  for (int64_t e = 0; e < op.n_active; ++e) {
    if (op.act_type[e] == 1) {
      op.flags[e] |= kCellCut;
      op.cut_of[e] = (int32_t)op.n_cut++;
      op.cut_cells.push_back((int32_t)e);
      if (op.ls_kind == UF_LS_SPHERES) {
        int64_t flat = 0, stride = 1;
        for (int a = 0; a < d; ++a) {
          flat += (int64_t)op.act_index[e * 3 + a] * stride;
          stride *= op.N[a];
        }
        while (cross_pos < bg_cross.size() && bg_cross[cross_pos].first < flat) ++cross_pos;
        for (; cross_pos < bg_cross.size() && bg_cross[cross_pos].first == flat; ++cross_pos)
          op.cut_sph.push_back(bg_cross[cross_pos].second);
        op.cut_sph_off.push_back((int64_t)op.cut_sph.size());
      }
    } else {
      ++op.n_inside;
    }
  }
  const bool use_gp = prm.gp_max_order > 0;
  const bool volume_gp = use_gp && prm.gp_kind == UF_GP_VOLUME;  // patches chosen after quadrature
  auto face_box = [&](int64_t e_minus, int axis) {
    Box b;
    b.m = d;
    for (int a = 0; a < d; ++a) {
      const int64_t I = op.act_index[e_minus * 3 + a];
      b.lo[a] = op.lo[a] + (double)I * hv[a];
      b.hi[a] = op.lo[a] + (double)(I + 1) * hv[a];
    }
    b.lo[axis] = b.hi[axis];
    return b;
  };
  for (int64_t e = 0; e < op.n_active; ++e) {
    for (int axis = 0; axis < d; ++axis)
      for (int side = 0; side < 2; ++side) {
        int64_t I[kMaxDim];
        for (int a = 0; a < d; ++a) I[a] = op.act_index[e * 3 + a];
        I[axis] += side ? 1 : -1;
        if (I[axis] < 0 || I[axis] >= op.N[axis]) continue;
        int64_t flat = 0, stride = 1;
        for (int a = 0; a < d; ++a) {
          flat += I[a] * stride;
          stride *= op.N[a];
        }
        const int32_t nb = op.id_map[flat];
        if (nb < 0) continue;
        const int f = 2 * axis + side;
        op.nbr[e * nf + f] = nb;
        const int64_t e_minus = side ? e : nb;
        int ftype;  // 0 full, 1 cut, 2 empty
        if (op.ls_kind == UF_LS_SPHERES) {
          // a face lies in a closed inside cell, or meets (or lies in) only the spheres of its two
          // cut cells
          ftype = union_face_type(op, face_box(e_minus, axis), e, nb);
        } else {
          ftype = classify(face_box(e_minus, axis));
        }
        const bool gp = use_gp && !volume_gp && (op.act_type[e] == 1 || op.act_type[nb] == 1);
        // the continuous space has no SIPG term
        if (ftype == 0 && !op.cg) op.flags[e] |= face_bit_sipg_full(f);
        if (ftype == 1 && !op.cg) op.flags[e] |= face_bit_sipg_cut(f);
        if (gp) op.flags[e] |= face_bit_gp(f);
        if (ftype == 1 && op.act_type[e] == 0 && !op.cg) {
          msg = "internal: an inside cell has a cut face";
          return UF_EGEOMETRY;
        }
        if (side == 1) {
          ++op.n_faces;
          if (ftype == 0) ++op.n_faces_full;
          if (ftype == 1) ++op.n_faces_cut;
          if (ftype == 2) ++op.n_faces_empty;
          if (gp) ++op.n_faces_gp;
        }
      }
  }

  // ---- quadrature of cut cells and their cut faces
  Gauss1 g;
  g.q = op.q;
  gauss_rule(op.q, g.x, g.w);
  op.vol_off.assign(1, 0);
  op.surf_off.assign(1, 0);
  op.cface_off.assign(1, 0);
  op.vline_off.assign(1, 0);
  op.fline_off.assign(1, 0);
  std::vector<QPoint> vol, surf, fq;
  std::vector<QLine> lines;
  std::vector<Fn> balls;
  std::vector<int32_t> cand;
  try {
    for (int64_t c = 0; c < op.n_cut; ++c) {
      const int64_t e = op.cut_cells[c];
      Box b;
      b.m = d;
      for (int a = 0; a < d; ++a) {
        const int64_t I = op.act_index[e * 3 + a];
        b.lo[a] = op.lo[a] + (double)I * hv[a];
        b.hi[a] = op.lo[a] + (double)(I + 1) * hv[a];
      }
      vol.clear();
      surf.clear();
      lines.clear();
      if (op.ls_kind == UF_LS_PLANE) {
        plane_box_rules(b, op.normal, op.offset, g, true, vol, surf, &lines);
      } else if (op.ls_kind == UF_LS_SPHERES) {
        balls.clear();
        for (int64_t i = op.cut_sph_off[c]; i < op.cut_sph_off[c + 1]; ++i) {
          const double *sp = &op.spheres[4 * (size_t)op.cut_sph[i]];
          Fn f{};
          for (int a = 0; a < d; ++a) f.c[a] = sp[a];
          f.rho = sp[3] * sp[3];
          balls.push_back(f);
        }
        union_box_rules(b, balls, g, 0, true, vol, surf, &lines);
      } else {
        sphere_box_rules(b, op.center, op.radius * op.radius, g, 0, true, vol, surf, &lines);
      }
      const int64_t vbase = (int64_t)op.vol_w.size(), sbase = (int64_t)op.surf_w.size();
      for (const QLine &ln : lines)
        op.vol_lines.push_back(QLine{ln.k, vbase + ln.vbeg, ln.vcnt, ln.sidx >= 0 ? sbase + ln.sidx : -1});
      op.vline_off.push_back((int64_t)op.vol_lines.size());
      for (const QPoint &p : vol) {
        for (int a = 0; a < d; ++a) op.vol_xi[a].push_back((p.x[a] - b.lo[a]) / op.h);
        op.vol_w.push_back(p.w);
      }
      for (const QPoint &p : surf) {
        for (int a = 0; a < d; ++a) {
          op.surf_xi[a].push_back((p.x[a] - b.lo[a]) / op.h);
          op.surf_n[a].push_back(p.nrm[a]);
        }
        op.surf_w.push_back(p.w);
      }
      op.vol_off.push_back((int64_t)op.vol_w.size());
      op.surf_off.push_back((int64_t)op.surf_w.size());
      for (int f = 0; f < nf; ++f) {
        if (op.flags[e] & face_bit_sipg_cut(f)) {
          const int axis = f / 2, side = f % 2;
          const int64_t e_minus = side ? e : op.nbr[e * nf + f];
          Box fb = face_box(e_minus, axis);
          const double xa = fb.lo[axis];
          Box sub = drop_dim(fb, axis);
          fq.clear();
          lines.clear();
          std::vector<QPoint> dummy;
          if (op.ls_kind == UF_LS_PLANE) {
            double nsub[kMaxDim];
            drop_vec(op.normal, d, axis, nsub);
            plane_box_rules(sub, nsub, op.offset - op.normal[axis] * xa, g, false, fq, dummy, &lines);
          } else if (op.ls_kind == UF_LS_SPHERES) {
            // the balls whose sphere meets the face, cut by the face's plane
            union_face_candidates(op, e, op.nbr[e * nf + f], cand);
            bool contained = false;
            balls.clear();
            for (int32_t i : cand) {
              const double *sp = &op.spheres[4 * (size_t)i];
              double dmin2, dmax2;
              box_dist2(sp, fb, dmin2, dmax2);
              const double r2 = sp[3] * sp[3];
              if (dmax2 <= r2) {
                contained = true;
              } else if (dmin2 < r2) {
                Fn disc{};
                drop_vec(sp, d, axis, disc.c);
                const double da = xa - sp[axis];
                disc.rho = r2 - da * da;
                balls.push_back(disc);
              }
            }
            if (contained)
              tensor_rule(sub, g, fq, &lines);
            else
              union_box_rules(sub, balls, g, 0, false, fq, dummy, &lines);
          } else {
            const double *cen = op.center;
            double R = op.radius;
            const double da = xa - cen[axis];
            const double rho = R * R - da * da;
            double csub[kMaxDim];
            drop_vec(cen, d, axis, csub);
            sphere_box_rules(sub, csub, rho, g, 0, false, fq, dummy, &lines);
          }
          const int64_t fbase = (int64_t)op.cface_w.size();
          for (const QLine &ln : lines) op.face_lines.push_back(QLine{ln.k, fbase + ln.vbeg, ln.vcnt, -1});
          Box sb = drop_dim(b, axis);
          for (const QPoint &p : fq) {
            for (int a = 0; a < d - 1; ++a) op.cface_eta[a].push_back((p.x[a] - sb.lo[a]) / op.h);
            op.cface_w.push_back(p.w);
          }
          if (side == 1) op.n_face_points_unique += (int64_t)fq.size();
        }
        op.cface_off.push_back((int64_t)op.cface_w.size());
        op.fline_off.push_back((int64_t)op.face_lines.size());
      }
    }
  } catch (const QuadError &) {
    msg = "quadrature subdivision depth exceeded";
    return UF_EGEOMETRY;
  }
  if (volume_gp) {
    // stable-neighbour patches: every cut cell pairs with its active face neighbour of largest
    // volume fraction (inside cells 1; compared after rounding to 12 decimals; first face in
    // the order axis 0 lower, axis 0 upper, ... on ties); a pair chosen twice is one patch
    const double hd = std::pow(op.h, d);
    std::vector<double> key(op.n_active, std::floor(1.0 * 1e12 + 0.5));
    for (int64_t c = 0; c < op.n_cut; ++c) {
      double vol = 0.0;
      for (int64_t p = op.vol_off[c]; p < op.vol_off[c + 1]; ++p) vol += op.vol_w[p];
      key[op.cut_cells[c]] = std::floor(vol / hd * 1e12 + 0.5);
    }
    for (int64_t c = 0; c < op.n_cut; ++c) {
      const int64_t e = op.cut_cells[c];
      int best_f = -1;
      for (int f = 0; f < nf; ++f) {
        const int32_t nb = op.nbr[e * nf + f];
        if (nb >= 0 && (best_f < 0 || key[nb] > key[op.nbr[e * nf + best_f]])) best_f = f;
      }
      if (best_f < 0) continue;
      const int32_t nb = op.nbr[e * nf + best_f];
      const int f_nb = best_f ^ 1;  // the same face seen from the neighbour
      if (!(op.flags[e] & face_bit_gp(best_f))) ++op.n_faces_gp;
      op.flags[e] |= face_bit_gp(best_f);
      op.flags[nb] |= face_bit_gp(f_nb);
    }
  }
  if (op.cg) {
    // lattice point p I_a + i_a of every cell-local DoF; used points numbered in lexicographic
    // order (x fastest), which is the order of their linear lattice index
    int64_t ldim[kMaxDim] = {1, 1, 1};
    for (int a = 0; a < d; ++a) ldim[a] = op.p * op.N[a] + 1;
    const int64_t n_loc = op.n_active * op.ndof;
    std::vector<int64_t> lat(n_loc);
    for (int64_t e = 0; e < op.n_active; ++e)
      for (int l = 0; l < op.ndof; ++l) {
        int64_t key = 0, stride = 1, rem = l;
        for (int a = 0; a < d; ++a) {
          const int64_t ia = rem % op.n;
          rem /= op.n;
          key += (op.act_index[e * 3 + a] * op.p + ia) * stride;
          stride *= ldim[a];
        }
        lat[e * op.ndof + l] = key;
      }
    std::vector<int64_t> order(n_loc);
    for (int64_t i = 0; i < n_loc; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return lat[a] < lat[b]; });
    op.cg_l2g.assign(n_loc, -1);
    op.cg_own_idx.assign(n_loc, 0);
    op.cg_own_off.clear();
    int64_t g = -1;
    for (int64_t k = 0; k < n_loc; ++k) {
      const int64_t i = order[k];
      if (k == 0 || lat[i] != lat[order[k - 1]]) {
        ++g;
        op.cg_own_off.push_back((int32_t)k);
      }
      op.cg_l2g[i] = (int32_t)g;
      op.cg_own_idx[k] = (int32_t)i;  // owners ascending (stable sort of ascending indices)
    }
    op.n_cg = g + 1;
    op.cg_own_off.push_back((int32_t)n_loc);
  }
  return UF_OK;
}

}  // namespace uf
