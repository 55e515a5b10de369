// Sphere accuracy benchmark (arXiv 2404.07911, Sec. 4): load vector of the manufactured
// right-hand side and L2 error of a discrete solution, on the operator's own quadrature (host,
// FP64).  Set-up and post-processing of the accuracy study; not on the operator's hot path.
//
// On the ball of radius R around c (the operator's sphere), with r = |x - c| and d the dimension,
//   u(r) = cos(omega R) - cos(omega r),   f(r) = -omega^2 (cos(omega r) + (d - 1) sinc(omega r)),
// so that -Lap u = f and u = 0 on the sphere (the Dirichlet data g = 0 of the Nitsche terms).
#include <cmath>
#include <string>
#include <vector>

#include "uf_operator.h"

namespace {

using uf::HostOperator;

double sphere_r(const HostOperator &H, const double *x) {
  double r2 = 0.0;
  for (int a = 0; a < H.dim; ++a) {
    const double t = x[a] - H.center[a];
    r2 += t * t;
  }
  return std::sqrt(r2);
}

double mf_solution(const HostOperator &H, double omega, const double *x) {
  return std::cos(omega * H.radius) - std::cos(omega * sphere_r(H, x));
}

double mf_rhs(const HostOperator &H, double omega, const double *x) {
  const double z = omega * sphere_r(H, x);
  const double sinc = (z == 0.0) ? 1.0 : std::sin(z) / z;
  return -omega * omega * (std::cos(z) + (H.dim - 1) * sinc);
}

// Calls fn(e, phi[ndof], w, x[3]) for every quadrature point of every active cell: the tensor
// Gauss rule with n points per direction on inside cells, the cut-cell volume rule on cut cells.
template <class F>
void for_each_point(const HostOperator &H, F &&fn) {
  const int d = H.dim, n = H.n, nd = H.ndof;
  std::vector<double> phi(nd);
  double hd = 1.0;
  for (int a = 0; a < d; ++a) hd *= H.h;
  auto eval = [&](const double *xi) {
    double v[3][uf::kMaxN], dv[uf::kMaxN];
    for (int a = 0; a < d; ++a) uf::lagrange_values(H.t, xi[a], v[a], dv);
    for (int l = 0; l < nd; ++l) {
      double prod = 1.0;
      int rem = l;
      for (int a = 0; a < d; ++a) {
        prod *= v[a][rem % n];
        rem /= n;
      }
      phi[l] = prod;
    }
  };
  for (int64_t e = 0; e < H.n_active; ++e) {
    double lo[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) lo[a] = H.lo[a] + (double)H.act_index[e * 3 + a] * H.h;
    double xi[3] = {0, 0, 0}, x[3] = {0, 0, 0};
    if (H.act_type[e] == 0) {
      int total = 1;
      for (int a = 0; a < d; ++a) total *= n;
      for (int flat = 0; flat < total; ++flat) {
        double w = hd;
        int rem = flat;
        for (int a = 0; a < d; ++a) {
          const int i = rem % n;
          rem /= n;
          xi[a] = H.t.gauss_x[i];
          w *= H.t.gauss_w[i];
          x[a] = lo[a] + H.h * xi[a];
        }
        eval(xi);
        fn(e, phi.data(), w, x);
      }
    } else {
      const int64_t c = H.cut_of[e];
      for (int64_t p = H.vol_off[c]; p < H.vol_off[c + 1]; ++p) {
        for (int a = 0; a < d; ++a) {
          xi[a] = H.vol_xi[a][p];
          x[a] = lo[a] + H.h * xi[a];
        }
        eval(xi);
        fn(e, phi.data(), H.vol_w[p], x);
      }
    }
  }
}

uf_status check(const uf_operator *op, double omega) {
  if (!op) return uf::fail(UF_EINVAL, "NULL argument");
  if (op->host.params.ls_kind != UF_LS_SPHERE)
    return uf::fail(UF_EUNSUPPORTED, "the manufactured solution is defined on the sphere only");
  if (!std::isfinite(omega)) return uf::fail(UF_EINVAL, "omega must be finite");
  return UF_OK;
}

}  // namespace

extern "C" {

uf_status uf_manufactured_rhs(const uf_operator *op, double omega, double *b) {
  uf_status st = check(op, omega);
  if (st != UF_OK) return st;
  if (!b) return uf::fail(UF_EINVAL, "NULL argument");
  const HostOperator &H = op->host;
  const int nd = H.ndof;
  std::vector<double> bloc((size_t)H.n_active * nd, 0.0);
  for_each_point(H, [&](int64_t e, const double *phi, double w, const double *x) {
    const double fw = w * mf_rhs(H, omega, x);
    double *be = &bloc[(size_t)e * nd];
    for (int l = 0; l < nd; ++l) be[l] += fw * phi[l];
  });
  if (!H.cg) {
    std::copy(bloc.begin(), bloc.end(), b);
    return UF_OK;
  }
  for (int64_t g = 0; g < H.n_cg; ++g) {
    double acc = 0.0;
    for (int32_t o = H.cg_own_off[g]; o < H.cg_own_off[g + 1]; ++o) acc += bloc[H.cg_own_idx[o]];
    b[g] = acc;
  }
  return UF_OK;
}

uf_status uf_l2_error(const uf_operator *op, double omega, const double *x, double *err,
                      double *norm) {
  uf_status st = check(op, omega);
  if (st != UF_OK) return st;
  if (!x || !err || !norm) return uf::fail(UF_EINVAL, "NULL argument");
  const HostOperator &H = op->host;
  const int nd = H.ndof;
  double e2 = 0.0, n2 = 0.0;
  for_each_point(H, [&](int64_t e, const double *phi, double w, const double *xp) {
    double uh = 0.0;
    for (int l = 0; l < nd; ++l) {
      const int64_t i = e * nd + l;
      uh += phi[l] * (H.cg ? x[H.cg_l2g[i]] : x[i]);
    }
    const double ue = mf_solution(H, omega, xp);
    e2 += w * (uh - ue) * (uh - ue);
    n2 += w * ue * ue;
  });
  *err = std::sqrt(e2);
  *norm = std::sqrt(n2);
  return UF_OK;
}

}  // extern "C"
