// C ABI of libunfitted: creation (host setup + device upload), vmult / adjoint dispatch,
// host-buffer vmult, exports.  Declarations and contracts: include/unfitted.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/unfitted.h"
#include "uf_device.h"
#include "uf_host.h"
#include "uf_operator.h"

namespace {
thread_local std::string g_last_error;

// Bump allocator over a byte count (256-byte aligned sub-arrays).
struct Layout {
  size_t bytes = 0;
  size_t take(size_t n) {
    size_t off = bytes;
    bytes += (n + 255) / 256 * 256;
    return off;
  }
};
}  // namespace

namespace uf {
uf_status fail(uf_status st, const std::string &msg) {
  g_last_error = msg;
  return st;
}

namespace {
// allocations that succeed before the injected failure (-1: none armed), and the live count
std::atomic<int64_t> g_fail_after{-1};
std::atomic<int64_t> g_live_allocations{0};

// True once, for the allocation that the armed hook makes fail; the hook then disarms.
bool injected_failure() {
  int64_t v = g_fail_after.load();
  while (v >= 0)
    if (g_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;
  return false;
}
}  // namespace

cudaError_t dev_malloc_raw(void **p, size_t bytes) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  const cudaError_t err = cudaMalloc(p, bytes);
  if (err == cudaSuccess && *p) ++g_live_allocations;
  return err;
}

cudaError_t pinned_malloc_raw(void **p, size_t bytes) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  const cudaError_t err = cudaMallocHost(p, bytes);
  if (err == cudaSuccess && *p) ++g_live_allocations;
  return err;
}

void dev_free(void *p) {
  if (!p) return;
  cudaFree(p);
  --g_live_allocations;
}

void pinned_free(void *p) {
  if (!p) return;
  cudaFreeHost(p);
  --g_live_allocations;
}

uf_operator *new_operator() {
  if (injected_failure()) return nullptr;
  uf_operator *op = new (std::nothrow) uf_operator();
  if (op) ++g_live_allocations;
  return op;
}

void delete_operator(uf_operator *op) {
  if (!op) return;
  delete op;
  --g_live_allocations;
}
}  // namespace uf

using uf::fail;
using uf::PrecisionData;
using uf::ProfSlot;
using uf::DeviceGuard;

// ------------------------------------------------------------------------------------------
// Constant 1D matrices of the structured terms (see uf_device.h for their meaning).
// ------------------------------------------------------------------------------------------
void uf::structured_matrices(const uf::HostOperator &op, std::vector<double> &out) {
  // layout of uf::StructTables: 16 matrices (n x n), then dow[2][n], dnb[2][n]
  const int n = op.n, nn = n * n, d = op.dim;
  const uf::Tables1D &t = op.t;
  const double h = op.h;
  const double hf = std::pow(h, d - 1);
  const double sig = op.params.sipg_gamma / h;
  out.assign(16 * nn + 4 * n, 0.0);
  double *kv = &out[0], *mass = &out[nn];
  for (int s = 0; s < 2; ++s) {
    const double sgn = s ? 1.0 : -1.0;
    for (int i = 0; i < n; ++i) {
      out[16 * nn + s * n + i] = sgn * t.deriv_end[s][1][i] / h;          // dow[s]
      out[16 * nn + 2 * n + s * n + i] = sgn * t.deriv_end[1 - s][1][i] / h;  // dnb[s]
    }
  }
  const double hv = std::pow(h, d - 2);
  for (int i = 0; i < nn; ++i) {
    kv[i] = hv * t.stiff[i];
    mass[i] = t.mass[i];
  }
  double gam[uf::kMaxN] = {0};
  for (int j = 1; j <= op.params.gp_max_order; ++j) {
    double fact = 1.0;
    for (int k = 2; k <= j; ++k) fact *= k;
    gam[j] = op.params.gp_gamma * std::pow(h, 2 * j - 1) / (fact * fact);
  }
  for (int s = 0; s < 2; ++s) {
    const double sgn = s ? 1.0 : -1.0;  // outward normal of the own face along the axis
    double e_own[uf::kMaxN], d_own[uf::kMaxN], e_nb[uf::kMaxN], d_nb[uf::kMaxN];
    double t_own[uf::kMaxN][uf::kMaxN], t_nb[uf::kMaxN][uf::kMaxN];  // [j][i]
    for (int i = 0; i < n; ++i) {
      e_own[i] = t.deriv_end[s][0][i];
      e_nb[i] = t.deriv_end[1 - s][0][i];
      d_own[i] = sgn * t.deriv_end[s][1][i] / h;
      d_nb[i] = sgn * t.deriv_end[1 - s][1][i] / h;
      double sj = 1.0, hj = 1.0;
      for (int j = 1; j <= op.p; ++j) {
        sj *= sgn;
        hj *= h;
        t_own[j][i] = sj * t.deriv_end[s][j][i] / hj;
        t_nb[j][i] = sj * t.deriv_end[1 - s][j][i] / hj;
      }
    }
    double *A = &out[(2 + s) * nn], *P = &out[(4 + s) * nn], *G = &out[(6 + s) * nn];
    double *B = &out[(8 + s) * nn], *C = &out[(10 + s) * nn], *Q = &out[(12 + s) * nn];
    double *H = &out[(14 + s) * nn];
    for (int r = 0; r < n; ++r)
      for (int m = 0; m < n; ++m) {
        const int k = r * n + m;
        A[k] = hf * -0.5 * (d_own[r] * e_own[m] + e_own[r] * d_own[m]);
        P[k] = hf * sig * e_own[r] * e_own[m];
        B[k] = hf * 0.5 * d_own[r] * e_nb[m];
        C[k] = hf * -0.5 * e_own[r] * d_nb[m];
        Q[k] = hf * -sig * e_own[r] * e_nb[m];
        double g = 0.0, hh = 0.0;
        for (int j = 1; j <= op.params.gp_max_order; ++j) {
          g += gam[j] * t_own[j][r] * t_own[j][m];
          hh += gam[j] * t_own[j][r] * t_nb[j][m];
        }
        G[k] = hf * g;
        H[k] = -hf * hh;
      }
    if (op.params.gp_kind == UF_GP_VOLUME && op.params.gp_max_order > 0) {
      // Volume ghost penalty on the patch with the neighbour across face s (Kronecker form: the
      // in-face mass sweeps supply the other axes).  Along the axis, with the neighbour's cell at
      // xi + sigma (sigma = +-1) and Gauss points x_q of [0, 1]:
      //   own-own  tau h^{d-2} (M + sum_q w_q phi_r(x_q + sigma) phi_m(x_q + sigma))
      //   own-nb  -tau h^{d-2} (sum_q w_q phi_r(x_q) phi_m(x_q - sigma)
      //                         + sum_q w_q phi_r(x_q + sigma) phi_m(x_q))
      const double sigma = s ? 1.0 : -1.0, c = op.params.gp_tau * std::pow(h, d - 2);
      double vq[uf::kMaxN][uf::kMaxN], vp[uf::kMaxN][uf::kMaxN], vm[uf::kMaxN][uf::kMaxN], dd[uf::kMaxN];
      for (int q = 0; q < n; ++q) {
        uf::lagrange_values(t, t.gauss_x[q], vq[q], dd);
        uf::lagrange_values(t, t.gauss_x[q] + sigma, vp[q], dd);
        uf::lagrange_values(t, t.gauss_x[q] - sigma, vm[q], dd);
      }
      for (int r = 0; r < n; ++r)
        for (int m = 0; m < n; ++m) {
          double ee = 0.0, x1 = 0.0, x2 = 0.0;
          for (int q = 0; q < n; ++q) {
            ee += t.gauss_w[q] * vp[q][r] * vp[q][m];
            x1 += t.gauss_w[q] * vq[q][r] * vm[q][m];
            x2 += t.gauss_w[q] * vp[q][r] * vq[q][m];
          }
          G[r * n + m] = c * (t.mass[r * n + m] + ee);
          H[r * n + m] = -c * (x1 + x2);
        }
    }
  }
}

namespace {
using uf::structured_matrices;

// Inverse of a small SPD matrix (n x n, row-major) by Gauss-Jordan elimination with partial
// pivoting.
std::vector<double> invert_small(std::vector<double> a, int n) {
  std::vector<double> inv(n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(a[r * n + col]) > std::fabs(a[piv * n + col])) piv = r;
    for (int c2 = 0; c2 < n; ++c2) {
      std::swap(a[col * n + c2], a[piv * n + c2]);
      std::swap(inv[col * n + c2], inv[piv * n + c2]);
    }
    const double dinv = 1.0 / a[col * n + col];
    for (int c2 = 0; c2 < n; ++c2) {
      a[col * n + c2] *= dinv;
      inv[col * n + c2] *= dinv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = a[r * n + col];
      if (f == 0.0) continue;
      for (int c2 = 0; c2 < n; ++c2) {
        a[r * n + c2] -= f * a[col * n + c2];
        inv[r * n + c2] -= f * inv[col * n + c2];
      }
    }
  }
  return inv;
}

// kappa = 1 variants of the per-axis self matrix (32, indexed by inside | full_lo << 1 |
// gp_lo << 2 | full_hi << 3 | gp_hi << 4) and of a ghost-penalty neighbour coupling
// (4, indexed by 2 * side + full), from the constant matrices of structured_matrices.
void variant_tables(const uf::HostOperator &op, const std::vector<double> &m,
                    std::vector<double> &lself, std::vector<double> &lnbgp) {
  const int nn = op.n * op.n;
  auto M = [&](int which, int s) { return &m[(which + s) * nn]; };  // which: 2 a, 4 pen, ...
  lself.assign(32 * nn, 0.0);
  for (int v = 0; v < 32; ++v)
    for (int i = 0; i < nn; ++i) {
      double acc = (v & 1) ? m[i] : 0.0;  // kv
      for (int s = 0; s < 2; ++s) {
        const bool full = (v >> (1 + 2 * s)) & 1, gp = (v >> (2 + 2 * s)) & 1;
        if (full) acc += M(2, s)[i] + M(4, s)[i];
        if (gp) acc += M(6, s)[i];
      }
      lself[v * nn + i] = acc;
    }
  lnbgp.assign(4 * nn, 0.0);
  for (int s = 0; s < 2; ++s)
    for (int full = 0; full < 2; ++full)
      for (int i = 0; i < nn; ++i)
        lnbgp[(2 * s + full) * nn + i] =
            (full ? M(8, s)[i] + M(10, s)[i] + M(12, s)[i] : 0.0) + M(14, s)[i];
}

// Outer reference coordinate `which` (0: lower other axis, 1: upper) of a line along axis k.
double line_outer(const uf::HostOperator &H, const uf::QLine &ln, int which) {
  const int d = H.dim, k = ln.k;
  int ob = (k == 0) ? 1 : 0, oc = (k == 2) ? 1 : 2;
  if (d == 2) ob = 1 - k;
  if (which == 1 && d == 2) return 0.0;
  const bool from_vol = ln.vcnt > 0;
  const int64_t p0 = from_vol ? ln.vbeg : ln.sidx;
  const std::vector<double> *xi = from_vol ? H.vol_xi : H.surf_xi;
  return xi[which == 0 ? ob : oc][p0];
}

// Groups of the lines of one cut cell along one axis (3D): lines that share one outer
// coordinate (the points of one line of the (d-1)-dimensional outer rule) form a group, so the
// contraction along the shared axis is done once per group.  The shared axis is the one with
// fewer distinct values; `lines` is reordered so that groups are contiguous, and
// group_start[i] = index in `lines` of the first line of line i's group.  Returns 1 if the
// lines share the lower outer coordinate, 0 if the upper one (2D: no groups, returns 0).
int group_lines(const uf::HostOperator &H, std::vector<const uf::QLine *> &lines,
                std::vector<int> &group_start) {
  group_start.resize(lines.size());
  if (H.dim != 3 || lines.empty()) {
    for (size_t i = 0; i < lines.size(); ++i) group_start[i] = (int)i;
    return 0;
  }
  auto distinct = [&](int which) {
    std::vector<double> v;
    for (const uf::QLine *l : lines) v.push_back(line_outer(H, *l, which));
    std::sort(v.begin(), v.end());
    return std::unique(v.begin(), v.end()) - v.begin();
  };
  const int shared_lo = distinct(0) < distinct(1) ? 1 : 0;
  const int which = shared_lo ? 0 : 1;
  std::stable_sort(lines.begin(), lines.end(), [&](const uf::QLine *a, const uf::QLine *b) {
    return line_outer(H, *a, which) < line_outer(H, *b, which);
  });
  for (size_t i = 0; i < lines.size(); ++i)
    group_start[i] = (i > 0 && line_outer(H, *lines[i], which) == line_outer(H, *lines[i - 1], which))
                         ? group_start[i - 1]
                         : (int)i;
  return shared_lo;
}

// Number of line groups of all cut cells (group_lines), for the as-built operation count.
int64_t count_line_groups(const uf::HostOperator &H) {
  int64_t groups = 0;
  std::vector<int> gs;
  for (int64_t c = 0; c < H.n_cut; ++c)
    for (int k = 0; k < H.dim; ++k) {
      std::vector<const uf::QLine *> lk;
      for (int64_t li = H.vline_off[c]; li < H.vline_off[c + 1]; ++li)
        if (H.vol_lines[li].k == k) lk.push_back(&H.vol_lines[li]);
      group_lines(H, lk, gs);
      for (size_t i = 0; i < gs.size(); ++i) groups += (gs[i] == (int)i) ? 1 : 0;
    }
  return groups;
}

bool kappa_is_uniform(const std::vector<double> &k) {
  for (double v : k)
    if (v != k[0]) return false;
  return true;
}

template <typename T>
uf_status upload(uf_operator *op, PrecisionData<T> &pd) {
  const uf::HostOperator &H = op->host;
  const int d = H.dim, nf = 2 * d, n = H.n;
  const int64_t na = H.n_active, nc = H.n_cut;
  const int64_t nv = (int64_t)H.vol_w.size(), ns = (int64_t)H.surf_w.size();
  const int64_t nfp = (int64_t)H.cface_w.size();
  if (nv > INT32_MAX || ns > INT32_MAX || nfp > INT32_MAX)
    return fail(UF_EUNSUPPORTED, "too many quadrature points for 32-bit offsets");

  // cut cells ordered by decreasing work (points of volume, surface and cut faces)
  std::vector<int32_t> order(nc);
  std::iota(order.begin(), order.end(), 0);
  // lane class of a cut cell (32, 16 or 8 lanes: the class's chunk holds all its volume lines and
  // all its cut-face lines), then decreasing work within a class; classes are contiguous
  std::vector<int64_t> cost(nc);
  std::vector<int> lanes(nc);
  for (int64_t c = 0; c < nc; ++c) {
    cost[c] = (H.vol_off[c + 1] - H.vol_off[c]) + (H.surf_off[c + 1] - H.surf_off[c]) +
              (H.cface_off[(c + 1) * nf] - H.cface_off[c * nf]);
    lanes[c] = uf::cut_lanes_of_cell(H, c);
    // FP32: the 16-lane groups measured slower than full warps (the 8-lane ones faster)
    if (sizeof(T) == sizeof(float) && lanes[c] == 16) lanes[c] = 32;
  }
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return lanes[a] != lanes[b] ? lanes[a] > lanes[b] : cost[a] > cost[b];
  });
  std::vector<int32_t> cut_list(nc), cut_idx(nc);
  for (int64_t i = 0; i < nc; ++i) {
    cut_idx[i] = order[i];
    cut_list[i] = H.cut_cells[order[i]];
  }
  // parts of the host-buffer pipeline: kPipeParts runs of consecutive cells (discontinuous
  // operators with enough cells); the cut cells of each part keep the order above, so each part
  // has the same three lane classes; all parts' lists are stored one after the other
  const int n_parts = (!H.cg && na >= 8 * 1024) ? uf::kPipeParts : 1;
  std::vector<int32_t> part_list, part_idx;
  std::vector<std::array<int32_t, 6>> part_meta;  // cell_begin, cell_end, 4 slot bounds
  {
    std::vector<std::vector<int32_t>> bucket(n_parts);
    auto part_of = [&](int64_t e) { return (int)((e * n_parts) / na); };
    for (int64_t i = 0; i < nc; ++i) bucket[part_of(H.cut_cells[order[i]])].push_back(order[i]);
    for (int pi = 0; pi < n_parts; ++pi) {
      std::array<int32_t, 6> m{};
      // the cells with part_of(e) == pi: ceil(pi na / n_parts) <= e < ceil((pi + 1) na / n_parts)
      const int64_t cb = (na * pi + n_parts - 1) / n_parts, ce = (na * (pi + 1) + n_parts - 1) / n_parts;
      m[0] = (int32_t)cb;
      m[1] = (int32_t)ce;
      m[2] = (int32_t)part_list.size();
      int cls[3] = {0, 0, 0};
      for (int32_t c : bucket[pi]) {
        part_list.push_back(H.cut_cells[c]);
        part_idx.push_back(c);
        ++cls[lanes[c] == 32 ? 0 : (lanes[c] == 16 ? 1 : 2)];
      }
      m[3] = m[2] + cls[0];
      m[4] = m[3] + cls[1];
      m[5] = m[4] + cls[2];
      part_meta.push_back(m);
    }
  }

  // ---- line-structured point data (lines of a cell sorted by axis)
  std::vector<int32_t> vline_koff(nc * 4), vpt_off, lsurf, fline_koff(nc * nf * 3), fpt_off, vline_grp;
  std::vector<double> vline_o0, vline_o1, vpt_t, vpt_w, spt_t, spt_w, spt_n[3];
  std::vector<double> fline_o, fpt_t, fpt_w;
  vpt_off.push_back(0);
  fpt_off.push_back(0);
  for (int64_t c = 0; c < nc; ++c) {
    std::vector<uf::QLine> ls(H.vol_lines.begin() + H.vline_off[c],
                              H.vol_lines.begin() + H.vline_off[c + 1]);
    std::stable_sort(ls.begin(), ls.end(), [](const uf::QLine &a, const uf::QLine &b) { return a.k < b.k; });
    for (int k = 0; k < 4; ++k) {
      vline_koff[c * 4 + k] = (int32_t)lsurf.size();
      std::vector<const uf::QLine *> lk;
      if (k < d)
        for (const uf::QLine &ln : ls)
          if (ln.k == k) lk.push_back(&ln);
      std::vector<int> gstart;
      const int shared_lo = group_lines(H, lk, gstart);
      const int32_t first = (int32_t)lsurf.size();
      for (size_t i = 0; i < lk.size(); ++i) {
        const uf::QLine &ln = *lk[i];
        vline_grp.push_back(((first + gstart[i]) << 1) | shared_lo);
        vline_o0.push_back(line_outer(H, ln, 0));
        vline_o1.push_back(line_outer(H, ln, 1));
        for (int64_t p = ln.vbeg; p < ln.vbeg + ln.vcnt; ++p) {
          vpt_t.push_back(H.vol_xi[k][p]);
          vpt_w.push_back(H.vol_w[p]);
        }
        vpt_off.push_back((int32_t)vpt_t.size());
        if (ln.sidx >= 0) {
          lsurf.push_back((int32_t)spt_t.size());
          spt_t.push_back(H.surf_xi[k][ln.sidx]);
          spt_w.push_back(H.surf_w[ln.sidx]);
          for (int a = 0; a < 3; ++a) spt_n[a].push_back(a < d ? H.surf_n[a][ln.sidx] : 0.0);
        } else {
          lsurf.push_back(-1);
        }
      }
    }
    for (int f = 0; f < nf; ++f) {
      std::vector<uf::QLine> fls(H.face_lines.begin() + H.fline_off[c * nf + f],
                                 H.face_lines.begin() + H.fline_off[c * nf + f + 1]);
      std::stable_sort(fls.begin(), fls.end(), [](const uf::QLine &a, const uf::QLine &b) { return a.k < b.k; });
      for (int kk = 0; kk < 3; ++kk) {
        fline_koff[(c * nf + f) * 3 + kk] = (int32_t)fline_o.size();
        if (kk < d - 1)
          for (const uf::QLine &ln : fls) {
            if (ln.k != kk) continue;
            fline_o.push_back(d == 3 ? H.cface_eta[1 - kk][ln.vbeg] : 0.0);
            for (int64_t p = ln.vbeg; p < ln.vbeg + ln.vcnt; ++p) {
              fpt_t.push_back(H.cface_eta[kk][p]);
              fpt_w.push_back(H.cface_w[p]);
            }
            fpt_off.push_back((int32_t)fpt_t.size());
          }
      }
    }
  }
  const int64_t nvl = (int64_t)lsurf.size(), nfl = (int64_t)fline_o.size();
  if ((int64_t)vpt_t.size() != nv || (int64_t)spt_t.size() != ns || (int64_t)fpt_t.size() != nfp)
    return fail(UF_EGEOMETRY, "internal: line structure does not cover every quadrature point");

  Layout L;
  const size_t o_nbr = L.take(sizeof(int32_t) * na * nf);
  const size_t o_flags = L.take(sizeof(uint32_t) * na);
  const size_t o_kappa = L.take(sizeof(T) * na);
  const size_t o_clist = L.take(sizeof(int32_t) * std::max<int64_t>(nc, 1));
  const size_t o_cidx = L.take(sizeof(int32_t) * std::max<int64_t>(nc, 1));
  const size_t o_plist = L.take(sizeof(int32_t) * std::max<int64_t>(nc, 1));
  const size_t o_pidx = L.take(sizeof(int32_t) * std::max<int64_t>(nc, 1));
  const size_t o_vlk = L.take(sizeof(int32_t) * std::max<int64_t>(nc * 4, 1));
  const size_t o_vo0 = L.take(sizeof(T) * std::max<int64_t>(nvl, 1));
  const size_t o_vo1 = L.take(sizeof(T) * std::max<int64_t>(nvl, 1));
  const size_t o_vpo = L.take(sizeof(int32_t) * (nvl + 1));
  const size_t o_lsf = L.take(sizeof(int32_t) * std::max<int64_t>(nvl, 1));
  const size_t o_vlg = L.take(sizeof(int32_t) * std::max<int64_t>(nvl, 1));
  const size_t o_vpt = L.take(sizeof(T) * std::max<int64_t>(nv, 1));
  const size_t o_vpw = L.take(sizeof(T) * std::max<int64_t>(nv, 1));
  const size_t o_spt = L.take(sizeof(T) * std::max<int64_t>(ns, 1));
  const size_t o_spw = L.take(sizeof(T) * std::max<int64_t>(ns, 1));
  size_t o_spn[3];
  for (int a = 0; a < 3; ++a) o_spn[a] = L.take(sizeof(T) * std::max<int64_t>(ns, 1));
  const size_t o_flk = L.take(sizeof(int32_t) * std::max<int64_t>(nc * nf * 3, 1));
  const size_t o_flo = L.take(sizeof(T) * std::max<int64_t>(nfl, 1));
  const size_t o_fpo = L.take(sizeof(int32_t) * (nfl + 1));
  const size_t o_fpt = L.take(sizeof(T) * std::max<int64_t>(nfp, 1));
  const size_t o_fpw = L.take(sizeof(T) * std::max<int64_t>(nfp, 1));
  std::vector<double> mats, lself0, lnbgp0;
  structured_matrices(H, mats);
  // The structured kernel evaluates sum_a (M .. L_a .. M) u as (M (x) M (x) M) sum_a M_a^{-1} L_a u
  // (3 mass sweeps in 3D instead of 5), so every per-axis 1D table is premultiplied by M^{-1}.
  const int nn = n * n;
  const std::vector<double> minv = invert_small(std::vector<double>(mats.begin() + nn, mats.begin() + 2 * nn), n);
  auto premul = [&](const std::vector<double> &m, size_t blocks, bool transpose) {
    std::vector<double> out(blocks * nn);
    for (size_t b = 0; b < blocks; ++b)
      for (int r = 0; r < n; ++r)
        for (int c2 = 0; c2 < n; ++c2) {
          double acc = 0.0;
          for (int k = 0; k < n; ++k)
            acc += minv[r * n + k] * (transpose ? m[b * nn + c2 * n + k] : m[b * nn + k * n + c2]);
          out[b * nn + r * n + c2] = acc;
        }
    return out;
  };
  const std::vector<double> smat = premul(mats, 16, false), smatT = premul(mats, 16, true);
  const size_t o_smat = L.take(sizeof(T) * smat.size());
  const size_t o_smatT = L.take(sizeof(T) * smatT.size());
  const size_t o_smat0 = L.take(sizeof(T) * 16 * nn);
  variant_tables(H, mats, lself0, lnbgp0);
  const std::vector<double> lself = premul(lself0, 32, false), lnbgp = premul(lnbgp0, 4, false);
  const size_t o_lself = L.take(sizeof(T) * lself.size());
  const size_t o_lnbgp = L.take(sizeof(T) * lnbgp.size());
  const std::vector<double> lselfT = premul(lself0, 32, true), lnbgpT = premul(lnbgp0, 4, true);
  auto transposed = [&](const std::vector<double> &m) {
    std::vector<double> t(m.size());
    for (size_t b = 0; b < m.size() / nn; ++b)
      for (int r = 0; r < n; ++r)
        for (int c2 = 0; c2 < n; ++c2) t[b * nn + r * n + c2] = m[b * nn + c2 * n + r];
    return t;
  };
  const std::vector<double> lselfxT = transposed(lself0), lnbgpxT = transposed(lnbgp0);
  const size_t o_lselfx = L.take(sizeof(T) * lself0.size());
  const size_t o_lnbgpx = L.take(sizeof(T) * lnbgp0.size());
  const size_t o_lselfxT = L.take(sizeof(T) * lselfxT.size());
  const size_t o_lnbgpxT = L.take(sizeof(T) * lnbgpxT.size());
  const size_t o_lselfT = L.take(sizeof(T) * lselfT.size());
  const size_t o_lnbgpT = L.take(sizeof(T) * lnbgpT.size());
  // FP64: the 1D basis at every line and point (the FP64 pipe is the bottleneck there, HBM is not)
  const bool pre = sizeof(T) == sizeof(double);
  std::vector<double> vline_b, vpt_b, spt_b, fline_b, fpt_b;
  if (pre) {
    double v[uf::kMaxN], dv[uf::kMaxN];
    vline_b.assign((size_t)std::max<int64_t>(nvl, 1) * 4 * n, 0.0);
    for (int64_t l = 0; l < nvl; ++l) {
      uf::lagrange_values(H.t, vline_o0[l], v, dv);
      for (int i = 0; i < n; ++i) {
        vline_b[l * 4 * n + i] = v[i];
        vline_b[l * 4 * n + n + i] = dv[i];
      }
      if (d == 3) {
        uf::lagrange_values(H.t, vline_o1[l], v, dv);
        for (int i = 0; i < n; ++i) {
          vline_b[l * 4 * n + 2 * n + i] = v[i];
          vline_b[l * 4 * n + 3 * n + i] = dv[i];
        }
      }
    }
    auto pts = [&](const std::vector<double> &tt, std::vector<double> &out, bool deriv) {
      const int w = deriv ? 2 * n : n;
      out.assign((size_t)std::max<size_t>(tt.size(), 1) * w, 0.0);
      for (size_t p = 0; p < tt.size(); ++p) {
        uf::lagrange_values(H.t, tt[p], v, dv);
        for (int i = 0; i < n; ++i) {
          out[p * w + i] = v[i];
          if (deriv) out[p * w + n + i] = dv[i];
        }
      }
    };
    pts(vpt_t, vpt_b, true);
    pts(spt_t, spt_b, true);
    pts(fpt_t, fpt_b, false);
    fline_b.assign((size_t)std::max<int64_t>(nfl, 1) * n, 0.0);
    if (d == 3)
      for (int64_t l = 0; l < nfl; ++l) {
        uf::lagrange_values(H.t, fline_o[l], v, dv);
        for (int i = 0; i < n; ++i) fline_b[l * n + i] = v[i];
      }
  }
  // FP64, per volume line: stiffness and mass integrals of the 1D basis over the line's points
  std::vector<double> vline_km(pre ? (size_t)std::max<int64_t>(nvl, 1) * 2 * nn : 0, 0.0);
  if (pre) {
    double v[uf::kMaxN], dv[uf::kMaxN];
    const double ih2 = 1.0 / (H.h * H.h);
    for (int64_t l = 0; l < nvl; ++l) {
      double *K = vline_km.data() + (size_t)l * 2 * nn, *M = K + nn;
      for (int32_t p = vpt_off[l]; p < vpt_off[l + 1]; ++p) {
        uf::lagrange_values(H.t, vpt_t[p], v, dv);
        const double w = vpt_w[p] * ih2;
        for (int i = 0; i < n; ++i)
          for (int j = 0; j < n; ++j) {
            K[i * n + j] += w * dv[i] * dv[j];
            M[i * n + j] += w * v[i] * v[j];
          }
      }
    }
  }
  // FP64, 3D, n <= kFaceMatrixMaxN: per cut cell and cut face, the face's mass matrix over its
  // points in the in-face tensor basis, tl = i_b' + n i_c' (the index of the cut-cell kernel's
  // trace arrays: along the line m, along the outer coordinate io, tl = m + n io for lines along
  // b', io + n m for lines along c'); w (phi_a phi_b) keeps it symmetric bit for bit
  const bool fmats = pre && d == 3 && n <= uf::kFaceMatrixMaxN;
  std::vector<int32_t> fmat_idx;
  std::vector<double> fmat;
  if (fmats) {
    const int nl2 = n * n;
    fmat_idx.assign((size_t)std::max<int64_t>(nc * nf, 1), -1);
    double v[uf::kMaxN], dv[uf::kMaxN], vo[uf::kMaxN], phi[uf::kMaxN * uf::kMaxN];
    int32_t cnt = 0;
    for (int64_t c = 0; c < nc; ++c)
      for (int f = 0; f < nf; ++f) {
        const int32_t *ko = &fline_koff[(size_t)(c * nf + f) * 3];
        if (ko[2] == ko[0]) continue;
        fmat_idx[c * nf + f] = cnt++;
        fmat.resize((size_t)cnt * nl2 * nl2, 0.0);
        double *Mf = fmat.data() + (size_t)(cnt - 1) * nl2 * nl2;
        for (int32_t l = ko[0]; l < ko[2]; ++l) {
          const bool along_b = l < ko[1];
          uf::lagrange_values(H.t, fline_o[l], vo, dv);
          for (int32_t q = fpt_off[l]; q < fpt_off[l + 1]; ++q) {
            uf::lagrange_values(H.t, fpt_t[q], v, dv);
            for (int io = 0; io < n; ++io)
              for (int m = 0; m < n; ++m) phi[along_b ? m + n * io : io + n * m] = v[m] * vo[io];
            for (int a = 0; a < nl2; ++a)
              for (int b = 0; b < nl2; ++b) Mf[a * nl2 + b] += fpt_w[q] * (phi[a] * phi[b]);
          }
        }
      }
    // a cut face with an empty rule (none on the workloads scanned) reads a zero matrix: an
    // empty rule adds nothing to the face integrals
    int32_t zero = -1;
    for (int64_t c = 0; c < nc; ++c)
      for (int f = 0; f < nf; ++f)
        if (fmat_idx[c * nf + f] < 0 && (H.flags[H.cut_cells[c]] & uf::face_bit_sipg_cut(f))) {
          if (zero < 0) {
            zero = cnt++;
            fmat.resize((size_t)cnt * nl2 * nl2, 0.0);
          }
          fmat_idx[c * nf + f] = zero;
        }
  }
  const size_t o_fm = fmats ? L.take(sizeof(T) * fmat.size()) : 0;
  const size_t o_fmi = fmats ? L.take(sizeof(int32_t) * fmat_idx.size()) : 0;
  const size_t o_vkm = pre ? L.take(sizeof(T) * vline_km.size()) : 0;
  const size_t o_vlb = pre ? L.take(sizeof(T) * vline_b.size()) : 0;
  const size_t o_vpb = pre ? L.take(sizeof(T) * vpt_b.size()) : 0;
  const size_t o_spb = pre ? L.take(sizeof(T) * spt_b.size()) : 0;
  const size_t o_flb = pre ? L.take(sizeof(T) * fline_b.size()) : 0;
  const size_t o_fpb = pre ? L.take(sizeof(T) * fpt_b.size()) : 0;

  std::vector<unsigned char> img(L.bytes, 0);
  auto put = [&](size_t off, const void *src, size_t bytes) {
    if (bytes) std::memcpy(img.data() + off, src, bytes);
  };
  auto put_t = [&](size_t off, const std::vector<double> &v) {
    T *dst = reinterpret_cast<T *>(img.data() + off);
    for (size_t i = 0; i < v.size(); ++i) dst[i] = (T)v[i];
  };
  auto put_i = [&](size_t off, const std::vector<int32_t> &v) {
    put(off, v.data(), sizeof(int32_t) * v.size());
  };
  put(o_nbr, H.nbr.data(), sizeof(int32_t) * na * nf);
  put(o_flags, H.flags.data(), sizeof(uint32_t) * na);
  put_t(o_kappa, H.kappa);
  put(o_clist, cut_list.data(), sizeof(int32_t) * nc);
  put(o_cidx, cut_idx.data(), sizeof(int32_t) * nc);
  put(o_plist, part_list.data(), sizeof(int32_t) * nc);
  put(o_pidx, part_idx.data(), sizeof(int32_t) * nc);
  put_i(o_vlk, vline_koff);
  put_t(o_vo0, vline_o0);
  put_t(o_vo1, vline_o1);
  put_i(o_vpo, vpt_off);
  put_i(o_lsf, lsurf);
  put_i(o_vlg, vline_grp);
  put_t(o_vpt, vpt_t);
  put_t(o_vpw, vpt_w);
  put_t(o_spt, spt_t);
  put_t(o_spw, spt_w);
  for (int a = 0; a < 3; ++a) put_t(o_spn[a], spt_n[a]);
  put_i(o_flk, fline_koff);
  put_t(o_flo, fline_o);
  put_i(o_fpo, fpt_off);
  put_t(o_fpt, fpt_t);
  put_t(o_fpw, fpt_w);
  put_t(o_lself, lself);
  put_t(o_smat, smat);
  put_t(o_smatT, smatT);
  put_t(o_smat0, std::vector<double>(mats.begin(), mats.begin() + 16 * nn));
  put_t(o_lnbgp, lnbgp);
  put_t(o_lselfT, lselfT);
  put_t(o_lnbgpT, lnbgpT);
  put_t(o_lselfx, lself0);
  put_t(o_lnbgpx, lnbgp0);
  put_t(o_lselfxT, lselfxT);
  put_t(o_lnbgpxT, lnbgpxT);
  if (fmats) {
    put_t(o_fm, fmat);
    put_i(o_fmi, fmat_idx);
  }
  if (pre) {
    put_t(o_vkm, vline_km);
    put_t(o_vlb, vline_b);
    put_t(o_vpb, vpt_b);
    put_t(o_spb, spt_b);
    put_t(o_flb, fline_b);
    put_t(o_fpb, fpt_b);
  }

  cudaError_t err = uf::dev_malloc(&pd.base, L.bytes);
  if (err != cudaSuccess) return fail(UF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(err));
  const size_t vec_bytes = sizeof(T) * (size_t)H.n_active * H.ndof;
  err = uf::dev_malloc(&pd.xbuf, vec_bytes);
  if (err == cudaSuccess) err = uf::dev_malloc(&pd.ybuf, vec_bytes);
  // the second staging set and the set events exist for pipelined operators (several parts)
  const bool piped = part_meta.size() > 1;
  if (err == cudaSuccess && piped) err = uf::dev_malloc(&pd.xbuf2, vec_bytes);
  if (err == cudaSuccess && piped) err = uf::dev_malloc(&pd.ybuf2, vec_bytes);
  for (int b = 0; b < 2 && err == cudaSuccess && piped; ++b)
    err = cudaEventCreateWithFlags(&pd.set_free[b], cudaEventDisableTiming);
  if (err != cudaSuccess) return fail(UF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(err));
  err = cudaMemcpy(pd.base, img.data(), L.bytes, cudaMemcpyHostToDevice);
  if (err != cudaSuccess) return fail(UF_ECUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(err));
  pd.device_bytes = L.bytes;
  if (H.cg) {
    const int64_t n_loc = H.n_active * H.ndof;
    err = uf::dev_malloc(&pd.cg_l2g, n_loc * sizeof(int32_t));
    if (err == cudaSuccess) err = uf::dev_malloc(&pd.cg_own_off, (H.n_cg + 1) * sizeof(int32_t));
    if (err == cudaSuccess) err = uf::dev_malloc(&pd.cg_own_idx, n_loc * sizeof(int32_t));
    if (err == cudaSuccess) err = uf::dev_malloc(&pd.x_loc, n_loc * sizeof(T));
    if (err == cudaSuccess) err = uf::dev_malloc(&pd.y_loc, n_loc * sizeof(T));
    if (err != cudaSuccess) return fail(UF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(err));
    cudaMemcpy(pd.cg_l2g, H.cg_l2g.data(), n_loc * sizeof(int32_t), cudaMemcpyHostToDevice);
    cudaMemcpy(pd.cg_own_off, H.cg_own_off.data(), (H.n_cg + 1) * sizeof(int32_t), cudaMemcpyHostToDevice);
    err = cudaMemcpy(pd.cg_own_idx, H.cg_own_idx.data(), n_loc * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return fail(UF_ECUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(err));
  }

  unsigned char *b = static_cast<unsigned char *>(pd.base);
  auto I32 = [&](size_t off) { return reinterpret_cast<const int32_t *>(b + off); };
  auto TP = [&](size_t off) { return reinterpret_cast<const T *>(b + off); };
  uf::DevArrays<T> &A = pd.arrays;
  A.nbr = I32(o_nbr);
  A.flags = reinterpret_cast<const uint32_t *>(b + o_flags);
  pd.kappa_dev = reinterpret_cast<T *>(b + o_kappa);
  A.kappa = pd.kappa_dev;
  A.cut_list = I32(o_clist);
  A.cut_idx = I32(o_cidx);
  {
    // parts: face neighbours lie within `halo` cells of a cell
    int64_t halo = 0;
    for (int64_t e = 0; e < na; ++e)
      for (int f = 0; f < nf; ++f) {
        const int32_t nb = H.nbr[e * nf + f];
        if (nb >= 0) halo = std::max<int64_t>(halo, std::llabs((long long)(nb - e)));
      }
    pd.parts.clear();
    pd.part_needs.clear();
    for (size_t pi = 0; pi < part_meta.size(); ++pi) {
      const auto &m = part_meta[pi];
      uf::LaunchRange r{};
      r.cell_begin = m[0];
      r.cell_end = m[1];
      r.cut_list = I32(o_plist);
      r.cut_idx = I32(o_pidx);
      for (int i = 0; i < 4; ++i) r.split[i] = m[2 + i];
      pd.parts.push_back(r);
    }
    for (size_t pi = 0; pi < part_meta.size(); ++pi) {
      const int64_t last = std::min<int64_t>(part_meta[pi][1] + halo, na) - 1;
      int need = (int)pi;
      while (need + 1 < (int)part_meta.size() && part_meta[need + 1][0] <= last) ++need;
      pd.part_needs.push_back(need);
    }
  }
  A.vline_koff = I32(o_vlk);
  A.vline_o0 = TP(o_vo0);
  A.vline_o1 = TP(o_vo1);
  A.vpt_off = I32(o_vpo);
  A.lsurf = I32(o_lsf);
  A.vline_grp = I32(o_vlg);
  A.vpt_t = TP(o_vpt);
  A.vpt_w = TP(o_vpw);
  A.spt_t = TP(o_spt);
  A.spt_w = TP(o_spw);
  for (int a = 0; a < 3; ++a) A.spt_n[a] = TP(o_spn[a]);
  A.fline_koff = I32(o_flk);
  A.fline_o = TP(o_flo);
  A.fpt_off = I32(o_fpo);
  A.fpt_t = TP(o_fpt);
  A.fpt_w = TP(o_fpw);
  A.lself = TP(o_lself);
  A.smat = TP(o_smat);
  A.smatT = TP(o_smatT);
  A.smat0 = TP(o_smat0);
  A.lnbgp = TP(o_lnbgp);
  A.lselfT = TP(o_lselfT);
  A.lnbgpT = TP(o_lnbgpT);
  A.lselfx = TP(o_lselfx);
  A.lnbgpx = TP(o_lnbgpx);
  A.lselfxT = TP(o_lselfxT);
  A.lnbgpxT = TP(o_lnbgpxT);
  A.vline_km = pre ? TP(o_vkm) : nullptr;
  A.fmat = fmats ? TP(o_fm) : nullptr;
  A.fmat_idx = fmats ? I32(o_fmi) : nullptr;
  A.vline_b = pre ? TP(o_vlb) : nullptr;
  A.vpt_b = pre ? TP(o_vpb) : nullptr;
  A.spt_b = pre ? TP(o_spb) : nullptr;
  A.fline_b = pre ? TP(o_flb) : nullptr;
  A.fpt_b = pre ? TP(o_fpb) : nullptr;
  if (sizeof(T) == sizeof(double)) {
    // kappa gradient (FP64): derivative tables and the per-cell partial buffer
    std::vector<double> kg;
    uf::kgrad_tables(H.n, mats, kg);
    err = uf::dev_malloc(&op->kg_tables, kg.size() * sizeof(double));
    if (err == cudaSuccess) err = uf::dev_malloc(&op->kg_scratch, (size_t)na * (1 + nf) * sizeof(double));
    if (err != cudaSuccess) return fail(UF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(err));
    err = cudaMemcpy(op->kg_tables, kg.data(), kg.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return fail(UF_ECUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(err));
  }
  A.kappa_uniform = kappa_is_uniform(H.kappa) ? 1 : 0;
  A.n_active = (int32_t)na;
  A.n_cut = (int32_t)nc;
  {
    // cut_list ranges of the three lane classes (32, then 16, then 8 lanes per cut cell)
    int32_t split[2] = {(int32_t)nc, (int32_t)nc};
    for (int64_t i = nc - 1; i >= 0; --i) {
      const int l = lanes[order[i]];
      if (l <= 16) split[0] = (int32_t)i;
      if (l <= 8) split[1] = (int32_t)i;
    }
    A.cut_split[0] = split[0];
    A.cut_split[1] = split[1];
  }
  pd.n_vlines = nvl;
  pd.n_flines = nfl;

  // constant tables (layout of StructTables): the 16 matrices, M^{-1} dow and dnb (both with
  // h^{d-1} / 2), and the columns of M^{-1} at the two face nodes
  {
    const double half_hf = 0.5 * std::pow(H.h, d - 1);
    std::vector<double> tabs(mats.begin(), mats.begin() + 16 * nn);
    for (int s2 = 0; s2 < 2; ++s2)
      for (int r = 0; r < n; ++r) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += minv[r * n + k] * (half_hf * mats[16 * nn + s2 * n + k]);
        tabs.push_back(acc);
      }
    for (int i = 0; i < 2 * n; ++i) tabs.push_back(half_hf * mats[16 * nn + 2 * n + i]);
    for (int s2 = 0; s2 < 2; ++s2)
      for (int r = 0; r < n; ++r) tabs.push_back(minv[r * n + (s2 ? n - 1 : 0)]);
    for (int i = 0; i < 2 * n; ++i) tabs.push_back(half_hf * mats[16 * nn + i]);  // dowx
    pd.struct_tables.assign(sizeof(T) * tabs.size(), 0);
    T *st = reinterpret_cast<T *>(pd.struct_tables.data());
    for (size_t i = 0; i < tabs.size(); ++i) st[i] = (T)tabs[i];
  }
  pd.point_tables.assign(sizeof(T) * 6 * n, 0);
  T *ptab = reinterpret_cast<T *>(pd.point_tables.data());
  for (int i = 0; i < n; ++i) {
    ptab[i] = (T)H.t.z[i];
    ptab[n + i] = (T)H.t.den_inv[i];
    ptab[2 * n + i] = (T)H.t.deriv_end[0][0][i];
    ptab[3 * n + i] = (T)H.t.deriv_end[1][0][i];
    ptab[4 * n + i] = (T)H.t.deriv_end[0][1][i];
    ptab[5 * n + i] = (T)H.t.deriv_end[1][1][i];
  }
  pd.scalars.h = (T)H.h;
  pd.scalars.inv_h = (T)(1.0 / H.h);
  pd.scalars.inv_h2 = (T)(1.0 / (H.h * H.h));
  pd.scalars.sipg_over_h = (T)(H.params.sipg_gamma / H.h);
  pd.scalars.nitsche_over_h = (T)(H.params.nitsche_gamma / H.h);
  pd.scalars.hf = (T)std::pow(H.h, d - 1);
  pd.scalars.hf_sigma = (T)(std::pow(H.h, d - 1) * H.params.sipg_gamma / H.h);
  pd.present = true;
  return UF_OK;
}

template <typename T>
void release(PrecisionData<T> &pd) {
  void *cg[] = {pd.cg_l2g, pd.cg_own_off, pd.cg_own_idx, pd.x_loc, pd.y_loc};
  for (void *p : cg)
    if (p) uf::dev_free(p);
  pd.cg_l2g = pd.cg_own_off = pd.cg_own_idx = nullptr;
  pd.x_loc = pd.y_loc = nullptr;
  if (pd.base) uf::dev_free(pd.base);
  if (pd.xbuf) uf::dev_free(pd.xbuf);
  if (pd.ybuf) uf::dev_free(pd.ybuf);
  if (pd.xbuf2) uf::dev_free(pd.xbuf2);
  if (pd.ybuf2) uf::dev_free(pd.ybuf2);
  for (cudaEvent_t &e : pd.set_free)
    if (e) cudaEventDestroy(e);
  pd.set_free[0] = pd.set_free[1] = nullptr;
  pd.base = pd.xbuf = pd.ybuf = pd.xbuf2 = pd.ybuf2 = nullptr;
  pd.present = false;
}


template <typename T>
uf_status vmult_t(uf_operator *op, PrecisionData<T> &pd, void *y, const void *x, void *stream,
                  bool adjoint, const uf::LaunchRange *rg = nullptr) {
  if (!pd.present) return fail(UF_EINVAL, "operator was not created with this precision");
  const bool cg = op->host.cg;
  const int64_t nvec = cg ? op->host.n_cg : op->host.n_active * op->host.ndof;
  const size_t bytes = sizeof(T) * (size_t)nvec;
  const char *xb = static_cast<const char *>(x);
  const char *yb = static_cast<const char *>(y);
  if (xb < yb + bytes && yb < xb + bytes) return fail(UF_EINVAL, "x and y overlap");
  DeviceGuard guard(op->device);
  void *const *ev = nullptr;
  if (!rg && op->prof_next < op->prof.size()) {
    ProfSlot &slot = op->prof[op->prof_next++];
    slot.prec = sizeof(T) == 8 ? 0 : 1;
    slot.adjoint = adjoint ? 1 : 0;
    slot.used = true;
    ev = reinterpret_cast<void *const *>(slot.ev);
  }
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n_loc = op->host.n_active * op->host.ndof;
  int err = 0;
  if (cg) err = uf::cg_gather<T>(pd.x_loc, static_cast<const T *>(x), pd.cg_l2g, n_loc, cs);
  if (err == 0)
    err = uf::launch_vmult<T>(op->host.dim, op->host.n, pd.arrays, pd.struct_tables.data(),
                              pd.point_tables.data(), pd.scalars, cg ? pd.y_loc : static_cast<T *>(y),
                              cg ? pd.x_loc : static_cast<const T *>(x), adjoint, stream, ev, rg);
  if (err == 0 && cg)
    err = uf::cg_node_sum<T>(static_cast<T *>(y), pd.y_loc, pd.cg_own_off, pd.cg_own_idx, op->host.n_cg, cs);
  if (err != 0)
    return fail(UF_ECUDA, std::string("kernel launch: ") + cudaGetErrorString((cudaError_t)err));
  return UF_OK;
}

uf_status check_vmult_args(uf_operator *op, int precision, void *y, const void *x) {
  if (!op || !y || !x) return fail(UF_EINVAL, "NULL argument");
  if (op->device < 0) return fail(UF_ENODEVICE, "operator was created host-only");
  if (precision != UF_FP64 && precision != UF_FP32) return fail(UF_EINVAL, "bad precision");
  return UF_OK;
}

}  // namespace

namespace uf {
// out rows of the listed cells = in rows widened to FP64 (one thread per DoF).
__global__ void k_rows_to_f64(double *__restrict__ out, const float *__restrict__ in,
                              const int32_t *__restrict__ cells, int64_t n_cells, int nd) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cells * nd) return;
  const int64_t r = (int64_t)cells[i / nd] * nd + i % nd;
  out[r] = (double)in[r];
}
// y32 rows of the listed cells = the FP64 rows rounded once (one thread per DoF).
__global__ void k_rows_to_f32(float *__restrict__ y32, const double *__restrict__ y64,
                              const int32_t *__restrict__ cells, int64_t n_cells, int nd) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cells * nd) return;
  const int64_t r = (int64_t)cells[i / nd] * nd + i % nd;
  y32[r] = (float)y64[r];
}
}  // namespace uf

uf_status uf::vmult_split(uf_operator *op, float *y, const float *x, cudaStream_t s) {
  PrecisionData<float> &p32 = op->f32;
  PrecisionData<double> &p64 = op->f64;
  if (!p32.present || !p64.present) return fail(UF_EINVAL, "the split operator needs FP32 and FP64");
  const CgSolveData &w = op->cgs;
  const bool cg = op->host.cg;
  const int64_t n_loc = op->host.n_active * op->host.ndof;
  DeviceGuard guard(op->device);
  // cell-local input in both precisions (the FP64 copy is the FP32 input widened, exactly)
  int err = 0;
  if (cg) err = cg_gather<float>(p32.x_loc, x, p32.cg_l2g, n_loc, s);
  const float *xl32 = cg ? p32.x_loc : x;
  float *yl32 = cg ? p32.y_loc : y;
  double *xl64 = cg ? p64.x_loc : static_cast<double *>(p64.xbuf);
  double *yl64 = cg ? p64.y_loc : static_cast<double *>(p64.ybuf);
  const int nd = op->host.ndof;
  if (err == 0 && w.n_halo > 0) {
    const int64_t m = w.n_halo * nd;
    k_rows_to_f64<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(xl64, xl32, w.halo_cells, w.n_halo, nd);
    err = (int)cudaGetLastError();
  }
  if (err == 0)
    err = launch_vmult<float>(op->host.dim, op->host.n, p32.arrays, p32.struct_tables.data(),
                              p32.point_tables.data(), p32.scalars, yl32, xl32, false, s, nullptr);
  if (err == 0 && w.n_split > 0) {
    // FP64 rows of the split cells only: the structured kernel on their list, the cut-cell
    // kernel on the cut cells among them
    const DevArrays<double> &a = p64.arrays;
    LaunchRange rg{};
    rg.cell_begin = 0;
    rg.cell_end = (int32_t)w.n_split;
    rg.cut_list = w.split_cut_list;
    rg.cut_idx = w.split_cut_idx;
    rg.split[0] = 0;
    rg.split[1] = w.split_cut_class[0];
    rg.split[2] = w.split_cut_class[1];
    rg.split[3] = w.split_cut_class[2];
    rg.cells = w.split_cells;
    err = launch_vmult<double>(op->host.dim, op->host.n, a, p64.struct_tables.data(),
                               p64.point_tables.data(), p64.scalars, yl64, xl64, false, s, nullptr, &rg);
    if (err == 0) {
      const int64_t m = w.n_split * nd;
      k_rows_to_f32<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(yl32, yl64, w.split_cells, w.n_split, nd);
      err = (int)cudaGetLastError();
    }
  }
  if (err == 0 && cg) err = cg_node_sum<float>(y, p32.y_loc, p32.cg_own_off, p32.cg_own_idx, op->host.n_cg, s);
  if (err != 0) return fail(UF_ECUDA, std::string("kernel launch: ") + cudaGetErrorString((cudaError_t)err));
  return UF_OK;
}

uf_status uf::vmult_launch(uf_operator *op, int precision, void *y, const void *x, void *stream,
                           bool adjoint) {
  if (precision == UF_FP64) return vmult_t<double>(op, op->f64, y, x, stream, adjoint);
  return vmult_t<float>(op, op->f32, y, x, stream, adjoint);
}

namespace {

uf_status vmult_dispatch(uf_operator *op, int precision, void *y, const void *x, void *stream,
                         bool adjoint) {
  uf_status st = check_vmult_args(op, precision, y, x);
  if (st != UF_OK) return st;
  if (precision == UF_FP64) return vmult_t<double>(op, op->f64, y, x, stream, adjoint);
  return vmult_t<float>(op, op->f32, y, x, stream, adjoint);
}

}  // namespace

namespace {

// Host-buffer y = A x of a discontinuous operator as a pipeline over consecutive-cell parts: all
// parts of x are copied in on one stream, part i's kernels start on a stream of their own once x
// reaches its face neighbours (the parts write disjoint rows of y, so their kernels may overlap
// one another), and its rows of y are copied out on a third stream, so the copies overlap the
// kernels.  The results equal the single-launch path bit for bit (every cell is evaluated by the
// same code from the same data).
template <typename T>
uf_status host_pipeline(uf_operator *op, PrecisionData<T> &pd, T *y_host, const T *x_host,
                        cudaStream_t s, bool adjoint, bool wait) {
  const int np = (int)pd.parts.size();
  cudaError_t err = cudaSuccess;
  if (!op->pipe_in) err = cudaStreamCreateWithFlags(&op->pipe_in, cudaStreamNonBlocking);
  if (err == cudaSuccess && !op->pipe_out) err = cudaStreamCreateWithFlags(&op->pipe_out, cudaStreamNonBlocking);
  // earlier parts run at higher priority: the parts overlap where one alone would leave SMs idle,
  // but finish roughly in order, so the copies out start early
  int prio_low = 0, prio_high = 0;
  if (err == cudaSuccess) err = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  while (err == cudaSuccess && op->pipe_run.size() < (size_t)uf::kPipeParts) {
    const int i = (int)op->pipe_run.size();
    const int levels = prio_low - prio_high + 1;  // priorities run from prio_high (most urgent) up
    const int prio = prio_high + (levels > 1 ? (i * levels) / uf::kPipeParts : 0);
    cudaStream_t r;
    err = cudaStreamCreateWithPriority(&r, cudaStreamNonBlocking, prio);
    if (err == cudaSuccess) op->pipe_run.push_back(r);
  }
  while (err == cudaSuccess && op->pipe_ev.size() < (size_t)(1 + 2 * uf::kPipeParts)) {
    cudaEvent_t e;
    err = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (err == cudaSuccess) op->pipe_ev.push_back(e);
  }
  if (err != cudaSuccess) return fail(UF_ECUDA, std::string("pipeline setup: ") + cudaGetErrorString(err));
  const size_t nd = (size_t)op->host.ndof;
  // staging set of this call; it is reused once the latest call on it has copied y out
  const int set = pd.next_set;
  pd.next_set ^= 1;
  T *xb = static_cast<T *>(set ? pd.xbuf2 : pd.xbuf);
  T *yb = static_cast<T *>(set ? pd.ybuf2 : pd.ybuf);
  const bool reuse = pd.set_used[set];
  cudaEvent_t *ev = op->pipe_ev.data();
  // the copies start after the work already queued on the caller's stream
  err = cudaEventRecord(ev[0], s);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(op->pipe_in, ev[0], 0);
  if (err == cudaSuccess && reuse) err = cudaStreamWaitEvent(op->pipe_in, pd.set_free[set], 0);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(op->pipe_out, ev[0], 0);
  for (int j = 0; j < np && err == cudaSuccess; ++j) {
    const size_t off = nd * (size_t)pd.parts[j].cell_begin;
    const size_t cnt = nd * (size_t)(pd.parts[j].cell_end - pd.parts[j].cell_begin);
    err = cudaMemcpyAsync(xb + off, x_host + off, sizeof(T) * cnt, cudaMemcpyHostToDevice, op->pipe_in);
    if (err == cudaSuccess) err = cudaEventRecord(ev[1 + j], op->pipe_in);
  }
  if (err != cudaSuccess) return fail(UF_ECUDA, std::string("H2D copy: ") + cudaGetErrorString(err));
  for (int i = 0; i < np; ++i) {
    cudaStream_t run = op->pipe_run[i];
    err = cudaStreamWaitEvent(run, ev[0], 0);
    if (err == cudaSuccess && reuse) err = cudaStreamWaitEvent(run, pd.set_free[set], 0);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(run, ev[1 + pd.part_needs[i]], 0);
    if (err != cudaSuccess) return fail(UF_ECUDA, std::string("pipeline wait: ") + cudaGetErrorString(err));
    const uf_status st = vmult_t<T>(op, pd, yb, xb, run, adjoint, &pd.parts[i]);
    if (st != UF_OK) return st;
    const size_t off = nd * (size_t)pd.parts[i].cell_begin;
    const size_t cnt = nd * (size_t)(pd.parts[i].cell_end - pd.parts[i].cell_begin);
    err = cudaEventRecord(ev[1 + uf::kPipeParts + i], run);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(op->pipe_out, ev[1 + uf::kPipeParts + i], 0);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(y_host + off, yb + off, sizeof(T) * cnt, cudaMemcpyDeviceToHost, op->pipe_out);
    if (err != cudaSuccess) return fail(UF_ECUDA, std::string("D2H copy: ") + cudaGetErrorString(err));
  }
  // every part's kernels precede its copy out on pipe_out, so set_free marks the end of the
  // call; a synchronous call also orders later work on the caller's stream after it (an
  // asynchronous one does not, so that the next call's copies can start: uf_host_wait joins)
  err = cudaEventRecord(pd.set_free[set], op->pipe_out);
  pd.set_used[set] = true;
  if (err == cudaSuccess && wait) err = cudaStreamWaitEvent(s, pd.set_free[set], 0);
  if (err == cudaSuccess && wait) err = cudaEventSynchronize(pd.set_free[set]);
  if (err != cudaSuccess) return fail(UF_ECUDA, std::string("D2H copy: ") + cudaGetErrorString(err));
  return UF_OK;
}

}  // namespace

extern "C" {

uf_status uf_create_unfitted_operator(const uf_params *params, uf_operator **out) {
  if (!params || !out) return fail(UF_EINVAL, "NULL argument");
  *out = nullptr;
  if ((params->precisions & ~(UF_FP64 | UF_FP32)) != 0)
    return fail(UF_EINVAL, "precisions must be a mask of UF_FP64 | UF_FP32");
  uf_operator *op = uf::new_operator();
  if (!op) return fail(UF_ENOMEM, "host allocation failed");
  std::string msg;
  uf_status st;
  try {
    st = uf::build_host_operator(*params, op->host, msg);
  } catch (const std::bad_alloc &) {
    st = UF_ENOMEM;
    msg = "host allocation failed during setup";
  }
  if (st != UF_OK) {
    uf::delete_operator(op);
    return fail(st, msg);
  }
  if (params->kappa) {
    for (int64_t e = 0; e < op->host.n_active; ++e) {
      if (!(params->kappa[e] > 0.0) || !std::isfinite(params->kappa[e])) {
        uf::delete_operator(op);
        return fail(UF_EINVAL, "kappa must be positive and finite");
      }
      op->host.kappa[e] = params->kappa[e];
    }
  }
  if (op->host.cg) {
    try {
      uf::cg_host_vectors(op->host);
    } catch (const std::bad_alloc &) {
      uf::delete_operator(op);
      return fail(UF_ENOMEM, "host allocation failed during setup");
    }
  }
  op->device = params->device;
  if (op->device >= 0) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || op->device >= ndev) {
      uf::delete_operator(op);
      return fail(UF_EINVAL, "CUDA device not available");
    }
    DeviceGuard guard(op->device);
    cudaDeviceGetAttribute(&op->num_sms, cudaDevAttrMultiProcessorCount, op->device);
    try {
      if (params->precisions & UF_FP64) st = upload<double>(op, op->f64);
      if (st == UF_OK && (params->precisions & UF_FP32)) st = upload<float>(op, op->f32);
      if (st == UF_OK && op->host.cg) st = uf::cg_alloc(op);
    } catch (const std::bad_alloc &) {
      st = fail(UF_ENOMEM, "host allocation failed during upload");
    }
    if (st != UF_OK) {
      release(op->f64);
      release(op->f32);
      uf::cg_free(op);
      if (op->kg_tables) uf::dev_free(op->kg_tables);
      if (op->kg_scratch) uf::dev_free(op->kg_scratch);
      uf::delete_operator(op);
      return st;
    }
  }
  *out = op;
  return UF_OK;
}

uf_status uf_get_info(const uf_operator *op, uf_info *info) {
  if (!op || !info) return fail(UF_EINVAL, "NULL argument");
  const uf::HostOperator &H = op->host;
  std::memset(info, 0, sizeof(*info));
  info->n_active = H.n_active;
  info->n_inside = H.n_inside;
  info->n_cut = H.n_cut;
  info->n_dofs = H.cg ? H.n_cg : H.n_active * H.ndof;
  info->n_faces = H.n_faces;
  info->n_faces_full = H.n_faces_full;
  info->n_faces_cut = H.n_faces_cut;
  info->n_faces_empty = H.n_faces_empty;
  info->n_faces_gp = H.n_faces_gp;
  info->n_vol_points = (int64_t)H.vol_w.size();
  info->n_surf_points = (int64_t)H.surf_w.size();
  info->n_face_points = H.n_face_points_unique;
  info->n_vol_lines = (int64_t)H.vol_lines.size();
  info->n_face_lines = (int64_t)H.face_lines.size();
  info->n_vol_groups = count_line_groups(H);
  for (int k = 0; k < 3; ++k) info->cut_lane_classes[k] = 0;
  for (int64_t c = 0; c < H.n_cut; ++c) {
    const int l = uf::cut_lanes_of_cell(H, c);
    ++info->cut_lane_classes[l == 32 ? 0 : (l == 16 ? 1 : 2)];
  }
  info->dim = H.dim;
  info->degree = H.p;
  info->dofs_per_cell = H.ndof;
  info->quad_order = H.q;
  info->h = H.h;
  const int d = H.dim, nf = 2 * d;
  // Per-kernel algorithmic bytes: the structured kernel reads x of every cell once (neighbour
  // lines are L2 hits) and writes y once, plus neighbours / flags / kappa; the cut-cell kernel
  // reads x of the cut cells (own and cut-face neighbours are L2 hits), reads and writes their y
  // rows, and reads the line-structured point data and offsets once.
  // FP64 in 3D up to kFaceMatrixMaxN reads one n^2 x n^2 mass matrix per cut cell and cut face
  // (and its index) instead of the face lines and points.
  const double vl = (double)info->n_vol_lines, flh = 0.5 * (double)info->n_face_lines;
  const bool fmats = d == 3 && H.n <= uf::kFaceMatrixMaxN;
  const double nl2 = (double)H.n * H.n;
  for (int s = 0; s < 2; ++s) {
    const double S = s == 0 ? 8.0 : 4.0;
    double *kb = s == 0 ? info->kernel_bytes_fp64 : info->kernel_bytes_fp32;
    kb[0] = 2.0 * S * (double)info->n_dofs + (double)H.n_active * (4.0 * nf + 4.0 + S);
    const double face_bytes = (s == 0 && fmats)
                                  ? 2.0 * H.n_faces_cut * nl2 * nl2 * S + (double)H.n_cut * nf * 4.0
                                  : S * 2.0 * info->n_face_points + flh * (S + 4.0);
    kb[1] = 3.0 * S * (double)H.n_cut * H.ndof +
            (double)H.n_cut * (4.0 * 2 + 4.0 * 4 + 4.0 * 3 * nf + S) +
            S * ((S == 8.0 ? 2.0 * H.n * H.n * info->n_vol_lines : 2.0 * info->n_vol_points) +
                 (2.0 + d) * info->n_surf_points) +
            vl * (2.0 * S + 8.0) + face_bytes;
    (s == 0 ? info->bytes_fp64 : info->bytes_fp32) = kb[0] + kb[1];
  }
  // Floating-point operations of the kernels as built (FMA = 2, every FP op counted once).
  const double n = H.n, nd = H.ndof, nline = nd / n;
  int64_t nb_faces = 0, struct_faces = 0;
  for (int64_t e = 0; e < H.n_active; ++e)
    for (int f = 0; f < nf; ++f) {
      const uint32_t fl = H.flags[e];
      if (fl & (uf::face_bit_sipg_full(f) | uf::face_bit_gp(f))) {
        ++nb_faces;
        if (f % 2 == 1) ++struct_faces;  // count each interior face once (from its lower cell)
      }
    }
  // structured kernel: per cell and axis one M^{-1} L line sweep (n^{d+1} FMA), ghost-penalty
  // neighbour couplings as full line sweeps (n^{d+1} FMA), SIPG-only neighbour couplings in
  // rank-2 form, the sum of the axes ((d - 1) n^d adds) and one mass sweep per direction
  // (n^{d+1} FMA each); plus the per-cell matrix build if kappa varies.
  int64_t gp_faces_cell = 0, r2_faces_cell = 0, r2_faces_axis0 = 0;
  for (int64_t e = 0; e < H.n_active; ++e)
    for (int f = 0; f < nf; ++f) {
      const uint32_t fl = H.flags[e];
      if (fl & uf::face_bit_gp(f)) {
        ++gp_faces_cell;
      } else if (fl & uf::face_bit_sipg_full(f)) {
        ++r2_faces_cell;
        if (f < 2) ++r2_faces_axis0;
      }
    }
  const double sweep = nline * n * n;  // FMA per line sweep of a cell
  const bool uni = kappa_is_uniform(H.kappa);
  // uniform kappa: lines for kappa = 1, rows scaled once (not at all for kappa = 1); rank-2
  // couplings per line: the neighbour's derivative (n FMA), two rank-1 updates (2n FMA) and the
  // coefficient (1 FMA; 2 multiplies more when kappa varies); with uniform kappa axis 0 is
  // applied after its mass sweep in W space: one rank-1 update and a single-entry correction
  // (4n + 2 flops per line) and one axis fewer in the sum
  double fl_struct = 2.0 * ((double)H.n_active * (d * sweep + d * sweep) +
                            (double)gp_faces_cell * sweep) +
                     (double)H.n_active * (uni ? d - 2 : d - 1) * nd;
  if (uni)
    fl_struct += (double)(r2_faces_cell - r2_faces_axis0) * nline * (6 * n + 2) +
                 (double)r2_faces_axis0 * nline * (4 * n + 2);
  else
    fl_struct += (double)r2_faces_cell * nline * (6 * n + 5);
  // FP32 keeps the form without M^{-1}: every axis in phase 1, rank-2 couplings in W space
  // (2n FMA + 2 flops per line; 3 more when kappa varies), 5 in-face mass sweeps in 3D (2 in 2D)
  double fl_struct32 = 2.0 * ((double)H.n_active * (d * sweep + (d == 3 ? 5 : 2) * sweep) +
                              (double)gp_faces_cell * sweep) +
                       (double)r2_faces_cell * nline * (uni ? 4 * n + 3 : 4 * n + 6);
  if (uni && H.kappa[0] != 1.0) {
    fl_struct += (double)H.n_active * nd;
    fl_struct32 += (double)H.n_active * nd;
  }
  if (!uni) {
    fl_struct += (double)H.n_active * d * n * n * 2.0 * 13.0;
    fl_struct32 += (double)H.n_active * d * n * n * 2.0 * 13.0;
  }
  // cut-cell kernel: 1D basis (values and derivatives) 14n - 8, values only 6n - 4 flops when
  // evaluated (FP32); the FP64 kernels read them from tables (fb = fbv = 0)
  const double vlines = (double)H.vol_lines.size(), flines = (double)H.face_lines.size();
  const double vgroups = (double)info->n_vol_groups;
  auto cut_flops = [&](bool tables) {
    const double fb = tables ? 0.0 : 14 * n - 8, fbv = tables ? 0.0 : 6 * n - 4;
    double fl = 0.0;
    if (d == 3) {
      // per group: contraction along the shared axis and expansion back (2 n^3 FMA each);
      // per line: its own outer axis, evaluation and integration (3 n^2 FMA each)
      // per line: its own outer axis and the integration back (3 n^2 FMA each), and the
      // line integrals of its volume points (3 n^2 FMA)
      fl += vgroups * (fb + 8 * n * n * n) + vlines * (fb + 12 * n * n);
      if (tables)
        fl += vlines * 6 * n * n;
      else
        fl += (double)info->n_vol_points * (fb + 2 * 3 * n + 4 + 2 * 3 * n);
      fl += (double)info->n_surf_points * (fb + 2 * 4 * n + 16 + 2 * 3 * n + 6);
      if (!(tables && fmats)) fl += flines * (fbv + 2 * 2 * n * n + 2 * 2 * n * n);
    } else {
      fl += vlines * (fb + 2 * 2 * n * n + 2 * 2 * n * n);
      if (tables)
        fl += vlines * 2 * 2 * n * n;
      else
        fl += (double)info->n_vol_points * (fb + 2 * 2 * n + 3 + 2 * 2 * n);
      fl += (double)info->n_surf_points * (fb + 2 * 3 * n + 12 + 2 * 2 * n + 4);
      fl += flines * (2 * 2 * n);
    }
    if (tables && fmats)  // two products with the face's mass matrix, 7 flops per row
      fl += 2.0 * (double)H.n_faces_cut * (2 * 2 * nl2 * nl2 + 7 * nl2);
    else
      fl += 2.0 * (double)info->n_face_points * (fbv + 2 * 2 * n + 8 + 2 * 2 * n);
    // traces (jump and flux; Lobatto face values need no arithmetic) and expansion
    fl += 2.0 * (double)H.n_faces_cut * (2 * 2 * nd + 4 * nd / n + 2 * nd + nd / n);
    return fl;
  };
  info->kernel_flops_built[0] = fl_struct;
  info->kernel_flops_built[1] = cut_flops(true);
  info->kernel_flops_built_fp32[0] = fl_struct32;
  info->kernel_flops_built_fp32[1] = cut_flops(false);

  // Algorithmic FMAs from the paper's complexity model (evaluation + integration = x2).
  const double k = n;
  double c_cell, c_face, c_order, c_upt, c_fpt, c_fside;
  if (d == 3) {
    c_cell = 6 * k * k * k * k;
    c_face = 7 * k * k * k;
    c_order = k * k * k;              // one more normal derivative interpolated into a face
    c_upt = 2 * k * k * k + 3 * k * k + 4 * k;
    c_fpt = 3 * k * k + 4 * k;
    c_fside = k * k * k;
  } else {
    c_cell = 4 * k * k * k;
    c_face = 4 * k * k;
    c_order = k * k;
    c_upt = 2 * k * k + 3 * k;
    c_fpt = 3 * k;
    c_fside = k * k;
  }
  const int J = H.params.gp_max_order;
  const double alg_struct = 2.0 * ((double)H.n_inside * c_cell +
                                   (double)struct_faces * 2.0 * c_face +
                                   (double)H.n_faces_gp * 2.0 * std::max(J - 1, 0) * c_order);
  const double alg_cut = 2.0 * ((double)(info->n_vol_points + info->n_surf_points) * c_upt +
                                (double)info->n_face_points * 2.0 * c_fpt +
                                (double)H.n_faces_cut * 2.0 * c_fside);
  info->kernel_flops[0] = 2.0 * alg_struct;
  info->kernel_flops[1] = 2.0 * alg_cut;
  info->flops = info->kernel_flops[0] + info->kernel_flops[1];
  return UF_OK;
}

uf_status uf_vmult(uf_operator *op, int precision, void *y, const void *x, void *stream) {
  return vmult_dispatch(op, precision, y, x, stream, false);
}

uf_status uf_vmult_split(uf_operator *op, float *y, const float *x, void *stream) {
  uf_status st = check_vmult_args(op, UF_FP32, y, x);
  if (st != UF_OK) return st;
  if (!op->f32.present || !op->f64.present)
    return fail(UF_EINVAL, "the split operator needs the FP32 and the FP64 operator");
  const int64_t nvec = op->host.cg ? op->host.n_cg : op->host.n_active * op->host.ndof;
  const char *xb = reinterpret_cast<const char *>(x), *yb = reinterpret_cast<const char *>(y);
  const size_t bytes = sizeof(float) * (size_t)nvec;
  if (xb < yb + bytes && yb < xb + bytes) return fail(UF_EINVAL, "x and y overlap");
  DeviceGuard guard(op->device);
  st = uf::split_cells_alloc(op);
  if (st != UF_OK) return st;
  return uf::vmult_split(op, y, x, reinterpret_cast<cudaStream_t>(stream));
}

uf_status uf_set_split_fraction(uf_operator *op, double fraction) {
  if (!op) return fail(UF_EINVAL, "NULL argument");
  if (!(fraction > 0.0)) return fail(UF_EINVAL, "the split fraction must be positive");
  if (fraction != op->split_fraction) {
    if (op->device >= 0) {
      DeviceGuard guard(op->device);
      uf::split_cells_free(op);
    }
    op->split_fraction = fraction;
  }
  return UF_OK;
}

uf_status uf_vmult_adjoint(uf_operator *op, int precision, void *y, const void *g, void *stream) {
  return vmult_dispatch(op, precision, y, g, stream, true);
}

static uf_status vmult_host_impl(uf_operator *op, int precision, void *y_host,
                                 const void *x_host, void *stream, bool adjoint, bool wait) {
  uf_status st = check_vmult_args(op, precision, y_host, x_host);
  if (st != UF_OK) return st;
  DeviceGuard guard(op->device);
  if (!op->host.cg) {
    if (precision == UF_FP64 && op->f64.present && op->f64.parts.size() > 1)
      return host_pipeline<double>(op, op->f64, static_cast<double *>(y_host),
                                   static_cast<const double *>(x_host), reinterpret_cast<cudaStream_t>(stream),
                                   adjoint, wait);
    if (precision == UF_FP32 && op->f32.present && op->f32.parts.size() > 1)
      return host_pipeline<float>(op, op->f32, static_cast<float *>(y_host),
                                  static_cast<const float *>(x_host), reinterpret_cast<cudaStream_t>(stream),
                                  adjoint, wait);
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t elem = precision == UF_FP64 ? sizeof(double) : sizeof(float);
  const size_t bytes = elem * (size_t)(op->host.cg ? op->host.n_cg : op->host.n_active * op->host.ndof);
  void *xb = precision == UF_FP64 ? op->f64.xbuf : op->f32.xbuf;
  void *yb = precision == UF_FP64 ? op->f64.ybuf : op->f32.ybuf;
  if (!xb || !yb) return fail(UF_EINVAL, "operator was not created with this precision");
  cudaError_t err = cudaMemcpyAsync(xb, x_host, bytes, cudaMemcpyHostToDevice, s);
  if (err != cudaSuccess) return fail(UF_ECUDA, std::string("H2D copy: ") + cudaGetErrorString(err));
  st = vmult_dispatch(op, precision, yb, xb, stream, adjoint);
  if (st != UF_OK) return st;
  err = cudaMemcpyAsync(y_host, yb, bytes, cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess && wait) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return fail(UF_ECUDA, std::string("D2H copy: ") + cudaGetErrorString(err));
  return UF_OK;
}

uf_status uf_vmult_host(uf_operator *op, int precision, void *y_host, const void *x_host,
                        void *stream) {
  return vmult_host_impl(op, precision, y_host, x_host, stream, false, true);
}

uf_status uf_vmult_adjoint_host(uf_operator *op, int precision, void *y_host, const void *g_host,
                                void *stream) {
  return vmult_host_impl(op, precision, y_host, g_host, stream, true, true);
}

uf_status uf_host_wait(uf_operator *op, void *stream) {
  if (!op) return fail(UF_EINVAL, "NULL operator");
  if (op->device < 0) return fail(UF_ENODEVICE, "operator was created host-only");
  DeviceGuard guard(op->device);
  cudaError_t err = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  if (err == cudaSuccess && op->pipe_out) err = cudaStreamSynchronize(op->pipe_out);
  if (err != cudaSuccess) return fail(UF_ECUDA, std::string("uf_host_wait: ") + cudaGetErrorString(err));
  return UF_OK;
}

uf_status uf_vmult_host_async(uf_operator *op, int precision, void *y_host, const void *x_host,
                              void *stream) {
  return vmult_host_impl(op, precision, y_host, x_host, stream, false, false);
}

uf_status uf_vmult_adjoint_host_async(uf_operator *op, int precision, void *y_host,
                                      const void *g_host, void *stream) {
  return vmult_host_impl(op, precision, y_host, g_host, stream, true, false);
}

uf_status uf_profile_begin(uf_operator *op, int capacity) {
  if (!op || capacity < 1) return fail(UF_EINVAL, "NULL operator or capacity < 1");
  if (op->device < 0) return fail(UF_ENODEVICE, "operator was created host-only");
  if (!op->prof.empty()) return fail(UF_EINVAL, "profiling already active");
  DeviceGuard guard(op->device);
  op->prof.resize(capacity);
  for (ProfSlot &slot : op->prof) {
    slot.used = false;
    for (int k = 0; k < 4; ++k) {
      cudaError_t err = cudaEventCreate(&slot.ev[k]);
      if (err != cudaSuccess) {
        op->prof.clear();
        return fail(UF_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(err));
      }
    }
  }
  op->prof_next = 0;
  return UF_OK;
}

uf_status uf_profile_end(uf_operator *op, uf_kernel_times *out) {
  if (!op || !out) return fail(UF_EINVAL, "NULL argument");
  if (op->prof.empty()) return fail(UF_EINVAL, "profiling not active");
  DeviceGuard guard(op->device);
  std::memset(out, 0, sizeof(*out));
  cudaError_t first_err = cudaSuccess;
  for (ProfSlot &slot : op->prof) {
    if (slot.used) {
      for (int kern = 0; kern < 2; ++kern) {
        float ms = 0.f;
        cudaError_t err = cudaEventSynchronize(slot.ev[2 * kern + 1]);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, slot.ev[2 * kern], slot.ev[2 * kern + 1]);
        if (err != cudaSuccess && first_err == cudaSuccess) first_err = err;
        out->ms_total[slot.prec][kern][slot.adjoint] += ms;
        out->launches[slot.prec][kern][slot.adjoint] += 1;
        int64_t nk = 1;
        if (kern == 1) {
          // FP64: one launch for all lane classes; FP32: one per non-empty class
          const int32_t *sp = slot.prec == 0 ? op->f64.arrays.cut_split : op->f32.arrays.cut_split;
          const int64_t nc = op->host.n_cut;
          nk = slot.prec == 0 ? (nc > 0 ? 1 : 0)
                              : (sp[0] > 0 ? 1 : 0) + (sp[1] > sp[0] ? 1 : 0) + (nc > sp[1] ? 1 : 0);
        } else if (op->host.n_active == 0) {
          nk = 0;
        }
        out->kernel_launches[slot.prec][kern][slot.adjoint] += nk;
      }
    }
    for (int k = 0; k < 4; ++k) cudaEventDestroy(slot.ev[k]);
  }
  op->prof.clear();
  op->prof_next = 0;
  if (first_err != cudaSuccess) return fail(UF_ECUDA, cudaGetErrorString(first_err));
  return UF_OK;
}

uf_status uf_set_kappa(uf_operator *op, const double *kappa_host) {
  if (!op || !kappa_host) return fail(UF_EINVAL, "NULL argument");
  for (int64_t e = 0; e < op->host.n_active; ++e)
    if (!(kappa_host[e] > 0.0) || !std::isfinite(kappa_host[e]))
      return fail(UF_EINVAL, "kappa must be positive and finite");
  std::copy(kappa_host, kappa_host + op->host.n_active, op->host.kappa.begin());
  if (op->host.cg) uf::cg_host_vectors(op->host);
  if (!op->host.cg && op->cgs.ready) uf::dg_host_diagonal(op->host);
  const int32_t uni = kappa_is_uniform(op->host.kappa) ? 1 : 0;
  op->f64.arrays.kappa_uniform = uni;
  op->f32.arrays.kappa_uniform = uni;
  if (op->device < 0) return UF_OK;
  DeviceGuard guard(op->device);
  const int64_t na = op->host.n_active;
  if (op->f64.present) {
    cudaError_t err = cudaMemcpy(op->f64.kappa_dev, kappa_host, sizeof(double) * na, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return fail(UF_ECUDA, cudaGetErrorString(err));
  }
  if (op->f32.present) {
    std::vector<float> k32(kappa_host, kappa_host + na);
    cudaError_t err = cudaMemcpy(op->f32.kappa_dev, k32.data(), sizeof(float) * na, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return fail(UF_ECUDA, cudaGetErrorString(err));
  }
  if (op->cgs.ready) return uf::cg_upload_diag(op);
  return UF_OK;
}

uf_status uf_export_cells(const uf_operator *op, int32_t *type, int32_t *index) {
  if (!op) return fail(UF_EINVAL, "NULL argument");
  const uf::HostOperator &H = op->host;
  for (int64_t e = 0; e < H.n_active; ++e) {
    if (type) type[e] = H.act_type[e];
    if (index)
      for (int a = 0; a < 3; ++a) index[e * 3 + a] = H.act_index[e * 3 + a];
  }
  return UF_OK;
}

uf_status uf_export_cut_cell_rule(const uf_operator *op, int64_t c, int kind, double *xi,
                                  double *w, double *normal, int64_t *count) {
  if (!op || !count) return fail(UF_EINVAL, "NULL argument");
  const uf::HostOperator &H = op->host;
  if (c < 0 || c >= H.n_cut || (kind != 0 && kind != 1)) return fail(UF_EINVAL, "index out of range");
  const std::vector<int64_t> &off = kind == 0 ? H.vol_off : H.surf_off;
  const int64_t b = off[c], e = off[c + 1];
  *count = e - b;
  if (!xi) return UF_OK;
  const int d = H.dim;
  for (int64_t i = b; i < e; ++i) {
    for (int a = 0; a < d; ++a) {
      xi[(i - b) * d + a] = kind == 0 ? H.vol_xi[a][i] : H.surf_xi[a][i];
      if (kind == 1 && normal) normal[(i - b) * d + a] = H.surf_n[a][i];
    }
    if (w) w[i - b] = kind == 0 ? H.vol_w[i] : H.surf_w[i];
  }
  return UF_OK;
}

uf_status uf_export_cut_face_rule(const uf_operator *op, int64_t e, int axis, int side,
                                  double *eta, double *w, int64_t *count) {
  if (!op || !count) return fail(UF_EINVAL, "NULL argument");
  const uf::HostOperator &H = op->host;
  if (e < 0 || e >= H.n_active || axis < 0 || axis >= H.dim || (side != 0 && side != 1))
    return fail(UF_EINVAL, "index out of range");
  *count = 0;
  const int c = H.cut_of[e];
  const int f = 2 * axis + side, nf = 2 * H.dim;
  if (c < 0) return UF_OK;
  const int64_t b = H.cface_off[c * nf + f], en = H.cface_off[c * nf + f + 1];
  *count = en - b;
  if (!eta) return UF_OK;
  for (int64_t i = b; i < en; ++i) {
    for (int a = 0; a < H.dim - 1; ++a) eta[(i - b) * (H.dim - 1) + a] = H.cface_eta[a][i];
    if (w) w[i - b] = H.cface_w[i];
  }
  return UF_OK;
}

uf_status uf_export_cut_cell_counts(const uf_operator *op, int32_t *vol_points, int32_t *vol_lines,
                                    int32_t *face_lines, int32_t *lanes) {
  if (!op) return fail(UF_EINVAL, "NULL argument");
  const uf::HostOperator &H = op->host;
  const int nf = 2 * H.dim;
  for (int64_t c = 0; c < H.n_cut; ++c) {
    if (vol_points) vol_points[c] = (int32_t)(H.vol_off[c + 1] - H.vol_off[c]);
    if (vol_lines) vol_lines[c] = (int32_t)(H.vline_off[c + 1] - H.vline_off[c]);
    if (face_lines) face_lines[c] = (int32_t)(H.fline_off[(c + 1) * nf] - H.fline_off[c * nf]);
    if (lanes) lanes[c] = uf::cut_lanes_of_cell(H, c);
  }
  return UF_OK;
}

uf_status uf_export_cut_cell_lines(const uf_operator *op, int64_t c, int32_t *axis,
                                   int32_t *group_start, int32_t *points, int64_t *count) {
  if (!op || !count) return fail(UF_EINVAL, "NULL argument");
  const uf::HostOperator &H = op->host;
  if (c < 0 || c >= H.n_cut) return fail(UF_EINVAL, "index out of range");
  *count = H.vline_off[c + 1] - H.vline_off[c];
  if (!axis) return UF_OK;
  // the order of the device arrays: lines sorted by axis, then contiguous groups per axis
  std::vector<uf::QLine> ls(H.vol_lines.begin() + H.vline_off[c], H.vol_lines.begin() + H.vline_off[c + 1]);
  std::stable_sort(ls.begin(), ls.end(), [](const uf::QLine &a, const uf::QLine &b) { return a.k < b.k; });
  int64_t i = 0;
  for (int k = 0; k < H.dim; ++k) {
    std::vector<const uf::QLine *> lk;
    for (const uf::QLine &ln : ls)
      if (ln.k == k) lk.push_back(&ln);
    std::vector<int> gstart;
    group_lines(H, lk, gstart);
    for (size_t j = 0; j < lk.size(); ++j, ++i) {
      axis[i] = k;
      if (group_start) group_start[i] = gstart[j] == (int)j ? 1 : 0;
      if (points) points[i] = (int32_t)lk[j]->vcnt;
    }
  }
  return UF_OK;
}

uf_status uf_export_cg(const uf_operator *op, int32_t *l2g, double *rhs, double *diag) {
  if (!op) return fail(UF_EINVAL, "NULL argument");
  const uf::HostOperator &H = op->host;
  if (!H.cg) return fail(UF_EINVAL, "not a continuous (UF_CG) operator");
  if (l2g) std::copy(H.cg_l2g.begin(), H.cg_l2g.end(), l2g);
  if (rhs) std::copy(H.cg_rhs.begin(), H.cg_rhs.end(), rhs);
  if (diag) std::copy(H.cg_diag.begin(), H.cg_diag.end(), diag);
  return UF_OK;
}

uf_status uf_destroy(uf_operator *op) {
  if (!op) return UF_OK;
  if (op->device >= 0) {
    DeviceGuard guard(op->device);
    // queued asynchronous host-buffer products finish before their buffers go
    for (cudaStream_t r : op->pipe_run) cudaStreamSynchronize(r);
    if (op->pipe_in) cudaStreamSynchronize(op->pipe_in);
    if (op->pipe_out) cudaStreamSynchronize(op->pipe_out);
    uf::release_csr(op->csr64);
    uf::release_csr(op->csr32);
    uf::cg_free(op);
    if (op->kg_tables) uf::dev_free(op->kg_tables);
    if (op->kg_scratch) uf::dev_free(op->kg_scratch);
    for (ProfSlot &slot : op->prof)
      for (int k = 0; k < 4; ++k) cudaEventDestroy(slot.ev[k]);
    for (cudaEvent_t e : op->pipe_ev) cudaEventDestroy(e);
    for (cudaStream_t r : op->pipe_run) cudaStreamDestroy(r);
    if (op->pipe_in) cudaStreamDestroy(op->pipe_in);
    if (op->pipe_out) cudaStreamDestroy(op->pipe_out);
    release(op->f64);
    release(op->f32);
  }
  uf::delete_operator(op);
  return UF_OK;
}

const char *uf_last_error(void) { return g_last_error.c_str(); }

uf_status uf_debug_fail_allocation(int64_t after) {
  uf::g_fail_after.store(after < 0 ? -1 : after);
  return UF_OK;
}

uf_status uf_debug_live_allocations(int64_t *live) {
  if (!live) return fail(UF_EINVAL, "NULL argument");
  *live = uf::g_live_allocations.load();
  return UF_OK;
}

}  // extern "C"
