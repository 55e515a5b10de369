// Host-side setup product of the unfitted DG operator (internal to libunfitted).
//
// The setup follows arXiv 2404.07911, Sec. 2.3 (quadrature classification): background cells
// are classified as inside / cut / outside against the level set, interior faces as full / cut /
// empty, and the cut cells and cut faces receive dimension-reduction quadrature (Saye's method,
// cited in Sec. 1) generated once; Sec. 6.2 excludes this setup from the timed operator.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/unfitted.h"

namespace uf {

constexpr int kMaxDim = 3;
constexpr int kMaxN = 9;  // degree <= 8

// Per-cell flag bits.  Bit 0: the cell is cut.  For face f = 2 * axis + side (side 0 = lower):
enum : uint32_t {
  kCellCut = 1u,
};
inline uint32_t face_bit_sipg_full(int f) { return 1u << (1 + 3 * f); }
inline uint32_t face_bit_sipg_cut(int f) { return 1u << (2 + 3 * f); }
inline uint32_t face_bit_gp(int f) { return 1u << (3 + 3 * f); }

// 1D tables (all FP64), n = p + 1 Gauss-Lobatto Lagrange polynomials on [0, 1].
struct Tables1D {
  int n = 0, p = 0;
  double z[kMaxN];              // Gauss-Lobatto nodes
  double den_inv[kMaxN];        // 1 / prod_{m != i} (z_i - z_m)
  double gauss_x[kMaxN], gauss_w[kMaxN];
  double mass[kMaxN * kMaxN];   // int_0^1 phi_i phi_j
  double stiff[kMaxN * kMaxN];  // int_0^1 phi_i' phi_j'
  // deriv_end[s][j][i] = phi_i^(j)(s), s = 0, 1, j = 0..p
  double deriv_end[2][kMaxN][kMaxN];
};

struct Fn {  // psi(x) = |x - c|^2 - rho on an m-dimensional box
  double c[kMaxDim];
  double rho;
};

struct QPoint {
  double x[kMaxDim];
  double w;
  double nrm[kMaxDim];
};

// A line of the dimension-reduction rule: points that share every coordinate except the one
// along axis k (the height direction of the box, or axis 0 of a tensor box).  vbeg / vcnt index
// volume points, sidx the surface point of the line (-1 if none).
struct QLine {
  int k;
  int64_t vbeg, vcnt, sidx;
};

struct HostOperator {
  uf_params params{};
  int dim = 0, p = 0, n = 0, ndof = 0, q = 0;
  int64_t N[kMaxDim] = {1, 1, 1};
  double lo[kMaxDim] = {0, 0, 0};
  double h = 0;
  double center[kMaxDim] = {0, 0, 0};
  double radius = 0;
  int ls_kind = 0;                      // UF_LS_SPHERE or UF_LS_PLANE
  double normal[kMaxDim] = {0, 0, 0};   // plane: phi = normal . x - offset
  double offset = 0;
  std::vector<double> spheres;          // union of balls: [n][4] = (cx, cy, cz, R)
  std::vector<int64_t> cut_sph_off;     // [n_cut + 1] union of balls: spheres meeting each cut
  std::vector<int32_t> cut_sph;         //   cell, cut_sph[cut_sph_off[c] .. cut_sph_off[c + 1])

  Tables1D t;

  // classification / numbering
  int64_t n_background = 0;
  std::vector<int32_t> id_map;    // background flat index (x fastest) -> active id, -1 outside
  std::vector<int32_t> act_index; // [n_active * 3] multi-index of each active cell
  std::vector<int8_t> act_type;   // 0 inside, 1 cut
  int64_t n_active = 0, n_inside = 0, n_cut = 0;

  // per active cell
  std::vector<int32_t> nbr;       // [n_active * 2 * dim], -1 = none
  std::vector<uint32_t> flags;    // kCellCut | face bits
  std::vector<double> kappa;      // [n_active]

  // cut cells (active order)
  std::vector<int32_t> cut_cells; // active id of each cut cell
  std::vector<int32_t> cut_of;    // [n_active] -> cut index or -1
  std::vector<int64_t> vol_off, surf_off;   // [n_cut + 1]
  std::vector<double> vol_xi[kMaxDim], vol_w;                 // reference coordinates, weights
  std::vector<double> surf_xi[kMaxDim], surf_w, surf_n[kMaxDim];
  // cut-face rules, stored per (cut cell, face) side: [n_cut * 2 * dim + 1]
  std::vector<int64_t> cface_off;
  std::vector<double> cface_eta[kMaxDim - 1], cface_w;
  // line structure of the rules (indices into the arrays above): volume/surface lines of cut
  // cell c are vol_lines[vline_off[c] .. vline_off[c + 1]); face lines of (c, face f) are
  // face_lines[fline_off[c * 2d + f] .. ], with k an in-face axis (0 = lower of the two).
  std::vector<QLine> vol_lines, face_lines;
  std::vector<int64_t> vline_off, fline_off;

  // continuous Q_p (discretization == UF_CG): global node of every cell-local DoF and, per global
  // node, its owners (cell * n^d + l, ascending); load vector (f = 1) and diagonal of A (FP64)
  bool cg = false;
  int64_t n_cg = 0;
  std::vector<int32_t> cg_l2g;            // [n_active * n^d]
  std::vector<int32_t> cg_own_off;        // [n_cg + 1]
  std::vector<int32_t> cg_own_idx;        // [n_active * n^d]
  std::vector<double> cg_rhs, cg_diag;    // [n_cg]
  std::vector<double> dg_diag;            // DG: diagonal of A [n_active * ndof], built on demand

  // counts
  int64_t n_faces = 0, n_faces_full = 0, n_faces_cut = 0, n_faces_empty = 0, n_faces_gp = 0;
  int64_t n_face_points_unique = 0;
};

// Builds everything above from params (no device work).  Returns UF_OK or an error with msg.
uf_status build_host_operator(const uf_params &params, HostOperator &op, std::string &msg);

// 1D tables (exposed for the device upload).
void build_tables_1d(int p, Tables1D &t);

// phi_i(x) and phi_i'(x), i = 0..n-1, of the Lobatto Lagrange basis of t.
void lagrange_values(const Tables1D &t, double x, double *val, double *der);

}  // namespace uf
