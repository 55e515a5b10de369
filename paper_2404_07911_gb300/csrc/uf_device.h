// Device-side data of the unfitted DG operator (internal to libunfitted).
#pragma once

#include <cstdint>

namespace uf {

constexpr int kMaxNdev = 9;
// Largest n (= p + 1) whose FP64 cut faces use per-face mass matrices: at n = 4 a face's matrix
// (256 values) costs 2 n^4 = 512 FMA against about 760 for its lines and points on a ball; at
// n = 5 the two are even, and above it the lines are cheaper.
constexpr int kFaceMatrixMaxN = 4;

// Constant 1D matrices of the structured (tensor-product) terms, all scalings folded in
// (arXiv 2404.07911, Sec. 3.2, Eq. sum_factorization_cell / Eq. sum_factorization_face: on a
// Cartesian cell the cell and face operators are Kronecker products of 1D matrices).
// Row index = test function, column index = trial function; side s = 0 lower, 1 upper face.
//   kv      h^{d-2} K        (cell stiffness along the axis; mass along the others)
//   mass    M                (1D reference mass, applied along the d-1 other axes)
//   a[s]    SIPG consistency of the own trace          (x kappa_K)
//   pen[s]  SIPG penalty, own-own                      (x {kappa})
//   gp[s]   ghost penalty, own-own, orders 1..J        (x {kappa})
//   b[s]    SIPG, own derivative x neighbour value     (x kappa_K)
//   c[s]    SIPG, own value x neighbour derivative     (x kappa_nb)
//   qn[s]   SIPG penalty, own-neighbour                (x {kappa})
//   hn[s]   ghost penalty, own-neighbour               (x {kappa})
// Face matrices carry the face measure h^{d-1} and the normal-derivative scalings 1/h^j.
//   dow[s]  h^{d-1}/2 sgn_s phi'(s) / h       (own outward normal derivative at the face)
//   dnb[s]  h^{d-1}/2 sgn_s phi'(1 - s) / h   (neighbour's derivative along the own normal)
// A full face without ghost penalty couples to the neighbour through rank 2 only:
//   (kappa_K b + kappa_nb c + {kappa} qn) u_nb
//     = kappa_K dow (u_nb at its face node) - e_own (kappa_nb dnb.u_nb
//       + h^{d-1} sigma/h {kappa} u_nb at its face node)   (delta property of the basis).
template <typename T, int N>
struct StructTables {
  T kv[N * N];
  T mass[N * N];
  T a[2][N * N], pen[2][N * N], gp[2][N * N];
  T b[2][N * N], c[2][N * N], qn[2][N * N], hn[2][N * N];
  T dow[2][N], dnb[2][N];  // dow premultiplied by M^{-1}; both carry h^{d-1} / 2
  T me[2][N];              // column of M^{-1} at the face node of side s (0 or N - 1)
  T dowx[2][N];            // dow without M^{-1} (axis 0 of the uniform-kappa path), h^{d-1} / 2
};

// 1D data for point evaluation of the Lagrange basis at arbitrary reference coordinates.
template <typename T, int N>
struct PointTables {
  T z[N];            // Gauss-Lobatto nodes
  T den_inv[N];      // 1 / prod_{m != i} (z_i - z_m)
  T end_val[2][N];   // phi_i(s), s = 0, 1
  T end_der[2][N];   // phi_i'(s)
};

// Per-operator scalars.
template <typename T>
struct Scalars {
  T h, inv_h, inv_h2;
  T sipg_over_h;     // sigma / h
  T nitsche_over_h;  // tau / h
  T hf;              // face measure scaling h^{d-1}
  T hf_sigma;        // h^{d-1} sigma / h
};

// Pointers into device memory (one allocation per precision).
//
// Unstructured points are stored line by line: a line of the dimension-reduction rule holds the
// points that share every reference coordinate except the one along its axis k.  Lines of a cut
// cell are sorted by k; vline_koff[ci * 4 + k] .. vline_koff[ci * 4 + k + 1] are the lines of
// cut cell ci along axis k (entries beyond the dimension repeat the end).  Line l owns volume
// points vpt_off[l] .. vpt_off[l + 1] (coordinate along k and weight) and surface point
// lsurf[l] (-1 if none).  Cut faces: fline_koff[(ci * 2d + f) * 3 + k'] for the two in-face
// axes k' (0 = lower one), same scheme with face points.
template <typename T>
struct DevArrays {
  const int32_t *nbr;       // [n_active * 2d]
  const uint32_t *flags;    // [n_active]
  const T *kappa;           // [n_active]
  const int32_t *cut_list;  // [n_cut] active ids, most expensive first
  const int32_t *cut_idx;   // [n_cut] cut index of cut_list[i] (row of the offset arrays)
  // volume / surface lines
  const int32_t *vline_koff;  // [n_cut * 4]
  const T *vline_o0, *vline_o1;  // outer reference coordinates (lower, upper other axis)
  const int32_t *vpt_off;     // [n_vlines + 1]
  const int32_t *lsurf;       // [n_vlines]
  // [n_vlines] (first line of the line's group) << 1 | shared_lo: the lines of a group are
  // contiguous and share the outer coordinate along the lower (shared_lo = 1) or upper other
  // axis, so the kernel contracts along that axis once per group (3D)
  const int32_t *vline_grp;
  const T *vpt_t, *vpt_w;     // [n_vol_points] coordinate along the line, weight
  const T *spt_t, *spt_w, *spt_n[3];  // [n_surf_points]
  // cut-face lines
  const int32_t *fline_koff;  // [n_cut * 2d * 3]
  const T *fline_o;           // outer in-face reference coordinate (3D)
  const int32_t *fpt_off;     // [n_flines + 1]
  const T *fpt_t, *fpt_w;     // [n_face_points]
  // Structured 1D matrices for kappa = 1, indexed by the face flags of one axis, all
  // premultiplied by M^{-1} (the structured kernel applies M (x) M (x) M once to the sum of the
  // axes' line results): lself[v], v = inside | full_lo << 1 | gp_lo << 2 | full_hi << 3 |
  // gp_hi << 4, and lnbgp[2 * s + full] for a ghost-penalty face on side s.  When kappa is
  // uniform (kappa_uniform != 0) every structured term scales with that value.
  const T *lself, *lnbgp;
  const T *lselfT, *lnbgpT;  // M^{-1} times the transposed tables (adjoint)
  // the same tables without M^{-1}: axis 0 of the FP64 uniform-kappa path (its lines are applied
  // in the first mass sweep, where M_0 M_0^{-1} cancels) and every axis of FP32
  const T *lselfx, *lnbgpx, *lselfxT, *lnbgpxT;
  // the 16 constant 1D matrices Q_k of StructTables (same order) premultiplied by M^{-1}, for
  // the per-cell matrices when kappa varies (read with a per-thread index)
  const T *smat;   // M^{-1} Q_k
  const T *smatT;  // M^{-1} Q_k^T (adjoint)
  const T *smat0;  // Q_k themselves (FP32, which keeps the form without M^{-1})
  // FP64 only (null otherwise): the 1D basis at every line and point, precomputed at creation
  // (values and derivatives; faces values only): vline_b [line][4n] = phi, phi' of the lower and
  // upper outer coordinate; vpt_b / spt_b [point][2n]; fline_b [face line][n]; fpt_b [point][n].
  const T *vline_b, *vpt_b, *spt_b, *fline_b, *fpt_b;
  // FP64 only (null otherwise), per volume line l: the line's quadrature integrals of 1D basis
  // products,
  // vline_km[l][0][i][j] = h^{-2} sum_p w_p phi_i'(t_p) phi_j'(t_p) and
  // vline_km[l][1][i][j] = h^{-2} sum_p w_p phi_i(t_p) phi_j(t_p) over the line's volume points:
  // the Poisson integrand of a line is linear in the line's contracted values, so evaluating at
  // its points and integrating back is these two n x n products (3 n^2 FMA per line instead of
  // 6 n FMA per point).
  const T *vline_km;
  // FP64, 3D, n <= kFaceMatrixMaxN only (null otherwise), per cut cell ci and cut face f with
  // index i = fmat_idx[ci * 2d + f] (-1: no lines): the cut face's mass matrix in the in-face
  // tensor basis over the face's quadrature points,
  // fmat[i][a][b] = sum_p w_p phi_a(p) phi_b(p), a, b = i_b' + n i_c' (b' < c' the in-face axes),
  // symmetric bit for bit.  The SIPG integrand of a cut face is linear in the traces' values at
  // its points, so the point loop of the face's lines is the product of this n^2 x n^2 matrix
  // with the jump and the flux traces (2 n^4 FMA per face).
  const T *fmat;
  const int32_t *fmat_idx;
  int32_t kappa_uniform;
  int32_t n_active, n_cut;
  // the cut-cell kernel gives cut_list[0 .. cut_split[0]) 32 lanes per cell, [cut_split[0] ..
  // cut_split[1]) 16 lanes (2 cells per warp) and the rest 8 lanes (4 cells per warp)
  int32_t cut_split[2];
};

// Lanes of the cut-cell kernel for one cut cell: the smallest group (8, 16 or 32 lanes) whose
// chunk holds all volume lines and all cut-face lines of the cell, so that small cut cells share
// a warp; groups of 8 or 16 only for n <= 5.
inline int cut_lanes_for(int n, int64_t lines) {
  return (n > 5 || lines > 16) ? 32 : (lines > 8 ? 16 : 8);
}

// A part of y = A x: the active cells [cell_begin, cell_end) and, of the cut cells among them,
// the slots [split[0], split[3]) of cut_list / cut_idx (32-lane class up to split[1], 16-lane
// class up to split[2], then 8 lanes).  The parts of the host-buffer pipeline.
struct LaunchRange {
  int32_t cell_begin, cell_end;
  const int32_t *cut_list, *cut_idx;
  int32_t split[4];
  // when set (FP64 only): the structured kernel takes the cells cells[cell_begin .. cell_end)
  const int32_t *cells;
};

// Launchers (uf_kernels_*.cu).  Return cudaError_t as int.
// ev: optional events recorded around the structured kernel (ev[0], ev[1]) and the cut-cell
// kernel (ev[2], ev[3]); nullptr when not profiling.  rg: nullptr for the whole operator.
template <typename T>
int launch_vmult(int dim, int n, const DevArrays<T> &d, const void *tables_struct,
                 const void *tables_point, const Scalars<T> &s, T *y, const T *x, bool adjoint,
                 void *stream, void *const *ev, const LaunchRange *rg = nullptr);

}  // namespace uf
