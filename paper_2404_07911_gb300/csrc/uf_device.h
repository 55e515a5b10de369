// Device-side data of the unfitted DG operator (internal to libunfitted).
#pragma once

#include <cstdint>

namespace uf {

constexpr int kMaxNdev = 9;

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
template <typename T, int N>
struct StructTables {
  T kv[N * N];
  T mass[N * N];
  T a[2][N * N], pen[2][N * N], gp[2][N * N];
  T b[2][N * N], c[2][N * N], qn[2][N * N], hn[2][N * N];
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
};

// Pointers into device memory (one allocation per precision).
template <typename T>
struct DevArrays {
  const int32_t *nbr;       // [n_active * 2d]
  const uint32_t *flags;    // [n_active]
  const T *kappa;           // [n_active]
  const int32_t *cut_list;  // [n_cut] active ids, most expensive first
  const int32_t *cut_idx;   // [n_cut] cut index of cut_list[i] (row of the offset arrays)
  const int32_t *vol_off, *surf_off, *cface_off;  // [n_cut + 1], [n_cut + 1], [n_cut * 2d + 1]
  const T *vol_xi[3], *vol_w;
  const T *surf_xi[3], *surf_w, *surf_n[3];
  const T *cface_eta[2], *cface_w;
  int32_t n_active, n_cut;
};

// Launchers (uf_kernels_*.cu).  Return cudaError_t as int.
// ev: optional events recorded around the structured kernel (ev[0], ev[1]) and the cut-cell
// kernel (ev[2], ev[3]); nullptr when not profiling.
template <typename T>
int launch_vmult(int dim, int n, const DevArrays<T> &d, const void *tables_struct,
                 const void *tables_point, const Scalars<T> &s, T *y, const T *x, bool adjoint,
                 void *stream, void *const *ev);

}  // namespace uf
