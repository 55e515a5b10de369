// Kernels of the matrix-free unfitted DG operator (arXiv 2404.07911), written for sm_103a.
//
// y = A x is evaluated cell-centrically: every active cell computes all terms whose test
// function lives on it and writes only its own n^d rows (no atomics), reading its neighbours'
// DoFs from global memory (they stay L2 resident).  Two kernels share the work:
//
//  * struct_kernel (all active cells): the structured terms of Sec. 3.2 (Eq.
//    sum_factorization_cell, Eq. sum_factorization_face): on a Cartesian cell every structured
//    term is a Kronecker product of 1D matrices, so
//        y_K = sum_a M (x) .. (x) L_a (x) .. (x) M  u_K  +  sum_faces  M (x) .. L_f .. (x) M  u_nb,
//    where L_a collects the cell stiffness (inside cells) and the own-trace parts of the SIPG
//    (full faces) and ghost-penalty terms, and L_f the neighbour couplings.  Per axis a the
//    kernel applies L along a-lines (registers, one line per thread), then the 1D mass along the
//    other axes (lines read back through shared memory).
//  * cut_kernel (one CTA per cut cell): the unstructured terms of Sec. 3.2 (Eq.
//    unstructured_cell, Eq. unstructured_face): Poisson volume term at the dimension-reduction
//    volume points, the Nitsche term at the surface points, and SIPG on cut faces.  Each point
//    evaluates the 1D basis in each direction and contracts the cell's DoFs one direction at a
//    time; integration accumulates the transposed contraction into the cell's rows.  The
//    kernel adds to y after struct_kernel (stream order), so no atomics are needed.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "uf_device.h"

namespace uf {

template <int DIM, int N>
struct Geo {
  static constexpr int ND = (DIM == 2) ? N * N : N * N * N;  // DoFs per cell
  static constexpr int NL = (DIM == 2) ? N : N * N;          // lines per direction
  static constexpr int NF = 2 * DIM;                         // faces per cell
};

// Stride of the local index l = i + n j + n^2 k along `axis`.
template <int N>
__device__ __forceinline__ int stride_of(int axis) {
  return axis == 0 ? 1 : (axis == 1 ? N : N * N);
}

// Offset of the first DoF of line t along `axis` (t enumerates the other axes, lowest first).
template <int DIM, int N>
__device__ __forceinline__ int line_base(int axis, int t) {
  if constexpr (DIM == 2) {
    return (axis == 0) ? t * N : t;
  } else {
    const int tb = t % N, tc = t / N;
    if (axis == 0) return tb * N + tc * N * N;
    if (axis == 1) return tb + tc * N * N;
    return tb + tc * N;
  }
}

__device__ __forceinline__ bool bit(uint32_t f, uint32_t b) { return (f & b) != 0u; }
__device__ __forceinline__ uint32_t bit_full(int f) { return 1u << (1 + 3 * f); }
__device__ __forceinline__ uint32_t bit_cut(int f) { return 1u << (2 + 3 * f); }
__device__ __forceinline__ uint32_t bit_gp(int f) { return 1u << (3 + 3 * f); }

template <int N>
__host__ __device__ constexpr int struct_cells_per_block(int NL) {
  return (NL >= 128) ? 1 : (128 / NL);
}

// ------------------------------------------------------------------------------------------
// Structured terms
// ------------------------------------------------------------------------------------------
template <typename T, int DIM, int N, bool ADJ>
__global__ void __launch_bounds__(128) struct_kernel(const __grid_constant__ StructTables<T, N> tab,
                                                     const DevArrays<T> d, T *__restrict__ y,
                                                     const T *__restrict__ x) {
  using G = Geo<DIM, N>;
  constexpr int ND = G::ND, NL = G::NL, NF = G::NF, NN = N * N;
  constexpr int CPB = struct_cells_per_block<N>(NL);
  constexpr int TPC = NL;

  __shared__ T s_tab[16 * NN];
  __shared__ T s_u[CPB][ND];
  __shared__ T s_w[CPB][ND];
  __shared__ T s_y[CPB][ND];
  __shared__ T s_l[CPB][3][NN];

  const int tid = threadIdx.x;
  // Copy the constant 1D matrices to shared memory (the L-build reads them per entry).
  {
    const T *src = reinterpret_cast<const T *>(&tab);
    for (int i = tid; i < 16 * NN; i += blockDim.x) s_tab[i] = src[i];
  }
  const T *kv = s_tab;
  const T *mass = s_tab + NN;
  auto A = [&](int s) { return s_tab + (2 + s) * NN; };
  auto P = [&](int s) { return s_tab + (4 + s) * NN; };
  auto GP = [&](int s) { return s_tab + (6 + s) * NN; };
  auto B = [&](int s) { return s_tab + (8 + s) * NN; };
  auto C = [&](int s) { return s_tab + (10 + s) * NN; };
  auto Q = [&](int s) { return s_tab + (12 + s) * NN; };
  auto H = [&](int s) { return s_tab + (14 + s) * NN; };

  const int first = blockIdx.x * CPB;
  const int c = tid / TPC;
  const int t = tid % TPC;
  const bool active_thread = (c < CPB);
  const int e = first + c;
  const bool has_cell = active_thread && (e < d.n_active);

  // Cooperative, coalesced load of the block's contiguous cells.
  {
    const int ncell = min(CPB, d.n_active - first);
    const T *src = x + (size_t)first * ND;
    for (int i = tid; i < ncell * ND; i += blockDim.x) (&s_u[0][0])[i] = src[i];
    for (int i = tid; i < CPB * ND; i += blockDim.x) (&s_y[0][0])[i] = T(0);
  }

  uint32_t fl = 0;
  int nb[NF];
  T kap = T(0), kavg[NF], knb[NF];
  if (has_cell) {
    fl = __ldg(d.flags + e);
    kap = __ldg(d.kappa + e);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      nb[f] = __ldg(d.nbr + (size_t)e * NF + f);
      knb[f] = (nb[f] >= 0) ? __ldg(d.kappa + nb[f]) : T(0);
      kavg[f] = T(0.5) * (kap + knb[f]);
    }
  } else {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      nb[f] = -1;
      knb[f] = T(0);
      kavg[f] = T(0);
    }
  }
  const bool inside = has_cell && !(fl & 1u);
  __syncthreads();

#pragma unroll 1
  for (int axis = 0; axis < DIM; ++axis) {
    // ---- per-cell 1D matrices for this axis: s_l[c][0] self, [1] lower neighbour, [2] upper
    if (active_thread) {
      for (int idx = t; idx < NN; idx += TPC) {
        const int r = idx / N, m = idx % N;
        const int tr = ADJ ? (m * N + r) : idx;  // transposed entry for the adjoint
        T self = inside ? kap * kv[tr] : T(0);
        T ln[2] = {T(0), T(0)};
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int f = 2 * axis + s;
          if (nb[f] < 0) continue;
          const bool full = bit(fl, bit_full(f));
          const bool gp = bit(fl, bit_gp(f));
          if (full) self += kap * A(s)[tr] + kavg[f] * P(s)[tr];
          if (gp) self += kavg[f] * GP(s)[tr];
          if (!ADJ) {
            if (full) ln[s] += kap * B(s)[idx] + knb[f] * C(s)[idx] + kavg[f] * Q(s)[idx];
            if (gp) ln[s] += kavg[f] * H(s)[idx];
          } else {
            // transpose of the neighbour's coupling toward this cell (its face 1 - s)
            const int so = 1 - s;
            if (full) ln[s] += knb[f] * B(so)[tr] + kap * C(so)[tr] + kavg[f] * Q(so)[tr];
            if (gp) ln[s] += kavg[f] * H(so)[tr];
          }
        }
        s_l[c][0][idx] = self;
        s_l[c][1][idx] = ln[0];
        s_l[c][2][idx] = ln[1];
      }
    }
    __syncthreads();

    // ---- L along `axis` (own line from shared memory, neighbour lines from global memory)
    if (has_cell) {
      const int base = line_base<DIM, N>(axis, t);
      const int st = stride_of<N>(axis);
      T u[N], w[N];
#pragma unroll
      for (int m = 0; m < N; ++m) u[m] = s_u[c][base + m * st];
#pragma unroll
      for (int r = 0; r < N; ++r) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < N; ++m) acc = fma(s_l[c][0][r * N + m], u[m], acc);
        w[r] = acc;
      }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int f = 2 * axis + s;
        if (nb[f] >= 0 && (bit(fl, bit_full(f)) || bit(fl, bit_gp(f)))) {
          const T *xn = x + (size_t)nb[f] * ND + base;
#pragma unroll
          for (int m = 0; m < N; ++m) u[m] = __ldg(xn + m * st);
#pragma unroll
          for (int r = 0; r < N; ++r) {
            T acc = w[r];
#pragma unroll
            for (int m = 0; m < N; ++m) acc = fma(s_l[c][1 + s][r * N + m], u[m], acc);
            w[r] = acc;
          }
        }
      }
#pragma unroll
      for (int r = 0; r < N; ++r) s_w[c][base + r * st] = w[r];
    }
    __syncthreads();

    // ---- 1D mass along the other axes, accumulate into s_y
#pragma unroll 1
    for (int ob = 0; ob < DIM; ++ob) {
      if (ob == axis) continue;
      const bool last = (ob == DIM - 1) || (axis == DIM - 1 && ob == DIM - 2);
      if (has_cell) {
        const int base = line_base<DIM, N>(ob, t);
        const int st = stride_of<N>(ob);
        T v[N];
#pragma unroll
        for (int m = 0; m < N; ++m) v[m] = s_w[c][base + m * st];
#pragma unroll
        for (int r = 0; r < N; ++r) {
          T acc = T(0);
#pragma unroll
          for (int m = 0; m < N; ++m) acc = fma(mass[r * N + m], v[m], acc);
          if (last)
            s_y[c][base + r * st] += acc;
          else
            s_w[c][base + r * st] = acc;
        }
      }
      __syncthreads();
    }
  }

  {
    const int ncell = min(CPB, d.n_active - first);
    T *dst = y + (size_t)first * ND;
    for (int i = tid; i < ncell * ND; i += blockDim.x) dst[i] = (&s_y[0][0])[i];
  }
}

// ------------------------------------------------------------------------------------------
// Unstructured terms on cut cells
// ------------------------------------------------------------------------------------------

// phi_i(xi) and phi_i'(xi) by prefix / suffix products of (xi - z_m).
template <typename T, int N>
__device__ __forceinline__ void basis_1d(const PointTables<T, N> &pt, T xi, T *val, T *der) {
  T pre[N], dpre[N], suf[N], dsuf[N];
  pre[0] = T(1);
  dpre[0] = T(0);
#pragma unroll
  for (int i = 1; i < N; ++i) {
    const T f = xi - pt.z[i - 1];
    dpre[i] = fma(dpre[i - 1], f, pre[i - 1]);
    pre[i] = pre[i - 1] * f;
  }
  suf[N - 1] = T(1);
  dsuf[N - 1] = T(0);
#pragma unroll
  for (int i = N - 2; i >= 0; --i) {
    const T f = xi - pt.z[i + 1];
    dsuf[i] = fma(dsuf[i + 1], f, suf[i + 1]);
    suf[i] = suf[i + 1] * f;
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    val[i] = pre[i] * suf[i] * pt.den_inv[i];
    der[i] = fma(dpre[i], suf[i], pre[i] * dsuf[i]) * pt.den_inv[i];
  }
}

template <int N>
__host__ __device__ constexpr int cut_chunk() {
  return (N <= 5) ? 128 : (N <= 8 ? 64 : 32);
}

template <typename T, int DIM, int N>
__global__ void __launch_bounds__(cut_chunk<N>()) cut_kernel(const __grid_constant__ PointTables<T, N> pt,
                                                            const DevArrays<T> d, const Scalars<T> sc,
                                                            T *__restrict__ y,
                                                            const T *__restrict__ x) {
  using G = Geo<DIM, N>;
  constexpr int ND = G::ND, NL = G::NL, NF = G::NF;
  constexpr int CH = cut_chunk<N>();
  constexpr int PSTRIDE = 2 * DIM * N + DIM + 1;  // per point: values, derivatives, coefficients

  __shared__ T s_u[ND];
  __shared__ T s_un[ND];
  __shared__ T s_acc[ND];
  __shared__ T s_pts[CH * PSTRIDE];
  __shared__ T s_tr[4][NL];   // traces: own value, own d/dn, neighbour value, neighbour d/dn
  __shared__ T s_ft[2][NL];   // face accumulators: value, d/dn

  const int tid = threadIdx.x;
  const int slot = blockIdx.x;
  if (slot >= d.n_cut) return;
  const int e = __ldg(d.cut_list + slot);
  const int ci = __ldg(d.cut_idx + slot);
  const T kap = __ldg(d.kappa + e);
  const uint32_t fl = __ldg(d.flags + e);

  for (int i = tid; i < ND; i += CH) {
    s_u[i] = __ldg(x + (size_t)e * ND + i);
    s_acc[i] = T(0);
  }
  __syncthreads();

  // ---- volume (Poisson) and surface (Nitsche) points
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    const int beg = __ldg((pass == 0 ? d.vol_off : d.surf_off) + ci);
    const int end = __ldg((pass == 0 ? d.vol_off : d.surf_off) + ci + 1);
#pragma unroll 1
    for (int p0 = beg; p0 < end; p0 += CH) {
      const int q = p0 + tid;
      T *mine = s_pts + tid * PSTRIDE;
      if (q < end) {
        T val[DIM][N], der[DIM][N];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          const T xi = __ldg((pass == 0 ? d.vol_xi[a] : d.surf_xi[a]) + q);
          basis_1d<T, N>(pt, xi, val[a], der[a]);
        }
        // value and reference gradient at the point, one direction at a time
        T u = T(0), g[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) g[a] = T(0);
        if constexpr (DIM == 3) {
#pragma unroll
          for (int k = 0; k < N; ++k) {
            T t0 = T(0), t1 = T(0), t2 = T(0);
#pragma unroll
            for (int j = 0; j < N; ++j) {
              T s0 = T(0), s1 = T(0);
#pragma unroll
              for (int i = 0; i < N; ++i) {
                const T v = s_u[i + N * j + N * N * k];
                s0 = fma(val[0][i], v, s0);
                s1 = fma(der[0][i], v, s1);
              }
              t0 = fma(val[1][j], s0, t0);
              t1 = fma(der[1][j], s0, t1);
              t2 = fma(val[1][j], s1, t2);
            }
            u = fma(val[2][k], t0, u);
            g[2] = fma(der[2][k], t0, g[2]);
            g[1] = fma(val[2][k], t1, g[1]);
            g[0] = fma(val[2][k], t2, g[0]);
          }
        } else {
#pragma unroll
          for (int j = 0; j < N; ++j) {
            T s0 = T(0), s1 = T(0);
#pragma unroll
            for (int i = 0; i < N; ++i) {
              const T v = s_u[i + N * j];
              s0 = fma(val[0][i], v, s0);
              s1 = fma(der[0][i], v, s1);
            }
            u = fma(val[1][j], s0, u);
            g[1] = fma(der[1][j], s0, g[1]);
            g[0] = fma(val[1][j], s1, g[0]);
          }
        }
        T cv, cg[DIM];
        if (pass == 0) {
          // kappa int grad v . grad u: reference gradients carry 1/h each
          const T wk = kap * __ldg(d.vol_w + q) * sc.inv_h2;
          cv = T(0);
#pragma unroll
          for (int a = 0; a < DIM; ++a) cg[a] = wk * g[a];
        } else {
          // kappa int_Gamma [ -d_n v u - v d_n u + tau/h v u ]
          const T wk = kap * __ldg(d.surf_w + q);
          T nr[DIM];
          T dn = T(0);
#pragma unroll
          for (int a = 0; a < DIM; ++a) {
            nr[a] = __ldg(d.surf_n[a] + q);
            dn = fma(nr[a], g[a], dn);
          }
          dn *= sc.inv_h;
          cv = wk * (sc.nitsche_over_h * u - dn);
#pragma unroll
          for (int a = 0; a < DIM; ++a) cg[a] = -wk * u * nr[a] * sc.inv_h;
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
          for (int i = 0; i < N; ++i) {
            mine[a * N + i] = val[a][i];
            mine[DIM * N + a * N + i] = der[a][i];
          }
        mine[2 * DIM * N] = cv;
#pragma unroll
        for (int a = 0; a < DIM; ++a) mine[2 * DIM * N + 1 + a] = cg[a];
      } else {
        for (int i = 0; i < PSTRIDE; ++i) mine[i] = T(0);
      }
      __syncthreads();
      const int npt = min(CH, end - p0);
      // integrate: every DoF gathers the chunk's points (transposed contraction)
      for (int l = tid; l < ND; l += CH) {
        const int i0 = l % N;
        const int i1 = (l / N) % N;
        T acc = T(0);
        if constexpr (DIM == 3) {
          const int i2 = l / (N * N);
#pragma unroll 4
          for (int pidx = 0; pidx < npt; ++pidx) {
            const T *pp = s_pts + pidx * PSTRIDE;
            const T v0 = pp[i0], v1 = pp[N + i1], v2 = pp[2 * N + i2];
            const T d0 = pp[3 * N + i0], d1 = pp[4 * N + i1], d2 = pp[5 * N + i2];
            const T cv = pp[6 * N], c0 = pp[6 * N + 1], c1 = pp[6 * N + 2], c2 = pp[6 * N + 3];
            const T v12 = v1 * v2;
            acc = fma(fma(cv, v0, c0 * d0), v12, acc);
            acc = fma(v0, fma(c1 * d1, v2, c2 * v1 * d2), acc);
          }
        } else {
#pragma unroll 4
          for (int pidx = 0; pidx < npt; ++pidx) {
            const T *pp = s_pts + pidx * PSTRIDE;
            const T v0 = pp[i0], v1 = pp[N + i1];
            const T d0 = pp[2 * N + i0], d1 = pp[3 * N + i1];
            const T cv = pp[4 * N], c0 = pp[4 * N + 1], c1 = pp[4 * N + 2];
            acc = fma(fma(cv, v0, c0 * d0), v1, acc);
            acc = fma(v0 * c1, d1, acc);
          }
        }
        s_acc[l] += acc;
      }
      __syncthreads();
    }
  }

  // ---- SIPG on cut faces: F cap Omega with unstructured in-face points (Eq. unstructured_face)
#pragma unroll 1
  for (int f = 0; f < NF; ++f) {
    if (!bit(fl, bit_cut(f))) continue;
    const int beg = __ldg(d.cface_off + (size_t)ci * NF + f);
    const int end = __ldg(d.cface_off + (size_t)ci * NF + f + 1);
    if (end <= beg) continue;
    const int axis = f / 2, side = f % 2;
    const int nbe = __ldg(d.nbr + (size_t)e * NF + f);
    const T knb = __ldg(d.kappa + nbe);
    const T kavg = T(0.5) * (kap + knb);
    const T sgn = side ? T(1) : T(-1);
    const int st = stride_of<N>(axis);
    for (int i = tid; i < ND; i += CH) s_un[i] = __ldg(x + (size_t)nbe * ND + i);
    __syncthreads();
    // traces on the face: values (delta property of the Lobatto basis) and n_K-derivatives
    for (int tl = tid; tl < NL; tl += CH) {
      const int base = line_base<DIM, N>(axis, tl);
      T ov = T(0), od = T(0), nv = T(0), nd = T(0);
#pragma unroll
      for (int m = 0; m < N; ++m) {
        const T uo = s_u[base + m * st];
        const T un = s_un[base + m * st];
        ov = fma(pt.end_val[side][m], uo, ov);
        od = fma(pt.end_der[side][m], uo, od);
        nv = fma(pt.end_val[1 - side][m], un, nv);
        nd = fma(pt.end_der[1 - side][m], un, nd);
      }
      s_tr[0][tl] = ov;
      s_tr[1][tl] = sgn * sc.inv_h * od;
      s_tr[2][tl] = nv;
      s_tr[3][tl] = sgn * sc.inv_h * nd;
      s_ft[0][tl] = T(0);
      s_ft[1][tl] = T(0);
    }
    __syncthreads();
    constexpr int FSTRIDE = 2 * N + 2;
#pragma unroll 1
    for (int p0 = beg; p0 < end; p0 += CH) {
      const int q = p0 + tid;
      T *mine = s_pts + tid * FSTRIDE;
      if (q < end) {
        T vb[N], vc[N], dummy[N];
        basis_1d<T, N>(pt, __ldg(d.cface_eta[0] + q), vb, dummy);
        if constexpr (DIM == 3) {
          basis_1d<T, N>(pt, __ldg(d.cface_eta[1] + q), vc, dummy);
        } else {
#pragma unroll
          for (int i = 0; i < N; ++i) vc[i] = (i == 0) ? T(1) : T(0);
        }
        T ev[4] = {T(0), T(0), T(0), T(0)};
        constexpr int NC = (DIM == 3) ? N : 1;
#pragma unroll
        for (int tc = 0; tc < NC; ++tc) {
          T part[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
          for (int tb = 0; tb < N; ++tb) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) part[kk] = fma(vb[tb], s_tr[kk][tb + N * tc], part[kk]);
          }
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) ev[kk] = fma(vc[tc], part[kk], ev[kk]);
        }
        const T w = __ldg(d.cface_w + q);
        const T jump = ev[0] - ev[2];
        const T avg = T(0.5) * (kap * ev[1] + knb * ev[3]);
        // coefficients of the own trace value and own normal derivative of the test function
        const T cvv = w * (sc.sipg_over_h * kavg * jump - avg);
        const T cdd = w * (T(-0.5) * kap * jump);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          mine[i] = vb[i];
          mine[N + i] = vc[i];
        }
        mine[2 * N] = cvv;
        mine[2 * N + 1] = cdd;
      } else {
        for (int i = 0; i < FSTRIDE; ++i) mine[i] = T(0);
      }
      __syncthreads();
      const int npt = min(CH, end - p0);
      for (int tl = tid; tl < NL; tl += CH) {
        const int tb = tl % N, tc = tl / N;
        T av = T(0), ad = T(0);
        for (int pidx = 0; pidx < npt; ++pidx) {
          const T *pp = s_pts + pidx * FSTRIDE;
          const T phi = pp[tb] * pp[N + tc];
          av = fma(pp[2 * N], phi, av);
          ad = fma(pp[2 * N + 1], phi, ad);
        }
        s_ft[0][tl] += av;
        s_ft[1][tl] += ad;
      }
      __syncthreads();
    }
    // expand the face accumulators into the cell: phi_l = phi_{i_a}(side) x in-face product
    for (int l = tid; l < ND; l += CH) {
      const int ia = (l / stride_of<N>(axis)) % N;
      int tl;
      if constexpr (DIM == 2) {
        tl = (axis == 0) ? l / N : l % N;
      } else {
        const int i0 = l % N, i1 = (l / N) % N, i2 = l / (N * N);
        tl = (axis == 0) ? (i1 + N * i2) : (axis == 1) ? (i0 + N * i2) : (i0 + N * i1);
      }
      s_acc[l] += pt.end_val[side][ia] * s_ft[0][tl] +
                  sgn * sc.inv_h * pt.end_der[side][ia] * s_ft[1][tl];
    }
    __syncthreads();
  }

  for (int i = tid; i < ND; i += CH) y[(size_t)e * ND + i] += s_acc[i];
}

// ------------------------------------------------------------------------------------------
// Launch
// ------------------------------------------------------------------------------------------
template <typename T, int DIM, int N>
int launch_vmult_t(const DevArrays<T> &d, const void *tables_struct, const void *tables_point,
                   const Scalars<T> &s, T *y, const T *x, bool adjoint, cudaStream_t stream,
                   void *const *ev) {
  using G = Geo<DIM, N>;
  constexpr int CPB = struct_cells_per_block<N>(G::NL);
  const int threads = ((CPB * G::NL + 31) / 32) * 32;
  const int blocks = (d.n_active + CPB - 1) / CPB;
  const auto &tab = *reinterpret_cast<const StructTables<T, N> *>(tables_struct);
  if (ev) cudaEventRecord(static_cast<cudaEvent_t>(ev[0]), stream);
  if (blocks > 0) {
    if (adjoint)
      struct_kernel<T, DIM, N, true><<<blocks, threads, 0, stream>>>(tab, d, y, x);
    else
      struct_kernel<T, DIM, N, false><<<blocks, threads, 0, stream>>>(tab, d, y, x);
  }
  if (ev) cudaEventRecord(static_cast<cudaEvent_t>(ev[1]), stream);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return (int)err;
  if (ev) cudaEventRecord(static_cast<cudaEvent_t>(ev[2]), stream);
  if (d.n_cut > 0) {
    const auto &ptab = *reinterpret_cast<const PointTables<T, N> *>(tables_point);
    cut_kernel<T, DIM, N><<<d.n_cut, cut_chunk<N>(), 0, stream>>>(ptab, d, s, y, x);
  }
  if (ev) cudaEventRecord(static_cast<cudaEvent_t>(ev[3]), stream);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_vmult_impl(int dim, int n, const DevArrays<T> &d, const void *ts, const void *tp,
                      const Scalars<T> &s, T *y, const T *x, bool adjoint, cudaStream_t st,
                      void *const *ev) {
#define UF_CASE(D, NN)                                                         \
  if (dim == D && n == NN) return launch_vmult_t<T, D, NN>(d, ts, tp, s, y, x, adjoint, st, ev);
  UF_CASE(2, 2) UF_CASE(2, 3) UF_CASE(2, 4) UF_CASE(2, 5) UF_CASE(2, 6) UF_CASE(2, 7)
  UF_CASE(2, 8) UF_CASE(2, 9) UF_CASE(3, 2) UF_CASE(3, 3) UF_CASE(3, 4) UF_CASE(3, 5)
  UF_CASE(3, 6) UF_CASE(3, 7) UF_CASE(3, 8) UF_CASE(3, 9)
#undef UF_CASE
  return (int)cudaErrorInvalidValue;
}

}  // namespace uf
