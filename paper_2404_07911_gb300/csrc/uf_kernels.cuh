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
#include <type_traits>

#include "uf_device.h"
#include "uf_struct_planes.cuh"

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

// Shared-memory layout of a cell in the structured kernel: element (i, j, k) at i + P j + P n k
// with the odd line stride P = n | 1, so that the lanes of a warp working on neighbouring x-lines
// (and the two cells a warp holds for n = 4) fall into different banks.
template <int N>
__host__ __device__ constexpr int spad() {
  return N | 1;
}
template <int DIM, int N>
__host__ __device__ constexpr int snd() {
  return (DIM == 2) ? spad<N>() * N : spad<N>() * N * N;
}
template <int N>
__device__ __forceinline__ int sstride(int axis) {
  return axis == 0 ? 1 : (axis == 1 ? spad<N>() : spad<N>() * N);
}
template <int DIM, int N>
__device__ __forceinline__ int sline_base(int axis, int t) {
  constexpr int P = spad<N>();
  if constexpr (DIM == 2) {
    return (axis == 0) ? t * P : t;
  } else {
    const int tb = t % N, tc = t / N;
    if (axis == 0) return tb * P + tc * P * N;
    if (axis == 1) return tb + tc * P * N;
    return tb + tc * P;
  }
}

// Row of an n x n row-major matrix whose rows start on multiples of n elements of a 16-byte
// aligned table: loaded with the widest vector the row length allows.
__device__ __forceinline__ void unpack(const float4 &v, float *o) {
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
__device__ __forceinline__ void unpack(const float2 &v, float *o) {
  o[0] = v.x;
  o[1] = v.y;
}
__device__ __forceinline__ void unpack(const double2 &v, double *o) {
  o[0] = v.x;
  o[1] = v.y;
}
template <typename T, int N>
__device__ __forceinline__ void load_row(const T *row, T *out) {
  constexpr int B = N * (int)sizeof(T);
  if constexpr (B % 16 == 0) {
    using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
    constexpr int W = 16 / (int)sizeof(T);
#pragma unroll
    for (int i = 0; i < N / W; ++i) unpack(reinterpret_cast<const V *>(row)[i], out + W * i);
  } else if constexpr (sizeof(T) == 4 && B % 8 == 0) {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) unpack(reinterpret_cast<const float2 *>(row)[i], out + 2 * i);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = row[i];
  }
}

__device__ __forceinline__ bool bit(uint32_t f, uint32_t b) { return (f & b) != 0u; }
__device__ __forceinline__ uint32_t bit_full(int f) { return 1u << (1 + 3 * f); }
__device__ __forceinline__ uint32_t bit_cut(int f) { return 1u << (2 + 3 * f); }
__device__ __forceinline__ uint32_t bit_gp(int f) { return 1u << (3 + 3 * f); }

// FP64 at n = 9 in 3D: the structured kernel's cells live in dynamic shared memory, so that a
// CTA can hold three of them (243 of 256 lanes busy; one cell in 48 KB of static arrays leaves
// 15 of 96 lanes idle).
template <typename T, int DIM, int N>
__host__ __device__ constexpr bool struct_dynamic_smem() {
  return DIM == 3 && N == 9 && sizeof(T) == 8;
}

// Cells per CTA of the structured kernel: one thread per line (n^{d-1} per cell), at most 128
// threads, and the shared memory of the cells (u, W per axis, per-cell matrices) under 40 KB.
template <typename T, int DIM, int N>
__host__ __device__ constexpr int struct_cells_per_block() {
  constexpr int NL = (DIM == 2) ? N : N * N;
  constexpr int by_threads = (NL >= 128) ? 1 : (128 / NL);
  constexpr int SND = (DIM == 2) ? (N | 1) * N : (N | 1) * N * N;
  constexpr int cell_bytes = (int)sizeof(T) * (SND * (1 + DIM) + DIM * 3 * N * N);
  constexpr int by_smem = 40960 / cell_bytes;
  int cpb = by_threads < by_smem ? by_threads : by_smem;
  if (cpb < 1) cpb = 1;
  // The warps of a CTA issue for all their lanes: when the cells leave more than 10 % of the
  // lanes idle (n = 6, 7 in 3D: 36 and 49 lines per cell), take the cell count up to 256 threads
  // and the 48 KB of static shared memory with the fewest idle lanes.
  auto idle = [](int c) { return ((c * NL + 31) / 32) * 32 - c * NL; };
  if (idle(cpb) * 10 > ((cpb * NL + 31) / 32) * 32) {
    int best = cpb;
    constexpr int smem_cap = struct_dynamic_smem<T, DIM, N>() ? 96 * 1024 : 48 * 1024;
    for (int c = 1; c * NL <= 256 && c * cell_bytes <= smem_cap; ++c)
      if (idle(c) * ((best * NL + 31) / 32) * 32 < idle(best) * ((c * NL + 31) / 32) * 32) best = c;
    cpb = best;
  }
  return cpb;
}

// Threads of a structured-kernel CTA (whole warps).
template <typename T, int DIM, int N>
__host__ __device__ constexpr int struct_threads() {
  constexpr int NL = (DIM == 2) ? N : N * N;
  return ((struct_cells_per_block<T, DIM, N>() * NL + 31) / 32) * 32;
}

// ------------------------------------------------------------------------------------------
// Structured terms
// ------------------------------------------------------------------------------------------
//
// y_K = sum_a (M .. L_a .. M) u_K + sum_faces (M .. L_f .. M) u_nb = (M (x) .. (x) M) Z with
// Z = sum_a Z_a, Z_a = M^{-1} (L_a u_K + sum_{faces along a} L_f u_nb): the 1D tables carry
// M^{-1}, so phase 1 computes every Z_a line by line and phase 2 sums the axes and applies the
// mass matrix once per direction (3 sweeps in 3D, 2 in 2D, instead of 5 and 2 for
// M_z (M_y W_x + M_x W_y) + M_y M_x W_z with W_a = M_a Z_a).
template <typename T, int N>
__device__ __forceinline__ void apply_line(const T *__restrict__ Lm, const T *u, T *w, bool accumulate) {
#pragma unroll
  for (int r = 0; r < N; ++r) {
    T lr[N];
    load_row<T, N>(Lm + r * N, lr);
    T acc = accumulate ? w[r] : T(0);
#pragma unroll
    for (int m = 0; m < N; ++m) acc = fma(lr[m], u[m], acc);
    w[r] = acc;
  }
}

template <typename T, int N>
__device__ __forceinline__ void mass_line(const T *__restrict__ M, T *v, int base, int st) {
  T a[N], b[N];
#pragma unroll
  for (int m = 0; m < N; ++m) a[m] = v[base + m * st];
#pragma unroll
  for (int r = 0; r < N; ++r) {
    T acc = T(0);
#pragma unroll
    for (int m = 0; m < N; ++m) acc = fma(M[r * N + m], a[m], acc);
    b[r] = acc;
  }
#pragma unroll
  for (int r = 0; r < N; ++r) v[base + r * st] = b[r];
}

// Axis 0 of the uniform-kappa path in W space (tables without M^{-1}), for the x-line whose
// DoFs are u: w += L_0 u + the couplings of the two axis-0 neighbours (ghost penalty: full 1D
// matrix; SIPG only: rank 2).  Added after the mass sweep along axis 0, which is then the only
// sweep that sees these terms' M_0 M_0^{-1} = I.
template <typename T, int DIM, int N, bool ADJ>
__device__ __forceinline__ void axis0_lines(const StructTables<T, N> &tab, const DevArrays<T> &d,
                                            const Scalars<T> &sc, const T *__restrict__ x,
                                            const int *nb, uint32_t fl, bool inside, int t,
                                            const T *u, T *w) {
  constexpr int ND = Geo<DIM, N>::ND, NN = N * N;
  int v = inside ? 1 : 0;
  v |= bit(fl, bit_full(0)) ? 2 : 0;
  v |= bit(fl, bit_gp(0)) ? 4 : 0;
  v |= bit(fl, bit_full(1)) ? 8 : 0;
  v |= bit(fl, bit_gp(1)) ? 16 : 0;
  apply_line<T, N>((ADJ ? d.lselfxT : d.lselfx) + v * NN, u, w, true);
  const int base = line_base<DIM, N>(0, t);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    if (nb[s] < 0) continue;
    const bool full = bit(fl, bit_full(s));
    const bool gp = bit(fl, bit_gp(s));
    if (!full && !gp) continue;
    T un[N];
    const T *xn = x + (size_t)nb[s] * ND + base;
#pragma unroll
    for (int m = 0; m < N; ++m) un[m] = __ldg(xn + m);
    if (gp) {
      const T *Lg = ADJ ? d.lnbgpxT + (2 * (1 - s) + (full ? 1 : 0)) * NN
                        : d.lnbgpx + (2 * s + (full ? 1 : 0)) * NN;
      apply_line<T, N>(Lg, un, w, true);
    } else {
      // rank-2 SIPG coupling: dow times the neighbour's face value, minus the neighbour's normal
      // derivative and penalty at the own face node
      const T alpha = un[s ? 0 : N - 1];
      T beta = T(0);
#pragma unroll
      for (int m = 0; m < N; ++m) beta = fma(tab.dnb[s][m], un[m], beta);
#pragma unroll
      for (int r = 0; r < N; ++r) w[r] = fma(alpha, tab.dowx[s][r], w[r]);
      w[s ? N - 1 : 0] -= fma(sc.hf_sigma, alpha, beta);
    }
  }
}

// LIST: the cells are cell_list[cell_begin .. cell_end) instead of cell_begin .. cell_end.
template <typename T, int DIM, int N, bool ADJ, bool UNI, bool LIST = false>
__global__ void __launch_bounds__(struct_threads<T, DIM, N>()) struct_kernel(const __grid_constant__ StructTables<T, N> tab,
                                                     const DevArrays<T> d, const Scalars<T> sc,
                                                     T *__restrict__ y, const T *__restrict__ x,
                                                     int cell_begin, int cell_end,
                                                     const int32_t *__restrict__ cell_list = nullptr) {
  using G = Geo<DIM, N>;
  constexpr int ND = G::ND, NL = G::NL, NF = G::NF, NN = N * N;
  constexpr int CPB = struct_cells_per_block<T, DIM, N>();
  constexpr int TPC = NL;
  constexpr int P = spad<N>(), SND = snd<DIM, N>();

  // u, W per axis and the per-cell matrices (non-uniform kappa): static arrays, or the dynamic
  // shared memory in the same order (struct_smem_bytes)
  constexpr bool DYN = struct_dynamic_smem<T, DIM, N>();
  __shared__ __align__(16) T s_u_st[DYN ? 1 : CPB][SND];
  __shared__ __align__(16) T s_w_st[DIM][DYN ? 1 : CPB][SND];
  __shared__ __align__(16) T s_l_st[DYN ? 1 : CPB][DIM][3][NN];
  extern __shared__ __align__(16) unsigned char struct_dyn[];
  auto &s_u = *reinterpret_cast<T (*)[CPB][SND]>(DYN ? static_cast<void *>(struct_dyn)
                                                     : static_cast<void *>(s_u_st));
  auto &s_w = *reinterpret_cast<T (*)[DIM][CPB][SND]>(
      DYN ? static_cast<void *>(struct_dyn + sizeof(T) * CPB * SND) : static_cast<void *>(s_w_st));
  auto &s_l = *reinterpret_cast<T (*)[CPB][DIM][3][NN]>(
      DYN ? static_cast<void *>(struct_dyn + sizeof(T) * (1 + DIM) * CPB * SND) : static_cast<void *>(s_l_st));
  // FP32 keeps the form without M^{-1} (W_a = L_a u + couplings, then the shared in-face mass
  // sweeps y = M_z (M_y W_x + M_x W_y) + M_y M_x W_z): its rounding errors are not amplified by
  // M^{-1}, which the FP32 solves inside iterative refinement depend on
  constexpr bool WS = sizeof(T) == 4;

  const int tid = threadIdx.x;
  const int first = cell_begin + blockIdx.x * CPB;
  const int c = tid / TPC;
  const int t = tid % TPC;
  const bool active_thread = (c < CPB);
  const bool has_cell = active_thread && (first + c < cell_end);
  const int e = LIST ? (has_cell ? __ldg(cell_list + first + c) : 0) : first + c;
  constexpr bool uniform = UNI;  // kappa uniform (d.kappa_uniform != 0)

  {
    const int ncell = min(CPB, cell_end - first);
    if constexpr (LIST) {
      for (int i = tid; i < ncell * ND; i += blockDim.x) {
        const int l = i % ND;
        s_u[i / ND][l + (P - N) * (l / N)] = x[(size_t)__ldg(cell_list + first + i / ND) * ND + l];
      }
    } else {
      const T *src = x + (size_t)first * ND;
      for (int i = tid; i < ncell * ND; i += blockDim.x) {
        const int l = i % ND;
        s_u[i / ND][l + (P - N) * (l / N)] = src[i];
      }
    }
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
  // Uniform kappa: every structured term scales with it, so the lines are computed for kappa = 1
  // and the cell's rows are scaled once at the end (not at all when kappa = 1).
  const T yscale = uniform ? kap : T(1);
  if (uniform) {
    kap = T(1);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      knb[f] = T(1);
      kavg[f] = T(1);
    }
  }
  const bool scale_rows = yscale != T(1);

  if (!uniform && has_cell) {
    // per-cell 1D matrices from the constant ones and kappa; the constant matrices are read from
    // their global-memory copy (each thread reads its own entry: coalesced through L1), matrix
    // `which` (kv 0, mass 1, a 2, pen 4, gp 6, b 8, c 10, qn 12, hn 14, + side) at which * NN
    // FP64: M^{-1} Q_k (adjoint: M^{-1} Q_k^T); FP32: Q_k, transposed by the index (adjoint)
    const T *Q = WS ? d.smat0 : (ADJ ? d.smatT : d.smat);
    for (int a = 0; a < DIM; ++a)
      for (int idx = t; idx < NN; idx += TPC) {
        const int tr = (WS && ADJ) ? ((idx % N) * N + idx / N) : idx;
        T self = inside ? kap * __ldg(Q + tr) : T(0);
        T ln[2] = {T(0), T(0)};
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int f = 2 * a + s;
          if (nb[f] < 0) continue;
          const bool full = bit(fl, bit_full(f));
          const bool gp = bit(fl, bit_gp(f));
          if (full) self += kap * __ldg(Q + (2 + s) * NN + tr) + kavg[f] * __ldg(Q + (4 + s) * NN + tr);
          if (gp) self += kavg[f] * __ldg(Q + (6 + s) * NN + tr);
          if (gp) {
            if (!ADJ) {
              if (full)
                ln[s] += kap * __ldg(Q + (8 + s) * NN + idx) + knb[f] * __ldg(Q + (10 + s) * NN + idx) +
                         kavg[f] * __ldg(Q + (12 + s) * NN + idx);
              ln[s] += kavg[f] * __ldg(Q + (14 + s) * NN + idx);
            } else {
              // transpose of the neighbour's coupling toward this cell (its face 1 - s)
              const int so = 1 - s;
              if (full)
                ln[s] += knb[f] * __ldg(Q + (8 + so) * NN + tr) + kap * __ldg(Q + (10 + so) * NN + tr) +
                         kavg[f] * __ldg(Q + (12 + so) * NN + tr);
              ln[s] += kavg[f] * __ldg(Q + (14 + so) * NN + tr);
            }
          }
        }
        s_l[c][a][0][idx] = self;
        s_l[c][a][1][idx] = ln[0];
        s_l[c][a][2][idx] = ln[1];
      }
  }
  __syncthreads();

  // ---- phase 1: Z_a = M^{-1} (L_a u + neighbour couplings), one line per thread and axis (the
  // uniform-kappa path leaves axis 0 to the first mass sweep)
  if (has_cell) {
#pragma unroll 1
    for (int a = (uniform && !WS) ? 1 : 0; a < DIM; ++a) {
      const int base = line_base<DIM, N>(a, t);  // global layout (neighbour lines)
      const int st = stride_of<N>(a);
      const int sb = sline_base<DIM, N>(a, t);   // shared-memory layout
      const int ss = sstride<N>(a);
      T u[N], w[N];
#pragma unroll
      for (int m = 0; m < N; ++m) u[m] = s_u[c][sb + m * ss];
      if (uniform) {
        int v = inside ? 1 : 0;
        v |= bit(fl, bit_full(2 * a)) ? 2 : 0;
        v |= bit(fl, bit_gp(2 * a)) ? 4 : 0;
        v |= bit(fl, bit_full(2 * a + 1)) ? 8 : 0;
        v |= bit(fl, bit_gp(2 * a + 1)) ? 16 : 0;
        apply_line<T, N>((WS ? (ADJ ? d.lselfxT : d.lselfx) : (ADJ ? d.lselfT : d.lself)) + v * NN, u, w, false);
      } else {
        apply_line<T, N>(s_l[c][a][0], u, w, false);
      }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int f = 2 * a + s;
        if (nb[f] < 0) continue;
        const bool full = bit(fl, bit_full(f));
        const bool gp = bit(fl, bit_gp(f));
        if (!full && !gp) continue;
        T un[N];
        const T *xn = x + (size_t)nb[f] * ND + base;
#pragma unroll
        for (int m = 0; m < N; ++m) un[m] = __ldg(xn + m * st);
        if (gp) {
          if (uniform) {
            // transpose of the neighbour's table entry (its face 1 - s) for the adjoint
            const T *Lg = ADJ ? (WS ? d.lnbgpxT : d.lnbgpT) + (2 * (1 - s) + (full ? 1 : 0)) * NN
                              : (WS ? d.lnbgpx : d.lnbgp) + (2 * s + (full ? 1 : 0)) * NN;
            apply_line<T, N>(Lg, un, w, true);
          } else {
            apply_line<T, N>(s_l[c][a][1 + s], un, w, true);
          }
        } else {
          // rank-2 SIPG coupling (the transposed coupling of a symmetric flux is the same form):
          // M^{-1} (ca dow - g e_own) with the device tables M^{-1} dow and me = M^{-1} e_own;
          // dow and dnb carry the factor h^{d-1} / 2
          const T alpha = un[s ? 0 : N - 1];
          T beta = T(0);
#pragma unroll
          for (int m = 0; m < N; ++m) beta = fma(tab.dnb[s][m], un[m], beta);
          const T ca = uniform ? alpha : kap * alpha;
          T g;
          if constexpr (uniform) {
            g = fma(sc.hf_sigma, alpha, beta);
          } else {
            g = fma(knb[f], beta, (sc.hf_sigma * kavg[f]) * alpha);
          }
          if constexpr (WS) {
            // W space: ca dow - g e_own
#pragma unroll
            for (int r = 0; r < N; ++r) w[r] = fma(ca, tab.dowx[s][r], w[r]);
            w[s ? N - 1 : 0] -= g;
          } else {
#pragma unroll
            for (int r = 0; r < N; ++r) w[r] = fma(-g, tab.me[s][r], fma(ca, tab.dow[s][r], w[r]));
          }
        }
      }
#pragma unroll
      for (int r = 0; r < N; ++r) s_w[a][c][sb + r * ss] = w[r];
    }
  }
  __syncthreads();

  // ---- phase 2: y = (M (x) .. (x) M) sum_a Z_a (M symmetric: the adjoint uses the same sweeps)
  const T *M = tab.mass;
  if constexpr (WS && DIM == 2) {
    // FP32: y = M_y W_x + M_x W_y
    if (has_cell) {
      mass_line<T, N>(M, s_w[0][c], sline_base<DIM, N>(1, t), P);  // M_y W_x
      mass_line<T, N>(M, s_w[1][c], sline_base<DIM, N>(0, t), 1);  // M_x W_y
    }
    __syncthreads();
    if (has_cell) {
      // y = W_x + W_y; thread t writes the x-line t
      const int base = line_base<DIM, N>(0, t), sb = sline_base<DIM, N>(0, t);
#pragma unroll
      for (int r = 0; r < N; ++r) {
        const T v = s_w[0][c][sb + r] + s_w[1][c][sb + r];
        y[(size_t)e * ND + base + r] = scale_rows ? yscale * v : v;
      }
    }
  } else if constexpr (WS) {
    // FP32: y = M_z (M_y W_x + M_x W_y) + M_y M_x W_z
    if (has_cell) {
      mass_line<T, N>(M, s_w[0][c], sline_base<DIM, N>(1, t), P);  // W_x <- M_y W_x
      mass_line<T, N>(M, s_w[2][c], sline_base<DIM, N>(0, t), 1);  // W_z <- M_x W_z
    }
    __syncthreads();
    if (has_cell) {
      // W_x += M_x W_y (x-lines)
      const int bx = sline_base<DIM, N>(0, t);
      T a[N];
#pragma unroll
      for (int m = 0; m < N; ++m) a[m] = s_w[1][c][bx + m];
#pragma unroll
      for (int r = 0; r < N; ++r) {
        T acc = s_w[0][c][bx + r];
#pragma unroll
        for (int m = 0; m < N; ++m) acc = fma(M[r * N + m], a[m], acc);
        s_w[0][c][bx + r] = acc;
      }
      mass_line<T, N>(M, s_w[2][c], sline_base<DIM, N>(1, t), P);  // W_z <- M_y W_z
    }
    __syncthreads();
    if (has_cell) {
      // y = M_z W_x + W_z along z-lines
      const int bz = line_base<DIM, N>(2, t), sbz = sline_base<DIM, N>(2, t);
      T a[N];
#pragma unroll
      for (int m = 0; m < N; ++m) a[m] = s_w[0][c][sbz + m * P * N];
#pragma unroll
      for (int r = 0; r < N; ++r) {
        T acc = s_w[2][c][sbz + r * P * N];
#pragma unroll
        for (int m = 0; m < N; ++m) acc = fma(M[r * N + m], a[m], acc);
        y[(size_t)e * ND + bz + r * N * N] = scale_rows ? yscale * acc : acc;
      }
    }
  } else if constexpr (DIM == 2) {
    if (has_cell) {
      // Z_x <- M_x (Z_x + Z_y) along x-lines (uniform kappa: M_x Z_y + L_x u + x-neighbours)
      const int bx = sline_base<DIM, N>(0, t);
      T a[N], o[N];
#pragma unroll
      for (int m = 0; m < N; ++m) a[m] = uniform ? s_w[1][c][bx + m] : s_w[0][c][bx + m] + s_w[1][c][bx + m];
#pragma unroll
      for (int r = 0; r < N; ++r) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < N; ++m) acc = fma(M[r * N + m], a[m], acc);
        o[r] = acc;
      }
      if constexpr (uniform) {
        T u[N];
#pragma unroll
        for (int m = 0; m < N; ++m) u[m] = s_u[c][bx + m];
        axis0_lines<T, DIM, N, ADJ>(tab, d, sc, x, nb, fl, inside, t, u, o);
      }
#pragma unroll
      for (int r = 0; r < N; ++r) s_w[0][c][bx + r] = o[r];
    }
    __syncthreads();
    if (has_cell) {
      // y = M_y Z_x along y-lines
      const int by = line_base<DIM, N>(1, t), sby = sline_base<DIM, N>(1, t);
      T a[N];
#pragma unroll
      for (int m = 0; m < N; ++m) a[m] = s_w[0][c][sby + m * P];
#pragma unroll
      for (int r = 0; r < N; ++r) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < N; ++m) acc = fma(M[r * N + m], a[m], acc);
        y[(size_t)e * ND + by + r * N] = scale_rows ? yscale * acc : acc;
      }
    }
  } else {
    if (has_cell) {
      // Z_x <- M_x (Z_x + Z_y + Z_z) along x-lines (uniform kappa: M_x (Z_y + Z_z) + L_x u +
      // x-neighbours)
      const int bx = sline_base<DIM, N>(0, t);
      T a[N], o[N];
#pragma unroll
      for (int m = 0; m < N; ++m)
        a[m] = uniform ? s_w[1][c][bx + m] + s_w[2][c][bx + m]
                       : (s_w[0][c][bx + m] + s_w[1][c][bx + m]) + s_w[2][c][bx + m];
#pragma unroll
      for (int r = 0; r < N; ++r) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < N; ++m) acc = fma(M[r * N + m], a[m], acc);
        o[r] = acc;
      }
      if constexpr (uniform) {
        T u[N];
#pragma unroll
        for (int m = 0; m < N; ++m) u[m] = s_u[c][bx + m];
        axis0_lines<T, DIM, N, ADJ>(tab, d, sc, x, nb, fl, inside, t, u, o);
      }
#pragma unroll
      for (int r = 0; r < N; ++r) s_w[0][c][bx + r] = o[r];
    }
    __syncthreads();
    if (has_cell) mass_line<T, N>(M, s_w[0][c], sline_base<DIM, N>(1, t), P);  // Z_x <- M_y Z_x
    __syncthreads();
    if (has_cell) {
      // y = M_z Z_x along z-lines
      const int bz = line_base<DIM, N>(2, t), sbz = sline_base<DIM, N>(2, t);
      T a[N];
#pragma unroll
      for (int m = 0; m < N; ++m) a[m] = s_w[0][c][sbz + m * P * N];
#pragma unroll
      for (int r = 0; r < N; ++r) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < N; ++m) acc = fma(M[r * N + m], a[m], acc);
        y[(size_t)e * ND + bz + r * N * N] = scale_rows ? yscale * acc : acc;
      }
    }
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

// phi_i(xi) only.
template <typename T, int N>
__device__ __forceinline__ void basis_1d_val(const PointTables<T, N> &pt, T xi, T *val) {
  T pre[N], suf[N];
  pre[0] = T(1);
#pragma unroll
  for (int i = 1; i < N; ++i) pre[i] = pre[i - 1] * (xi - pt.z[i - 1]);
  suf[N - 1] = T(1);
#pragma unroll
  for (int i = N - 2; i >= 0; --i) suf[i] = suf[i + 1] * (xi - pt.z[i + 1]);
#pragma unroll
  for (int i = 0; i < N; ++i) val[i] = pre[i] * suf[i] * pt.den_inv[i];
}

// FP64 reads the 1D basis values at lines and points from tables built at creation (the FP64 pipe
// runs at 1/64 of the FP32 rate on this part, so loading 2n values is cheaper than evaluating
// them); FP32 evaluates them in registers.
template <typename T>
constexpr bool kPrecomputedBasis = sizeof(T) == sizeof(double);

template <typename T, int N>
__device__ __forceinline__ void point_basis(const PointTables<T, N> &pt, const T *tab, const T *tt,
                                            int p, T *val, T *der) {
  if constexpr (kPrecomputedBasis<T>) {
    const T *bp = tab + (size_t)p * 2 * N;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      val[i] = __ldg(bp + i);
      der[i] = __ldg(bp + N + i);
    }
  } else {
    basis_1d<T, N>(pt, __ldg(tt + p), val, der);
  }
}

// The volume points of a line enter only through the line integrals K, M (FP64: read from the
// precomputed vline_km, which takes 3 n^2 FMA per line instead of 6 n per point on the FP64 pipe),
// or point by point with the 1D basis evaluated in registers (FP32: the latency-bound FP32 kernel
// measured faster without the extra table reads).
template <typename T>
constexpr bool kLineIntegrals = sizeof(T) == sizeof(double);
// FP64 cut faces in 3D through their mass matrices (DevArrays::fmat) up to kFaceMatrixMaxN
template <typename T, int DIM, int N>
constexpr bool kFaceMatrices = sizeof(T) == sizeof(double) && DIM == 3 && N <= kFaceMatrixMaxN;

// z += cf w_p (phi'(t_p) phi'(t_p)^T w0, phi phi^T w1, phi phi^T w2) over the line's points.
template <typename T, int N>
__device__ __forceinline__ void point_integrals(const PointTables<T, N> &pt, const DevArrays<T> &d,
                                                T cfv, int line, const T *w0, const T *w1,
                                                const T *w2, T *z0, T *z1, T *z2, bool third) {
#pragma unroll
  for (int m = 0; m < N; ++m) {
    z0[m] = T(0);
    z1[m] = T(0);
    z2[m] = T(0);
  }
  const int pb = __ldg(d.vpt_off + line), pe = __ldg(d.vpt_off + line + 1);
#pragma unroll 1
  for (int p = pb; p < pe; ++p) {
    T cv[N], cd[N];
    point_basis<T, N>(pt, d.vpt_b, d.vpt_t, p, cv, cd);
    T gk = T(0), gb = T(0), gc = T(0);
#pragma unroll
    for (int m = 0; m < N; ++m) {
      gk = fma(cd[m], w0[m], gk);
      gb = fma(cv[m], w1[m], gb);
      if (third) gc = fma(cv[m], w2[m], gc);
    }
    // kappa int grad v . grad u: reference gradients carry 1/h each
    const T cf = cfv * __ldg(d.vpt_w + p);
    gk *= cf;
    gb *= cf;
    gc *= cf;
#pragma unroll
    for (int m = 0; m < N; ++m) {
      z0[m] = fma(gk, cd[m], z0[m]);
      z1[m] = fma(gb, cv[m], z1[m]);
      if (third) z2[m] = fma(gc, cv[m], z2[m]);
    }
  }
}

// z0 = kappa K w0, z1 = kappa M w1 (and z2 = kappa M w2 when `third`) with the n x n line
// integrals K, M stored one after the other at km (rows start on multiples of n elements).
template <typename T, int N>
__device__ __forceinline__ void line_products(const T *km, T kap, const T *w0, const T *w1,
                                              const T *w2, T *z0, T *z1, T *z2, bool third) {
#pragma unroll
  for (int r = 0; r < N; ++r) {
    T kr[N], mr[N];
    load_row<T, N>(km + r * N, kr);
    load_row<T, N>(km + N * N + r * N, mr);
    T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
    for (int m = 0; m < N; ++m) {
      a0 = fma(kr[m], w0[m], a0);
      a1 = fma(mr[m], w1[m], a1);
      if (third) a2 = fma(mr[m], w2[m], a2);
    }
    z0[r] = a0;
    z1[r] = a1;
    z2[r] = a2;
  }
  if (kap != T(1)) {
#pragma unroll
    for (int r = 0; r < N; ++r) {
      z0[r] *= kap;
      z1[r] *= kap;
      z2[r] *= kap;
    }
  }
}

// The cut-cell kernel runs one warp per CTA; each cut cell is handled by a group of S lanes
// (S = 32, 16 or 8: the CTA then holds 32 / S cells), and S lines form a chunk.  A chunk of the
// 3D volume part holds at most cut_gmax line groups (it ends early at the next group start once
// it has that many; the per-group partial contractions take GMAX n^2 values each).
template <int N>
__host__ __device__ constexpr int cut_gmax() {
  return (N <= 5) ? 16 : (N <= 8) ? 8 : 6;
}


// Other axes of a line along axis k (lower first) in 3D.
__device__ __forceinline__ void other_axes(int k, int &b, int &c) {
  b = (k == 0) ? 1 : 0;
  c = (k == 2) ? 1 : 2;
}

// Dynamic shared memory of the cut-cell kernel (offsets in elements of T, then ints).  The
// volume phase and the cut-face phase run one after the other, so the per-group partial
// contractions (3D), the per-line partial integrals (2D) and the face arrays share one region.
template <typename T, int DIM, int N, int S>
struct CutSmem {
  static constexpr int ND = Geo<DIM, N>::ND, NL = Geo<DIM, N>::NL, NF = Geo<DIM, N>::NF;
  static constexpr int CH = S;
  // at most GMAX groups per chunk: cut_gmax, and half the lanes for the 16- and 8-lane classes
  // (their cells have few groups; the smaller partial arrays raise residency)
  static constexpr int GMAX = cut_gmax<N>() < (S >= 32 ? S : S / 2) ? cut_gmax<N>() : (S >= 32 ? S : S / 2);
  static constexpr int cmax(int a, int b) { return a > b ? a : b; }
  static constexpr int u = 0;                    // [ND] the cell's DoFs
  static constexpr int acc = u + ND;             // [ND] accumulated output rows
  static constexpr int shared = acc + ND;        // region of size `region`:
  //   3D volume: P0, P1 = [GMAX][NL] per group (then Q0, Q1)
  //   2D volume: lt0, lt1 = [CH][NL] per line partial integrals
  //   faces:     tr = [FB][2][NL] trace jump and flux, ft = [FB][2][NL] face accumulators
  // cut faces per batch of the face phase: all of them, except at n = 9 in 3D, where batches of
  // three keep the face arrays as small as the volume phase's with GMAX 6 (FP64: 32.1 KB per
  // one-warp CTA, 7 CTAs per SM instead of 5 with all faces and GMAX 8)
  static constexpr int FB = (DIM == 3 && N >= 9) ? 3 : NF;
  static constexpr int region = cmax(cmax(2 * GMAX * NL, 2 * CH * NL * (DIM == 2 ? 1 : 0)), 4 * FB * NL);
  static constexpr int p0 = shared, p1 = shared + GMAX * NL;
  static constexpr int lt0 = shared, lt1 = shared + CH * NL;
  static constexpr int tr = shared, ft = shared + 2 * FB * NL;
  static constexpr int lvb = shared + region;    // [CH][N] per line basis (values)
  static constexpr int ldb = lvb + CH * N;       // [CH][N] (derivatives)
  static constexpr int zz = ldb + CH * N;        // [3][CH][N] per line point integrals
  static constexpr int gcv = zz + 3 * CH * N;    // [GMAX][N] per group shared-axis basis (3D)
  static constexpr int gcd = gcv + GMAX * N;
  static constexpr int total = gcd + GMAX * N;
  // ints after the T data: line tags (faces) [CH], group of each line [CH], first line of
  // each group [GMAX + 1], shared axis of each group [GMAX]
  static constexpr int itag = 0, ilgrp = CH, igline = 2 * CH, igax = 2 * CH + GMAX + 1;
  static constexpr size_t bytes = (size_t)total * sizeof(T) + (2 * CH + 2 * GMAX + 1) * sizeof(int);
  static constexpr size_t stride = (bytes + 15) / 16 * 16;  // per cell in the CTA
};

// Volume (Poisson) and surface (Nitsche) points of a 3D cut cell (Eq. unstructured_cell), in a
// two-level hierarchy of the dimension-reduction rule: a line holds the points that share both
// outer coordinates, and a group holds the lines that share one of them (the points of one
// line of the 2D outer rule).  Per chunk of CH lines (one thread per line):
//   A  (per group)  P0 = (phi_c x I x I) u, P1 = (phi_c' x I x I) u along the shared axis c;
//   B  (per line)   w0, w1, w2 = (phi_b | phi_b') contractions of P0 / P1 along the line's own
//                   outer axis b, then values and gradients at the line's points and the
//                   integration back along the line (z0, z1, z2);
//   C1 (per group)  Q0 = sum_lines phi_b z0 + phi_b' z1, Q1 = sum_lines phi_b z2;
//   C2 (per DoF)    acc += sum_groups phi_c Q0 + phi_c' Q1.
// Per line this costs 6 n^2 FMA and per group 4 n^3, against 4 n^3 + 6 n^2 per line when
// every line contracts both outer axes itself.
template <typename T, int N, int S>
__device__ __forceinline__ void cut_volume_3d(const PointTables<T, N> &pt, const DevArrays<T> &d,
                                              const Scalars<T> &sc, unsigned char *smem_raw, int ci,
                                              T kap, int tid, unsigned gmask, int gshift) {
  using G = Geo<3, N>;
  using SM = CutSmem<T, 3, N, S>;
  constexpr int ND = G::ND, NL = G::NL;
  constexpr int CH = SM::CH, GMAX = SM::GMAX;
  T *sm = reinterpret_cast<T *>(smem_raw);
  const T *s_u = sm + SM::u;
  T *s_acc = sm + SM::acc;
  T (*s_p0)[NL] = reinterpret_cast<T (*)[NL]>(sm + SM::p0);  // P0, then Q0
  T (*s_p1)[NL] = reinterpret_cast<T (*)[NL]>(sm + SM::p1);  // P1, then Q1
  T (*s_vb)[N] = reinterpret_cast<T (*)[N]>(sm + SM::lvb);
  T (*s_db)[N] = reinterpret_cast<T (*)[N]>(sm + SM::ldb);
  T (*s_z)[CH][N] = reinterpret_cast<T (*)[CH][N]>(sm + SM::zz);
  T (*s_gcv)[N] = reinterpret_cast<T (*)[N]>(sm + SM::gcv);
  T (*s_gcd)[N] = reinterpret_cast<T (*)[N]>(sm + SM::gcd);
  int *s_ints = reinterpret_cast<int *>(sm + SM::total);
  int *s_lgrp = s_ints + SM::ilgrp;
  int *s_gline = s_ints + SM::igline;
  int *s_gax = s_ints + SM::igax;

#pragma unroll 1
  for (int k = 0; k < 3; ++k) {
    const int lbeg = __ldg(d.vline_koff + ci * 4 + k);
    const int lend = __ldg(d.vline_koff + ci * 4 + k + 1);
    int ob, oc;
    other_axes(k, ob, oc);
    const int sk = stride_of<N>(k), sob = stride_of<N>(ob), soc = stride_of<N>(oc);
    int nl = 0;
#pragma unroll 1
    for (int l0 = lbeg; l0 < lend; l0 += nl) {
      const int line = l0 + tid;
      const bool in_range = tid < min(CH, lend - l0);
      const int gword = in_range ? __ldg(d.vline_grp + line) : 0;
      const int shared_lo = gword & 1;  // the group shares the coordinate along ob
      // groups of this chunk (a group cut by the chunk boundary restarts at its first thread);
      // the chunk ends before the start of group GMAX
      const bool start0 = in_range && (tid == 0 || (gword >> 1) == line);
      const unsigned starts0 = __ballot_sync(gmask, start0) >> gshift;  // bits of this group
      const int gl = __popc(starts0 & ((2u << tid) - 1u)) - 1;
      const unsigned over = __ballot_sync(gmask, start0 && gl >= GMAX) >> gshift;
      nl = over ? (__ffs(over) - 1) : min(CH, lend - l0);
      const bool act = tid < nl;
      const bool start = start0 && act;
      const int ng = __popc(starts0 & ((nl >= 32) ? 0xffffffffu : ((1u << nl) - 1u)));
      if (start) {
        s_gline[gl] = tid;
        s_gax[gl] = shared_lo;
        T cv[N], cd[N];
        if constexpr (kPrecomputedBasis<T>) {
          const T *bp = d.vline_b + (size_t)line * 4 * N + (shared_lo ? 0 : 2 * N);
#pragma unroll
          for (int i = 0; i < N; ++i) {
            cv[i] = __ldg(bp + i);
            cd[i] = __ldg(bp + N + i);
          }
        } else {
          basis_1d<T, N>(pt, __ldg((shared_lo ? d.vline_o0 : d.vline_o1) + line), cv, cd);
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
          s_gcv[gl][i] = cv[i];
          s_gcd[gl][i] = cd[i];
        }
      }
      if (tid == 0) s_gline[ng] = nl;
      if (act) s_lgrp[tid] = gl;
      __syncwarp(gmask);
      // A: contraction along the shared axis, per group; P[g][ib * N + m], ib along the
      // group's line axis, m along k
      for (int item = tid; item < ng * NL; item += CH) {
        const int g = item / NL, r = item % NL, ib = r / N, m = r % N;
        const int lo = s_gax[g];
        const int sb = lo ? soc : sob, scs = lo ? sob : soc;
        const T *up = s_u + ib * sb + m * sk;
        T p0 = T(0), p1 = T(0);
#pragma unroll
        for (int ic = 0; ic < N; ++ic) {
          const T v = up[ic * scs];
          p0 = fma(s_gcv[g][ic], v, p0);
          p1 = fma(s_gcd[g][ic], v, p1);
        }
        s_p0[g][r] = p0;
        s_p1[g][r] = p1;
      }
      __syncwarp(gmask);
      // B: one thread per line
      if (act) {
        const int ab = shared_lo ? oc : ob;  // the line's own outer axis
        const int ac = shared_lo ? ob : oc;  // the shared one
        T vb[N], db[N];
        if constexpr (kPrecomputedBasis<T>) {
          const T *bp = d.vline_b + (size_t)line * 4 * N + (shared_lo ? 2 * N : 0);
#pragma unroll
          for (int i = 0; i < N; ++i) {
            vb[i] = __ldg(bp + i);
            db[i] = __ldg(bp + N + i);
          }
        } else {
          basis_1d<T, N>(pt, __ldg((shared_lo ? d.vline_o1 : d.vline_o0) + line), vb, db);
        }
        // w0 = phi_b phi_c u, w1 = phi_b' phi_c u, w2 = phi_b phi_c' u along the line
        T w0[N], w1[N], w2[N];
#pragma unroll
        for (int m = 0; m < N; ++m) {
          T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
          for (int ib = 0; ib < N; ++ib) {
            const T q0 = s_p0[gl][ib * N + m];
            a0 = fma(vb[ib], q0, a0);
            a1 = fma(db[ib], q0, a1);
            a2 = fma(vb[ib], s_p1[gl][ib * N + m], a2);
          }
          w0[m] = a0;
          w1[m] = a1;
          w2[m] = a2;
        }
        // kappa int grad v . grad u over the line's volume points: with the line's integrals
        // K_l (derivatives along the line) and M_l (values), z0 = kappa K_l w0, z1 = kappa M_l w1,
        // z2 = kappa M_l w2 (both carry h^{-2}: a reference gradient has 1/h per factor)
        T z0[N], z1[N], z2[N];
        if constexpr (kLineIntegrals<T>) {
          line_products<T, N>(d.vline_km + (size_t)line * 2 * N * N, kap, w0, w1, w2, z0, z1, z2, true);
        } else {
#pragma unroll
          for (int m = 0; m < N; ++m) {
            z0[m] = T(0);
            z1[m] = T(0);
            z2[m] = T(0);
          }
          const int pb = __ldg(d.vpt_off + line), pe = __ldg(d.vpt_off + line + 1);
          const T cfv = kap * sc.inv_h2;
#pragma unroll 1
          for (int p = pb; p < pe; ++p) {
            T cv[N], cd[N];
            point_basis<T, N>(pt, d.vpt_b, d.vpt_t, p, cv, cd);
            T gk = T(0), gb = T(0), gc = T(0);
#pragma unroll
            for (int m = 0; m < N; ++m) {
              gk = fma(cd[m], w0[m], gk);
              gb = fma(cv[m], w1[m], gb);
              gc = fma(cv[m], w2[m], gc);
            }
            // kappa int grad v . grad u: reference gradients carry 1/h each
            const T cf = cfv * __ldg(d.vpt_w + p);
            gk *= cf;
            gb *= cf;
            gc *= cf;
#pragma unroll
            for (int m = 0; m < N; ++m) {
              z0[m] = fma(gk, cd[m], z0[m]);
              z1[m] = fma(gb, cv[m], z1[m]);
              z2[m] = fma(gc, cv[m], z2[m]);
            }
          }
        }
        const int sp = __ldg(d.lsurf + line);
        if (sp >= 0) {
          // kappa int_Gamma [ -d_n v u - v d_n u + tau/h v u ]
          T cv[N], cd[N];
          point_basis<T, N>(pt, d.spt_b, d.spt_t, sp, cv, cd);
          T u = T(0), gk = T(0), gb = T(0), gc = T(0);
#pragma unroll
          for (int m = 0; m < N; ++m) {
            u = fma(cv[m], w0[m], u);
            gk = fma(cd[m], w0[m], gk);
            gb = fma(cv[m], w1[m], gb);
            gc = fma(cv[m], w2[m], gc);
          }
          const T nk = __ldg(d.spt_n[k] + sp), nb = __ldg(d.spt_n[ab] + sp), nc = __ldg(d.spt_n[ac] + sp);
          const T wk = kap * __ldg(d.spt_w + sp);
          const T dn = (nk * gk + nb * gb + nc * gc) * sc.inv_h;
          const T cval = wk * (sc.nitsche_over_h * u - dn);
          const T cu = -wk * u * sc.inv_h;
#pragma unroll
          for (int m = 0; m < N; ++m) {
            z0[m] = fma(cval, cv[m], fma(cu * nk, cd[m], z0[m]));
            z1[m] = fma(cu * nb, cv[m], z1[m]);
            z2[m] = fma(cu * nc, cv[m], z2[m]);
          }
        }
#pragma unroll
        for (int m = 0; m < N; ++m) {
          s_z[0][tid][m] = z0[m];
          s_z[1][tid][m] = z1[m];
          s_z[2][tid][m] = z2[m];
          s_vb[tid][m] = vb[m];
          s_db[tid][m] = db[m];
        }
      }
      __syncwarp(gmask);
      // C1: sum over the lines of each group, Q[g][ib * N + m] (P is no longer read)
      for (int item = tid; item < ng * NL; item += CH) {
        const int g = item / NL, r = item % NL, ib = r / N, m = r % N;
        T q0 = T(0), q1 = T(0);
        for (int t = s_gline[g]; t < s_gline[g + 1]; ++t) {
          q0 = fma(s_vb[t][ib], s_z[0][t][m], fma(s_db[t][ib], s_z[1][t][m], q0));
          q1 = fma(s_vb[t][ib], s_z[2][t][m], q1);
        }
        s_p0[g][r] = q0;
        s_p1[g][r] = q1;
      }
      __syncwarp(gmask);
      // C2: expansion along the shared axis into the cell's rows
      for (int l = tid; l < ND; l += CH) {
        const int im = (l / sk) % N, iob = (l / sob) % N, ioc = (l / soc) % N;
        T acc = T(0);
        for (int g = 0; g < ng; ++g) {
          const int lo = s_gax[g];
          const int ib = lo ? ioc : iob, ic = lo ? iob : ioc;
          acc = fma(s_gcv[g][ic], s_p0[g][ib * N + im], fma(s_gcd[g][ic], s_p1[g][ib * N + im], acc));
        }
        s_acc[l] += acc;
      }
      __syncwarp(gmask);
    }
  }
}

// The cut cells of one lane class handled by CTA `block` of that class (one warp; 32 / S cells).
template <typename T, int DIM, int N, int S>
__device__ __forceinline__ void cut_cells(const PointTables<T, N> &pt, const DevArrays<T> &d,
                                          const Scalars<T> &sc, T *__restrict__ y,
                                          const T *__restrict__ x, int slot_begin, int slot_end,
                                          int block) {
  using G = Geo<DIM, N>;
  using SM = CutSmem<T, DIM, N, S>;
  constexpr int ND = G::ND, NL = G::NL, NF = G::NF;
  constexpr int CH = SM::CH;
  constexpr int CPW = 32 / S;  // cut cells per CTA

  // lane group of this thread: lanes [gshift, gshift + S) work on one cut cell
  const int grp = threadIdx.x / S;
  const int gshift = grp * S;
  const unsigned gmask = (S == 32) ? 0xffffffffu : (((1u << S) - 1u) << gshift);
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char *smem_raw = smem_all + grp * SM::stride;
  T *sm = reinterpret_cast<T *>(smem_raw);
  T *s_u = sm + SM::u;
  T *s_acc = sm + SM::acc;
  T (*s_lt0)[NL] = reinterpret_cast<T (*)[NL]>(sm + SM::lt0);
  T (*s_lt1)[NL] = reinterpret_cast<T (*)[NL]>(sm + SM::lt1);
  T (*s_lvb)[N] = reinterpret_cast<T (*)[N]>(sm + SM::lvb);
  T (*s_ldb)[N] = reinterpret_cast<T (*)[N]>(sm + SM::ldb);
  T (*s_tr)[2][NL] = reinterpret_cast<T (*)[2][NL]>(sm + SM::tr);
  T (*s_ft)[2][NL] = reinterpret_cast<T (*)[2][NL]>(sm + SM::ft);
  T (*s_fz)[CH][N] = reinterpret_cast<T (*)[CH][N]>(sm + SM::zz);  // face lines: zv, zd
  int *s_tag = reinterpret_cast<int *>(sm + SM::total) + SM::itag;

  const int tid = threadIdx.x - gshift;
  const int slot = slot_begin + block * CPW + grp;  // cut_list range of this lane class
  if (slot >= slot_end) return;  // a whole lane group leaves together
  const int e = __ldg(d.cut_list + slot);
  const int ci = __ldg(d.cut_idx + slot);
  const T kap = __ldg(d.kappa + e);
  const uint32_t fl = __ldg(d.flags + e);

  for (int i = tid; i < ND; i += CH) {
    s_u[i] = __ldg(x + (size_t)e * ND + i);
    s_acc[i] = T(0);
  }
  __syncwarp(gmask);

  if constexpr (DIM == 3) {
    cut_volume_3d<T, N, S>(pt, d, sc, smem_raw, ci, kap, tid, gmask, gshift);
  } else {
    // ---- volume (Poisson) and surface (Nitsche) points, line by line (Eq. unstructured_cell:
    // the contractions along the two outer axes are shared by every point of a line)
  #pragma unroll 1
    for (int k = 0; k < DIM; ++k) {
      const int lbeg = __ldg(d.vline_koff + ci * 4 + k);
      const int lend = __ldg(d.vline_koff + ci * 4 + k + 1);
      int ob = 0, oc = 0;
      if constexpr (DIM == 3) {
        other_axes(k, ob, oc);
      } else {
        ob = 1 - k;
      }
      const int sk = stride_of<N>(k), sb = stride_of<N>(ob), scc = stride_of<N>(oc);
  #pragma unroll 1
      for (int l0 = lbeg; l0 < lend; l0 += CH) {
        const int line = l0 + tid;
        if (line < lend) {
          T vb[N], db[N], vc[N], dc[N];
          if constexpr (kPrecomputedBasis<T>) {
            const T *bp = d.vline_b + (size_t)line * 4 * N;
  #pragma unroll
            for (int i = 0; i < N; ++i) {
              vb[i] = __ldg(bp + i);
              db[i] = __ldg(bp + N + i);
              if constexpr (DIM == 3) {
                vc[i] = __ldg(bp + 2 * N + i);
                dc[i] = __ldg(bp + 3 * N + i);
              }
            }
          } else {
            basis_1d<T, N>(pt, __ldg(d.vline_o0 + line), vb, db);
            if constexpr (DIM == 3) basis_1d<T, N>(pt, __ldg(d.vline_o1 + line), vc, dc);
          }
          // w0 = (phi_b phi_c) u, w1 = (phi_b' phi_c) u, w2 = (phi_b phi_c') u along the line
          T w0[N], w1[N], w2[N];
  #pragma unroll
          for (int m = 0; m < N; ++m) {
            w0[m] = T(0);
            w1[m] = T(0);
            w2[m] = T(0);
          }
          constexpr int NC = (DIM == 3) ? N : 1;
  #pragma unroll
          for (int m = 0; m < N; ++m) {
  #pragma unroll
            for (int ic = 0; ic < NC; ++ic) {
              T s0 = T(0), s1 = T(0);
  #pragma unroll
              for (int ib = 0; ib < N; ++ib) {
                const T v = s_u[ib * sb + ic * scc + m * sk];
                s0 = fma(vb[ib], v, s0);
                s1 = fma(db[ib], v, s1);
              }
              if constexpr (DIM == 3) {
                w0[m] = fma(vc[ic], s0, w0[m]);
                w1[m] = fma(vc[ic], s1, w1[m]);
                w2[m] = fma(dc[ic], s0, w2[m]);
              } else {
                w0[m] = s0;
                w1[m] = s1;
              }
            }
          }
          // volume points of the line through its integrals K_l, M_l (see cut_volume_3d)
          T z0[N], z1[N], z2[N];
          if constexpr (kLineIntegrals<T>) {
            line_products<T, N>(d.vline_km + (size_t)line * 2 * N * N, kap, w0, w1, w2, z0, z1, z2,
                                DIM == 3);
          } else {
            point_integrals<T, N>(pt, d, kap * sc.inv_h2, line, w0, w1, w2, z0, z1, z2, DIM == 3);
          }
          const int sp = __ldg(d.lsurf + line);
          if (sp >= 0) {
            // kappa int_Gamma [ -d_n v u - v d_n u + tau/h v u ]
            T cv[N], cd[N];
            point_basis<T, N>(pt, d.spt_b, d.spt_t, sp, cv, cd);
            T u = T(0), gk = T(0), gb = T(0), gc = T(0);
  #pragma unroll
            for (int m = 0; m < N; ++m) {
              u = fma(cv[m], w0[m], u);
              gk = fma(cd[m], w0[m], gk);
              gb = fma(cv[m], w1[m], gb);
              if constexpr (DIM == 3) gc = fma(cv[m], w2[m], gc);
            }
            const T nk = __ldg(d.spt_n[k] + sp), nb = __ldg(d.spt_n[ob] + sp);
            const T nc = (DIM == 3) ? __ldg(d.spt_n[oc] + sp) : T(0);
            const T wk = kap * __ldg(d.spt_w + sp);
            const T dn = (nk * gk + nb * gb + nc * gc) * sc.inv_h;
            const T cval = wk * (sc.nitsche_over_h * u - dn);
            const T cu = -wk * u * sc.inv_h;
  #pragma unroll
            for (int m = 0; m < N; ++m) {
              z0[m] = fma(cval, cv[m], fma(cu * nk, cd[m], z0[m]));
              z1[m] = fma(cu * nb, cv[m], z1[m]);
              if constexpr (DIM == 3) z2[m] = fma(cu * nc, cv[m], z2[m]);
            }
          }
          // partial integration along the upper other axis; the lower one is done by the DoFs
  #pragma unroll
          for (int ic = 0; ic < NC; ++ic)
  #pragma unroll
            for (int m = 0; m < N; ++m) {
              if constexpr (DIM == 3) {
                s_lt0[tid][ic * N + m] = fma(vc[ic], z0[m], dc[ic] * z2[m]);
                s_lt1[tid][ic * N + m] = vc[ic] * z1[m];
              } else {
                s_lt0[tid][m] = z0[m];
                s_lt1[tid][m] = z1[m];
              }
            }
  #pragma unroll
          for (int ib = 0; ib < N; ++ib) {
            s_lvb[tid][ib] = vb[ib];
            s_ldb[tid][ib] = db[ib];
          }
        }
        __syncwarp(gmask);
        const int nlines = min(CH, lend - l0);
        for (int l = tid; l < ND; l += CH) {
          const int ib = (l / sb) % N, m = (l / sk) % N;
          const int col = (DIM == 3) ? (((l / scc) % N) * N + m) : m;
          T acc = T(0);
          for (int q = 0; q < nlines; ++q)
            acc = fma(s_lvb[q][ib], s_lt0[q][col], fma(s_ldb[q][ib], s_lt1[q][col], acc));
          s_acc[l] += acc;
        }
        __syncwarp(gmask);
      }
    }
  }

  // ---- SIPG on cut faces: F cap Omega, in-face lines (Eq. unstructured_face).  The cut faces
  // of the cell are processed together (in batches of SM::FB faces, the size of the face
  // arrays) so that the warp's lanes stay busy.
  int cfl[NF];
  int ncf = 0;
#pragma unroll
  for (int f = 0; f < NF; ++f)
    if (bit(fl, bit_cut(f))) cfl[ncf++] = f;
  const int *koff_cell = d.fline_koff + (size_t)ci * NF * 3;
  // the cut faces cfl[b0 .. b0 + nbf) (ascending face index: their lines are contiguous)
  auto face_batch = [&](const int b0, const int nbf) {
    // per cut face, indexed by the in-face DoF tl = i_b' + n i_c' (b' < c' in-face axes): the
    // jump of the traces [u] = u_K - u_nb (the trace of a Lobatto basis is its face-node value)
    // and the average normal flux {kappa d_n u} along the own outward normal; the neighbour's
    // lines are read from global memory (L2)
    for (int item = tid; item < nbf * NL; item += CH) {
      const int fi = item / NL, tl = item % NL;
      const int f = cfl[b0 + fi], axis = f / 2, side = f % 2;
      const int nbe = __ldg(d.nbr + (size_t)e * NF + f);
      const T knb = __ldg(d.kappa + nbe);
      const int base = line_base<DIM, N>(axis, tl);
      const int st = stride_of<N>(axis);
      const T *xn = x + (size_t)nbe * ND + base;
      const int end_own = side ? N - 1 : 0, end_nb = side ? 0 : N - 1;
      T od = T(0), nd = T(0);
#pragma unroll
      for (int m = 0; m < N; ++m) {
        od = fma(pt.end_der[side][m], s_u[base + m * st], od);
        nd = fma(pt.end_der[1 - side][m], __ldg(xn + m * st), nd);
      }
      const T sgn = side ? T(1) : T(-1);
      s_tr[fi][0][tl] = s_u[base + end_own * st] - __ldg(xn + end_nb * st);
      s_tr[fi][1][tl] = (T(0.5) * sgn * sc.inv_h) * fma(kap, od, knb * nd);
      s_ft[fi][0][tl] = T(0);
      s_ft[fi][1][tl] = T(0);
    }
    __syncwarp(gmask);
    if constexpr (kFaceMatrices<T, DIM, N>) {
      // with the face's mass matrix Mf: ft0 = sigma/h {kappa} Mf [u] - Mf {kappa d_n u} and
      // ft1 = -kappa/2 Mf [u] (Mf is symmetric: lanes read its columns, consecutive rows)
      for (int item = tid; item < nbf * NL; item += CH) {
        const int fi = item / NL, row = item % NL;
        const int f = cfl[b0 + fi];
        const T knb = __ldg(d.kappa + __ldg(d.nbr + (size_t)e * NF + f));
        const T *mf = d.fmat + (size_t)__ldg(d.fmat_idx + (size_t)ci * NF + f) * NL * NL + row;
        T a = T(0), b = T(0);
#pragma unroll
        for (int col = 0; col < NL; ++col) {
          const T m = __ldg(mf + col * NL);
          a = fma(m, s_tr[fi][0][col], a);
          b = fma(m, s_tr[fi][1][col], b);
        }
        s_ft[fi][0][row] = fma(sc.sipg_over_h * (T(0.5) * (kap + knb)), a, -b);
        s_ft[fi][1][row] = T(-0.5) * kap * a;
      }
      __syncwarp(gmask);
    } else {
      const int fl_beg = (SM::FB >= NF) ? __ldg(koff_cell) : __ldg(koff_cell + cfl[b0] * 3);
      const int fl_end = (SM::FB >= NF) ? __ldg(koff_cell + (NF - 1) * 3 + 2)
                                        : __ldg(koff_cell + cfl[b0 + nbf - 1] * 3 + 2);
#pragma unroll 1
      for (int l0 = fl_beg; l0 < fl_end; l0 += CH) {
        const int line = l0 + tid;
        int tag = -1;
        if (line < fl_end) {
          int fi = 0, kk = 0;
          for (int j = 0; j < nbf; ++j) {
            const int *ko = koff_cell + cfl[b0 + j] * 3;
            if (line >= __ldg(ko) && line < __ldg(ko + 2)) {
              fi = j;
              kk = (line < __ldg(ko + 1)) ? 0 : 1;
            }
          }
          tag = 2 * fi + kk;
          const int f = cfl[b0 + fi];
          const int nbe = __ldg(d.nbr + (size_t)e * NF + f);
          const T knb = __ldg(d.kappa + nbe);
          const T kavg = T(0.5) * (kap + knb);
          // in-face strides of the line axis and of the outer axis in tl = i_b' + n i_c'
          const int s_line = (kk == 0) ? 1 : N, s_out = (kk == 0) ? N : 1;
          T vo[N];
          if constexpr (DIM == 3) {
            if constexpr (kPrecomputedBasis<T>) {
#pragma unroll
              for (int i = 0; i < N; ++i) vo[i] = __ldg(d.fline_b + (size_t)line * N + i);
            } else {
              basis_1d_val<T, N>(pt, __ldg(d.fline_o + line), vo);
            }
          }
          // jump and flux contracted along the outer in-face axis
          T r[2][N];
#pragma unroll
          for (int m = 0; m < N; ++m) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              if constexpr (DIM == 3) {
                T acc = T(0);
#pragma unroll
                for (int io = 0; io < N; ++io) acc = fma(vo[io], s_tr[fi][q][io * s_out + m * s_line], acc);
                r[q][m] = acc;
              } else {
                r[q][m] = s_tr[fi][q][m];
              }
            }
          }
          T zv[N], zd[N];
#pragma unroll
          for (int m = 0; m < N; ++m) {
            zv[m] = T(0);
            zd[m] = T(0);
          }
          const int pb = __ldg(d.fpt_off + line), pe = __ldg(d.fpt_off + line + 1);
#pragma unroll 1
          for (int p = pb; p < pe; ++p) {
            T cv[N];
            if constexpr (kPrecomputedBasis<T>) {
#pragma unroll
              for (int i = 0; i < N; ++i) cv[i] = __ldg(d.fpt_b + (size_t)p * N + i);
            } else {
              basis_1d_val<T, N>(pt, __ldg(d.fpt_t + p), cv);
            }
            T jump = T(0), avg = T(0);
#pragma unroll
            for (int m = 0; m < N; ++m) {
              jump = fma(cv[m], r[0][m], jump);
              avg = fma(cv[m], r[1][m], avg);
            }
            const T w = __ldg(d.fpt_w + p);
            // coefficients of the own trace value and own normal derivative of the test function
            const T cvv = w * (sc.sipg_over_h * kavg * jump - avg);
            const T cdd = w * (T(-0.5) * kap * jump);
#pragma unroll
            for (int m = 0; m < N; ++m) {
              zv[m] = fma(cvv, cv[m], zv[m]);
              zd[m] = fma(cdd, cv[m], zd[m]);
            }
          }
#pragma unroll
          for (int m = 0; m < N; ++m) {
            s_fz[0][tid][m] = zv[m];
            s_fz[1][tid][m] = zd[m];
            s_lvb[tid][m] = (DIM == 3) ? vo[m] : T(1);
          }
        }
        s_tag[tid] = tag;
        __syncwarp(gmask);
        const int nlines = min(CH, fl_end - l0);
        for (int item = tid; item < nbf * NL; item += CH) {
          const int fi = item / NL, tl = item % NL;
          T av = T(0), ad = T(0);
          for (int q = 0; q < nlines; ++q) {
            const int tg = s_tag[q];
            if ((tg >> 1) != fi) continue;
            const int kk = tg & 1;
            int m, io;
            if constexpr (DIM == 3) {
              m = (kk == 0) ? (tl % N) : (tl / N);
              io = (kk == 0) ? (tl / N) : (tl % N);
            } else {
              m = tl;
              io = 0;
            }
            av = fma(s_lvb[q][io], s_fz[0][q][m], av);
            ad = fma(s_lvb[q][io], s_fz[1][q][m], ad);
          }
          s_ft[fi][0][tl] += av;
          s_ft[fi][1][tl] += ad;
        }
        __syncwarp(gmask);
      }
    }
    // expand the face accumulators into the cell: phi_l = phi_{i_a}(side) x in-face product
    for (int l = tid; l < ND; l += CH) {
      T add = T(0);
      for (int fi = 0; fi < nbf; ++fi) {
        const int f = cfl[b0 + fi], axis = f / 2, side = f % 2;
        const T sgn = side ? T(1) : T(-1);
        const int ia = (l / stride_of<N>(axis)) % N;
        int tl;
        if constexpr (DIM == 2) {
          tl = (axis == 0) ? l / N : l % N;
        } else {
          const int i0 = l % N, i1 = (l / N) % N, i2 = l / (N * N);
          tl = (axis == 0) ? (i1 + N * i2) : (axis == 1) ? (i0 + N * i2) : (i0 + N * i1);
        }
        add = fma(sgn * sc.inv_h * pt.end_der[side][ia], s_ft[fi][1][tl], add);
        if (ia == (side ? N - 1 : 0)) add += s_ft[fi][0][tl];
      }
      s_acc[l] += add;
    }
  };
  if constexpr (SM::FB >= NF) {
    if (ncf > 0) face_batch(0, ncf);
  } else {
#pragma unroll 1
    for (int b0 = 0; b0 < ncf; b0 += SM::FB) {
      face_batch(b0, min(SM::FB, ncf - b0));
      __syncwarp(gmask);  // the next batch overwrites the face arrays that this one read
    }
  }

  for (int i = tid; i < ND; i += CH) y[(size_t)e * ND + i] += s_acc[i];
}

// Cut cells of the lane classes in CLS (bit 0: 32 lanes, bit 1: 16, bit 2: 8) in one launch: the
// first CTAs take the 32-lane class (one cell each, most expensive first), then the 16-lane class
// (two cells per CTA), then the 8-lane class (four).  FP64 launches all classes together, so
// that they fill each other's tails instead of ending in partial waves (the 64^3 Q3 ball: 0.377
// -> 0.356 ms); FP32, whose kernel is latency-bound, keeps one launch per class (a kernel holding
// every class's code measured 17 % slower there), and so do the parts of the host-buffer
// pipeline, whose launches overlap on several streams (merged: end-to-end 8.92 -> 8.62 GDoF/s).
template <typename T, int DIM, int N, int CLS>
__global__ void __launch_bounds__(32) cut_kernel(const __grid_constant__ PointTables<T, N> pt,
                                                 const DevArrays<T> d, const Scalars<T> sc,
                                                 T *__restrict__ y, const T *__restrict__ x,
                                                 int s0, int s1, int s2, int s3) {
  int b = blockIdx.x;
  if constexpr ((CLS & 1) != 0) {
    const int b32 = s1 - s0;
    if (b < b32) {
      cut_cells<T, DIM, N, 32>(pt, d, sc, y, x, s0, s1, b);
      return;
    }
    b -= b32;
  }
  if constexpr (N <= 5 && (CLS & 2) != 0) {
    const int b16 = (s2 - s1 + 1) / 2;
    if (b < b16) {
      cut_cells<T, DIM, N, 16>(pt, d, sc, y, x, s1, s2, b);
      return;
    }
    b -= b16;
  }
  if constexpr (N <= 5 && (CLS & 4) != 0) cut_cells<T, DIM, N, 8>(pt, d, sc, y, x, s2, s3, b);
}

// Dynamic shared memory of a launch of the classes in CLS: the largest need among its non-empty
// classes (sp: the slot bounds of the 32-, 16- and 8-lane classes).
template <typename T, int DIM, int N, int CLS>
size_t cut_smem_bytes(const int *sp) {
  size_t m = ((CLS & 1) && sp[1] > sp[0]) ? CutSmem<T, DIM, N, 32>::stride : 0;
  if constexpr (N <= 5) {
    const size_t m16 = ((CLS & 2) && sp[2] > sp[1]) ? 2 * CutSmem<T, DIM, N, 16>::stride : 0;
    const size_t m8 = ((CLS & 4) && sp[3] > sp[2]) ? 4 * CutSmem<T, DIM, N, 8>::stride : 0;
    m = m16 > m ? m16 : m;
    m = m8 > m ? m8 : m;
  }
  return m;
}

// ------------------------------------------------------------------------------------------
// Launch
// ------------------------------------------------------------------------------------------
template <typename T, int DIM, int N, int CLS>
int launch_cut_classes(const PointTables<T, N> &ptab, const DevArrays<T> &d, const Scalars<T> &s,
                       T *y, const T *x, cudaStream_t stream, const int *sp) {
  int blocks = 0;
  if (CLS & 1) blocks += sp[1] - sp[0];
  if (N <= 5 && (CLS & 2)) blocks += (sp[2] - sp[1] + 1) / 2;
  if (N <= 5 && (CLS & 4)) blocks += (sp[3] - sp[2] + 3) / 4;
  if (blocks <= 0) return 0;
  const size_t smem = cut_smem_bytes<T, DIM, N, CLS>(sp);
  if (smem > 48 * 1024) {
    const cudaError_t err = cudaFuncSetAttribute(cut_kernel<T, DIM, N, CLS>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
  }
  cut_kernel<T, DIM, N, CLS><<<blocks, 32, smem, stream>>>(ptab, d, s, y, x, sp[0], sp[1], sp[2], sp[3]);
  return (int)cudaGetLastError();
}

// merged: all lane classes in one launch (FP64 products of the whole operator; the parts of the
// host-buffer pipeline, which run on several streams at once, keep one launch per class)
template <typename T, int DIM, int N>
int launch_cut(const PointTables<T, N> &ptab, const DevArrays<T> &d, const Scalars<T> &s, T *y,
               const T *x, cudaStream_t stream, const int *sp, bool merged) {
  if (merged) {
    return launch_cut_classes<T, DIM, N, 7>(ptab, d, s, y, x, stream, sp);
  } else {
    int e = launch_cut_classes<T, DIM, N, 1>(ptab, d, s, y, x, stream, sp);
    if (e == 0) e = launch_cut_classes<T, DIM, N, 2>(ptab, d, s, y, x, stream, sp);
    if (e == 0) e = launch_cut_classes<T, DIM, N, 4>(ptab, d, s, y, x, stream, sp);
    return e;
  }
}

// Dynamic shared memory of a structured-kernel launch (struct_dynamic_smem: u, W per axis and,
// for non-uniform kappa, the per-cell matrices of CPB cells), with the kernel's limit raised to
// it; 0 for the instances with static arrays.
template <typename T, int DIM, int N, bool UNI, typename K>
size_t struct_smem_setup(K kernel) {
  if constexpr (!struct_dynamic_smem<T, DIM, N>()) {
    (void)kernel;
    return 0;
  } else {
    constexpr int CPB = struct_cells_per_block<T, DIM, N>(), SND = snd<DIM, N>();
    constexpr size_t bytes = sizeof(T) * CPB * (SND * (1 + DIM) + (UNI ? 0 : DIM * 3 * N * N));
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return bytes;
  }
}

template <typename T, int DIM, int N>
int launch_vmult_t(const DevArrays<T> &d0, const void *tables_struct, const void *tables_point,
                   const Scalars<T> &s, T *y, const T *x, bool adjoint, cudaStream_t stream,
                   void *const *ev, const LaunchRange *rg) {
  using G = Geo<DIM, N>;
  constexpr int CPB = struct_cells_per_block<T, DIM, N>();
  // whole operator, or one part of it (its cells and its cut-cell slots in the part's own list)
  DevArrays<T> d = d0;
  int cb = 0, ce = d.n_active;
  int sp[4] = {0, d.cut_split[0], d.cut_split[1], d.n_cut};
  if (rg) {
    cb = rg->cell_begin;
    ce = rg->cell_end;
    d.cut_list = rg->cut_list;
    d.cut_idx = rg->cut_idx;
    for (int i = 0; i < 4; ++i) sp[i] = rg->split[i];
  }
  const int threads = ((CPB * G::NL + 31) / 32) * 32;
  const int blocks = (ce - cb + CPB - 1) / CPB;
  const auto &tab = *reinterpret_cast<const StructTables<T, N> *>(tables_struct);
  if (ev) cudaEventRecord(static_cast<cudaEvent_t>(ev[0]), stream);
  bool planes = false;  // FP32, 3D, n <= 5, uniform kappa: one thread per z-plane of a cell
  if constexpr (std::is_same<T, float>::value && DIM == 3 && N <= 5)
    planes = d.kappa_uniform != 0 && !(rg && rg->cells) &&
             (N != 4 || ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) % 16 == 0));
  if (rg && rg->cells) {
    // a list of cells (FP64, y = A x rows of those cells)
    if constexpr (sizeof(T) == sizeof(double)) {
      if (blocks > 0) {
        if (d.kappa_uniform != 0)
          struct_kernel<T, DIM, N, false, true, true>
              <<<blocks, threads, struct_smem_setup<T, DIM, N, true>(struct_kernel<T, DIM, N, false, true, true>),
                 stream>>>(tab, d, s, y, x, cb, ce, rg->cells);
        else
          struct_kernel<T, DIM, N, false, false, true>
              <<<blocks, threads, struct_smem_setup<T, DIM, N, false>(struct_kernel<T, DIM, N, false, false, true>),
                 stream>>>(tab, d, s, y, x, cb, ce, rg->cells);
      }
    } else {
      return (int)cudaErrorInvalidValue;
    }
  } else if (planes) {
    if constexpr (std::is_same<T, float>::value && DIM == 3 && N <= 5)
      launch_struct_planes<N>(tab, d, s, y, x, adjoint, stream, cb, ce);
  } else if (blocks > 0) {
    const bool uni = d.kappa_uniform != 0;
    if (adjoint && uni)
      struct_kernel<T, DIM, N, true, true>
          <<<blocks, threads, struct_smem_setup<T, DIM, N, true>(struct_kernel<T, DIM, N, true, true>), stream>>>(
              tab, d, s, y, x, cb, ce, nullptr);
    else if (adjoint)
      struct_kernel<T, DIM, N, true, false>
          <<<blocks, threads, struct_smem_setup<T, DIM, N, false>(struct_kernel<T, DIM, N, true, false>), stream>>>(
              tab, d, s, y, x, cb, ce, nullptr);
    else if (uni)
      struct_kernel<T, DIM, N, false, true>
          <<<blocks, threads, struct_smem_setup<T, DIM, N, true>(struct_kernel<T, DIM, N, false, true>), stream>>>(
              tab, d, s, y, x, cb, ce, nullptr);
    else
      struct_kernel<T, DIM, N, false, false>
          <<<blocks, threads, struct_smem_setup<T, DIM, N, false>(struct_kernel<T, DIM, N, false, false>), stream>>>(
              tab, d, s, y, x, cb, ce, nullptr);
  }
  if (ev) cudaEventRecord(static_cast<cudaEvent_t>(ev[1]), stream);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return (int)err;
  if (ev) cudaEventRecord(static_cast<cudaEvent_t>(ev[2]), stream);
  if (sp[3] > sp[0]) {
    const auto &ptab = *reinterpret_cast<const PointTables<T, N> *>(tables_point);
    // the three lane classes are contiguous in cut_list (32, 16, 8 lanes per cell)
    const bool merged = sizeof(T) == sizeof(double) && (!rg || rg->cells);
    const int e2 = launch_cut<T, DIM, N>(ptab, d, s, y, x, stream, sp, merged);
    if (e2 != 0) return e2;
  }
  if (ev) cudaEventRecord(static_cast<cudaEvent_t>(ev[3]), stream);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_vmult_impl(int dim, int n, const DevArrays<T> &d, const void *ts, const void *tp,
                      const Scalars<T> &s, T *y, const T *x, bool adjoint, cudaStream_t st,
                      void *const *ev, const LaunchRange *rg) {
#define UF_CASE(D, NN)                                                         \
  if (dim == D && n == NN) return launch_vmult_t<T, D, NN>(d, ts, tp, s, y, x, adjoint, st, ev, rg);
  UF_CASE(2, 2) UF_CASE(2, 3) UF_CASE(2, 4) UF_CASE(2, 5) UF_CASE(2, 6) UF_CASE(2, 7)
  UF_CASE(2, 8) UF_CASE(2, 9) UF_CASE(3, 2) UF_CASE(3, 3) UF_CASE(3, 4) UF_CASE(3, 5)
  UF_CASE(3, 6) UF_CASE(3, 7) UF_CASE(3, 8) UF_CASE(3, 9)
#undef UF_CASE
  return (int)cudaErrorInvalidValue;
}

}  // namespace uf
