// FP32 structured kernel with one thread per z-plane of a cell (3D, n <= 5, uniform kappa).
//
// The structured terms of a Cartesian cell are Kronecker products of 1D matrices (arXiv
// 2404.07911, Sec. 3.2, Eq. sum_factorization_cell / Eq. sum_factorization_face):
//     y = M_z (M_y W_x + M_x W_y) + M_x M_y W_z,   W_a = L_a u + neighbour couplings along a,
// with L_a the kappa = 1 line matrices of the cell's face configuration (no M^{-1}: FP32 keeps the
// unpremultiplied form, whose rounding errors are not amplified by M^{-1}).
//
// A cell is handled by n threads of one warp.  Thread t first owns the z-plane k = t of the cell
// (its n^2 DoFs in registers): the x- and y-lines of a plane lie in it, so W_x, W_y and
// P = M_y W_x + M_x W_y need no data from other threads.  The planes of P are exchanged through
// shared memory once for the sweep along z.  Thread t then owns the row j = t of every plane: the
// z-lines (i, t, :) lie in it, so W_z and M_x W_z are local again, and one exchange of rows
// gives M_y.  Each thread finally holds the output plane t.
//
// Memory: the CTA's own cells are one contiguous block of x, loaded with coalesced 16-byte reads
// into a padded shared layout (cell stride n^3 + 4 words for n = 4: the 16-byte reads of plane t
// or row t by the 8 cells of a warp fall into distinct bank groups); x-neighbours inside the block
// come from there, other neighbours from global memory (L2) as whole planes (x-, y-faces) or rows
// (z-faces).  Compared with one thread per line and shared-memory transposes for every sweep, the
// cell's data crosses shared memory twice instead of about ten times.
#pragma once

#include "uf_device.h"

namespace uf {

template <int N>
struct PlaneCfg {
  static constexpr int NN = N * N, ND = N * N * N;
  static constexpr int CPW = 32 / N;      // cells per warp (a cell never straddles two warps)
  static constexpr int CPB = 4 * CPW;     // cells per CTA (4 warps)
  static constexpr int THREADS = 128;
  static constexpr int SC = (N == 4) ? ND + 4 : ND + 1;  // padded cell stride in shared memory
  // registers capped for 6 CTAs (24 warps) per SM: the kernel waits on neighbour reads from L2,
  // and 24 warps hide them better than 20 with the uncapped 96 registers (n = 4: 36 us against
  // 39 us on the 64^3 Q3 workload; an asynchronous prefetch of the neighbour data into shared
  // memory, which cuts residency to 4 CTAs, took 54 us)
  static constexpr int MINB = 6;
};

// n consecutive floats at p: one 16-byte access for n = 4 (every such p in the kernel is a multiple
// of 4 floats past a 16-byte aligned base: shared arrays, and x / y, which the host checks), scalar
// accesses otherwise.
template <int N>
__device__ __forceinline__ void ld_run(const float *p, float *o) {
  if constexpr (N == 4) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
  } else {
#pragma unroll
    for (int m = 0; m < N; ++m) o[m] = p[m];
  }
}
template <int N>
__device__ __forceinline__ void ldg_run(const float *p, float *o) {
  if constexpr (N == 4) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
  } else {
#pragma unroll
    for (int m = 0; m < N; ++m) o[m] = __ldg(p + m);
  }
}
template <int N>
__device__ __forceinline__ void st_run(float *p, const float *v) {
  if constexpr (N == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int m = 0; m < N; ++m) p[m] = v[m];
  }
}

// Line-matrix selector of axis a: inside | full_lo << 1 | gp_lo << 2 | full_hi << 3 | gp_hi << 4.
__device__ __forceinline__ int plane_vsel(uint32_t fl, bool inside, int a) {
  int v = inside ? 1 : 0;
  v |= (fl & (1u << (1 + 3 * (2 * a)))) ? 2 : 0;
  v |= (fl & (1u << (3 + 3 * (2 * a)))) ? 4 : 0;
  v |= (fl & (1u << (1 + 3 * (2 * a + 1)))) ? 8 : 0;
  v |= (fl & (1u << (3 + 3 * (2 * a + 1)))) ? 16 : 0;
  return v;
}

// w += coupling of one line to its neighbour line un across the face on side s (ghost penalty:
// the full 1D matrix G; SIPG only: rank 2 through the neighbour's face value and derivative).
template <int N>
__device__ __forceinline__ void plane_couple(const StructTables<float, N> &tab, float hf_sigma,
                                             bool gp, const float *G, int s, const float *un,
                                             float *w) {
  if (gp) {
#pragma unroll
    for (int r = 0; r < N; ++r) {
      float acc = w[r];
#pragma unroll
      for (int m = 0; m < N; ++m) acc = fmaf(G[r * N + m], un[m], acc);
      w[r] = acc;
    }
  } else {
    const float alpha = un[s ? 0 : N - 1];
    float beta = 0.f;
#pragma unroll
    for (int m = 0; m < N; ++m) beta = fmaf(tab.dnb[s][m], un[m], beta);
#pragma unroll
    for (int r = 0; r < N; ++r) w[r] = fmaf(alpha, tab.dowx[s][r], w[r]);
    w[s ? N - 1 : 0] -= fmaf(hf_sigma, alpha, beta);
  }
}

template <int N, bool ADJ>
__global__ void __launch_bounds__(PlaneCfg<N>::THREADS, PlaneCfg<N>::MINB) struct_plane_kernel(
    const __grid_constant__ StructTables<float, N> tab, const DevArrays<float> d,
    const Scalars<float> sc, float *__restrict__ y, const float *__restrict__ x, int cell_begin,
    int cell_end) {
  using C = PlaneCfg<N>;
  constexpr int NN = C::NN, ND = C::ND, CPW = C::CPW, CPB = C::CPB, SC = C::SC;
  __shared__ __align__(16) float s_self[32 * NN];  // line matrices by face configuration
  __shared__ __align__(16) float s_gp[4 * NN];     // ghost-penalty neighbour couplings
  __shared__ __align__(16) float s_u[CPB * SC];    // the CTA's own cells
  __shared__ __align__(16) float s_x[CPB * SC];    // plane / row exchange

  const int tid = threadIdx.x;
  const int first = cell_begin + blockIdx.x * CPB;
  const int ncell = min(CPB, cell_end - first);
  {
    const float *selfsrc = ADJ ? d.lselfxT : d.lselfx;
    const float *gpsrc = ADJ ? d.lnbgpxT : d.lnbgpx;
    for (int i = tid; i < 32 * NN; i += C::THREADS) s_self[i] = __ldg(selfsrc + i);
    for (int i = tid; i < 4 * NN; i += C::THREADS) s_gp[i] = __ldg(gpsrc + i);
    const float *src = x + (size_t)first * ND;
    if constexpr (N == 4) {
      const float4 *s4 = reinterpret_cast<const float4 *>(src);
      for (int i = tid; i < ncell * (ND / 4); i += C::THREADS) {
        const int cc = i / (ND / 4), o = (i % (ND / 4)) * 4;
        *reinterpret_cast<float4 *>(s_u + cc * SC + o) = __ldg(s4 + i);
      }
    } else {
      for (int i = tid; i < ncell * ND; i += C::THREADS) s_u[(i / ND) * SC + i % ND] = __ldg(src + i);
    }
  }
  __syncthreads();

  const int lane = tid & 31, cw = lane / N, t = lane % N;
  const int c = (tid >> 5) * CPW + cw;
  const int e = first + c;
  if (cw >= CPW || c >= ncell) return;  // the n threads of a cell leave together
  const unsigned cm = ((1u << N) - 1u) << (cw * N);

  const uint32_t fl = __ldg(d.flags + e);
  const bool inside = !(fl & 1u);
  const float yscale = __ldg(d.kappa + e);  // uniform kappa scales every structured term
  int nb[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) nb[f] = __ldg(d.nbr + (size_t)e * 6 + f);
  const float *su = s_u + c * SC;
  float *sx = s_x + c * SC;

  // the cell's own data or a neighbour's (shared memory when it is one of the CTA's cells)
  auto cell_src = [&](int cell, const float *&p, bool &shared) {
    const int r = cell - first;
    shared = (r >= 0 && r < ncell);
    p = shared ? s_u + r * SC : x + (size_t)cell * ND;
  };
  auto ld_any = [&](const float *p, bool shared, float *o) {
    if (shared)
      ld_run<N>(p, o);
    else
      ldg_run<N>(p, o);
  };

  // ---- plane k = t: W_x and W_y, P = M_y W_x + M_x W_y
  float U[NN];
#pragma unroll
  for (int j = 0; j < N; ++j) ld_run<N>(su + t * NN + j * N, U + j * N);
  float P[NN];
  {
    float L[NN], W[NN];
#pragma unroll
    for (int q = 0; q < N; ++q) ld_run<N>(s_self + plane_vsel(fl, inside, 0) * NN + q * N, L + q * N);
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
      for (int r = 0; r < N; ++r) {
        float acc = 0.f;
#pragma unroll
        for (int m = 0; m < N; ++m) acc = fmaf(L[r * N + m], U[j * N + m], acc);
        W[j * N + r] = acc;
      }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const bool full = fl & (1u << (1 + 3 * s)), gp = fl & (1u << (3 + 3 * s));
      if (nb[s] < 0 || !(full || gp)) continue;
      const float *p;
      bool shr;
      cell_src(nb[s], p, shr);
      float V[NN], G[NN];
#pragma unroll
      for (int j = 0; j < N; ++j) ld_any(p + t * NN + j * N, shr, V + j * N);
      if (gp) {
        const int gi = ADJ ? 2 * (1 - s) + (full ? 1 : 0) : 2 * s + (full ? 1 : 0);
#pragma unroll
        for (int q = 0; q < N; ++q) ld_run<N>(s_gp + gi * NN + q * N, G + q * N);
      }
#pragma unroll
      for (int j = 0; j < N; ++j) plane_couple<N>(tab, sc.hf_sigma, gp, G, s, V + j * N, W + j * N);
    }
    // P = M_y W_x
#pragma unroll
    for (int jo = 0; jo < N; ++jo)
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) acc = fmaf(tab.mass[jo * N + j], W[j * N + i], acc);
        P[jo * N + i] = acc;
      }
  }
  {
    float L[NN], W[NN];  // W[i * N + j]: the y-line (i, :, t)
#pragma unroll
    for (int q = 0; q < N; ++q) ld_run<N>(s_self + plane_vsel(fl, inside, 1) * NN + q * N, L + q * N);
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int r = 0; r < N; ++r) {
        float acc = 0.f;
#pragma unroll
        for (int m = 0; m < N; ++m) acc = fmaf(L[r * N + m], U[m * N + i], acc);
        W[i * N + r] = acc;
      }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int f = 2 + s;
      const bool full = fl & (1u << (1 + 3 * f)), gp = fl & (1u << (3 + 3 * f));
      if (nb[f] < 0 || !(full || gp)) continue;
      const float *p;
      bool shr;
      cell_src(nb[f], p, shr);
      float V[NN], G[NN];
#pragma unroll
      for (int j = 0; j < N; ++j) ld_any(p + t * NN + j * N, shr, V + j * N);
      if (gp) {
        const int gi = ADJ ? 2 * (1 - s) + (full ? 1 : 0) : 2 * s + (full ? 1 : 0);
#pragma unroll
        for (int q = 0; q < N; ++q) ld_run<N>(s_gp + gi * NN + q * N, G + q * N);
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float un[N];
#pragma unroll
        for (int m = 0; m < N; ++m) un[m] = V[m * N + i];
        plane_couple<N>(tab, sc.hf_sigma, gp, G, s, un, W + i * N);
      }
    }
    // P += M_x W_y
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
      for (int io = 0; io < N; ++io) {
        float acc = P[j * N + io];
#pragma unroll
        for (int i = 0; i < N; ++i) acc = fmaf(tab.mass[io * N + i], W[i * N + j], acc);
        P[j * N + io] = acc;
      }
  }
  // ---- S = M_z P: exchange the planes
#pragma unroll
  for (int j = 0; j < N; ++j) st_run<N>(sx + t * NN + j * N, P + j * N);
  __syncwarp(cm);
  float S[NN];
#pragma unroll
  for (int q = 0; q < NN; ++q) S[q] = 0.f;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const float mk = tab.mass[t * N + k];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float Q[N];
      ld_run<N>(sx + k * NN + j * N, Q);
#pragma unroll
      for (int i = 0; i < N; ++i) S[j * N + i] = fmaf(mk, Q[i], S[j * N + i]);
    }
  }
  __syncwarp(cm);

  // ---- row j = t: W_z on the z-lines (i, t, :), T = M_x W_z, then M_y across the rows
  {
    float Ur[NN], L[NN], W[NN];  // Ur[k * N + i] = u(i, t, k); W[i * N + k]: the z-line (i, t, :)
#pragma unroll
    for (int k = 0; k < N; ++k) ld_run<N>(su + k * NN + t * N, Ur + k * N);
#pragma unroll
    for (int q = 0; q < N; ++q) ld_run<N>(s_self + plane_vsel(fl, inside, 2) * NN + q * N, L + q * N);
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int r = 0; r < N; ++r) {
        float acc = 0.f;
#pragma unroll
        for (int m = 0; m < N; ++m) acc = fmaf(L[r * N + m], Ur[m * N + i], acc);
        W[i * N + r] = acc;
      }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int f = 4 + s;
      const bool full = fl & (1u << (1 + 3 * f)), gp = fl & (1u << (3 + 3 * f));
      if (nb[f] < 0 || !(full || gp)) continue;
      const float *p;
      bool shr;
      cell_src(nb[f], p, shr);
      float V[NN], G[NN];  // V[k * N + i]: row t of the neighbour's plane k
#pragma unroll
      for (int k = 0; k < N; ++k) ld_any(p + k * NN + t * N, shr, V + k * N);
      if (gp) {
        const int gi = ADJ ? 2 * (1 - s) + (full ? 1 : 0) : 2 * s + (full ? 1 : 0);
#pragma unroll
        for (int q = 0; q < N; ++q) ld_run<N>(s_gp + gi * NN + q * N, G + q * N);
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float un[N];
#pragma unroll
        for (int m = 0; m < N; ++m) un[m] = V[m * N + i];
        plane_couple<N>(tab, sc.hf_sigma, gp, G, s, un, W + i * N);
      }
    }
    // T[k][io] = sum_i M[io][i] W_z(i, t, k), written as row t of plane k
#pragma unroll
    for (int k = 0; k < N; ++k) {
      float T[N];
#pragma unroll
      for (int io = 0; io < N; ++io) {
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < N; ++i) acc = fmaf(tab.mass[io * N + i], W[i * N + k], acc);
        T[io] = acc;
      }
      st_run<N>(sx + k * NN + t * N, T);
    }
  }
  __syncwarp(cm);
  // plane t again: S += M_y T (row j of plane t was written by thread j)
  {
    float Q[NN];
#pragma unroll
    for (int j = 0; j < N; ++j) ld_run<N>(sx + t * NN + j * N, Q + j * N);
#pragma unroll
    for (int jo = 0; jo < N; ++jo)
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float acc = S[jo * N + i];
#pragma unroll
        for (int j = 0; j < N; ++j) acc = fmaf(tab.mass[jo * N + j], Q[j * N + i], acc);
        S[jo * N + i] = acc;
      }
  }
  float *yp = y + (size_t)e * ND + t * NN;
  if (yscale != 1.f) {
#pragma unroll
    for (int q = 0; q < NN; ++q) S[q] *= yscale;
  }
#pragma unroll
  for (int j = 0; j < N; ++j) st_run<N>(yp + j * N, S + j * N);
}

// Launch of the plane kernel on cells [cb, ce) (uniform kappa, 3D, FP32, n <= 5; for n = 4, x and
// y 16-byte aligned).
template <int N>
void launch_struct_planes(const StructTables<float, N> &tab, const DevArrays<float> &d,
                          const Scalars<float> &s, float *y, const float *x, bool adjoint,
                          cudaStream_t stream, int cb, int ce) {
  using C = PlaneCfg<N>;
  const int blocks = (ce - cb + C::CPB - 1) / C::CPB;
  if (blocks <= 0) return;
  if (adjoint)
    struct_plane_kernel<N, true><<<blocks, C::THREADS, 0, stream>>>(tab, d, s, y, x, cb, ce);
  else
    struct_plane_kernel<N, false><<<blocks, C::THREADS, 0, stream>>>(tab, d, s, y, x, cb, ce);
}

}  // namespace uf
