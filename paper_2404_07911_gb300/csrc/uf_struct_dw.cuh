// FP64-accurate structured terms in double-word arithmetic on the FP32 pipe (3D, n = 4, uniform
// kappa): an alternative to the FP64 structured kernel for a part whose FP64 pipe runs at 1/64 of
// its FP32 rate.
//
// A double-word number is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2 (about
// 48 significant bits).  The kernel uses the error-free transformations TwoSum (Knuth: the exact
// rounding error of a float sum from six operations) and TwoProd by FMA (the exact error of a float
// product from one fused multiply-add), combined as in the double-word building blocks analysed by
// Joldes, Muller and Popescu (2017, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic"): a double-word product with the two cross terms, added to a
// double-word accumulator by TwoSum of the high parts and a renormalisation (TwoSum again).  Every
// operation uses the _rn intrinsics, which the compiler never contracts into fused operations.
//
// The kernel keeps the structure of the FP32 plane kernel (one thread per z-plane of a cell; the
// form y = M_z (M_y W_x + M_x W_y) + M_x M_y W_z with the unpremultiplied line matrices) and reads
// the FP64 operator's own tables, input and output (doubles, split into double words on load).
#pragma once

#include "uf_device.h"

namespace uf {

struct dw {
  float h, l;
};

__device__ __forceinline__ dw dw_of(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double dw_val(dw a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ dw dw_zero() { return {0.f, 0.f}; }

// s + t exactly as hi + lo (TwoSum, no ordering needed)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// hi + lo renormalised by TwoSum (FastTwoSum would need |s| >= |t|, which cancellation in the
// accumulations of this operator can break)
__device__ __forceinline__ dw renorm(float s, float t) {
  dw r;
  two_sum(s, t, r.h, r.l);
  return r;
}

// c + a b
__device__ __forceinline__ dw dw_fma(dw a, dw b, dw c) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);          // exact error of the high product
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  float s, t;
  two_sum(c.h, p, s, t);
  t = __fadd_rn(t, __fadd_rn(e, c.l));
  return renorm(s, t);
}
__device__ __forceinline__ dw dw_add(dw a, dw b) {
  float s, t;
  two_sum(a.h, b.h, s, t);
  t = __fadd_rn(t, __fadd_rn(a.l, b.l));
  return renorm(s, t);
}
__device__ __forceinline__ dw dw_neg(dw a) { return {-a.h, -a.l}; }

// sum_m a[m] b[m] over n terms: the high products summed by TwoSum, their rounding errors and the
// cross terms collected in one float, one renormalisation at the end (about 12 instead of 18
// operations per term)
template <int N>
__device__ __forceinline__ dw dw_dot(const dw *a, const dw *b) {
  float s = 0.f, c = 0.f;
#pragma unroll
  for (int m = 0; m < N; ++m) {
    const float p = __fmul_rn(a[m].h, b[m].h);
    float e = __fmaf_rn(a[m].h, b[m].h, -p);
    e = __fmaf_rn(a[m].h, b[m].l, e);
    e = __fmaf_rn(a[m].l, b[m].h, e);
    float t;
    two_sum(s, p, s, t);
    c = __fadd_rn(c, __fadd_rn(t, e));
  }
  return renorm(s, c);
}
__device__ __forceinline__ dw dw_mul(dw a, dw b) { return dw_fma(a, b, dw_zero()); }

template <int N>
struct DwCfg {
  static constexpr int NN = N * N, ND = N * N * N;
  static constexpr int CPW = 32 / N, CPB = 4 * CPW, THREADS = 128;
  static constexpr int SC = ND + 4;  // padded cell stride (in double words)
};

// n consecutive double words from shared memory.
template <int N>
__device__ __forceinline__ void ld_dw(const dw *p, dw *o) {
#pragma unroll
  for (int m = 0; m < N; ++m) o[m] = p[m];
}
// n consecutive doubles from global memory as double words.
template <int N>
__device__ __forceinline__ void ldg_dw(const double *p, dw *o) {
#pragma unroll
  for (int m = 0; m < N; ++m) o[m] = dw_of(__ldg(p + m));
}

// w += coupling of one line to its neighbour line un across the face on side s: ghost penalty
// through the full 1D matrix G, SIPG only through rank 2 (the neighbour's face value and normal
// derivative; dow, dnb and hs = h^{d-1} sigma / h as in the FP64 tables).
template <int N>
__device__ __forceinline__ void dw_couple(bool gp, const dw *G, const dw *dow, const dw *dnb,
                                          dw hs, int s, const dw *un, dw *w) {
  if (gp) {
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
      for (int m = 0; m < N; ++m) w[r] = dw_fma(G[r * N + m], un[m], w[r]);
  } else {
    const dw alpha = un[s ? 0 : N - 1];
    dw beta = dw_zero();
#pragma unroll
    for (int m = 0; m < N; ++m) beta = dw_fma(dnb[m], un[m], beta);
#pragma unroll
    for (int r = 0; r < N; ++r) w[r] = dw_fma(alpha, dow[r], w[r]);
    const int o = s ? N - 1 : 0;
    w[o] = dw_add(w[o], dw_neg(dw_fma(hs, alpha, beta)));
  }
}

template <int N, bool ADJ>
__global__ void __launch_bounds__(DwCfg<N>::THREADS, 2) struct_dw_kernel(
    const __grid_constant__ StructTables<double, N> tab, const DevArrays<double> d,
    const Scalars<double> sc, double *__restrict__ y, const dw *__restrict__ x,
    int cell_begin, int cell_end) {
  using C = DwCfg<N>;
  constexpr int NN = C::NN, ND = C::ND, CPW = C::CPW, CPB = C::CPB, SC = C::SC;
  __shared__ dw s_self[32 * NN];  // line matrices by face configuration (no M^{-1})
  __shared__ dw s_gp[4 * NN];     // ghost-penalty neighbour couplings
  __shared__ dw s_mass[NN];
  __shared__ dw s_aux[4 * N];     // dow[0], dow[1], dnb[0], dnb[1]
  __shared__ dw s_u[CPB * SC];    // the CTA's own cells
  __shared__ dw s_x[CPB * SC];    // plane / row exchange

  const int tid = threadIdx.x;
  const int first = cell_begin + blockIdx.x * CPB;
  const int ncell = min(CPB, cell_end - first);
  {
    const double *selfsrc = ADJ ? d.lselfxT : d.lselfx;
    const double *gpsrc = ADJ ? d.lnbgpxT : d.lnbgpx;
    for (int i = tid; i < 32 * NN; i += C::THREADS) s_self[i] = dw_of(__ldg(selfsrc + i));
    for (int i = tid; i < 4 * NN; i += C::THREADS) s_gp[i] = dw_of(__ldg(gpsrc + i));
    for (int i = tid; i < NN; i += C::THREADS) s_mass[i] = dw_of(tab.mass[i]);
    for (int i = tid; i < 2 * N; i += C::THREADS) {
      s_aux[i] = dw_of(tab.dowx[i / N][i % N]);
      s_aux[2 * N + i] = dw_of(tab.dnb[i / N][i % N]);
    }
    const dw *src = x + (size_t)first * ND;
    for (int i = tid; i < ncell * ND; i += C::THREADS) s_u[(i / ND) * SC + i % ND] = src[i];
  }
  __syncthreads();

  const int lane = tid & 31, cw = lane / N, t = lane % N;
  const int c = (tid >> 5) * CPW + cw;
  const int e = first + c;
  if (cw >= CPW || c >= ncell) return;  // the n threads of a cell leave together
  const unsigned cm = ((1u << N) - 1u) << (cw * N);

  const uint32_t fl = __ldg(d.flags + e);
  const bool inside = !(fl & 1u);
  const double kap = __ldg(d.kappa + e);  // uniform kappa scales every structured term
  int nb[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) nb[f] = __ldg(d.nbr + (size_t)e * 6 + f);
  const dw *su = s_u + c * SC;
  dw *sx = s_x + c * SC;
  const dw hs = dw_of(sc.hf_sigma);

  // n double words of a neighbour at element offset `off` with stride `st` (shared when the
  // neighbour is one of the CTA's cells)
  auto nb_line = [&](int cell, int off, int st, dw *o) {
    const int r = cell - first;
    if (r >= 0 && r < ncell) {
#pragma unroll
      for (int m = 0; m < N; ++m) o[m] = s_u[r * SC + off + m * st];
    } else {
      const dw *p = x + (size_t)cell * ND + off;
#pragma unroll
      for (int m = 0; m < N; ++m) o[m] = p[m * st];
    }
  };
  auto face_bits = [&](int f, bool &full, bool &gp) {
    full = (fl & (1u << (1 + 3 * f))) != 0u;
    gp = (fl & (1u << (3 + 3 * f))) != 0u;
  };

  // ---- plane k = t: P = M_y W_x + M_x W_y, accumulated line by line
  dw P[NN];
#pragma unroll
  for (int q = 0; q < NN; ++q) P[q] = dw_zero();
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const dw *L = s_self + plane_vsel(fl, inside, a) * NN;
#pragma unroll 1
    for (int q = 0; q < N; ++q) {  // x-line j = q (a = 0) or y-line i = q (a = 1)
      dw line[N], w[N];
#pragma unroll
      for (int m = 0; m < N; ++m) line[m] = su[t * NN + (a == 0 ? q * N + m : m * N + q)];
#pragma unroll
      for (int r = 0; r < N; ++r) {
        dw lr[N];
#pragma unroll
        for (int m = 0; m < N; ++m) lr[m] = L[r * N + m];
        w[r] = dw_dot<N>(lr, line);
      }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int f = 2 * a + s;
        bool full, gp;
        face_bits(f, full, gp);
        if (nb[f] < 0 || !(full || gp)) continue;
        dw un[N];
        if (a == 0)
          nb_line(nb[f], t * NN + q * N, 1, un);
        else
          nb_line(nb[f], t * NN + q, N, un);
        const int gi = ADJ ? 2 * (1 - s) + (full ? 1 : 0) : 2 * s + (full ? 1 : 0);
        dw_couple<N>(gp, s_gp + gi * NN, s_aux + s * N, s_aux + 2 * N + s * N, hs, s, un, w);
      }
      // a = 0: P[jo][i] += M[jo][q] w[i];  a = 1: P[j][io] += M[io][q] w[j]
#pragma unroll
      for (int o = 0; o < N; ++o) {
        const dw mo = s_mass[o * N + q];
#pragma unroll
        for (int r = 0; r < N; ++r) {
          const int idx = a == 0 ? o * N + r : r * N + o;
          P[idx] = dw_fma(mo, w[r], P[idx]);
        }
      }
    }
  }
  // ---- S = M_z P: exchange the planes
#pragma unroll
  for (int q = 0; q < NN; ++q) sx[t * NN + q] = P[q];
  __syncwarp(cm);
  dw S[NN];
#pragma unroll
  for (int q = 0; q < NN; ++q) S[q] = dw_zero();
#pragma unroll 1
  for (int k = 0; k < N; ++k) {
    const dw mk = s_mass[t * N + k];
#pragma unroll
    for (int q = 0; q < NN; ++q) S[q] = dw_fma(mk, sx[k * NN + q], S[q]);
  }
  __syncwarp(cm);
  // ---- row j = t: T = M_x W_z on the z-lines (i, t, :), written as row t of every plane
  {
    const dw *L = s_self + plane_vsel(fl, inside, 2) * NN;
    dw T[NN];  // T[k * N + io]
#pragma unroll
    for (int q = 0; q < NN; ++q) T[q] = dw_zero();
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
      dw line[N], w[N];
#pragma unroll
      for (int k = 0; k < N; ++k) line[k] = su[k * NN + t * N + i];
#pragma unroll
      for (int r = 0; r < N; ++r) {
        dw lr[N];
#pragma unroll
        for (int m = 0; m < N; ++m) lr[m] = L[r * N + m];
        w[r] = dw_dot<N>(lr, line);
      }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int f = 4 + s;
        bool full, gp;
        face_bits(f, full, gp);
        if (nb[f] < 0 || !(full || gp)) continue;
        dw un[N];
        nb_line(nb[f], t * N + i, NN, un);
        const int gi = ADJ ? 2 * (1 - s) + (full ? 1 : 0) : 2 * s + (full ? 1 : 0);
        dw_couple<N>(gp, s_gp + gi * NN, s_aux + s * N, s_aux + 2 * N + s * N, hs, s, un, w);
      }
#pragma unroll
      for (int io = 0; io < N; ++io) {
        const dw mo = s_mass[io * N + i];
#pragma unroll
        for (int k = 0; k < N; ++k) T[k * N + io] = dw_fma(mo, w[k], T[k * N + io]);
      }
    }
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
      for (int io = 0; io < N; ++io) sx[k * NN + t * N + io] = T[k * N + io];
  }
  __syncwarp(cm);
  // plane t: S += M_y T (row j of plane t was written by thread j)
#pragma unroll
  for (int jo = 0; jo < N; ++jo)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const dw mo = s_mass[jo * N + j];
#pragma unroll
      for (int i = 0; i < N; ++i) S[jo * N + i] = dw_fma(mo, sx[t * NN + j * N + i], S[jo * N + i]);
    }
  double *yp = y + (size_t)e * ND + t * NN;
#pragma unroll
  for (int q = 0; q < NN; ++q) yp[q] = kap == 1.0 ? dw_val(S[q]) : kap * dw_val(S[q]);
}

// x (doubles) to double words, once per product (the split takes FP64-pipe operations, which the
// kernel would otherwise repeat for every neighbour read).
static __global__ void k_to_dw(dw *__restrict__ out, const double *__restrict__ in, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = dw_of(in[i]);
}

// Launch of the double-word structured kernel on cells [cb, ce) (3D, uniform kappa); xw holds
// n_active * n^3 double words of scratch for the converted input.
template <int N>
void launch_struct_dw(const StructTables<double, N> &tab, const DevArrays<double> &d,
                      const Scalars<double> &s, double *y, const double *x, dw *xw, bool adjoint,
                      cudaStream_t stream, int cb, int ce) {
  using C = DwCfg<N>;
  const int blocks = (ce - cb + C::CPB - 1) / C::CPB;
  if (blocks <= 0) return;
  const int64_t nx = (int64_t)d.n_active * C::ND;
  k_to_dw<<<(unsigned)((nx + 255) / 256), 256, 0, stream>>>(xw, x, nx);
  if (adjoint)
    struct_dw_kernel<N, true><<<blocks, C::THREADS, 0, stream>>>(tab, d, s, y, xw, cb, ce);
  else
    struct_dw_kernel<N, false><<<blocks, C::THREADS, 0, stream>>>(tab, d, s, y, xw, cb, ce);
}

}  // namespace uf
