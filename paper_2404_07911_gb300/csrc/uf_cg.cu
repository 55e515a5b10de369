// Continuous Q_p operator (Eq. bilinear_cg with the face ghost penalty, no SIPG): load vector,
// Jacobi diagonal, global <-> cell-local maps, and the preconditioned CG solvers in FP64 and as
// FP32 inner iterations inside FP64 iterative refinement.
//
// The continuous operator is A = P^T A_loc P, with P the map from global lattice nodes to
// cell-local DoFs and A_loc the cell-local operator that the DG kernels evaluate when the face
// flags carry no SIPG term: y = A x is a gather (x_loc = P x), the cell-centric kernels
// (y_loc = A_loc x_loc), and a node sum (y = P^T y_loc) over each node's owners in a fixed order,
// so no floating-point atomics are needed and the result is deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "uf_operator.h"

namespace uf {

// ------------------------------------------------------------------------------------------
// Host: load vector (f = 1) and diagonal of A, FP64
// ------------------------------------------------------------------------------------------
// Cell-local load vector (f = 1) and diagonal of the cell-local operator of every active cell.
// discontinuous = false: the continuous space, where the couplings across a face act on the shared
// face nodes (they enter the diagonal); true: the discontinuous space, whose diagonal carries the
// SIPG self terms of full and cut faces and no neighbour coupling.
void local_vectors(const HostOperator &op, bool discontinuous, std::vector<double> &bloc,
                   std::vector<double> &dloc) {
  const int d = op.dim, n = op.n, nd = op.ndof, nf = 2 * d, nn = n * n;
  const Tables1D &t = op.t;
  const double h = op.h;
  std::vector<double> m;
  structured_matrices(op, m);
  const double *Kv = &m[0], *M = &m[nn];
  auto mat = [&](int which, int s) { return &m[(which + s) * nn]; };  // 2 a, 4 pen, 6 gp, 8 b, 10 c, 12 qn, 14 hn
  // integrals of the 1D basis: w_i = int_0^1 phi_i
  double wi[kMaxN] = {0};
  for (int q = 0; q < n; ++q)
    for (int i = 0; i < n; ++i) {
      double v[kMaxN], dv[kMaxN];
      lagrange_values(t, t.gauss_x[q], v, dv);
      wi[i] += t.gauss_w[q] * v[i];
    }
  const double hd = std::pow(h, d);
  bloc.assign((size_t)op.n_active * nd, 0.0);
  dloc.assign((size_t)op.n_active * nd, 0.0);
  auto idx3 = [&](int l, int *ia) {
    for (int a = 0; a < 3; ++a) {
      ia[a] = (a < d) ? l % n : 0;
      l /= n;
    }
  };
  for (int64_t e = 0; e < op.n_active; ++e) {
    double *b = &bloc[e * nd], *dg = &dloc[e * nd];
    const uint32_t fl = op.flags[e];
    const bool inside = op.act_type[e] == 0;
    const double kap = op.kappa[e];
    // ---- structured terms: diag of sum_a (L_a along a) (x) M (x) M and ghost-penalty cross terms
    double Lself[kMaxDim][kMaxN * kMaxN];
    double cross[kMaxDim][2];  // L_nb[own][nb] at the face node of each side (0 if no coupling)
    for (int a = 0; a < d; ++a) {
      for (int i = 0; i < nn; ++i) Lself[a][i] = inside ? kap * Kv[i] : 0.0;
      for (int s = 0; s < 2; ++s) {
        cross[a][s] = 0.0;
        const int f = 2 * a + s;
        const int nb = op.nbr[e * nf + f];
        if (nb < 0) continue;
        const double kavg = 0.5 * (kap + op.kappa[nb]);
        const bool full = fl & face_bit_sipg_full(f), gp = fl & face_bit_gp(f);
        const int io = s ? n - 1 : 0, inb = s ? 0 : n - 1;
        for (int i = 0; i < nn; ++i) {
          if (full) Lself[a][i] += kap * mat(2, s)[i] + kavg * mat(4, s)[i];
          if (gp) Lself[a][i] += kavg * mat(6, s)[i];
        }
        double c = 0.0;
        if (full) c += kap * mat(8, s)[io * n + inb] + op.kappa[nb] * mat(10, s)[io * n + inb] +
                       kavg * mat(12, s)[io * n + inb];
        if (gp) c += kavg * mat(14, s)[io * n + inb];
        cross[a][s] = c;
      }
    }
    for (int l = 0; l < nd; ++l) {
      int ia[3];
      idx3(l, ia);
      double acc = 0.0;
      for (int a = 0; a < d; ++a) {
        double mm = 1.0;
        for (int bb = 0; bb < d; ++bb)
          if (bb != a) mm *= M[ia[bb] * n + ia[bb]];
        acc += Lself[a][ia[a] * n + ia[a]] * mm;
        if (!discontinuous)
          for (int s = 0; s < 2; ++s)
            if (ia[a] == (s ? n - 1 : 0)) acc += cross[a][s] * mm;
      }
      dg[l] = acc;
      if (inside) {
        double v = hd;
        for (int a = 0; a < d; ++a) v *= wi[ia[a]];
        b[l] = v;
      }
    }
    if (inside) continue;
    // ---- unstructured terms of a cut cell, line by line
    const int64_t c = op.cut_of[e];
    for (int64_t li = op.vline_off[c]; li < op.vline_off[c + 1]; ++li) {
      const QLine &ln = op.vol_lines[li];
      const int k = ln.k;
      int ob = (k == 0) ? 1 : 0, oc = (k == 2) ? 1 : 2;
      if (d == 2) ob = 1 - k;
      const bool has_vol = ln.vcnt > 0;
      const int64_t p0 = has_vol ? ln.vbeg : ln.sidx;
      const std::vector<double> *xi = has_vol ? op.vol_xi : op.surf_xi;
      double A[kMaxN], Ad[kMaxN], B[kMaxN] = {1.0}, Bd[kMaxN] = {0.0};
      lagrange_values(t, xi[ob][p0], A, Ad);
      if (d == 3) lagrange_values(t, xi[oc][p0], B, Bd);
      const int nbm = (d == 3) ? n : 1;
      // volume: S0_k = sum w C_k, S1_k = sum w C_k^2, S2_k = sum w C_k'^2
      double S0[kMaxN] = {0}, S1[kMaxN] = {0}, S2[kMaxN] = {0};
      for (int64_t p = ln.vbeg; p < ln.vbeg + ln.vcnt; ++p) {
        double C[kMaxN], Cd[kMaxN];
        lagrange_values(t, op.vol_xi[k][p], C, Cd);
        const double w = op.vol_w[p];
        for (int q = 0; q < n; ++q) {
          S0[q] += w * C[q];
          S1[q] += w * C[q] * C[q];
          S2[q] += w * Cd[q] * Cd[q];
        }
      }
      const double sk = kap / (h * h);
      for (int ib = 0; ib < n; ++ib)
        for (int ic = 0; ic < nbm; ++ic)
          for (int q = 0; q < n; ++q) {
            int l = ib * (ob == 0 ? 1 : (ob == 1 ? n : n * n)) + q * (k == 0 ? 1 : (k == 1 ? n : n * n));
            if (d == 3) l += ic * (oc == 0 ? 1 : (oc == 1 ? n : n * n));
            const double a2 = A[ib] * A[ib], ad2 = Ad[ib] * Ad[ib];
            const double b2 = B[ic] * B[ic], bd2 = Bd[ic] * Bd[ic];
            dg[l] += sk * (ad2 * b2 * S1[q] + a2 * bd2 * S1[q] + a2 * b2 * S2[q]);
            b[l] += A[ib] * B[ic] * S0[q];
          }
      // Nitsche at the surface point of the line
      if (ln.sidx >= 0) {
        const int64_t sp = ln.sidx;
        double C[kMaxN], Cd[kMaxN];
        lagrange_values(t, op.surf_xi[k][sp], C, Cd);
        const double w = op.surf_w[sp] * kap, tau = op.params.nitsche_gamma / h;
        const double nk = op.surf_n[k][sp], nbn = op.surf_n[ob][sp], nc = (d == 3) ? op.surf_n[oc][sp] : 0.0;
        for (int ib = 0; ib < n; ++ib)
          for (int ic = 0; ic < nbm; ++ic)
            for (int q = 0; q < n; ++q) {
              int l = ib * (ob == 0 ? 1 : (ob == 1 ? n : n * n)) + q * (k == 0 ? 1 : (k == 1 ? n : n * n));
              if (d == 3) l += ic * (oc == 0 ? 1 : (oc == 1 ? n : n * n));
              const double phi = A[ib] * B[ic] * C[q];
              const double dn = (nbn * Ad[ib] * B[ic] * C[q] + nc * A[ib] * Bd[ic] * C[q] +
                                 nk * A[ib] * B[ic] * Cd[q]) / h;
              dg[l] += w * (-2.0 * phi * dn + tau * phi * phi);
            }
      }
    }
    if (!discontinuous) continue;
    // ---- SIPG on the cut faces of a cut cell (own-own terms): at a face point only the DoFs on
    // the own face-node layer are non-zero; with sgn = +1 on the upper face (own cell K^-) and
    // -1 on the lower one, a(phi, phi) += w (-sgn kappa_K d_axis phi phi + sigma/h {kappa} phi^2)
    for (int f = 0; f < nf; ++f) {
      if (!(fl & face_bit_sipg_cut(f))) continue;
      const int axis = f / 2, side = f % 2;
      const int nb = op.nbr[e * nf + f];
      const double kavg = 0.5 * (kap + op.kappa[nb]);
      const double sgn = side ? 1.0 : -1.0, sig = op.params.sipg_gamma / h;
      const int end = side ? n - 1 : 0;
      const double dend = t.deriv_end[side][1][end] / h;
      int oa[2] = {0, 0}, no = 0;
      for (int a = 0; a < d; ++a)
        if (a != axis) oa[no++] = a;
      for (int64_t p = op.cface_off[c * nf + f]; p < op.cface_off[c * nf + f + 1]; ++p) {
        double V[2][kMaxN], Dv[kMaxN];
        for (int j = 0; j < no; ++j) lagrange_values(t, op.cface_eta[j][p], V[j], Dv);
        const double w = op.cface_w[p];
        for (int l = 0; l < nd; ++l) {
          int ia[3];
          idx3(l, ia);
          if (ia[axis] != end) continue;
          double prod = 1.0;
          for (int j = 0; j < no; ++j) prod *= V[j][ia[oa[j]]];
          const double phi = prod, dphi = dend * prod;
          dg[l] += w * (-sgn * kap * dphi * phi + sig * kavg * phi * phi);
        }
      }
    }
  }
}

void dg_host_diagonal(HostOperator &op) {
  std::vector<double> bloc;
  local_vectors(op, true, bloc, op.dg_diag);
}

void cg_host_vectors(HostOperator &op) {
  std::vector<double> bloc, dloc;
  local_vectors(op, false, bloc, dloc);
  op.cg_rhs.assign(op.n_cg, 0.0);
  op.cg_diag.assign(op.n_cg, 0.0);
  for (int64_t g = 0; g < op.n_cg; ++g)
    for (int32_t o = op.cg_own_off[g]; o < op.cg_own_off[g + 1]; ++o) {
      op.cg_rhs[g] += bloc[op.cg_own_idx[o]];
      op.cg_diag[g] += dloc[op.cg_own_idx[o]];
    }
}

}  // namespace uf

// ------------------------------------------------------------------------------------------
// Device: gather, node sum, vector kernels
// ------------------------------------------------------------------------------------------
namespace uf {
namespace {

constexpr int kDotBlocks = 608;  // 4 x 152 SMs; partial sums reduced in a fixed order
constexpr int kDotThreads = 256;

template <typename T>
__global__ void k_gather(T *__restrict__ xl, const T *__restrict__ x, const int32_t *__restrict__ l2g,
                         int64_t n_loc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_loc) xl[i] = x[l2g[i]];
}

template <typename T>
__global__ void k_node_sum(T *__restrict__ y, const T *__restrict__ yl, const int32_t *__restrict__ off,
                           const int32_t *__restrict__ idx, int64_t n) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  T acc = T(0);
  for (int32_t o = off[g]; o < off[g + 1]; ++o) acc += yl[idx[o]];
  y[g] = acc;
}

// Block partial sums of sum_i a_i b_i (and of sum_i a_i a_i if two > 0) in FP64, fixed order.
template <typename T>
__global__ void __launch_bounds__(kDotThreads) k_dot_partial(const T *__restrict__ a, const T *__restrict__ b,
                                                             int64_t n, double *__restrict__ part, int two) {
  __shared__ double s0[kDotThreads], s1[kDotThreads];
  double acc0 = 0.0, acc1 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double av = (double)a[i];
    acc0 = fma(av, (double)b[i], acc0);
    if (two) acc1 = fma(av, av, acc1);
  }
  s0[threadIdx.x] = acc0;
  s1[threadIdx.x] = acc1;
  __syncthreads();
  for (int w = kDotThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s0[threadIdx.x] += s0[threadIdx.x + w];
      s1[threadIdx.x] += s1[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0[0];
    part[kDotBlocks + blockIdx.x] = s1[0];
  }
}

__global__ void k_dot_final(const double *__restrict__ part, double *__restrict__ out) {
  __shared__ double s0[kDotThreads], s1[kDotThreads];
  double a0 = 0.0, a1 = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += kDotThreads) {
    a0 += part[i];
    a1 += part[kDotBlocks + i];
  }
  s0[threadIdx.x] = a0;
  s1[threadIdx.x] = a1;
  __syncthreads();
  for (int w = kDotThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s0[threadIdx.x] += s0[threadIdx.x + w];
      s1[threadIdx.x] += s1[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s0[0];
    out[1] = s1[0];
  }
}

// z = invd * r
template <typename T>
__global__ void k_jacobi(T *__restrict__ z, const T *__restrict__ r, const T *__restrict__ invd, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = invd[i] * r[i];
}

// 16-byte packs of a vector (the solver's work vectors are separate cudaMalloc allocations, so
// their packs are aligned): V entries per pack.
template <typename T>
struct Pack;
template <>
struct Pack<float> {
  static constexpr int V = 4;
  __device__ __forceinline__ static void load(const float *a, int64_t j, float *o) {
    const float4 v = reinterpret_cast<const float4 *>(a)[j];
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
  }
  __device__ __forceinline__ static void store(float *a, int64_t j, const float *o) {
    reinterpret_cast<float4 *>(a)[j] = make_float4(o[0], o[1], o[2], o[3]);
  }
};
template <>
struct Pack<double> {
  static constexpr int V = 2;
  __device__ __forceinline__ static void load(const double *a, int64_t j, double *o) {
    const double2 v = reinterpret_cast<const double2 *>(a)[j];
    o[0] = v.x;
    o[1] = v.y;
  }
  __device__ __forceinline__ static void store(double *a, int64_t j, const double *o) {
    reinterpret_cast<double2 *>(a)[j] = make_double2(o[0], o[1]);
  }
};

// Block sums of (s0, s1) over kDotThreads threads, written to part[blockIdx.x] and
// part[kDotBlocks + blockIdx.x] (fixed order).
__device__ __forceinline__ void block_sums(double a0, double a1, double *__restrict__ part) {
  __shared__ double s0[kDotThreads], s1[kDotThreads];
  s0[threadIdx.x] = a0;
  s1[threadIdx.x] = a1;
  __syncthreads();
  for (int w = kDotThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s0[threadIdx.x] += s0[threadIdx.x + w];
      s1[threadIdx.x] += s1[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0[0];
    part[kDotBlocks + blockIdx.x] = s1[0];
  }
}

// PCG start: pcg_init_final reads the block sums of r.z and r.r.
__global__ void k_pcg_init_final(const double *__restrict__ part, PcgScalars *__restrict__ sc, double rtol) {
  __shared__ double s0[kDotThreads], s1[kDotThreads];
  double a0 = 0.0, a1 = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += kDotThreads) {
    a0 += part[i];
    a1 += part[kDotBlocks + i];
  }
  s0[threadIdx.x] = a0;
  s1[threadIdx.x] = a1;
  __syncthreads();
  for (int w = kDotThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s0[threadIdx.x] += s0[threadIdx.x + w];
      s1[threadIdx.x] += s1[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sc->rz = s0[0];
    sc->rr = s1[0];
    sc->rr_stop = rtol * rtol * s1[0];
    sc->pq = sc->alpha = sc->beta = 0.0;
    sc->its = 0;
    sc->status = (s1[0] == 0.0) ? 1 : 0;
  }
}

// alpha = rz / pq from the block sums of p.q (breakdown if pq <= 0).
__global__ void k_pcg_alpha(const double *__restrict__ part, PcgScalars *__restrict__ sc) {
  if (sc->status != 0) return;
  __shared__ double s0[kDotThreads];
  double a0 = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += kDotThreads) a0 += part[i];
  s0[threadIdx.x] = a0;
  __syncthreads();
  for (int w = kDotThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s0[threadIdx.x] += s0[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double pq = s0[0];
    sc->pq = pq;
    if (pq > 0.0) {
      sc->alpha = sc->rz / pq;
    } else {
      sc->alpha = 0.0;
      sc->status = 2;
    }
  }
}

// Block sums of p.q (grid of kDotBlocks), skipped once the run has stopped.
template <typename T>
__global__ void __launch_bounds__(kDotThreads) k_pcg_pq(const T *__restrict__ p, const T *__restrict__ q,
                                                        int64_t n, double *__restrict__ part,
                                                        const PcgScalars *__restrict__ sc) {
  if (sc->status != 0) return;
  constexpr int V = Pack<T>::V;
  const int64_t nv = n / V;
  double acc = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += (int64_t)gridDim.x * blockDim.x) {
    T pv[V], qv[V];
    Pack<T>::load(p, j, pv);
    Pack<T>::load(q, j, qv);
#pragma unroll
    for (int e = 0; e < V; ++e) acc = fma((double)pv[e], (double)qv[e], acc);
  }
  if (blockIdx.x == 0)  // the last n mod V entries
    for (int64_t i = nv * V + threadIdx.x; i < n; i += blockDim.x) acc = fma((double)p[i], (double)q[i], acc);
  block_sums(acc, 0.0, part);
}

// x += alpha p, r -= alpha q, z = invd r, and the block sums of r.z and r.r (grid of kDotBlocks).
template <typename T>
__global__ void __launch_bounds__(kDotThreads)
    k_pcg_update(T *__restrict__ x, T *__restrict__ r, T *__restrict__ z, const T *__restrict__ p,
                 const T *__restrict__ q, const T *__restrict__ invd, int64_t n, double *__restrict__ part,
                 const PcgScalars *__restrict__ sc) {
  if (sc->status != 0) return;
  const T alpha = (T)sc->alpha;
  constexpr int V = Pack<T>::V;
  const int64_t nv = n / V;
  double a0 = 0.0, a1 = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += (int64_t)gridDim.x * blockDim.x) {
    T xv[V], rv[V], pv[V], qv[V], dv[V], zv[V];
    Pack<T>::load(x, j, xv);
    Pack<T>::load(r, j, rv);
    Pack<T>::load(p, j, pv);
    Pack<T>::load(q, j, qv);
    Pack<T>::load(invd, j, dv);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      xv[e] = fma(alpha, pv[e], xv[e]);
      rv[e] = fma(-alpha, qv[e], rv[e]);
      zv[e] = dv[e] * rv[e];
      a0 = fma((double)rv[e], (double)zv[e], a0);
      a1 = fma((double)rv[e], (double)rv[e], a1);
    }
    Pack<T>::store(x, j, xv);
    Pack<T>::store(r, j, rv);
    Pack<T>::store(z, j, zv);
  }
  if (blockIdx.x == 0)  // the last n mod V entries
    for (int64_t i = nv * V + threadIdx.x; i < n; i += blockDim.x) {
      x[i] = fma(alpha, p[i], x[i]);
      const T ri = fma(-alpha, q[i], r[i]);
      const T zi = invd[i] * ri;
      r[i] = ri;
      z[i] = zi;
      a0 = fma((double)ri, (double)zi, a0);
      a1 = fma((double)ri, (double)ri, a1);
    }
  block_sums(a0, a1, part);
}

// New r.z and r.r: stop test, then beta = rz_new / rz.
__global__ void k_pcg_beta(const double *__restrict__ part, PcgScalars *__restrict__ sc) {
  if (sc->status != 0) return;
  __shared__ double s0[kDotThreads], s1[kDotThreads];
  double a0 = 0.0, a1 = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += kDotThreads) {
    a0 += part[i];
    a1 += part[kDotBlocks + i];
  }
  s0[threadIdx.x] = a0;
  s1[threadIdx.x] = a1;
  __syncthreads();
  for (int w = kDotThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s0[threadIdx.x] += s0[threadIdx.x + w];
      s1[threadIdx.x] += s1[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sc->its += 1;
    sc->rr = s1[0];
    if (s1[0] <= sc->rr_stop) {
      sc->status = 1;
    } else {
      sc->beta = s0[0] / sc->rz;
      sc->rz = s0[0];
    }
  }
}

// p = z + beta p (one 16-byte pack per thread; block 0 also takes the last n mod V entries)
template <typename T>
__global__ void k_pcg_direction(T *__restrict__ p, const T *__restrict__ z, int64_t n,
                                const PcgScalars *__restrict__ sc) {
  if (sc->status != 0) return;
  const T beta = (T)sc->beta;
  constexpr int V = Pack<T>::V;
  const int64_t nv = n / V;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nv) {
    T pv[V], zv[V];
    Pack<T>::load(p, j, pv);
    Pack<T>::load(z, j, zv);
#pragma unroll
    for (int e = 0; e < V; ++e) pv[e] = fma(beta, pv[e], zv[e]);
    Pack<T>::store(p, j, pv);
  }
  if (blockIdx.x == 0 && nv * V + threadIdx.x < n) {
    const int64_t i = nv * V + threadIdx.x;
    p[i] = fma(beta, p[i], z[i]);
  }
}

// r = b - q
__global__ void k_residual(double *__restrict__ r, const double *__restrict__ b, const double *__restrict__ q,
                           int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = b[i] - q[i];
}

// r32 = (float)(r * s)
__global__ void k_scale_to_f32(float *__restrict__ r32, const double *__restrict__ r, double s, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r32[i] = (float)(r[i] * s);
}

// x += s * d32
__global__ void k_refine(double *__restrict__ x, const float *__restrict__ d32, double s, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = fma(s, (double)d32[i], x[i]);
}

// x += d
__global__ void k_add(double *__restrict__ x, const double *__restrict__ d, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] += d[i];
}

template <typename T>
__global__ void k_fill(T *__restrict__ x, T v, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

template <typename T>
int cg_gather(T *x_loc, const T *x, const int32_t *l2g, int64_t n_loc, cudaStream_t s) {
  k_gather<T><<<nblk(n_loc), 256, 0, s>>>(x_loc, x, l2g, n_loc);
  return (int)cudaGetLastError();
}

template <typename T>
int cg_node_sum(T *y, const T *y_loc, const int32_t *off, const int32_t *idx, int64_t n, cudaStream_t s) {
  k_node_sum<T><<<nblk(n), 256, 0, s>>>(y, y_loc, off, idx, n);
  return (int)cudaGetLastError();
}

template int cg_gather<double>(double *, const double *, const int32_t *, int64_t, cudaStream_t);
template int cg_gather<float>(float *, const float *, const int32_t *, int64_t, cudaStream_t);
template int cg_node_sum<double>(double *, const double *, const int32_t *, const int32_t *, int64_t, cudaStream_t);
template int cg_node_sum<float>(float *, const float *, const int32_t *, const int32_t *, int64_t, cudaStream_t);

// ------------------------------------------------------------------------------------------
// Solvers
// ------------------------------------------------------------------------------------------
namespace {

struct SolveCtx {
  uf_operator *op;
  cudaStream_t s;
  int64_t n;
  double *dot_part;        // [2 * kDotBlocks]
  double *dot_out;         // [2] device
  double *dot_host;        // [2] pinned host
  PcgScalars *sc;          // device
  PcgScalars *sc_host;     // pinned host
};

// pcg's operator code for the split FP32 operator (rows of cut and ghost-penalty cells in FP64).
constexpr int kSplitPrecision = 3;

// Iterations enqueued between two reads of the stopping state.  The kernels of iterations
// after the stop are no-ops except the operator's own, so at most kChunk - 1 vmults are spent
// past convergence while the host never waits inside a chunk.
constexpr int kChunk = 32;

// One FP64 dot product (two fixed-order reduction passes), read back synchronously.
template <typename T>
uf_status host_dot(SolveCtx &c, const T *a, const T *b, double &ab) {
  k_dot_partial<T><<<kDotBlocks, kDotThreads, 0, c.s>>>(a, b, c.n, c.dot_part, 0);
  k_dot_final<<<1, kDotThreads, 0, c.s>>>(c.dot_part, c.dot_out);
  cudaError_t err = cudaMemcpyAsync(c.dot_host, c.dot_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(c.s);
  if (err != cudaSuccess) return fail(UF_ECUDA, std::string("reduction: ") + cudaGetErrorString(err));
  ab = c.dot_host[0];
  return UF_OK;
}

// Jacobi-preconditioned CG on A x = r (x starts at zero, r is overwritten by the residual) until
// ||r|| <= rtol ||r_0|| or `maxit` iterations; *its = iterations done, *rel = ||r|| / ||r_0|| of
// the recursive residual.  alpha, beta and the dot products stay on the device (PcgScalars).
template <typename T>
uf_status pcg(SolveCtx &c, int precision, const T *invd, T *x, T *r, T *z, T *p, T *q, double rtol,
              int maxit, int *its, double *rel) {
  const int64_t n = c.n;
  k_fill<T><<<nblk(n), 256, 0, c.s>>>(x, T(0), n);
  k_jacobi<T><<<nblk(n), 256, 0, c.s>>>(z, r, invd, n);
  cudaMemcpyAsync(p, z, n * sizeof(T), cudaMemcpyDeviceToDevice, c.s);
  k_dot_partial<T><<<kDotBlocks, kDotThreads, 0, c.s>>>(r, z, n, c.dot_part, 1);
  k_pcg_init_final<<<1, kDotThreads, 0, c.s>>>(c.dot_part, c.sc, rtol);
  *its = 0;
  *rel = 1.0;
  double rr0 = 0.0;
  bool started = false;  // the first pass only reads the state after the start
  for (int launched = 0;;) {
    const int chunk = started ? std::min(kChunk, maxit - launched) : 0;
    for (int i = 0; i < chunk; ++i) {
      uf_status st;
      if constexpr (std::is_same<T, float>::value) {
        st = precision == kSplitPrecision ? vmult_split(c.op, q, p, c.s)
                                          : vmult_launch(c.op, precision, q, p, c.s, false);
      } else {
        st = vmult_launch(c.op, precision, q, p, c.s, false);
      }
      if (st != UF_OK) return st;
      k_pcg_pq<T><<<kDotBlocks, kDotThreads, 0, c.s>>>(p, q, n, c.dot_part, c.sc);
      k_pcg_alpha<<<1, kDotThreads, 0, c.s>>>(c.dot_part, c.sc);
      k_pcg_update<T><<<kDotBlocks, kDotThreads, 0, c.s>>>(x, r, z, p, q, invd, n, c.dot_part, c.sc);
      k_pcg_beta<<<1, kDotThreads, 0, c.s>>>(c.dot_part, c.sc);
      k_pcg_direction<T><<<nblk(std::max<int64_t>(n / Pack<T>::V, 1)), 256, 0, c.s>>>(p, z, n, c.sc);
    }
    launched += chunk;
    cudaError_t err = cudaMemcpyAsync(c.sc_host, c.sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, c.s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(c.s);
    if (err != cudaSuccess) return fail(UF_ECUDA, std::string("PCG: ") + cudaGetErrorString(err));
    const PcgScalars &h = *c.sc_host;
    if (!started) rr0 = h.rr;
    started = true;
    *its = h.its;
    *rel = rr0 > 0.0 ? std::sqrt(h.rr / rr0) : 0.0;
    if (h.status == 2) return fail(UF_EINVAL, "CG breakdown: the operator is not positive definite");
    if (h.status == 1 || launched >= maxit) break;
  }
  return UF_OK;
}

}  // namespace
}  // namespace uf

using uf::fail;

extern "C" uf_status uf_solve(uf_operator *op, const uf_solve_params *prm, double *x, const double *b,
                              uf_solve_stats *stats, void *stream) {
  if (!op || !prm || !x || !b || !stats) return fail(UF_EINVAL, "NULL argument");
  if (op->device < 0) return fail(UF_ENODEVICE, "operator was created host-only");
  if (!op->host.cg && !op->cgs.ready) {
    // discontinuous operators: Jacobi diagonal and work vectors on the first solve
    uf::DeviceGuard g0(op->device);
    uf::dg_host_diagonal(op->host);
    const uf_status st0 = uf::cg_alloc(op);
    if (st0 != UF_OK) {
      uf::cg_free(op);
      return st0;
    }
  }
  if (!op->cgs.ready) return fail(UF_EINVAL, "the solver's work vectors are missing");
  if (prm->mode != UF_SOLVE_FP64 && prm->mode != UF_SOLVE_IR && prm->mode != UF_SOLVE_IR_SPLIT)
    return fail(UF_EINVAL, "bad solve mode");
  if (prm->mode != UF_SOLVE_FP64 && !op->f32.present) return fail(UF_EINVAL, "IR needs the FP32 operator");
  if (!op->f64.present) return fail(UF_EINVAL, "uf_solve needs the FP64 operator");
  if (!(prm->tol > 0.0) || prm->max_iter < 1) return fail(UF_EINVAL, "bad tolerance or iteration cap");
  uf::DeviceGuard guard(op->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = uf::solve_size(op->host);
  uf::CgSolveData &w = op->cgs;
  uf::SolveCtx c{op, s, n, w.dot_part, w.dot_out, w.dot_host, w.sc, w.sc_host};
  std::memset(stats, 0, sizeof(*stats));
  if (prm->mode == UF_SOLVE_IR_SPLIT) {
    const uf_status s0 = uf::split_cells_alloc(op);
    if (s0 != UF_OK) return s0;
  }
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventRecord(t0, s);
  uf_status st = UF_OK;
  double bb = 0.0;
  st = uf::host_dot<double>(c, b, b, bb);
  const double bnorm = std::sqrt(bb);
  auto residual64 = [&]() -> uf_status {  // r64 = b - A x (FP64)
    uf_status s2 = uf::vmult_launch(op, UF_FP64, w.q64, x, s, false);
    if (s2 != UF_OK) return s2;
    uf::k_residual<<<uf::nblk(n), 256, 0, s>>>(w.r64, b, w.q64, n);
    return UF_OK;
  };
  const bool ir = prm->mode == UF_SOLVE_IR || prm->mode == UF_SOLVE_IR_SPLIT;
  const int inner_op = prm->mode == UF_SOLVE_IR_SPLIT ? uf::kSplitPrecision : UF_FP32;
  int total_it = 0, outer = 0;
  double rel = 1.0;
  if (st == UF_OK && bnorm == 0.0) {
    uf::k_fill<double><<<uf::nblk(n), 256, 0, s>>>(x, 0.0, n);
    rel = 0.0;
  } else if (st == UF_OK) {
    // Correction steps on the FP64 residual r = b - A x:
    //   FP64 mode: PCG in FP64 on A d = r to the remaining reduction tol ||b|| / ||r||, x += d;
    //     it is repeated (restarted CG) while the recursive residual of the PCG has drifted
    //     from the true one, so both modes stop on the same true FP64 residual;
    //   IR mode: PCG in FP32 on A d = r / ||r|| to inner_tol, x += ||r|| d.
    st = residual64();
    for (outer = 0; st == UF_OK && outer < std::max(prm->max_outer, 1); ++outer) {
      double rr = 0.0;
      st = uf::host_dot<double>(c, w.r64, w.r64, rr);
      if (st != UF_OK) break;
      const double rn = std::sqrt(rr);
      rel = rn / bnorm;
      if (rel <= prm->tol || total_it >= prm->max_iter) break;
      int its = 0;
      double rel_in = 1.0;
      if (ir) {
        uf::k_scale_to_f32<<<uf::nblk(n), 256, 0, s>>>(w.r32, w.r64, 1.0 / rn, n);
        st = uf::pcg<float>(c, inner_op, w.invd32, w.d32, w.r32, w.z32, w.p32, w.q32,
                            prm->inner_tol > 0.0 ? prm->inner_tol : 1e-4, prm->max_iter - total_it,
                            &its, &rel_in);
        if (st != UF_OK) break;
        uf::k_refine<<<uf::nblk(n), 256, 0, s>>>(x, w.d32, rn, n);
      } else {
        st = uf::pcg<double>(c, UF_FP64, w.invd64, w.d64, w.r64, w.z64, w.p64, w.q64,
                             prm->tol * bnorm / rn, prm->max_iter - total_it, &its, &rel_in);
        if (st != UF_OK) break;
        uf::k_add<<<uf::nblk(n), 256, 0, s>>>(x, w.d64, n);
      }
      total_it += its;
      st = residual64();
    }
  }
  cudaEventRecord(t1, s);
  cudaEventSynchronize(t1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, t0, t1);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  stats->iterations = total_it;
  stats->outer = outer;
  stats->rel_residual = rel;
  stats->converged = (st == UF_OK && rel <= prm->tol) ? 1 : 0;
  stats->seconds = ms * 1e-3;
  return st;
}

namespace uf {

int64_t solve_size(const HostOperator &h) { return h.cg ? h.n_cg : h.n_active * h.ndof; }

uf_status cg_alloc(uf_operator *op) {
  CgSolveData &w = op->cgs;
  const int64_t n = solve_size(op->host);
  cudaError_t err = cudaSuccess;
  auto A = [&](void **p, size_t bytes) {
    if (err == cudaSuccess) err = uf::dev_malloc(p, bytes);
  };
  if (op->f64.present) {
    A((void **)&w.r64, n * 8);
    A((void **)&w.q64, n * 8);
    A((void **)&w.d64, n * 8);
    A((void **)&w.z64, n * 8);
    A((void **)&w.p64, n * 8);
    A((void **)&w.invd64, n * 8);
  }
  if (op->f32.present) {
    A((void **)&w.r32, n * 4);
    A((void **)&w.q32, n * 4);
    A((void **)&w.d32, n * 4);
    A((void **)&w.z32, n * 4);
    A((void **)&w.p32, n * 4);
    A((void **)&w.invd32, n * 4);
  }
  A((void **)&w.dot_part, 2 * kDotBlocks * sizeof(double));
  A((void **)&w.dot_out, 2 * sizeof(double));
  A((void **)&w.sc, sizeof(PcgScalars));
  if (err == cudaSuccess) err = uf::pinned_malloc((void **)&w.dot_host, 2 * sizeof(double));
  if (err == cudaSuccess) err = uf::pinned_malloc((void **)&w.sc_host, sizeof(PcgScalars));
  if (err != cudaSuccess) return fail(UF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(err));
  return cg_upload_diag(op);
}

uf_status split_cells_alloc(uf_operator *op) {
  CgSolveData &w = op->cgs;
  if (w.split_built) return UF_OK;
  const HostOperator &H = op->host;
  const int nf = 2 * H.dim;
  // T: the cut cells whose volume fraction |K cap Omega| / h^d is below the split fraction (all
  // cut cells for a fraction >= 1); the split cells are T and their active face neighbours,
  // whose rows hold the ghost-penalty couplings to T
  const double theta = op->split_fraction, hd = std::pow(H.h, H.dim);
  std::vector<char> in_split(H.n_active, 0), in_halo(H.n_active, 0);
  for (int64_t c = 0; c < H.n_cut; ++c) {
    double vol = 0.0;
    for (int64_t p = H.vol_off[c]; p < H.vol_off[c + 1]; ++p) vol += H.vol_w[p];
    if (theta < 1.0 && !(vol < theta * hd)) continue;
    const int32_t e = H.cut_cells[c];
    in_split[e] = 1;
    for (int f = 0; f < nf; ++f) {
      const int32_t nb = H.nbr[(size_t)e * nf + f];
      if (nb >= 0) in_split[nb] = 1;
    }
  }
  std::vector<int32_t> cells, halo, scut[3], sidx[3];
  for (int64_t e = 0; e < H.n_active; ++e)
    if (in_split[e]) {
      cells.push_back((int32_t)e);
      in_halo[e] = 1;
      for (int f = 0; f < nf; ++f) {
        const int32_t nb = H.nbr[(size_t)e * nf + f];
        if (nb >= 0) in_halo[nb] = 1;
      }
      const int32_t c = H.cut_of[e];
      if (c >= 0) {
        // the cut cells among the split cells, by lane class as in the full cut-cell list
        const int l = cut_lanes_of_cell(H, c), k = l == 32 ? 0 : (l == 16 ? 1 : 2);
        scut[k].push_back((int32_t)e);
        sidx[k].push_back(c);
      }
    }
  for (int64_t e = 0; e < H.n_active; ++e)
    if (in_halo[e]) halo.push_back((int32_t)e);
  std::vector<int32_t> all(cells);
  all.insert(all.end(), halo.begin(), halo.end());
  const size_t o_cut = all.size();
  for (int k = 0; k < 3; ++k) all.insert(all.end(), scut[k].begin(), scut[k].end());
  const size_t o_idx = all.size();
  for (int k = 0; k < 3; ++k) all.insert(all.end(), sidx[k].begin(), sidx[k].end());
  if (!all.empty()) {
    cudaError_t err = uf::dev_malloc((void **)&w.split_cells, all.size() * sizeof(int32_t));
    if (err == cudaSuccess)
      err = cudaMemcpy(w.split_cells, all.data(), all.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return fail(UF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(err));
  }
  w.n_split = (int64_t)cells.size();
  w.halo_cells = w.split_cells + cells.size();
  w.n_halo = (int64_t)halo.size();
  w.split_cut_list = w.split_cells + o_cut;
  w.split_cut_idx = w.split_cells + o_idx;
  w.split_cut_class[0] = (int32_t)scut[0].size();
  w.split_cut_class[1] = w.split_cut_class[0] + (int32_t)scut[1].size();
  w.split_cut_class[2] = w.split_cut_class[1] + (int32_t)scut[2].size();
  w.split_built = true;
  return UF_OK;
}

void split_cells_free(uf_operator *op) {
  CgSolveData &w = op->cgs;
  if (w.split_cells) uf::dev_free(w.split_cells);
  w.split_cells = w.halo_cells = w.split_cut_list = w.split_cut_idx = nullptr;
  w.n_split = w.n_halo = 0;
  w.split_cut_class[0] = w.split_cut_class[1] = w.split_cut_class[2] = 0;
  w.split_built = false;
}

uf_status cg_upload_diag(uf_operator *op) {
  CgSolveData &w = op->cgs;
  const int64_t n = solve_size(op->host);
  const std::vector<double> &diag = op->host.cg ? op->host.cg_diag : op->host.dg_diag;
  std::vector<double> inv(n);
  for (int64_t i = 0; i < n; ++i) inv[i] = 1.0 / diag[i];
  cudaError_t err = cudaSuccess;
  if (w.invd64) err = cudaMemcpy(w.invd64, inv.data(), n * 8, cudaMemcpyHostToDevice);
  if (err == cudaSuccess && w.invd32) {
    std::vector<float> inv32(inv.begin(), inv.end());
    err = cudaMemcpy(w.invd32, inv32.data(), n * 4, cudaMemcpyHostToDevice);
  }
  if (err != cudaSuccess) return fail(UF_ECUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(err));
  w.ready = true;
  return UF_OK;
}

void cg_free(uf_operator *op) {
  CgSolveData &w = op->cgs;
  void *ptrs[] = {w.r64, w.q64, w.d64, w.z64, w.p64, w.invd64, w.r32, w.q32, w.d32,
                  w.z32, w.p32, w.invd32, w.dot_part, w.dot_out, w.sc, w.split_cells};
  for (void *p : ptrs)
    if (p) uf::dev_free(p);
  if (w.dot_host) uf::pinned_free(w.dot_host);
  if (w.sc_host) uf::pinned_free(w.sc_host);
  w = CgSolveData{};
}

}  // namespace uf
