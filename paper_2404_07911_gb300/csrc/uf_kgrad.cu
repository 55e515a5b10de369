// Gradient of r^T A(kappa) x with respect to the per-cell coefficient kappa (FP64).
//
// A(kappa) = sum_K kappa_K A_K (every term of the form is linear in kappa), so
// dk_K = r^T A_K x = sum over row blocks R of r_R^T (d y_R / d kappa_K).  Each cell e computes
// for its own rows the parts that multiply kappa_e (slot 0) and the kappa of its neighbour across
// face f (slot 1 + f) and dots them with r_e, with the quadrature-point values recomputed from x
// and r (nothing is stored by the forward product).  A gather adds, for cell K, its own slot 0 and
// slot 1 + f' of every neighbour (f' = the neighbour's face toward K).  No atomics: the partials
// of one cell are written by one thread block, the gather reads them after the kernels finish.
//
//  * structured terms: r_e^T (L (x) M (x) M) u = (M_b M_c r_e)^T (L along a) u, so r is swept by
//    the 1D mass once per axis and each coupling contributes a line dot product;
//  * cut cells: volume, Nitsche and cut-face integrands evaluated at the dimension-reduction
//    points from the line contractions of both r and x (no integration back).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "uf_kernels.cuh"
#include "uf_operator.h"

namespace uf {
namespace {

// Offsets (in N*N matrices) of the kappa-derivative 1D matrices in the device table:
//  kself[32]  d(self matrix)/d kappa_e, same variant index as lself (inside | full_lo << 1 | ...)
//  knb[8]     d(neighbour coupling)/d kappa_e, index (2 s + full) * 2 + gp
//  nself[8]   d(self matrix)/d kappa_nb(s)
//  nnb[8]     d(neighbour coupling)/d kappa_nb(s)
constexpr int kKself = 0, kKnb = 32, kNself = 40, kNnb = 48, kKgMats = 56;

__device__ __forceinline__ int face_index(bool full, bool gp, int s) {
  return (2 * s + (full ? 1 : 0)) * 2 + (gp ? 1 : 0);
}

template <int DIM, int N>
__host__ __device__ constexpr int kg_cells_per_block() {
  constexpr int NL = (DIM == 2) ? N : N * N;
  return (NL >= 128) ? 1 : (128 / NL);
}

template <int DIM, int N>
struct KgSmem {
  static constexpr int ND = Geo<DIM, N>::ND, NL = Geo<DIM, N>::NL, NF = Geo<DIM, N>::NF;
  static constexpr int CPB = kg_cells_per_block<DIM, N>();
  static constexpr int cell = ND * (4 + DIM) + NL * (1 + NF);  // doubles per cell
  static constexpr size_t bytes = (size_t)CPB * cell * sizeof(double);
};

template <int N>
__device__ __forceinline__ double dot_apply(const double *__restrict__ L, const double *u,
                                            const double *rt) {
  double acc = 0.0;
#pragma unroll
  for (int r = 0; r < N; ++r) {
    double t = 0.0;
#pragma unroll
    for (int m = 0; m < N; ++m) t = fma(__ldg(L + r * N + m), u[m], t);
    acc = fma(rt[r], t, acc);
  }
  return acc;
}

template <int N>
__device__ __forceinline__ void mass_sweep(const double *M, const double *src, double *dst,
                                           int base, int st) {
  double a[N];
#pragma unroll
  for (int m = 0; m < N; ++m) a[m] = src[base + m * st];
#pragma unroll
  for (int r = 0; r < N; ++r) {
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < N; ++m) acc = fma(M[r * N + m], a[m], acc);
    dst[base + r * st] = acc;
  }
}

template <int DIM, int N>
__global__ void __launch_bounds__(128) kgrad_struct_kernel(const double *__restrict__ kg,
                                                           const __grid_constant__ StructTables<double, N> tab,
                                                           const DevArrays<double> d,
                                                           const Scalars<double> sc,
                                                           double *__restrict__ S,
                                                           const double *__restrict__ r,
                                                           const double *__restrict__ x) {
  using G = Geo<DIM, N>;
  using SM = KgSmem<DIM, N>;
  constexpr int ND = G::ND, NL = G::NL, NF = G::NF, NN = N * N;
  constexpr int CPB = SM::CPB, TPC = NL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *sm = reinterpret_cast<double *>(smem_raw);

  const int tid = threadIdx.x;
  const int first = blockIdx.x * CPB;
  const int c = tid / TPC, t = tid % TPC;
  const bool active_thread = c < CPB;
  const int e = first + c;
  const bool has_cell = active_thread && e < d.n_active;
  double *cs = sm + (active_thread ? c : 0) * SM::cell;
  double *s_x = cs, *s_r = cs + ND, *s_t1 = cs + 2 * ND, *s_t2 = cs + 3 * ND;
  double *s_rt = cs + 4 * ND;  // [DIM][ND]
  double *s_part = cs + (4 + DIM) * ND;  // [TPC][1 + NF]
  const double *M = kg + kKgMats * NN;

  if (has_cell)
    for (int i = t; i < ND; i += TPC) {
      s_x[i] = __ldg(x + (size_t)e * ND + i);
      s_r[i] = __ldg(r + (size_t)e * ND + i);
    }
  __syncthreads();
  // r swept by the mass along the other axes: rt_a = (prod_{b != a} M_b) r
  if (has_cell) {
    if constexpr (DIM == 3) {
      mass_sweep<N>(M, s_r, s_t1, line_base<DIM, N>(2, t), N * N);  // t1 = M_z r
      mass_sweep<N>(M, s_r, s_t2, line_base<DIM, N>(1, t), N);      // t2 = M_y r
    } else {
      mass_sweep<N>(M, s_r, s_rt, line_base<DIM, N>(1, t), N);       // rt_x = M_y r
      mass_sweep<N>(M, s_r, s_rt + ND, line_base<DIM, N>(0, t), 1);  // rt_y = M_x r
    }
  }
  __syncthreads();
  if constexpr (DIM == 3) {
    if (has_cell) {
      mass_sweep<N>(M, s_t1, s_rt, line_base<DIM, N>(1, t), N);           // rt_x = M_y M_z r
      mass_sweep<N>(M, s_t1, s_rt + ND, line_base<DIM, N>(0, t), 1);      // rt_y = M_x M_z r
      mass_sweep<N>(M, s_t2, s_rt + 2 * ND, line_base<DIM, N>(0, t), 1);  // rt_z = M_x M_y r
    }
    __syncthreads();
  }

  double p[1 + NF];
#pragma unroll
  for (int k = 0; k <= NF; ++k) p[k] = 0.0;
  if (has_cell) {
    const uint32_t fl = __ldg(d.flags + e);
    const bool inside = !(fl & 1u);
#pragma unroll 1
    for (int a = 0; a < DIM; ++a) {
      const int base = line_base<DIM, N>(a, t);
      const int st = stride_of<N>(a);
      double u[N], rt[N];
#pragma unroll
      for (int m = 0; m < N; ++m) {
        u[m] = s_x[base + m * st];
        rt[m] = s_rt[a * ND + base + m * st];
      }
      int v = inside ? 1 : 0;
      v |= bit(fl, bit_full(2 * a)) ? 2 : 0;
      v |= bit(fl, bit_gp(2 * a)) ? 4 : 0;
      v |= bit(fl, bit_full(2 * a + 1)) ? 8 : 0;
      v |= bit(fl, bit_gp(2 * a + 1)) ? 16 : 0;
      p[0] += dot_apply<N>(kg + (kKself + v) * NN, u, rt);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int f = 2 * a + s;
        const int nb = __ldg(d.nbr + (size_t)e * NF + f);
        if (nb < 0) continue;
        const bool full = bit(fl, bit_full(f)), gp = bit(fl, bit_gp(f));
        if (!full && !gp) continue;
        double un[N];
        const double *xn = x + (size_t)nb * ND + base;
#pragma unroll
        for (int m = 0; m < N; ++m) un[m] = __ldg(xn + m * st);
        if (gp) {
          const int fi = face_index(full, gp, s);
          p[0] += dot_apply<N>(kg + (kKnb + fi) * NN, un, rt);
          p[1 + f] += dot_apply<N>(kg + (kNself + fi) * NN, u, rt) +
                      dot_apply<N>(kg + (kNnb + fi) * NN, un, rt);
        } else {
          // SIPG only: the couplings are rank 2 (Lobatto delta property, as in the operator).
          // The neighbour's line enters through its face value alpha and the derivative
          // beta = dnb . un; d/dkappa_e of the coupling is alpha dow - (1/2) hf_sigma alpha e_own,
          // d/dkappa_nb of it is -(beta + (1/2) hf_sigma alpha) e_own, and the neighbour's share
          // of the own-own penalty adds (1/2) hf_sigma u_own e_own
          const double alpha = un[s ? 0 : N - 1];
          const double rto = rt[s ? N - 1 : 0], uo = u[s ? N - 1 : 0];
          double beta = 0.0, rdow = 0.0;
#pragma unroll
          for (int m = 0; m < N; ++m) {
            beta = fma(tab.dnb[s][m], un[m], beta);
            rdow = fma(tab.dowx[s][m], rt[m], rdow);
          }
          const double hs = 0.5 * sc.hf_sigma;
          p[0] += alpha * (rdow - hs * rto);
          p[1 + f] += rto * (hs * (uo - alpha) - beta);
        }
      }
    }
#pragma unroll
    for (int k = 0; k <= NF; ++k) s_part[t * (1 + NF) + k] = p[k];
  }
  __syncthreads();
  // thread k of the cell sums slot k over the cell's lines (the same order as one thread would)
  if (has_cell)
    for (int k = t; k <= NF; k += TPC) {
      double acc = 0.0;
      for (int q = 0; q < TPC; ++q) acc += s_part[q * (1 + NF) + k];
      S[(size_t)e * (1 + NF) + k] = acc;
    }
}

// Volume and surface integrands of r^T (dA/dkappa_K) x on a 3D cut cell, with the two-level line
// groups of the cut-cell rule (as in the operator's cut-cell kernel): per chunk of 32 lines, the
// contraction of x and r along each group's shared outer axis (2 n^3 FMA per field and group),
// then per line along its own outer axis (3 n^2 per field), then the points on the line.
template <int N>
__device__ __forceinline__ void kgrad_volume_grouped(const PointTables<double, N> &pt,
                                                     const DevArrays<double> &d,
                                                     const Scalars<double> &sc, int ci, int lane,
                                                     const double *s_x, const double *s_r,
                                                     double &p_self) {
  constexpr int NL = N * N, GMAX = 16;
  __shared__ double s_p[4][GMAX][NL];  // P0 x, P1 x, P0 r, P1 r per group
  __shared__ double s_gcv[GMAX][N], s_gcd[GMAX][N];
  __shared__ int s_gax[GMAX];
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
      const int line = l0 + lane;
      const bool in_range = lane < min(32, lend - l0);
      const int gword = in_range ? __ldg(d.vline_grp + line) : 0;
      const int shared_lo = gword & 1;  // the group shares the coordinate along ob
      const bool start0 = in_range && (lane == 0 || (gword >> 1) == line);
      const unsigned starts0 = __ballot_sync(0xffffffffu, start0);
      const int gl = __popc(starts0 & ((2u << lane) - 1u)) - 1;
      const unsigned over = __ballot_sync(0xffffffffu, start0 && gl >= GMAX);
      nl = over ? (__ffs(over) - 1) : min(32, lend - l0);
      const bool act = lane < nl;
      const int ng = __popc(starts0 & ((nl >= 32) ? 0xffffffffu : ((1u << nl) - 1u)));
      if (start0 && act) {
        s_gax[gl] = shared_lo;
        const double *bp = d.vline_b + (size_t)line * 4 * N + (shared_lo ? 0 : 2 * N);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          s_gcv[gl][i] = __ldg(bp + i);
          s_gcd[gl][i] = __ldg(bp + N + i);
        }
      }
      __syncwarp();
      for (int item = lane; item < ng * NL; item += 32) {
        const int g = item / NL, rr = item % NL, ib = rr / N, m = rr % N;
        const int lo = s_gax[g];
        const int sb = lo ? soc : sob, scs = lo ? sob : soc;
        double px0 = 0.0, px1 = 0.0, pr0 = 0.0, pr1 = 0.0;
#pragma unroll
        for (int ic = 0; ic < N; ++ic) {
          const int idx = ib * sb + ic * scs + m * sk;
          px0 = fma(s_gcv[g][ic], s_x[idx], px0);
          px1 = fma(s_gcd[g][ic], s_x[idx], px1);
          pr0 = fma(s_gcv[g][ic], s_r[idx], pr0);
          pr1 = fma(s_gcd[g][ic], s_r[idx], pr1);
        }
        s_p[0][g][rr] = px0;
        s_p[1][g][rr] = px1;
        s_p[2][g][rr] = pr0;
        s_p[3][g][rr] = pr1;
      }
      __syncwarp();
      if (act) {
        const int ab = shared_lo ? oc : ob, ac = shared_lo ? ob : oc;
        double vb[N], db[N];
        const double *bp = d.vline_b + (size_t)line * 4 * N + (shared_lo ? 2 * N : 0);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          vb[i] = __ldg(bp + i);
          db[i] = __ldg(bp + N + i);
        }
        // w[0] value, w[1] derivative along the own outer axis ab, w[2] along the shared one ac
        double wx[3][N], wr[3][N];
#pragma unroll
        for (int m = 0; m < N; ++m) {
          double a0 = 0.0, a1 = 0.0, a2 = 0.0, b0 = 0.0, b1 = 0.0, b2 = 0.0;
#pragma unroll
          for (int ib = 0; ib < N; ++ib) {
            const double qx = s_p[0][gl][ib * N + m], qr = s_p[2][gl][ib * N + m];
            a0 = fma(vb[ib], qx, a0);
            a1 = fma(db[ib], qx, a1);
            a2 = fma(vb[ib], s_p[1][gl][ib * N + m], a2);
            b0 = fma(vb[ib], qr, b0);
            b1 = fma(db[ib], qr, b1);
            b2 = fma(vb[ib], s_p[3][gl][ib * N + m], b2);
          }
          wx[0][m] = a0;
          wx[1][m] = a1;
          wx[2][m] = a2;
          wr[0][m] = b0;
          wr[1][m] = b1;
          wr[2][m] = b2;
        }
        // the line's volume points through its integrals K_l, M_l (h^{-2} folded in):
        // sum_p w_p grad r . grad x / h^2 = wr0 . K_l wx0 + wr1 . M_l wx1 + wr2 . M_l wx2
        {
          const double *km = d.vline_km + (size_t)line * 2 * N * N;
          double acc = 0.0;
#pragma unroll
          for (int q = 0; q < N; ++q) {
            double kr[N], mr[N];
            load_row<double, N>(km + q * N, kr);
            load_row<double, N>(km + N * N + q * N, mr);
            double t0 = 0.0, t1 = 0.0;
#pragma unroll
            for (int m = 0; m < N; ++m) {
              t0 = fma(kr[m], wx[0][m], t0);
              t1 = fma(mr[m], wx[1][m], t1);
            }
            double t2 = 0.0;
#pragma unroll
            for (int m = 0; m < N; ++m) t2 = fma(mr[m], wx[2][m], t2);
            acc = fma(wr[0][q], t0, fma(wr[1][q], t1, fma(wr[2][q], t2, acc)));
          }
          p_self += acc;
        }
        const int sp = __ldg(d.lsurf + line);
        if (sp >= 0) {
          double cv[N], cd[N];
          point_basis<double, N>(pt, d.spt_b, d.spt_t, sp, cv, cd);
          double ux = 0.0, ur = 0.0, gx[3] = {0, 0, 0}, gr[3] = {0, 0, 0};
#pragma unroll
          for (int m = 0; m < N; ++m) {
            ux = fma(cv[m], wx[0][m], ux);
            ur = fma(cv[m], wr[0][m], ur);
            gx[0] = fma(cd[m], wx[0][m], gx[0]);
            gx[1] = fma(cv[m], wx[1][m], gx[1]);
            gx[2] = fma(cv[m], wx[2][m], gx[2]);
            gr[0] = fma(cd[m], wr[0][m], gr[0]);
            gr[1] = fma(cv[m], wr[1][m], gr[1]);
            gr[2] = fma(cv[m], wr[2][m], gr[2]);
          }
          const double nk = __ldg(d.spt_n[k] + sp), nb = __ldg(d.spt_n[ab] + sp);
          const double nc = __ldg(d.spt_n[ac] + sp);
          const double dnx = (nk * gx[0] + nb * gx[1] + nc * gx[2]) * sc.inv_h;
          const double dnr = (nk * gr[0] + nb * gr[1] + nc * gr[2]) * sc.inv_h;
          p_self += __ldg(d.spt_w + sp) * (-dnr * ux - ur * dnx + sc.nitsche_over_h * ur * ux);
        }
      }
      __syncwarp();
    }
  }
}

// Cut cells: one warp per cut cell, adds its unstructured partials to S.
template <int DIM, int N>
__global__ void __launch_bounds__(32) kgrad_cut_kernel(const __grid_constant__ PointTables<double, N> pt,
                                                       const DevArrays<double> d,
                                                       const Scalars<double> sc,
                                                       double *__restrict__ S,
                                                       const double *__restrict__ r,
                                                       const double *__restrict__ x) {
  using G = Geo<DIM, N>;
  constexpr int ND = G::ND, NL = G::NL, NF = G::NF;
  __shared__ double s_x[ND], s_r[ND];
  __shared__ double s_tr[NF][6][NL];
  const int lane = threadIdx.x;
  const int slot = blockIdx.x;
  if (slot >= d.n_cut) return;
  const int e = __ldg(d.cut_list + slot);
  const int ci = __ldg(d.cut_idx + slot);
  const uint32_t fl = __ldg(d.flags + e);
  for (int i = lane; i < ND; i += 32) {
    s_x[i] = __ldg(x + (size_t)e * ND + i);
    s_r[i] = __ldg(r + (size_t)e * ND + i);
  }
  __syncwarp();
  double p_self = 0.0;
  double p_face[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) p_face[f] = 0.0;

  // volume and surface points
  if constexpr (DIM == 3 && N <= 6) {
    kgrad_volume_grouped<N>(pt, d, sc, ci, lane, s_x, s_r, p_self);
  } else {
    // volume and surface points, line by line
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
      constexpr int NC = (DIM == 3) ? N : 1;
  #pragma unroll 1
      for (int line = lbeg + lane; line < lend; line += 32) {
        double vb[N], db[N], vc[N], dc[N];
        {
          const double *bp = d.vline_b + (size_t)line * 4 * N;  // precomputed at creation (FP64)
  #pragma unroll
          for (int i = 0; i < N; ++i) {
            vb[i] = __ldg(bp + i);
            db[i] = __ldg(bp + N + i);
            if constexpr (DIM == 3) {
              vc[i] = __ldg(bp + 2 * N + i);
              dc[i] = __ldg(bp + 3 * N + i);
            }
          }
        }
        double wx[3][N], wr[3][N];
  #pragma unroll
        for (int m = 0; m < N; ++m)
  #pragma unroll
          for (int q = 0; q < 3; ++q) {
            wx[q][m] = 0.0;
            wr[q][m] = 0.0;
          }
  #pragma unroll
        for (int m = 0; m < N; ++m)
  #pragma unroll
          for (int ic = 0; ic < NC; ++ic) {
            double sx0 = 0.0, sx1 = 0.0, sr0 = 0.0, sr1 = 0.0;
  #pragma unroll
            for (int ib = 0; ib < N; ++ib) {
              const int idx = ib * sb + ic * scc + m * sk;
              sx0 = fma(vb[ib], s_x[idx], sx0);
              sx1 = fma(db[ib], s_x[idx], sx1);
              sr0 = fma(vb[ib], s_r[idx], sr0);
              sr1 = fma(db[ib], s_r[idx], sr1);
            }
            if constexpr (DIM == 3) {
              wx[0][m] = fma(vc[ic], sx0, wx[0][m]);
              wx[1][m] = fma(vc[ic], sx1, wx[1][m]);
              wx[2][m] = fma(dc[ic], sx0, wx[2][m]);
              wr[0][m] = fma(vc[ic], sr0, wr[0][m]);
              wr[1][m] = fma(vc[ic], sr1, wr[1][m]);
              wr[2][m] = fma(dc[ic], sr0, wr[2][m]);
            } else {
              wx[0][m] = sx0;
              wx[1][m] = sx1;
              wr[0][m] = sr0;
              wr[1][m] = sr1;
            }
          }
        const int pb = __ldg(d.vpt_off + line), pe = __ldg(d.vpt_off + line + 1);
  #pragma unroll 1
        for (int p = pb; p < pe; ++p) {
          double cv[N], cd[N];
          point_basis<double, N>(pt, d.vpt_b, d.vpt_t, p, cv, cd);
          double gx[3] = {0, 0, 0}, gr[3] = {0, 0, 0};
  #pragma unroll
          for (int m = 0; m < N; ++m) {
            gx[0] = fma(cd[m], wx[0][m], gx[0]);
            gx[1] = fma(cv[m], wx[1][m], gx[1]);
            gr[0] = fma(cd[m], wr[0][m], gr[0]);
            gr[1] = fma(cv[m], wr[1][m], gr[1]);
            if constexpr (DIM == 3) {
              gx[2] = fma(cv[m], wx[2][m], gx[2]);
              gr[2] = fma(cv[m], wr[2][m], gr[2]);
            }
          }
          p_self += __ldg(d.vpt_w + p) * sc.inv_h2 * (gx[0] * gr[0] + gx[1] * gr[1] + gx[2] * gr[2]);
        }
        const int sp = __ldg(d.lsurf + line);
        if (sp >= 0) {
          double cv[N], cd[N];
          point_basis<double, N>(pt, d.spt_b, d.spt_t, sp, cv, cd);
          double ux = 0.0, ur = 0.0, gx[3] = {0, 0, 0}, gr[3] = {0, 0, 0};
  #pragma unroll
          for (int m = 0; m < N; ++m) {
            ux = fma(cv[m], wx[0][m], ux);
            ur = fma(cv[m], wr[0][m], ur);
            gx[0] = fma(cd[m], wx[0][m], gx[0]);
            gx[1] = fma(cv[m], wx[1][m], gx[1]);
            gr[0] = fma(cd[m], wr[0][m], gr[0]);
            gr[1] = fma(cv[m], wr[1][m], gr[1]);
            if constexpr (DIM == 3) {
              gx[2] = fma(cv[m], wx[2][m], gx[2]);
              gr[2] = fma(cv[m], wr[2][m], gr[2]);
            }
          }
          const double nk = __ldg(d.spt_n[k] + sp), nb = __ldg(d.spt_n[ob] + sp);
          const double nc = (DIM == 3) ? __ldg(d.spt_n[oc] + sp) : 0.0;
          const double dnx = (nk * gx[0] + nb * gx[1] + nc * gx[2]) * sc.inv_h;
          const double dnr = (nk * gr[0] + nb * gr[1] + nc * gr[2]) * sc.inv_h;
          p_self += __ldg(d.spt_w + sp) * (-dnr * ux - ur * dnx + sc.nitsche_over_h * ur * ux);
        }
      }
    }
  }

  // cut faces: traces of r (own) and x (own, neighbour) on every cut face of the cell
  int cfl[NF];
  int ncf = 0;
#pragma unroll
  for (int f = 0; f < NF; ++f)
    if (bit(fl, bit_cut(f))) cfl[ncf++] = f;
  if (ncf > 0) {
    for (int item = lane; item < ncf * NL; item += 32) {
      const int fi = item / NL, tl = item % NL;
      const int f = cfl[fi], axis = f / 2, side = f % 2;
      const int nbe = __ldg(d.nbr + (size_t)e * NF + f);
      const int base = line_base<DIM, N>(axis, tl);
      const int st = stride_of<N>(axis);
      const double *xn = x + (size_t)nbe * ND + base;
      double rv = 0, rd = 0, xv = 0, xd = 0, nv = 0, nd = 0;
#pragma unroll
      for (int m = 0; m < N; ++m) {
        const double ro = s_r[base + m * st], xo = s_x[base + m * st], xb = __ldg(xn + m * st);
        rv = fma(pt.end_val[side][m], ro, rv);
        rd = fma(pt.end_der[side][m], ro, rd);
        xv = fma(pt.end_val[side][m], xo, xv);
        xd = fma(pt.end_der[side][m], xo, xd);
        nv = fma(pt.end_val[1 - side][m], xb, nv);
        nd = fma(pt.end_der[1 - side][m], xb, nd);
      }
      const double sg = (side ? 1.0 : -1.0) * sc.inv_h;
      s_tr[fi][0][tl] = rv;
      s_tr[fi][1][tl] = sg * rd;
      s_tr[fi][2][tl] = xv;
      s_tr[fi][3][tl] = sg * xd;
      s_tr[fi][4][tl] = nv;
      s_tr[fi][5][tl] = sg * nd;
    }
    __syncwarp();
    if constexpr (kFaceMatrices<double, DIM, N>) {
      // every face integrand is a product of two traces, so with the face's mass matrix Mf and
      // a = Mf r, b = Mf dr (J = [x] the jump): the points' sums are a.(sigma/h J / 2 - dx_e / 2)
      // - b.J / 2 (self) and a.(sigma/h J - dx_nb) / 2 (neighbour)
      for (int item = lane; item < ncf * NL; item += 32) {
        const int fi = item / NL, row = item % NL;
        const int f = cfl[fi];
        const double *mf = d.fmat + (size_t)__ldg(d.fmat_idx + (size_t)ci * NF + f) * NL * NL + row;
        double a = 0.0, b = 0.0;
#pragma unroll
        for (int col = 0; col < NL; ++col) {
          const double m = __ldg(mf + col * NL);
          a = fma(m, s_tr[fi][0][col], a);
          b = fma(m, s_tr[fi][1][col], b);
        }
        const double jump = s_tr[fi][2][row] - s_tr[fi][4][row];
        p_self += -0.5 * b * jump - 0.5 * a * s_tr[fi][3][row] + 0.5 * sc.sipg_over_h * a * jump;
        const double pnb = -0.5 * a * s_tr[fi][5][row] + 0.5 * sc.sipg_over_h * a * jump;
#pragma unroll
        for (int j = 0; j < NF; ++j)
          if (j == f) p_face[j] += pnb;
      }
    } else {
      const int *koff_cell = d.fline_koff + (size_t)ci * NF * 3;
      const int fl_beg = __ldg(koff_cell);
      const int fl_end = __ldg(koff_cell + (NF - 1) * 3 + 2);
#pragma unroll 1
      for (int line = fl_beg + lane; line < fl_end; line += 32) {
        int fi = 0, kk = 0;
        for (int j = 0; j < ncf; ++j) {
          const int *ko = koff_cell + cfl[j] * 3;
          if (line >= __ldg(ko) && line < __ldg(ko + 2)) {
            fi = j;
            kk = (line < __ldg(ko + 1)) ? 0 : 1;
          }
        }
        double vo[N];
        if constexpr (DIM == 3)
#pragma unroll
          for (int i = 0; i < N; ++i) vo[i] = __ldg(d.fline_b + (size_t)line * N + i);
        double rr[6][N];
#pragma unroll
        for (int m = 0; m < N; ++m)
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            if constexpr (DIM == 3) {
              double acc = 0.0;
#pragma unroll
              for (int io = 0; io < N; ++io) {
                const int tl = (kk == 0) ? (m + N * io) : (io + N * m);
                acc = fma(vo[io], s_tr[fi][q][tl], acc);
              }
              rr[q][m] = acc;
            } else {
              rr[q][m] = s_tr[fi][q][m];
            }
          }
        double pf_self = 0.0, pf_nb = 0.0;
        const int pb = __ldg(d.fpt_off + line), pe = __ldg(d.fpt_off + line + 1);
#pragma unroll 1
        for (int p = pb; p < pe; ++p) {
          double cv[N];
#pragma unroll
          for (int i = 0; i < N; ++i) cv[i] = __ldg(d.fpt_b + (size_t)p * N + i);
          double ev[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
          for (int m = 0; m < N; ++m)
#pragma unroll
            for (int q = 0; q < 6; ++q) ev[q] = fma(cv[m], rr[q][m], ev[q]);
          const double w = __ldg(d.fpt_w + p);
          const double jump = ev[2] - ev[4];
          // d/dkappa_e:  -1/2 dr J - 1/2 r dx_e + 1/2 sigma/h r J;  d/dkappa_nb: -1/2 r dx_nb + 1/2 sigma/h r J
          pf_self += w * (-0.5 * ev[1] * jump - 0.5 * ev[0] * ev[3] + 0.5 * sc.sipg_over_h * ev[0] * jump);
          pf_nb += w * (-0.5 * ev[0] * ev[5] + 0.5 * sc.sipg_over_h * ev[0] * jump);
        }
        p_self += pf_self;
#pragma unroll
        for (int j = 0; j < NF; ++j)
          if (j == fi) p_face[cfl[j]] += pf_nb;
      }
    }
  }
  // warp reductions, lane 0 adds to the structured partials of this cell
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) p_self += __shfl_xor_sync(0xffffffffu, p_self, off);
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) p_face[f] += __shfl_xor_sync(0xffffffffu, p_face[f], off);
  if (lane == 0) {
    S[(size_t)e * (1 + NF)] += p_self;
#pragma unroll
    for (int f = 0; f < NF; ++f) S[(size_t)e * (1 + NF) + 1 + f] += p_face[f];
  }
}

template <int DIM>
__global__ void kgrad_gather_kernel(const DevArrays<double> d, const double *__restrict__ S,
                                    double *__restrict__ dk) {
  constexpr int NF = 2 * DIM;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_active) return;
  double acc = S[(size_t)e * (1 + NF)];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int nb = __ldg(d.nbr + (size_t)e * NF + f);
    if (nb >= 0) acc += S[(size_t)nb * (1 + NF) + 1 + (f ^ 1)];
  }
  dk[e] = acc;
}

template <int DIM, int N>
int launch_kgrad_t(const double *kg, const DevArrays<double> &d, const void *tables_struct,
                   const void *tables_point, const Scalars<double> &s, double *S, double *dk,
                   const double *r, const double *x, cudaStream_t stream) {
  const auto &tab = *reinterpret_cast<const StructTables<double, N> *>(tables_struct);
  using SM = KgSmem<DIM, N>;
  constexpr int CPB = SM::CPB;
  const int threads = ((CPB * Geo<DIM, N>::NL + 31) / 32) * 32;
  const int blocks = (d.n_active + CPB - 1) / CPB;
  cudaError_t err = cudaSuccess;
  if (SM::bytes > 48 * 1024) {
    err = cudaFuncSetAttribute(kgrad_struct_kernel<DIM, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)SM::bytes);
    if (err != cudaSuccess) return (int)err;
  }
  kgrad_struct_kernel<DIM, N><<<blocks, threads, SM::bytes, stream>>>(kg, tab, d, s, S, r, x);
  if (d.n_cut > 0) {
    const auto &ptab = *reinterpret_cast<const PointTables<double, N> *>(tables_point);
    kgrad_cut_kernel<DIM, N><<<d.n_cut, 32, 0, stream>>>(ptab, d, s, S, r, x);
  }
  kgrad_gather_kernel<DIM><<<(d.n_active + 127) / 128, 128, 0, stream>>>(d, S, dk);
  return (int)cudaGetLastError();
}

int launch_kgrad(int dim, int n, const double *kg, const DevArrays<double> &d, const void *ts,
                 const void *tp, const Scalars<double> &s, double *S, double *dk, const double *r,
                 const double *x, cudaStream_t st) {
#define UF_KCASE(D, NN) \
  if (dim == D && n == NN) return launch_kgrad_t<D, NN>(kg, d, ts, tp, s, S, dk, r, x, st);
  UF_KCASE(2, 2) UF_KCASE(2, 3) UF_KCASE(2, 4) UF_KCASE(2, 5) UF_KCASE(2, 6) UF_KCASE(2, 7)
  UF_KCASE(2, 8) UF_KCASE(2, 9) UF_KCASE(3, 2) UF_KCASE(3, 3) UF_KCASE(3, 4) UF_KCASE(3, 5)
  UF_KCASE(3, 6) UF_KCASE(3, 7) UF_KCASE(3, 8) UF_KCASE(3, 9)
#undef UF_KCASE
  return (int)cudaErrorInvalidValue;
}

__global__ void k_kappa_to_f32(float *dst, const double *src, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

}  // namespace

// kappa-derivative 1D matrices (see the offsets above) and the 1D mass, from the constant
// matrices of the structured terms (layout of StructTables: kv, mass, a, pen, gp, b, c, qn, hn).
void kgrad_tables(int n, const std::vector<double> &m, std::vector<double> &out) {
  const int nn = n * n;
  auto Mx = [&](int which, int s) { return &m[(which + s) * nn]; };
  out.assign((kKgMats + 1) * nn, 0.0);
  for (int v = 0; v < 32; ++v)
    for (int i = 0; i < nn; ++i) {
      double acc = (v & 1) ? m[i] : 0.0;
      for (int s = 0; s < 2; ++s) {
        const bool full = (v >> (1 + 2 * s)) & 1, gp = (v >> (2 + 2 * s)) & 1;
        if (full) acc += Mx(2, s)[i] + 0.5 * Mx(4, s)[i];
        if (gp) acc += 0.5 * Mx(6, s)[i];
      }
      out[(kKself + v) * nn + i] = acc;
    }
  for (int s = 0; s < 2; ++s)
    for (int full = 0; full < 2; ++full)
      for (int gp = 0; gp < 2; ++gp) {
        const int fi = (2 * s + full) * 2 + gp;
        for (int i = 0; i < nn; ++i) {
          out[(kKnb + fi) * nn + i] =
              (full ? Mx(8, s)[i] + 0.5 * Mx(12, s)[i] : 0.0) + (gp ? 0.5 * Mx(14, s)[i] : 0.0);
          out[(kNself + fi) * nn + i] = (full ? 0.5 * Mx(4, s)[i] : 0.0) + (gp ? 0.5 * Mx(6, s)[i] : 0.0);
          out[(kNnb + fi) * nn + i] =
              (full ? Mx(10, s)[i] + 0.5 * Mx(12, s)[i] : 0.0) + (gp ? 0.5 * Mx(14, s)[i] : 0.0);
        }
      }
  for (int i = 0; i < nn; ++i) out[kKgMats * nn + i] = m[nn + i];
}

// ---- fixed partial buffer of uf_kappa_gradient_noalloc ----------------------------------
// 2^20 doubles (8 MiB), resident on every device that loads the library until the process exits.
// One slot per (cell, 1 + 2d): at most 149,796 active cells in 3D, 209,715 in 2D.
constexpr size_t kStaticPartialDoubles = (size_t)1 << 20;
static __device__ __align__(256) double g_kgrad_partials[kStaticPartialDoubles];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_partials_mutex;
double *g_partials_addr[kMaxDevices] = {};  // device address of g_kgrad_partials per device
}  // namespace

// Device address of the fixed buffer on `device` (which must be current).  The host-side name of
// the array is only a stand-in, so the address is looked up once per device and cached.
static uf_status static_partials(int device, double **out) {
  if (device < 0 || device >= kMaxDevices) return fail(UF_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_partials_mutex);
  if (!g_partials_addr[device]) {
    void *addr = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&addr, g_kgrad_partials);
    if (err != cudaSuccess)
      return fail(UF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(err));
    g_partials_addr[device] = static_cast<double *>(addr);
  }
  *out = g_partials_addr[device];
  return UF_OK;
}

}  // namespace uf

using uf::fail;

extern "C" {

uf_status uf_kappa_gradient_noalloc(uf_operator *op, double *dk, const double *r,
                                    const double *x, void *stream) {
  if (!op || !dk || !r || !x) return fail(UF_EINVAL, "NULL argument");
  if (op->device < 0) return fail(UF_ENODEVICE, "operator was created host-only");
  if (!op->f64.present || !op->kg_tables)
    return fail(UF_EINVAL, "the kappa gradient needs the FP64 operator");
  const size_t need = (size_t)op->host.n_active * (1 + 2 * op->host.dim);
  if (need > uf::kStaticPartialDoubles)
    return fail(UF_EINVAL, "operator too large for the fixed partial buffer: " +
                               std::to_string(need) + " doubles needed, " +
                               std::to_string(uf::kStaticPartialDoubles) + " available");
  uf::DeviceGuard guard(op->device);
  double *partials = nullptr;
  uf_status st = uf::static_partials(op->device, &partials);
  if (st != UF_OK) return st;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  const double *rl = r, *xl = x;
  if (op->host.cg) {
    const int64_t n_loc = op->host.n_active * op->host.ndof;
    uf::cg_gather<double>(op->f64.x_loc, x, op->f64.cg_l2g, n_loc, cs);
    uf::cg_gather<double>(op->f64.y_loc, r, op->f64.cg_l2g, n_loc, cs);
    xl = op->f64.x_loc;
    rl = op->f64.y_loc;
  }
  // Every slot the gather reads is written by the structured kernel of this call before any
  // other kernel reads or accumulates into it, so the buffer needs no clearing.
  int err = uf::launch_kgrad(op->host.dim, op->host.n, op->kg_tables, op->f64.arrays,
                             op->f64.struct_tables.data(), op->f64.point_tables.data(), op->f64.scalars, partials, dk, rl, xl, cs);
  if (err != 0)
    return fail(UF_ECUDA, std::string("kernel launch: ") + cudaGetErrorString((cudaError_t)err));
  return UF_OK;
}

uf_status uf_kappa_gradient(uf_operator *op, double *dk, const double *r, const double *x,
                            void *stream) {
  if (!op || !dk || !r || !x) return fail(UF_EINVAL, "NULL argument");
  if (op->device < 0) return fail(UF_ENODEVICE, "operator was created host-only");
  if (!op->f64.present || !op->kg_tables || !op->kg_scratch)
    return fail(UF_EINVAL, "the kappa gradient needs the FP64 operator");
  uf::DeviceGuard guard(op->device);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  const double *rl = r, *xl = x;
  if (op->host.cg) {
    // continuous space: dk_K = (P r)^T A_loc,K (P x) with the cell-local gathers of r and x
    const int64_t n_loc = op->host.n_active * op->host.ndof;
    uf::cg_gather<double>(op->f64.x_loc, x, op->f64.cg_l2g, n_loc, cs);
    uf::cg_gather<double>(op->f64.y_loc, r, op->f64.cg_l2g, n_loc, cs);
    xl = op->f64.x_loc;
    rl = op->f64.y_loc;
  }
  int err = uf::launch_kgrad(op->host.dim, op->host.n, op->kg_tables, op->f64.arrays,
                             op->f64.struct_tables.data(), op->f64.point_tables.data(), op->f64.scalars, op->kg_scratch, dk, rl,
                             xl, cs);
  if (err != 0)
    return fail(UF_ECUDA, std::string("kernel launch: ") + cudaGetErrorString((cudaError_t)err));
  return UF_OK;
}

uf_status uf_set_kappa_device(uf_operator *op, const double *kappa_dev, void *stream) {
  if (!op || !kappa_dev) return fail(UF_EINVAL, "NULL argument");
  if (op->device < 0) return fail(UF_ENODEVICE, "operator was created host-only");
  uf::DeviceGuard guard(op->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int na = (int)op->host.n_active;
  cudaError_t err = cudaSuccess;
  if (op->f64.present) {
    err = cudaMemcpyAsync(op->f64.kappa_dev, kappa_dev, sizeof(double) * na, cudaMemcpyDeviceToDevice, s);
    op->f64.arrays.kappa_uniform = 0;
  }
  if (err == cudaSuccess && op->f32.present) {
    uf::k_kappa_to_f32<<<(na + 255) / 256, 256, 0, s>>>(op->f32.kappa_dev, kappa_dev, na);
    err = cudaGetLastError();
    op->f32.arrays.kappa_uniform = 0;
  }
  if (err != cudaSuccess) return fail(UF_ECUDA, cudaGetErrorString(err));
  return UF_OK;
}

}  // extern "C"
