// Assembled-matrix baseline: the operator as a CSR matrix and its SpMV (arXiv 2404.07911,
// Sec. 3.1: the same element operators give the sparse matrix; Sec. 5.1 models the matrix-based
// evaluation at 12 bytes and 2 FLOPs per nonzero with 32-bit column indices).
//
// Assembly takes the matrix column by column from the matrix-free operator (Sec. 3.1: "local
// matrices ... computed column-by-column by applying I_e B_e E_e on element-wise unit vectors"):
// with a distance-2 colouring of the background cells (colour (i + 2j + 3k) mod 7 in 3D,
// (i + 2j) mod 5 in 2D: any two cells of one colour are more than two face steps apart), the
// vector with a one in local DoF j of every cell of colour c has, in the rows of a cell r, exactly
// the column (s, j) of the one coupled cell s of colour c.  n_colours x n^d operator applications
// fill every block.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "uf_operator.h"

namespace {

constexpr int kMaxCoupled = 8;  // self + 2d face neighbours (d <= 3) + padding

__global__ void k_indicator(double *x, const int8_t *color, int n_active, int nd, int c, int j) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)n_active * nd;
  if (i >= n) return;
  const int64_t e = i / nd;
  const int l = (int)(i % nd);
  x[i] = (l == j && color[e] == c) ? 1.0 : 0.0;
}

// One CTA per cell: tile T[i][j] = ystage[j][r nd + i] (the columns (s, j) of the cell's rows),
// written into the CSR rows of the block of the coupled cell s of colour c.
template <typename T>
__global__ void k_scatter(T *val, const double *ystage, const int64_t *row_ptr,
                          const int32_t *coupled, const int8_t *ncoupled, const int8_t *color,
                          int n_active, int nd, int64_t n_dofs, int c) {
  extern __shared__ double tile[];  // [nd][nd + 1]
  const int r = blockIdx.x;
  if (r >= n_active) return;
  int b = -1;
  for (int q = 0; q < ncoupled[r]; ++q)
    if (color[coupled[r * kMaxCoupled + q]] == c) b = q;
  if (b < 0) return;  // uniform over the block
  for (int idx = threadIdx.x; idx < nd * nd; idx += blockDim.x) {
    const int j = idx / nd, i = idx % nd;  // coalesced along i
    tile[i * (nd + 1) + j] = ystage[(int64_t)j * n_dofs + (int64_t)r * nd + i];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nd * nd; idx += blockDim.x) {
    const int i = idx / nd, j = idx % nd;  // coalesced along j
    val[row_ptr[(int64_t)r * nd + i] + (int64_t)b * nd + j] = (T)tile[i * (nd + 1) + j];
  }
}

__global__ void k_fill_cols(int32_t *col, const int64_t *row_ptr, const int32_t *coupled,
                            const int8_t *ncoupled, int n_active, int nd) {
  const int r = blockIdx.x;
  if (r >= n_active) return;
  const int nc = ncoupled[r];
  for (int idx = threadIdx.x; idx < nd * nc * nd; idx += blockDim.x) {
    const int i = idx / (nc * nd), rem = idx % (nc * nd);
    const int b = rem / nd, j = rem % nd;
    col[row_ptr[(int64_t)r * nd + i] + rem] = coupled[r * kMaxCoupled + b] * nd + j;
  }
}

// y = A x, one warp per row; matrix streamed with evict-first loads, x gathered through L2.
template <typename T>
__global__ void __launch_bounds__(256) k_spmv(T *__restrict__ y, const T *__restrict__ x,
                                              const int64_t *__restrict__ row_ptr,
                                              const int32_t *__restrict__ col,
                                              const T *__restrict__ val, int64_t n_rows) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n_rows) return;
  const int64_t b = row_ptr[row], e = row_ptr[row + 1];
  T acc = T(0);
  for (int64_t k = b + lane; k < e; k += 32) acc = fma(__ldcs(val + k), __ldg(x + __ldcs(col + k)), acc);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) y[row] = acc;
}

}  // namespace

namespace uf {

void release_csr(CsrData &c) {
  if (c.row_ptr) uf::dev_free(c.row_ptr);
  if (c.col) uf::dev_free(c.col);
  if (c.val) uf::dev_free(c.val);
  c = CsrData{};
}

}  // namespace uf

using uf::fail;

extern "C" {

uf_status uf_assemble_csr(uf_operator *op, int precision) {
  if (!op) return fail(UF_EINVAL, "NULL operator");
  if (op->device < 0) return fail(UF_ENODEVICE, "operator was created host-only");
  if (precision != UF_FP64 && precision != UF_FP32) return fail(UF_EINVAL, "bad precision");
  if (!op->f64.present) return fail(UF_EINVAL, "CSR assembly needs the FP64 operator");
  if (op->host.cg) return fail(UF_EUNSUPPORTED, "CSR assembly is built for the DG operator");
  uf::DeviceGuard guard(op->device);
  const uf::HostOperator &H = op->host;
  const int d = H.dim, nf = 2 * d, nd = H.ndof;
  const int64_t na = H.n_active, n = na * nd;
  uf::CsrData &csr = (precision == UF_FP64) ? op->csr64 : op->csr32;
  uf::release_csr(csr);

  // coupled cells of every row block (self and every neighbour with a face term), ascending
  std::vector<int32_t> coupled(na * kMaxCoupled, -1);
  std::vector<int8_t> ncoupled(na), color(na);
  std::vector<int64_t> row_ptr(n + 1);
  int64_t nnz = 0;
  for (int64_t r = 0; r < na; ++r) {
    std::vector<int32_t> list{(int32_t)r};
    for (int f = 0; f < nf; ++f) {
      const uint32_t bits = uf::face_bit_sipg_full(f) | uf::face_bit_sipg_cut(f) | uf::face_bit_gp(f);
      if (H.nbr[r * nf + f] >= 0 && (H.flags[r] & bits)) list.push_back(H.nbr[r * nf + f]);
    }
    std::sort(list.begin(), list.end());
    ncoupled[r] = (int8_t)list.size();
    for (size_t q = 0; q < list.size(); ++q) coupled[r * kMaxCoupled + q] = list[q];
    const int32_t *ix = &H.act_index[r * 3];
    color[r] = (int8_t)((d == 3) ? (ix[0] + 2 * ix[1] + 3 * ix[2]) % 7 : (ix[0] + 2 * ix[1]) % 5);
    for (int i = 0; i < nd; ++i) {
      row_ptr[r * nd + i] = nnz;
      nnz += (int64_t)list.size() * nd;
    }
  }
  row_ptr[n] = nnz;
  const int ncolors = (d == 3) ? 7 : 5;
  const size_t vsize = precision == UF_FP64 ? sizeof(double) : sizeof(float);

  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const size_t need = nnz * (vsize + sizeof(int32_t)) + (n + 1) * sizeof(int64_t) +
                      (size_t)nd * n * sizeof(double) + (size_t)na * (kMaxCoupled * 4 + 2);
  if (need + ((size_t)256 << 20) > free_b)
    return fail(UF_ENOMEM, "not enough device memory for the CSR matrix (" +
                               std::to_string(need >> 20) + " MiB needed)");

  cudaError_t err = cudaSuccess;
  double *ystage = nullptr, *xind = nullptr;
  int32_t *d_coupled = nullptr;
  int8_t *d_ncoupled = nullptr, *d_color = nullptr;
  auto cleanup = [&]() {
    if (ystage) uf::dev_free(ystage);
    if (xind) uf::dev_free(xind);
    if (d_coupled) uf::dev_free(d_coupled);
    if (d_ncoupled) uf::dev_free(d_ncoupled);
    if (d_color) uf::dev_free(d_color);
  };
  err = uf::dev_malloc(&csr.row_ptr, (n + 1) * sizeof(int64_t));
  if (err == cudaSuccess) err = uf::dev_malloc(&csr.col, nnz * sizeof(int32_t));
  if (err == cudaSuccess) err = uf::dev_malloc(&csr.val, nnz * vsize);
  if (err == cudaSuccess) err = uf::dev_malloc(&ystage, (size_t)nd * n * sizeof(double));
  if (err == cudaSuccess) err = uf::dev_malloc(&xind, n * sizeof(double));
  if (err == cudaSuccess) err = uf::dev_malloc(&d_coupled, na * kMaxCoupled * sizeof(int32_t));
  if (err == cudaSuccess) err = uf::dev_malloc(&d_ncoupled, na);
  if (err == cudaSuccess) err = uf::dev_malloc(&d_color, na);
  if (err != cudaSuccess) {
    cleanup();
    uf::release_csr(csr);
    return fail(UF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(err));
  }
  cudaMemcpy(csr.row_ptr, row_ptr.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
  cudaMemcpy(d_coupled, coupled.data(), na * kMaxCoupled * sizeof(int32_t), cudaMemcpyHostToDevice);
  cudaMemcpy(d_ncoupled, ncoupled.data(), na, cudaMemcpyHostToDevice);
  err = cudaMemcpy(d_color, color.data(), na, cudaMemcpyHostToDevice);
  k_fill_cols<<<(unsigned)na, 256>>>(csr.col, csr.row_ptr, d_coupled, d_ncoupled, (int)na, nd);
  const size_t tile_bytes = (size_t)nd * (nd + 1) * sizeof(double);
  if (tile_bytes > 48 * 1024) {
    cudaFuncSetAttribute(k_scatter<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_bytes);
    cudaFuncSetAttribute(k_scatter<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_bytes);
  }
  const unsigned nb_ind = (unsigned)((n + 255) / 256);
  uf_status st = UF_OK;
  for (int c = 0; c < ncolors && st == UF_OK; ++c) {
    for (int j = 0; j < nd && st == UF_OK; ++j) {
      k_indicator<<<nb_ind, 256>>>(xind, d_color, (int)na, nd, c, j);
      st = uf::vmult_launch(op, UF_FP64, ystage + (size_t)j * n, xind, nullptr, false);
    }
    if (st != UF_OK) break;
    if (precision == UF_FP64)
      k_scatter<double><<<(unsigned)na, 256, tile_bytes>>>(static_cast<double *>(csr.val), ystage,
                                                          csr.row_ptr, d_coupled, d_ncoupled,
                                                          d_color, (int)na, nd, n, c);
    else
      k_scatter<float><<<(unsigned)na, 256, tile_bytes>>>(static_cast<float *>(csr.val), ystage,
                                                         csr.row_ptr, d_coupled, d_ncoupled,
                                                         d_color, (int)na, nd, n, c);
  }
  if (st == UF_OK) {
    err = cudaDeviceSynchronize();
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err != cudaSuccess) st = fail(UF_ECUDA, std::string("CSR assembly: ") + cudaGetErrorString(err));
  }
  cleanup();
  if (st != UF_OK) {
    uf::release_csr(csr);
    return st;
  }
  csr.nnz = nnz;
  csr.present = true;
  return UF_OK;
}

uf_status uf_csr_info(const uf_operator *op, int precision, int64_t *nnz, double *bytes) {
  if (!op || !nnz) return fail(UF_EINVAL, "NULL argument");
  const uf::CsrData &csr = (precision == UF_FP64) ? op->csr64 : op->csr32;
  if (!csr.present) return fail(UF_EINVAL, "CSR matrix not assembled for this precision");
  *nnz = csr.nnz;
  if (bytes) {
    const double vs = precision == UF_FP64 ? 8.0 : 4.0;
    const double n = (double)op->host.n_active * op->host.ndof;
    *bytes = (double)csr.nnz * (vs + 4.0) + (n + 1) * 8.0 + 2.0 * n * vs;
  }
  return UF_OK;
}

uf_status uf_csr_spmv(uf_operator *op, int precision, void *y, const void *x, void *stream) {
  if (!op || !y || !x) return fail(UF_EINVAL, "NULL argument");
  if (op->device < 0) return fail(UF_ENODEVICE, "operator was created host-only");
  const uf::CsrData &csr = (precision == UF_FP64) ? op->csr64 : op->csr32;
  if (!csr.present) return fail(UF_EINVAL, "CSR matrix not assembled for this precision");
  const int64_t n = op->host.n_active * op->host.ndof;
  const size_t vs = precision == UF_FP64 ? 8 : 4;
  const char *xb = static_cast<const char *>(x);
  const char *yb = static_cast<const char *>(y);
  if (xb < yb + n * vs && yb < xb + n * vs) return fail(UF_EINVAL, "x and y overlap");
  uf::DeviceGuard guard(op->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const unsigned blocks = (unsigned)((n * 32 + 255) / 256);
  if (precision == UF_FP64)
    k_spmv<double><<<blocks, 256, 0, s>>>(static_cast<double *>(y), static_cast<const double *>(x),
                                          csr.row_ptr, csr.col, static_cast<const double *>(csr.val), n);
  else
    k_spmv<float><<<blocks, 256, 0, s>>>(static_cast<float *>(y), static_cast<const float *>(x),
                                         csr.row_ptr, csr.col, static_cast<const float *>(csr.val), n);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return fail(UF_ECUDA, std::string("SpMV launch: ") + cudaGetErrorString(err));
  return UF_OK;
}

uf_status uf_export_csr(const uf_operator *op, int precision, int64_t *row_ptr, int32_t *col,
                        double *val) {
  if (!op) return fail(UF_EINVAL, "NULL argument");
  const uf::CsrData &csr = (precision == UF_FP64) ? op->csr64 : op->csr32;
  if (!csr.present) return fail(UF_EINVAL, "CSR matrix not assembled for this precision");
  uf::DeviceGuard guard(op->device);
  const int64_t n = op->host.n_active * op->host.ndof;
  cudaError_t err = cudaSuccess;
  if (row_ptr) err = cudaMemcpy(row_ptr, csr.row_ptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost);
  if (err == cudaSuccess && col) err = cudaMemcpy(col, csr.col, csr.nnz * sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (err == cudaSuccess && val) {
    if (precision == UF_FP64) {
      err = cudaMemcpy(val, csr.val, csr.nnz * sizeof(double), cudaMemcpyDeviceToHost);
    } else {
      std::vector<float> tmp(csr.nnz);
      err = cudaMemcpy(tmp.data(), csr.val, csr.nnz * sizeof(float), cudaMemcpyDeviceToHost);
      for (int64_t i = 0; i < csr.nnz; ++i) val[i] = tmp[i];
    }
  }
  if (err != cudaSuccess) return fail(UF_ECUDA, cudaGetErrorString(err));
  return UF_OK;
}

uf_status uf_release_csr(uf_operator *op) {
  if (!op) return UF_OK;
  if (op->device >= 0) {
    uf::DeviceGuard guard(op->device);
    uf::release_csr(op->csr64);
    uf::release_csr(op->csr32);
  }
  return UF_OK;
}

}  // extern "C"
