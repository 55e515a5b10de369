// Internal definition of uf_operator (shared by uf_api.cu and uf_csr.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/unfitted.h"
#include "uf_device.h"
#include "uf_host.h"

namespace uf {

constexpr int kPipeParts = 16;  // parts of the host-buffer pipeline (large discontinuous operators)

// Sets the thread-local message returned by uf_last_error and returns st.
uf_status fail(uf_status st, const std::string &msg);

template <typename T>
struct PrecisionData {
  bool present = false;
  void *base = nullptr;        // one device allocation for all arrays of this precision
  void *xbuf = nullptr;        // device staging buffers of uf_vmult_host
  void *ybuf = nullptr;
  // second staging set (pipelined operators): consecutive host-buffer calls alternate sets, so
  // an asynchronous call's copies overlap the previous call's kernels; set_free[b] is recorded
  // after the last copy out of the latest call on set b
  void *xbuf2 = nullptr, *ybuf2 = nullptr;
  int next_set = 0;
  bool set_used[2] = {false, false};
  cudaEvent_t set_free[2] = {nullptr, nullptr};
  T *kappa_dev = nullptr;
  DevArrays<T> arrays{};
  std::vector<unsigned char> struct_tables;  // StructTables<T, n>
  std::vector<unsigned char> point_tables;   // PointTables<T, n>
  Scalars<T> scalars{};
  size_t device_bytes = 0;
  int64_t n_vlines = 0, n_flines = 0;
  // host-buffer pipeline (discontinuous operators): consecutive-cell parts of y = A x, and for
  // part i the last part whose x must be on the device before it runs (face neighbours)
  std::vector<LaunchRange> parts;
  std::vector<int> part_needs;
  // continuous operators: global node of every cell-local DoF, owners of every node, and the
  // cell-local work vectors of the gather / kernels / node-sum sequence
  int32_t *cg_l2g = nullptr, *cg_own_off = nullptr, *cg_own_idx = nullptr;
  T *x_loc = nullptr, *y_loc = nullptr;
};

// Scalars of one PCG run, kept in device memory so that the iterations need no host round trip.
struct PcgScalars {
  double rz;       // r . z of the current iterate
  double pq;       // p . A p
  double rr;       // r . r
  double alpha, beta;
  double rr_stop;  // converged once rr <= rr_stop
  int status;      // 0 running, 1 converged, 2 breakdown (p . A p <= 0)
  int its;         // iterations completed
};

// Work vectors of the CG solvers (continuous operators).
struct CgSolveData {
  bool ready = false;
  double *r64 = nullptr, *q64 = nullptr, *d64 = nullptr, *z64 = nullptr, *p64 = nullptr;
  double *invd64 = nullptr;
  float *r32 = nullptr, *q32 = nullptr, *d32 = nullptr, *z32 = nullptr, *p32 = nullptr;
  float *invd32 = nullptr;
  double *dot_part = nullptr, *dot_out = nullptr, *dot_host = nullptr;
  PcgScalars *sc = nullptr, *sc_host = nullptr;  // device / pinned host copy
  // cells whose rows the split FP32 operator evaluates in FP64 (cut cells and cells with a
  // ghost-penalty face): the Nitsche and ghost-penalty terms live there
  int32_t *split_cells = nullptr;
  int64_t n_split = 0;
  // the split cells and their active face neighbours (the FP64 kernels read those cells' input)
  int32_t *halo_cells = nullptr;
  int64_t n_halo = 0;
  // the cut cells among the split cells (active ids, cut indices), sorted by lane class; class
  // ends [32 lanes, 16 lanes, 8 lanes]
  int32_t *split_cut_list = nullptr, *split_cut_idx = nullptr;
  int32_t split_cut_class[3] = {0, 0, 0};
  bool split_built = false;
};

struct ProfSlot {
  cudaEvent_t ev[4];
  int prec;     // 0 FP64, 1 FP32
  int adjoint;  // 0 vmult, 1 adjoint
  bool used;
};

// Assembled CSR matrix of the operator (device memory, one precision).
struct CsrData {
  bool present = false;
  int64_t nnz = 0;
  int64_t *row_ptr = nullptr;  // [n_dofs + 1]
  int32_t *col = nullptr;      // [nnz]
  void *val = nullptr;         // [nnz] double or float
};

// Restores the calling thread's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = (cudaSetDevice(dev) == cudaSuccess);
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

}  // namespace uf

struct uf_operator {
  uf::HostOperator host;
  int device = -1;
  int num_sms = 0;
  uf::PrecisionData<double> f64;
  uf::PrecisionData<float> f32;
  std::vector<uf::ProfSlot> prof;  // non-empty while profiling
  size_t prof_next = 0;
  uf::CsrData csr64, csr32;
  uf::CgSolveData cgs;           // continuous operators: solver work vectors
  double split_fraction = 1.0;   // cut cells below this volume fraction get FP64 split rows
  cudaStream_t pipe_in = nullptr, pipe_out = nullptr;  // copy streams of the host-buffer path
  std::vector<cudaStream_t> pipe_run;                 // one kernel stream per part
  std::vector<cudaEvent_t> pipe_ev;                   // [start, per part: in, done]
  double *kg_tables = nullptr;   // kappa-derivative 1D matrices (FP64)
  double *kg_scratch = nullptr;  // [n_active][1 + 2d] per-cell partials of the kappa gradient
};

namespace uf {
// Lanes of the cut-cell kernel for cut cell c (cut_lanes_for of its volume / cut-face lines).
inline int cut_lanes_of_cell(const HostOperator &H, int64_t c) {
  const int nf = 2 * H.dim;
  const int64_t vl = H.vline_off[c + 1] - H.vline_off[c];
  const int64_t fl = H.fline_off[(c + 1) * nf] - H.fline_off[c * nf];
  return cut_lanes_for(H.n, vl > fl ? vl : fl);
}
// FP32 y = A x with the rows of the split cells (CgSolveData::split_cells) evaluated in FP64 from
// the FP32 input and rounded once: the inner operator of the split iterative refinement.
uf_status vmult_split(uf_operator *op, float *y, const float *x, cudaStream_t stream);
uf_status split_cells_alloc(uf_operator *op);  // builds CgSolveData::split_cells once
void split_cells_free(uf_operator *op);        // drops them (rebuilt on the next use)
// Launch y = A x (or A^T x) of the operator's kernels on `stream` (no argument checks).
uf_status vmult_launch(uf_operator *op, int precision, void *y, const void *x, void *stream,
                       bool adjoint);
void release_csr(CsrData &c);
// kappa-derivative 1D matrices from the constant matrices of the structured terms.
void kgrad_tables(int n, const std::vector<double> &m, std::vector<double> &out);
// Constant 1D matrices of the structured terms (layout of StructTables, FP64).
void structured_matrices(const HostOperator &op, std::vector<double> &out);
// Continuous Q_p: load vector (f = 1) and diagonal of A on the host, FP64 (uf_cg.cu).
void cg_host_vectors(HostOperator &op);
// Discontinuous space: diagonal of A on the host, FP64, into op.dg_diag (uf_cg.cu).
void dg_host_diagonal(HostOperator &op);
int64_t solve_size(const HostOperator &h);  // unknowns of the linear system (CG: nodes)
uf_status cg_alloc(uf_operator *op);        // solver work vectors + Jacobi diagonal upload
uf_status cg_upload_diag(uf_operator *op);  // (re)upload 1 / diag(A)
void cg_free(uf_operator *op);
template <typename T>
int cg_gather(T *x_loc, const T *x, const int32_t *l2g, int64_t n_loc, cudaStream_t s);
template <typename T>
int cg_node_sum(T *y, const T *y_loc, const int32_t *off, const int32_t *idx, int64_t n, cudaStream_t s);

// Every device and pinned-host allocation of the library, and every operator object, goes
// through these: a test can make one of them fail (uf_debug_fail_allocation) and count the live
// ones (uf_debug_live_allocations).
cudaError_t dev_malloc_raw(void **p, size_t bytes);
cudaError_t pinned_malloc_raw(void **p, size_t bytes);
void dev_free(void *p);     // NULL is ignored
void pinned_free(void *p);  // NULL is ignored
template <typename P>
inline cudaError_t dev_malloc(P **p, size_t bytes) {
  return dev_malloc_raw(reinterpret_cast<void **>(p), bytes);
}
template <typename P>
inline cudaError_t pinned_malloc(P **p, size_t bytes) {
  return pinned_malloc_raw(reinterpret_cast<void **>(p), bytes);
}
uf_operator *new_operator();           // NULL when the allocation fails
void delete_operator(uf_operator *op);  // NULL is ignored
}  // namespace uf
