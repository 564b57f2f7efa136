// Host-side workspace of the GB300 PDHG solver and the launchers shared by the
// translation units.
#pragma once

#include <string>
#include <vector>

#include "common.cuh"

namespace ucpdhg {

// Owning sliced-ELL matrix (device arrays).
struct DevSell {
  int32_t nslices = 0, rows = 0;
  int64_t nnz_pad = 0;
  int32_t* off = nullptr;
  int32_t* col = nullptr;
  int32_t* src = nullptr;  // CSR position of each slot, -1 for padding
  double* val64 = nullptr;
  float* val32 = nullptr;
  int32_t* chunks = nullptr;  // [nchunks + 1] slice boundaries of the staged chunks
  int32_t nchunks = 0;        // 0: a slice exceeds kStageEntries (no staged kernels)
  int32_t* chunks2 = nullptr;  // chunks of the row-staged kernels
  int32_t nchunks2 = 0;
  SellView<double> v64() const { return {off, col, val64, nslices, rows}; }
  SellView<float> v32() const { return {off, col, val32, nslices, rows}; }
};

// Iterate buffers of one precision.
template <class T>
struct IterBufs {
  T* x[2] = {nullptr, nullptr};
  T* y[2] = {nullptr, nullptr};
  T* KTy[2] = {nullptr, nullptr};
  T* Kx[2] = {nullptr, nullptr};  // FP64 only (StoresKx)
  T* xbar = nullptr;
  T* ybar = nullptr;
  double* xbar64 = nullptr;  // FP32 mode only
  double* ybar64 = nullptr;
  T* xa = nullptr;
  T* ya = nullptr;
  bool allocated = false;
};

// Host description of the internal layout, built once per workspace.
struct HostLayout {
  std::vector<int32_t> perm_row, perm_col;  // internal -> original
  std::vector<int32_t> k_off, k_col, k_src;
  std::vector<int32_t> t_off, t_col, t_src;
};

int build_layout(int64_t n, int64_t m, int64_t m_eq, const std::vector<int64_t>& row_ptr,
                 const std::vector<int32_t>& col, HostLayout* out, std::string* err);

// Per-round initialisation of the device state.
struct RoundInit {
  double eta, omega;       // used when reset_steps
  int32_t reset_steps;     // 1: take eta/omega from the values above
  int32_t first_round;     // 1: restart the clock and the tolerance stamps
  double tol, ir_red;
  int64_t max_k, max_checks, k_offset;
  uint64_t t_limit_ns;
  double inv_dp, inv_dd;
  double gap_w;  // Delta_0 / Delta: keeps KKT_w's gap term in round-0 units
  int32_t fixed, trace_on, art_total;
  int64_t trace_cap_a, trace_cap_c;
  int32_t refine;  // 1: refinement rounds (mixed precision)
  double beta_suff, beta_nec, beta_art, omega_smooth, red_exp, grow_exp;
  double infeas_eps;
  int32_t fold_every;
};

// Device-state update of a refinement fold that continues the iteration in
// new coordinates (Delta' = f Delta): scalings, restart-metric scale, the next
// round's target, attempt bookkeeping.
struct RoundContinue {
  double f;              // Delta' / Delta
  double inv_dp, inv_dd, gap_w;
  double rel;            // rel-KKT of the folded point
  int64_t max_k, max_checks, k_offset;
};

// Launch configuration of the two per-attempt kernels of one precision:
// variant (unroll: 1, 2, 4 slices per warp, 0 software-pipelined) and grid
// size, picked by timing.
struct Tune {
  int unroll_dual = 1, grid_dual = 0, unroll_adj = 1, grid_adj = 0;
  bool done = false;
};

struct Workspace {
  int device = 0;
  int num_sms = 0;
  bool overlap_refused = false;  // graph built without programmatic dependent launch
  pdhg_problem prob{};
  pdhg_opts opts{};
  int64_t n = 0, m = 0, m_eq = 0, nnz = 0;
  DevSell K, KT;
  int32_t* perm_row = nullptr;
  int32_t* perm_col = nullptr;
  // FP64 vectors, internal order
  double *Dr = nullptr, *Dc = nullptr, *fac_r = nullptr, *fac_c = nullptr;
  double *iDr = nullptr, *iDc = nullptr;
  double *c_s = nullptr, *l_s = nullptr, *u_s = nullptr, *q_s = nullptr;  // rescaled LP
  double *c_h = nullptr, *l_h = nullptr, *u_h = nullptr, *q_h = nullptr, *ylo_h = nullptr;
  float *c_f = nullptr, *l_f = nullptr, *u_f = nullptr, *q_f = nullptr, *ylo_f = nullptr;
  double *x_star = nullptr, *y_star = nullptr;
  double *Kz_avg = nullptr, *KTz_avg = nullptr;
  double *Kz_cur = nullptr, *KTz_cur = nullptr, *Kx_anc = nullptr, *KTy_anc = nullptr;
  double *scr_m = nullptr, *scr_n = nullptr;
  double* scalars = nullptr;  // [16] eta0, omega0, norms, consts
  IterBufs<double> b64;
  IterBufs<float> b32;
  DevState* st = nullptr;
  DevState* st_host = nullptr;  // pinned mirror
  DevState* st_backup = nullptr;
  double* partials = nullptr;  // 3 regions of kMaxBlocks * 16
  double* trace_a = nullptr;
  double* trace_c = nullptr;
  int64_t trace_cap_a = 0, trace_cap_c = 0;
  bool values_f32 = false;  // FP32 matrix copy up to date
  bool solved = false;      // x_star/y_star hold a solution
  int grid_k = 0, grid_kt = 0, grid_vec = 0;
  Tune tune[2];  // [0] FP64, [1] FP32
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<void*> allocs;
  // batched / adjoint resources are owned by their translation units
  void* batched = nullptr;
  void* adjoint = nullptr;
};

// message of the last failure on this thread (pdhg_last_error), pdhg_api.cu
extern thread_local std::string g_err;

// pdhg_layout.cu
void launch_prepare(Workspace* w, cudaStream_t s);
void launch_spmv64(const SellView<double>& A, const double* x, double* y, int grid, cudaStream_t s);
void launch_spmv32(const SellView<float>& A, const float* x, float* y, int grid, cudaStream_t s);
void launch_gather_perm(const int32_t* perm, const double* in, double* out, int64_t n, cudaStream_t s);
void launch_scatter_perm(const int32_t* perm, const double* in, double* out, int64_t n,
                         cudaStream_t s);
void launch_to_f32(const double* in, float* out, int64_t n, cudaStream_t s);
void launch_to_f64(const float* in, double* out, int64_t n, cudaStream_t s);

// pdhg_kernels.cu
template <class T>
void launch_init_iterates(const IterArgs<T>& a, int grid, cudaStream_t s);
template <class T>
void launch_dual(const IterArgs<T>& a, int grid, cudaStream_t s, int unroll);
template <class T>
void launch_adjoint(const IterArgs<T>& a, int grid, cudaStream_t s, int unroll);
void launch_state_init(DevState* st, const RoundInit& r, const double* scalars, cudaStream_t s);
int blocks_per_sm_iter();  // resident blocks per SM of the per-attempt kernels (both precisions)

// pdhg_staged.cu: per-attempt kernels with TMA-staged matrix chunks
template <class T>
void launch_dual_staged(const IterArgs<T>& a, int grid, cudaStream_t s, int pair);
template <class T>
void launch_adjoint_staged(const IterArgs<T>& a, int grid, cudaStream_t s, int pair);
int staged_setup();
// pdhg_rowstaged.cu: the same with the row (column) operands staged too
template <class T>
void launch_dual_rowstaged(const IterArgs<T>& a, int grid, cudaStream_t s, int pair);
template <class T>
void launch_adjoint_rowstaged(const IterArgs<T>& a, int grid, cudaStream_t s, int pair);
int rowstaged_setup();
// pdhg_ring.cu: per-warp rings of asynchronous copies (3 or 4 slots)
template <class T>
void launch_dual_ring(const IterArgs<T>& a, int grid, cudaStream_t s, int slots);
template <class T>
void launch_adjoint_ring(const IterArgs<T>& a, int grid, cudaStream_t s, int slots);
int ring_setup();
// chunks of consecutive slices with at most max_entries entries and max_slices
// slices each; false if a single slice is larger
bool build_chunks(const std::vector<int32_t>& off, std::vector<int32_t>* chunks, int max_entries,
                  int max_slices);

// pdhg_kkt.cu
template <class T>
void launch_check(const IterArgs<T>& a, int grid_k, int grid_kt, int init, cudaStream_t s);
template <class T>
void launch_accumulate(const IterArgs<T>& a, double* x_star, double* y_star, int grid,
                       cudaStream_t s);
template <class T>
void launch_recenter(const IterArgs<T>& a, double f, cudaStream_t s);
void launch_state_continue(DevState* st, const RoundContinue& rc, const double* scalars,
                           cudaStream_t s);
void launch_ir_build(Workspace* w, double dp, double dd, bool make_f32, cudaStream_t s);
void launch_output(Workspace* w, double* x_out, double* y_out, cudaStream_t s);

template <class T>
IterArgs<T> make_args(Workspace* w);

// pdhg_batched.cu: frees the batched buffers and graph of a workspace
void release_batched(Workspace* w);
// pdhg_batched.cu: rows per warp and grid of the batched sweeps (dual, adjoint)
void batched_tuning(Workspace* w, int32_t* out4);
// pdhg_adjoint.cu: frees the adjoint's scratch
void release_adjoint(Workspace* w);

}  // namespace ucpdhg
