// Shared device-side definitions of the GB300 PDHG solver.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "../../include/pdhg.h"

namespace ucpdhg {

constexpr int kSlice = 32;       // rows per sliced-ELL slice (one warp, one row per lane)
constexpr int kBlock = 256;      // threads per block of every streaming kernel
constexpr int kWarps = kBlock / 32;
constexpr int kCheckEvery = 64;  // step attempts between KKT checks (one graph body)
constexpr int kMaxBlocks = 8192; // upper bound of the persistent grid sizes
constexpr int kRowSums = 7;      // per-candidate sums of the row-side KKT kernel
constexpr int kColSums = 9;      // per-candidate sums of the column-side KKT kernel
constexpr int kRegionStride = 24;  // doubles per block in each partials region (>= 2 x sums)
constexpr int kStageEntries = 3072;  // sliced-ELL entries per shared-memory chunk (staged kernels)
constexpr int kRsEntries = 2048;     // entries per chunk of the row-staged kernels
constexpr int kRsSlices = 32;        // slices per chunk of the row-staged kernels
// Certificate tolerance floor for rays made of FP32 iterates: differences of
// FP32 vectors carry ~1e-7 relative noise, so their violation/objective ratio
// cannot fall below ~1e-7 however well the iteration has converged onto the
// infeasibility direction; FP32 iterations therefore test rays at
// max(infeas_tol, kFp32RayTol).
constexpr double kFp32RayTol = 1e-6;
constexpr int kTraceCheckCols = 12;  // values recorded per KKT check in the trace

// Sliced ELL with 32-row slices over the internal (length-sorted) row order.
// Entry k of row r = 32 s + lane sits at off[s] + 32 k + lane, so the warp
// owning a slice reads each k-column with one coalesced 128 B / 256 B access.
// Padding entries carry col = 0 and value 0.
template <class T>
struct SellView {
  const int32_t* off;  // [nslices + 1] element offsets (multiples of 32)
  const int32_t* col;  // [nnz_pad] internal column index
  const T* val;        // [nnz_pad]
  int32_t nslices;
  int32_t rows;        // logical rows (<= 32 * nslices)
};

// Device-resident solver state: every scalar decision of the PDHG loop lives
// here, so the loop never waits on the host.
struct DevState {
  // step control
  double eta, omega;
  double dx2;        // ||x' - x||^2 of the pending candidate
  double w_last;     // eta of the last attempt if accepted, else 0
  double pending_w;  // weight of the y-average update not yet applied
  double wsum;       // sum of average weights since the last restart
  double avg_div;    // wsum frozen for restart_apply
  int32_t par;       // parity of the current iterate buffers
  int32_t accepted_last;
  int64_t k;              // attempts this round
  int64_t since_restart;  // attempts since the last restart
  int64_t accepted;       // accepted attempts this round
  int64_t restarts;       // this round
  int64_t checks;         // this round
  // restart control
  double kkt0, kkt_prev;
  int32_t restart_now, restart_to_avg;
  // outcome of the last check (best candidate)
  int32_t done, status;  // status: 0 running/round target met, else PDHG_STATUS_*
  int32_t best_is_avg, numeric;
  double rel_p, rel_d, rel_gap, rel_kkt, pobj, dobj;
  // targets and limits
  double tol, round_target, ir_red;
  double round_rel0;  // rel_kkt of the current iterate when the round started
  int64_t max_k, max_checks;
  uint64_t t_start, t_limit_ns;
  double t_tol[3];
  int64_t k_tol[3];
  int64_t k_offset;  // attempts of earlier refinement rounds
  // constants of the method
  double beta_suff, beta_nec, beta_art, omega_smooth, red_exp, grow_exp;
  double infeas_eps;  // certificate tolerance of the infeasibility test (0: off)
  int32_t fold_every; // refinement: fold after this many checks of a round (0: off)
  int32_t wait_timeout;  // set by a kernel whose bounded wait gave up
  int32_t fixed;     // constant steps, no restarts
  int32_t art_total; // artificial restart against attempts of all rounds
  int32_t trace_on;
  int64_t trace_cap_a, trace_cap_c, n_trace_a, n_trace_c;
  // refinement rounds (mixed mode): a check whose current iterate meets
  // round_target ends the round; fold = 1 asks the host to fold that iterate
  // into x*, y* and continue the iteration in the new coordinates
  int32_t refine, fold;
  // norms of the unscaled data and refinement scalars
  double qnorm, cnorm;
  double inv_dp, inv_dd;      // 1/Delta_P, 1/Delta_D
  double gap_w;               // Delta of round 0 / Delta of this round (weights the gap in KKT_w)
  double const_p, const_d;    // c~^T x*, q~^T y*
  // last-block counters of the reducing kernels
  uint32_t counter;
  uint32_t counter2;
};

// Pointers of one precision's iteration.
template <class T>
struct IterArgs {
  SellView<T> K, KT;
  T* x[2];
  T* y[2];
  T* KTy[2];
  T* Kx[2];  // K x of x[0], x[1]: stored in FP64 mode (nullptr in FP32 mode, where
             // k_dual recomputes K x from the matrix pass it makes anyway)
  T* xbar;  // weighted sums (not divided) of the attempts since the last check
  T* ybar;
  // FP32 mode: the step-weighted sums since the last restart live in FP64; at
  // every check the window's FP32 sums (<= 64 terms) are added in and cleared.
  // The sums must stay exact through refinement folds, which re-express them
  // relative to the current iterate (a cancellation that FP32 sums of up to 10^6
  // terms cannot survive).  nullptr in FP64 mode (xbar, ybar are FP64 there).
  double* xbar64;
  double* ybar64;
  T* xa;    // anchors (last restart point)
  T* ya;
  const T* c;
  const T* l;
  const T* u;
  const T* q;
  const T* ylo;  // nullptr: -inf on equality rows, 0 on >= rows
  int32_t n, m, m_eq;
  DevState* st;
  double* partials;
  double* trace_a;  // [cap][5]
  double* trace_c;  // [cap][kTraceCheckCols]
  volatile int32_t* cancel;
  // chunks of slices staged in shared memory by the staged kernels: chunk c is
  // slices [kchunks[c], kchunks[c+1]) of K (tchunks: of K^T)
  const int32_t* kchunks;
  const int32_t* tchunks;
  int32_t kchunks_n, tchunks_n;
  // chunks of the row-staged kernels (<= kRsEntries entries, <= kRsSlices slices)
  const int32_t* kchunks2;
  const int32_t* tchunks2;
  int32_t kchunks2_n, tchunks2_n;
  unsigned long long cond;  // cudaGraphConditionalHandle
  int32_t in_graph;
  int32_t overlap;  // 1: per-attempt kernels launched with programmatic dependent launch
  // FP64 data of the KKT evaluation
  SellView<double> K64, KT64;
  const double* q_res;  // q^ (FP64)
  const double* c_res;  // c^ (FP64)
  const double* q_obj;  // q~
  const double* c_obj;  // c~
  const double* l_obj;  // l~
  const double* u_obj;  // u~
  const double* Dr;
  const double* Dc;
  const double* iDr;  // 1 / Dr (the KKT kernels multiply: FP64 division is slow)
  const double* iDc;  // 1 / Dc
  double* Kz_avg;   // [m] K~ xbar / wsum (FP64)
  double* KTz_avg;  // [n] K~^T ybar / wsum (FP64)
  double* Kz_cur;   // [m] K~ x of the current iterate at the last check (FP64)
  double* KTz_cur;  // [n] K~^T y of the same
  double* Kx_anc;   // [m] K~ x of the restart anchor (FP64): rays K~ (x - x_anchor)
  double* KTy_anc;  // [n] K~^T y of the restart anchor
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of NV values per thread; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem /* [kWarps*NV] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) smem[wid * NV + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int w = 0; w < kWarps; ++w) s += smem[w * NV + k];
      v[k] = s;
    }
  }
  __syncthreads();
}

// Writes this block's NV partial sums and returns true in every thread of the
// block that finished last.  That block then reads all partials with
// final_sum (fixed order, so the result does not depend on scheduling).
template <int NV>
__device__ __forceinline__ bool publish_partials(double (&v)[NV], double* partials,
                                                 uint32_t* counter) {
  __shared__ double smem[kWarps * NV];
  __shared__ int last;
  block_sum<NV>(v, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[(size_t)blockIdx.x * NV + k] = v[k];
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  return last != 0;
}

// Fixed-order sum over the partials of `nblocks` blocks; valid in thread 0.
template <int NV>
__device__ __forceinline__ void final_sum(const double* partials, int nblocks, double (&out)[NV]) {
  __shared__ double smem[kWarps * NV];
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] += __ldcg(partials + (size_t)b * NV + k);
  block_sum<NV>(v, smem);
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = v[k];
}

// The same last-block reduction with the partials kept in the iterate type T
// up to the final total: for T = float no FP64 instruction runs per warp (a
// warp-wide FP64 add holds GB300's narrow FP64 pipe for tens of cycles, which
// the per-attempt kernels would pay at every block's end).  The partials
// buffer is reused as T storage.
template <class T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int NV, class T>
__device__ __forceinline__ void block_sum_t(T (&v)[NV], T* smem /* [kWarps*NV] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum_t<T>(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) smem[wid * NV + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      T s = 0;
      for (int w = 0; w < kWarps; ++w) s += smem[w * NV + k];
      v[k] = s;
    }
  }
  __syncthreads();
}

template <int NV, class T>
__device__ __forceinline__ bool publish_partials_t(T (&v)[NV], double* partials, uint32_t* counter) {
  __shared__ T smem_t[kWarps * NV];
  __shared__ int last_t;
  block_sum_t<NV, T>(v, smem_t);
  if (threadIdx.x == 0) {
    T* pt = reinterpret_cast<T*>(partials);
#pragma unroll
    for (int k = 0; k < NV; ++k) pt[(size_t)blockIdx.x * NV + k] = v[k];
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    last_t = (t == gridDim.x - 1);
  }
  __syncthreads();
  return last_t != 0;
}

// Fixed-order total of the T partials; valid in thread 0, returned in FP64.
template <int NV, class T>
__device__ __forceinline__ void final_sum_t(const double* partials, int nblocks, double (&out)[NV]) {
  __shared__ T smem_f[kWarps * NV];
  const T* pt = reinterpret_cast<const T*>(partials);
  T v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] += __ldcg(pt + (size_t)b * NV + k);
  block_sum_t<NV, T>(v, smem_f);
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = (double)v[k];
}

// (k+1)^(-e) of the step-size rule in FP32 (relative error ~1e-6): an FP64
// pow on the serial tail of every attempt would cost microseconds on a GPU
// whose FP64 rate is ~1/60 of FP32, and the rule is a heuristic factor.
__device__ __forceinline__ double step_power(int64_t k1, double e) {
  return (double)exp2f(-(float)e * log2f((float)k1));
}

// FP32 iterations take tau = eta / omega and sigma = eta * omega in FP32.  The
// cap is applied once per check (k_control), where the FP64 division costs
// nothing per attempt; between checks eta grows by at most a factor ~1.3.  When
// the step-size rule finds no interaction (eta_max = inf, e.g. a primal iterate
// pinned at its bounds while the dual diverges on an infeasible LP) it grows eta
// by (1 + (k+1)^-0.6) per attempt, which leaves the FP32 range within ~10^4
// attempts; capping eta so both stay below 1e30 keeps the diverging iterates
// finite until the infeasibility certificate is read off them.  The cap is far
// above any step the rule accepts on a feasible LP (eta <= eta_max ~ 1/||K~||).
__device__ __forceinline__ double fp32_step_cap(double omega) {
  return 1e30 / fmax(omega, 1.0 / omega);
}

// Per-attempt scalars of the step kernels, read from the device state and
// converted by thread 0 of each block, then shared: GB300 retires FP64
// instructions at a small fraction of its FP32 rate, so an FP64 multiply,
// divide or conversion in every thread held every warp of a launch on the
// FP64 pipe before its first slice.
template <class T>
struct DualScalars {
  int done, p, has_pw;
  T pw, sigma;
};
template <class T>
__device__ __forceinline__ void dual_scalars(const DevState* st, DualScalars<T>& s) {
  s.done = st->done;
  s.p = st->par;
  const double pw = st->pending_w;
  s.has_pw = pw != 0.0;
  s.pw = (T)pw;
  s.sigma = (T)(st->eta * st->omega);
}
template <class T>
struct AdjScalars {
  int done, p, acc_last, upd_avg;
  T wl, tau;
};
template <class T>
__device__ __forceinline__ void adj_scalars(const DevState* st, AdjScalars<T>& s) {
  s.done = st->done;
  s.p = st->par;
  s.acc_last = st->accepted_last;
  const double wl = st->w_last;
  s.upd_avg = s.acc_last && wl != 0.0;
  s.wl = (T)wl;
  s.tau = (T)(st->eta / st->omega);
}

// Programmatic dependent launch (sm_90 and later).  A per-attempt kernel lets
// the next kernel in the stream start as soon as all of its own blocks are
// running (launch_dependents); the next kernel reads only the matrix (slice
// offsets, columns, values: constant for the whole solve) before
// griddepcontrol.wait, which returns once every earlier grid has finished and
// its writes are visible.  Both instructions are no-ops for a kernel launched
// without the attribute.
__device__ __forceinline__ void grid_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void grid_wait_prior() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// FP64 iterations store K x (an m-vector stream read and write per attempt)
// instead of recomputing it with a second product per matrix entry: GB300's
// FP64 pipe, not HBM, bounds the FP64 kernels, and the second product costs one
// FP64 FMA per entry.  FP32 iterations recompute it (FP32 FMAs are nearly free
// and the stream would cost bandwidth).
template <class T>
struct StoresKx {
  static constexpr bool value = sizeof(T) == 8;
};

template <class T>
__device__ __forceinline__ T dual_floor(const T* ylo, int i, int m_eq) {
  if (ylo) return ylo[i];
  return (i < m_eq) ? (T)(-INFINITY) : (T)0;
}

// Adaptive step rule on the device (thread 0 of the last block of k_dual).
template <class T>
__device__ void decide_step(DevState* st, const IterArgs<T>& a, double dy2, double inter) {
  const double eta = st->eta, omega = st->omega;
  const double movement = omega * st->dx2 + dy2 / omega;
  const double interaction = 2.0 * fabs(inter);
  const double eta_max = interaction > 0.0 ? movement / interaction : INFINITY;
  const int64_t k = st->k + 1;
  st->k = k;
  // attempts of all rounds: a refinement round is a change of coordinates,
  // not a new solve
  const int64_t kg = st->k_offset + k;
  double eta_next = fmin((1.0 - step_power(kg + 1, st->red_exp)) * eta_max,
                         (1.0 + step_power(kg + 1, st->grow_exp)) * eta);
  int accept = eta <= eta_max;
  if (st->fixed) {
    accept = 1;
    eta_next = eta;
  }
  if (st->trace_on && a.trace_a) {
    int64_t t = st->n_trace_a;
    if (t < st->trace_cap_a) {
      double* r = a.trace_a + t * 5;
      r[0] = eta;
      r[1] = omega;
      r[2] = (double)accept;
      r[3] = eta_max;
      r[4] = eta_next;
    }
    st->n_trace_a = t + 1;
  }
  if (accept) {
    st->par = 1 - st->par;
    st->w_last = eta;
    st->pending_w = eta;
    st->wsum += eta;
    st->accepted += 1;
  } else {
    st->w_last = 0.0;
    st->pending_w = 0.0;
  }
  st->accepted_last = accept;
  st->since_restart += 1;
  st->eta = eta_next;
}

// ---- host-side launchers (defined in the .cu files) ----------------------------
struct Workspace;

}  // namespace ucpdhg
