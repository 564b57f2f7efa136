// C ABI, workspace management and the solve driver.
//
// The PDHG loop of one refinement round runs as ONE CUDA graph: a conditional
// WHILE node whose body holds 64 step attempts (k_dual, k_adjoint) followed by
// the KKT check (k_kkt_row, k_kkt_col, k_control, k_restart_apply).  k_control
// clears the while condition on the device when the round is finished, so the
// host launches the graph once per round and waits once per round.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "internal.cuh"

namespace ucpdhg {

thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(PDHG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

template <class P>
static cudaError_t dalloc(Workspace* w, P** p, size_t count) {
  void* q = nullptr;
  // lengths rounded up to whole 32-row slices: the row-staged kernels copy the
  // operand rows of whole slices
  count = (count + 31) / 32 * 32;
  cudaError_t e = cudaMalloc(&q, count * sizeof(P) + 16);
  if (e == cudaSuccess) {
    w->allocs.push_back(q);
    *p = (P*)q;
  }
  return e;
}

#define DALLOC(ptr, count)                                                                 \
  do {                                                                                     \
    cudaError_t e_ = dalloc(w, &(ptr), (size_t)(count));                                   \
    if (e_ != cudaSuccess) return fail(PDHG_ERR_NOMEM, std::string("cudaMalloc: ") +       \
                                                           cudaGetErrorString(e_));         \
  } while (0)

template <class T>
IterArgs<T> make_args(Workspace* w) {
  IterArgs<T> a{};
  IterBufs<T>* b;
  if constexpr (sizeof(T) == 8) {
    b = (IterBufs<T>*)&w->b64;
    a.K = w->K.v64();
    a.KT = w->KT.v64();
    a.c = (const T*)w->c_h;
    a.l = (const T*)w->l_h;
    a.u = (const T*)w->u_h;
    a.q = (const T*)w->q_h;
    a.ylo = nullptr;
  } else {
    b = (IterBufs<T>*)&w->b32;
    a.K = w->K.v32();
    a.KT = w->KT.v32();
    a.c = (const T*)w->c_f;
    a.l = (const T*)w->l_f;
    a.u = (const T*)w->u_f;
    a.q = (const T*)w->q_f;
    a.ylo = (const T*)w->ylo_f;
  }
  for (int i = 0; i < 2; ++i) {
    a.x[i] = b->x[i];
    a.y[i] = b->y[i];
    a.KTy[i] = b->KTy[i];
    a.Kx[i] = b->Kx[i];
  }
  a.xbar = b->xbar;
  a.ybar = b->ybar;
  a.xbar64 = b->xbar64;
  a.ybar64 = b->ybar64;
  a.xa = b->xa;
  a.ya = b->ya;
  a.n = (int32_t)w->n;
  a.m = (int32_t)w->m;
  a.m_eq = (int32_t)w->m_eq;
  a.st = w->st;
  a.partials = w->partials;
  a.trace_a = w->trace_a;
  a.trace_c = w->trace_c;
  a.cancel = w->opts.cancel_flag;
  a.kchunks = w->K.chunks;
  a.kchunks_n = w->K.nchunks;
  a.tchunks = w->KT.chunks;
  a.tchunks_n = w->KT.nchunks;
  a.kchunks2 = w->K.chunks2;
  a.kchunks2_n = w->K.nchunks2;
  a.tchunks2 = w->KT.chunks2;
  a.tchunks2_n = w->KT.nchunks2;
  a.cond = 0;
  a.in_graph = 0;
  a.overlap = (w->opts.launch_overlap && !w->overlap_refused) ? 1 : 0;
  a.K64 = w->K.v64();
  a.KT64 = w->KT.v64();
  a.q_res = w->q_h;
  a.c_res = w->c_h;
  a.q_obj = w->q_s;
  a.c_obj = w->c_s;
  a.l_obj = w->l_s;
  a.u_obj = w->u_s;
  a.Dr = w->Dr;
  a.Dc = w->Dc;
  a.iDr = w->iDr;
  a.iDc = w->iDc;
  a.Kz_avg = w->Kz_avg;
  a.KTz_avg = w->KTz_avg;
  a.Kz_cur = w->Kz_cur;
  a.KTz_cur = w->KTz_cur;
  a.Kx_anc = w->Kx_anc;
  a.KTy_anc = w->KTy_anc;
  return a;
}

template IterArgs<double> make_args<double>(Workspace*);
template IterArgs<float> make_args<float>(Workspace*);

template <class T>
static int alloc_bufs(Workspace* w, IterBufs<T>* b) {
  if (b->allocated) return PDHG_OK;
  for (int i = 0; i < 2; ++i) {
    DALLOC(b->x[i], w->n);
    DALLOC(b->y[i], w->m);
    DALLOC(b->KTy[i], w->n);
    if (StoresKx<T>::value) DALLOC(b->Kx[i], w->m);
  }
  DALLOC(b->xbar, w->n);
  DALLOC(b->ybar, w->m);
  if (sizeof(T) == 4) {
    DALLOC(b->xbar64, w->n);
    DALLOC(b->ybar64, w->m);
  }
  DALLOC(b->xa, w->n);
  DALLOC(b->ya, w->m);
  b->allocated = true;
  return PDHG_OK;
}

static int grid_for(Workspace* w, int per_sm, int nslices) {
  if (per_sm < 1) per_sm = 4;
  int g = w->num_sms * per_sm;
  int need = (nslices + kWarps - 1) / kWarps;
  if (g > need) g = need;
  if (g > kMaxBlocks) g = kMaxBlocks;
  return g < 1 ? 1 : g;
}

__global__ void k_reopen_state(DevState* st) {
  st->done = 0;
  st->counter = 0;
  st->trace_on = 0;
}

template <class T>
static void run_dual(Workspace* w, const IterArgs<T>& a, cudaStream_t s) {
  const Tune& t = w->tune[sizeof(T) == 8 ? 0 : 1];
  launch_dual<T>(a, t.grid_dual, s, t.unroll_dual);
}

template <class T>
static void run_adjoint(Workspace* w, const IterArgs<T>& a, cudaStream_t s) {
  const Tune& t = w->tune[sizeof(T) == 8 ? 0 : 1];
  launch_adjoint<T>(a, t.grid_adj, s, t.unroll_adj);
}

// Picks, by timing on this workspace's matrix, the variant (1, 2 or 4 slices
// a warp sweeps together, or 0: the software-pipelined single-slice form) and
// the grid size (2 to 8 blocks per SM) of each per-attempt kernel.  The
// candidate launches run real attempts on scratch state; the caller
// re-initialises the iterates afterwards.
template <class T>
static int autotune(Workspace* w, const IterArgs<T>& a, cudaStream_t s) {
  const int pi = sizeof(T) == 8 ? 0 : 1;
  Tune& t = w->tune[pi];
  if (t.done) return PDHG_OK;
  const int fixed_variant = w->opts.kernel_variant;
  t.unroll_dual = t.unroll_adj = fixed_variant >= 0 ? fixed_variant : 1;
  t.grid_dual = w->grid_k;
  t.grid_adj = w->grid_kt;
  if (!w->opts.autotune || fixed_variant >= 0) {
    if ((fixed_variant == 16 || fixed_variant == 17) &&
        (w->K.nchunks == 0 || w->KT.nchunks == 0 || staged_setup() != 0))
      return fail(PDHG_ERR_UNSUPPORTED,
                  "kernel_variant 16/17: a slice exceeds the staged chunk size on this matrix");
    if ((fixed_variant == 18 || fixed_variant == 19) &&
        (w->K.nchunks2 == 0 || w->KT.nchunks2 == 0 || rowstaged_setup() != 0))
      return fail(PDHG_ERR_UNSUPPORTED,
                  "kernel_variant 18/19: a slice exceeds the row-staged chunk size on this matrix");
    if ((fixed_variant == 20 || fixed_variant == 21) && ring_setup() != 0)
      return fail(PDHG_ERR_CUDA, "kernel_variant 20/21: shared-memory opt-in refused");
    if (w->opts.kernel_grid > 0) t.grid_dual = t.grid_adj = w->opts.kernel_grid;
    t.done = true;
    return PDHG_OK;
  }
  // 1, 2, 4: slices a warp sweeps together; 0: one slice per warp, software
  // pipelined (the next slice's first entries and row operands load early);
  // 8, 9: the one-slice and pipelined forms limited to 32 registers (8 blocks
  // per SM); 16-19: TMA-staged chunks; 20, 21: per-warp cp.async rings
  const bool staged = w->K.nchunks > 0 && w->KT.nchunks > 0 && staged_setup() == 0;
  const bool rowstaged = w->K.nchunks2 > 0 && w->KT.nchunks2 > 0 && rowstaged_setup() == 0;
  const bool ring = ring_setup() == 0;
  const int unrolls[12] = {1, 2, 4, 0, 8, 9, 16, 17, 18, 19, 20, 21};
  // grids beyond one resident wave let blocks that finish early take the
  // remaining slices (the sweeps' slices are spread round-robin over warps)
  const int bps[7] = {2, 3, 4, 6, 8, 12, 16};
  // UCPDHG_TUNE_LOG=1 prints every timed candidate to stderr
  const char* log_env = std::getenv("UCPDHG_TUNE_LOG");
  const bool log = log_env && log_env[0] == '1';
  for (int which = 0; which < 2; ++which) {
    const int nsl = which == 0 ? w->K.nslices : w->KT.nslices;
    float best = 1e30f;
    int bu = 1, bg = which == 0 ? w->grid_k : w->grid_kt;
    for (int ui = 0; ui < 12; ++ui) {
      const int U = unrolls[ui];
      if ((U == 16 || U == 17) && !staged) continue;
      if ((U == 18 || U == 19) && !rowstaged) continue;
      if ((U == 20 || U == 21) && !ring) continue;
      const int Us = (U == 2 || U == 4) ? U : 1;
      const int need = (nsl + kWarps * Us - 1) / (kWarps * Us);
      for (int bi = 0; bi < 7; ++bi) {
        int g = std::min(w->num_sms * bps[bi], std::min(need, kMaxBlocks));
        if (g < 1) g = 1;
        k_reopen_state<<<1, 1, 0, s>>>(w->st);
        if (which == 0)
          launch_dual<T>(a, g, s, U);
        else
          launch_adjoint<T>(a, g, s, U);
        CK(cudaEventRecord(w->ev[2], s));
        for (int r = 0; r < 3; ++r) {
          if (which == 0)
            launch_dual<T>(a, g, s, U);
          else
            launch_adjoint<T>(a, g, s, U);
        }
        CK(cudaEventRecord(w->ev[3], s));
        CK(cudaEventSynchronize(w->ev[3]));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, w->ev[2], w->ev[3]));
        if (log)
          std::fprintf(stderr, "autotune %s %s variant %d grid %d: %.2f us\n", sizeof(T) == 8 ? "fp64" : "fp32",
                       which == 0 ? "dual" : "adjoint", U, g, ms * 1000.f / 3.f);
        if (ms < best * 0.98f) {
          best = ms;
          bu = U;
          bg = g;
        }
        if (g == need) break;  // larger grids add nothing
      }
    }
    if (which == 0) {
      t.unroll_dual = bu;
      t.grid_dual = bg;
    } else {
      t.unroll_adj = bu;
      t.grid_adj = bg;
    }
  }
  if (w->opts.kernel_grid > 0) t.grid_dual = t.grid_adj = w->opts.kernel_grid;
  CK(cudaGetLastError());
  t.done = true;
  return PDHG_OK;
}

template <class T>
static int build_graph_once(Workspace* w);

// The solve graph; built with programmatic dependent launches of the
// per-attempt kernels when enabled, and once more without them if the driver
// refuses that graph.
template <class T>
static int build_graph(Workspace* w) {
  const int pi = sizeof(T) == 8 ? 0 : 1;
  if (w->graph_exec[pi]) return PDHG_OK;
  int rc = build_graph_once<T>(w);
  if (rc != PDHG_OK && w->opts.launch_overlap && !w->overlap_refused) {
    cudaGetLastError();
    w->overlap_refused = true;
    g_err.clear();
    rc = build_graph_once<T>(w);
  }
  return rc;
}

template <class T>
static int build_graph_once(Workspace* w) {
  const int pi = sizeof(T) == 8 ? 0 : 1;
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  // cudaGraphNodeParams has no default constructor: zeroed storage instead
  alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
  std::memset(cp_raw, 0, sizeof(cp_raw));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(w->cap_stream, body, nullptr, nullptr, 0,
                                   cudaStreamCaptureModeThreadLocal));
  IterArgs<T> a = make_args<T>(w);
  a.in_graph = 1;
  a.cond = (unsigned long long)h;
  for (int k = 0; k < kCheckEvery; ++k) {
    run_dual<T>(w, a, w->cap_stream);
    run_adjoint<T>(w, a, w->cap_stream);
  }
  launch_check<T>(a, w->grid_k, w->grid_kt, 0, w->cap_stream);
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(w->cap_stream, &captured);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(PDHG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(PDHG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  w->graph[pi] = g;
  w->graph_exec[pi] = ex;
  return PDHG_OK;
}

static int validate_opts(const pdhg_opts* o) {
  if (!(o->tol > 0.0) || o->max_iters < 1 || !(o->time_limit_s > 0.0))
    return fail(PDHG_ERR_INVALID_ARG, "opts: tol, max_iters, time_limit_s must be > 0");
  if (o->precision != PDHG_PREC_FP64 && o->precision != PDHG_PREC_MIXED)
    return fail(PDHG_ERR_INVALID_ARG, "opts: precision must be PDHG_PREC_FP64 or PDHG_PREC_MIXED");
  if (o->check_every != kCheckEvery)
    return fail(PDHG_ERR_UNSUPPORTED, "opts: check_every must be 64");
  if (o->ruiz_iters < 0 || o->ruiz_iters > 100)
    return fail(PDHG_ERR_INVALID_ARG, "opts: ruiz_iters out of range");
  if (o->ir_max_rounds < 0 || !(o->ir_reduction > 0.0) || !(o->ir_reduction < 1.0))
    return fail(PDHG_ERR_INVALID_ARG, "opts: refinement settings out of range");
  if (o->fixed_eta < 0.0 || (o->fixed_eta > 0.0 && !(o->fixed_omega > 0.0)))
    return fail(PDHG_ERR_INVALID_ARG, "opts: fixed_eta needs fixed_omega > 0");
  if (!(o->kernel_variant == -1 || o->kernel_variant == 0 || o->kernel_variant == 1 ||
        o->kernel_variant == 2 || o->kernel_variant == 4 || o->kernel_variant == 8 ||
        o->kernel_variant == 9 || o->kernel_variant == 16 || o->kernel_variant == 17 ||
        o->kernel_variant == 18 || o->kernel_variant == 19 || o->kernel_variant == 20 ||
        o->kernel_variant == 21))
    return fail(PDHG_ERR_INVALID_ARG, "opts: kernel_variant must be -1, 0, 1, 2, 4, 8, 9 or 16-21");
  if (o->ir_fold_checks < 0)
    return fail(PDHG_ERR_INVALID_ARG, "opts: ir_fold_checks must be >= 0");
  if (o->launch_overlap != 0 && o->launch_overlap != 1)
    return fail(PDHG_ERR_INVALID_ARG, "opts: launch_overlap must be 0 or 1");
  if (!(o->infeas_tol >= 0.0))
    return fail(PDHG_ERR_INVALID_ARG, "opts: infeas_tol must be >= 0");
  if (o->kernel_grid < 0 || o->kernel_grid > kMaxBlocks)
    return fail(PDHG_ERR_INVALID_ARG, "opts: kernel_grid out of range");
  return PDHG_OK;
}

static int ensure_trace(Workspace* w) {
  if (!w->opts.trace || w->trace_a) return PDHG_OK;
  w->trace_cap_a = 1 << 16;
  w->trace_cap_c = 1 << 17;
  DALLOC(w->trace_a, w->trace_cap_a * 5);
  DALLOC(w->trace_c, w->trace_cap_c * kTraceCheckCols);
  return PDHG_OK;
}

static void release(Workspace* w) {
  release_batched(w);
  release_adjoint(w);
  for (int i = 0; i < 2; ++i) {
    if (w->graph_exec[i]) cudaGraphExecDestroy(w->graph_exec[i]);
    if (w->graph[i]) cudaGraphDestroy(w->graph[i]);
  }
  for (int i = 0; i < 4; ++i)
    if (w->ev[i]) cudaEventDestroy(w->ev[i]);
  if (w->cap_stream) cudaStreamDestroy(w->cap_stream);
  if (w->st_host) cudaFreeHost(w->st_host);
  for (void* p : w->allocs) cudaFree(p);
  w->allocs.clear();
}

// Runs one solve of precision T: prepare, refinement rounds, output.
template <class T>
static int solve_impl(Workspace* w, double* x_out, double* y_out, pdhg_result* res,
                      cudaStream_t s) {
  const bool mixed = sizeof(T) == 4;
  int rc;
  if (mixed) {
    if ((rc = alloc_bufs(w, &w->b32)) != PDHG_OK) return rc;
  } else {
    if ((rc = alloc_bufs(w, &w->b64)) != PDHG_OK) return rc;
  }
  if ((rc = ensure_trace(w)) != PDHG_OK) return rc;
  const pdhg_opts& o = w->opts;
  CK(cudaEventRecord(w->ev[0], s));
  launch_prepare(w, s);
  if (mixed) {
    launch_to_f32(w->K.val64, w->K.val32, w->K.nnz_pad, s);
    launch_to_f32(w->KT.val64, w->KT.val32, w->KT.nnz_pad, s);
    w->values_f32 = true;
  }
  CK(cudaMemsetAsync(w->x_star, 0, sizeof(double) * w->n, s));
  CK(cudaMemsetAsync(w->y_star, 0, sizeof(double) * w->m, s));
  const int max_rounds = mixed ? 1 + o.ir_max_rounds : 1;
  const bool fixed = o.fixed_eta > 0.0;
  int64_t k_done = 0, accepted = 0, restarts = 0, checks = 0;
  // kernels launched by this call: preparation (8 + 4 per rescaling pass),
  // FP32 copies, then per round: correction build 4; for the first round state
  // 1, init vectors 2, first primal step 1, initial check 3, for a continued
  // round re-centering 1 and state 1; one 64-attempt body (2 per attempt + a
  // 4-kernel check) per executed check, accumulate 1; output 1.
  const int passes = o.ruiz_iters + (o.pock_chambolle ? 1 : 0);
  int64_t launches = 8 + 4 * passes + (mixed ? 2 : 0) + 1;
  // Bound/objective rescaling is round 0 of the refinement form: the solver
  // iterates on q^ = dp0 q~, [l^,u^] = dp0 [l~,u~], c^ = dd0 c~.
  double dp0 = 1.0, dd0 = 1.0, omega0 = 0.0;
  if (o.bound_obj_rescale && !fixed) {
    double sc[16];
    CK(cudaMemcpyAsync(sc, w->scalars, sizeof(sc), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    dp0 = 1.0 / (1.0 + sc[5]);
    dd0 = 1.0 / (1.0 + sc[4]);
    const double cn = dd0 * sc[4], qn = dp0 * sc[5];
    omega0 = (cn > 1e-10 && qn > 1e-10) ? cn / qn : 1.0;
  }
  double dp = dp0, dd = dd0;
  int status = 0;
  int rounds = 0;
  IterArgs<T> a = make_args<T>(w);
  bool fold = false;  // the previous round ended in a refinement fold
  double fold_f = 1.0, fold_rel = 1.0;
  for (int r = 0; r < max_rounds; ++r) {
    launch_ir_build(w, dp, dd, mixed, s);
    if (fold) {
      // continue the iteration in the new coordinates (see k_recenter)
      launch_recenter<T>(a, fold_f, s);
      RoundContinue cont{};
      cont.f = fold_f;
      cont.inv_dp = 1.0 / dp;
      cont.inv_dd = 1.0 / dd;
      cont.gap_w = dp0 / dp;
      cont.rel = fold_rel;
      cont.max_k = o.max_iters - k_done;
      cont.max_checks = (cont.max_k + kCheckEvery - 1) / kCheckEvery + 1;
      cont.k_offset = k_done;
      launch_state_continue(w->st, cont, w->scalars, s);
      launches += 4 + 2;
    } else {
      RoundInit ri{};
      ri.reset_steps = (r == 0);
      ri.eta = fixed ? o.fixed_eta : 0.0;
      ri.omega = fixed ? o.fixed_omega : omega0;
      ri.art_total = o.artificial_total ? 1 : 0;
      ri.first_round = (r == 0);
      ri.tol = o.tol;
      ri.ir_red = o.ir_reduction;
      ri.max_k = o.max_iters - k_done;
      ri.max_checks = (ri.max_k + kCheckEvery - 1) / kCheckEvery + 1;
      ri.k_offset = k_done;
      ri.t_limit_ns = (uint64_t)(o.time_limit_s * 1e9);
      ri.inv_dp = 1.0 / dp;
      ri.inv_dd = 1.0 / dd;
      ri.gap_w = dp0 / dp;
      ri.fixed = fixed ? 1 : 0;
      ri.trace_on = o.trace ? 1 : 0;
      ri.trace_cap_a = w->trace_cap_a;
      ri.trace_cap_c = w->trace_cap_c;
      ri.refine = mixed ? 1 : 0;
      ri.beta_suff = o.beta_sufficient;
      ri.beta_nec = o.beta_necessary;
      ri.beta_art = o.beta_artificial;
      ri.omega_smooth = o.omega_smoothing;
      ri.red_exp = o.step_reduction_exp;
      ri.grow_exp = o.step_growth_exp;
      ri.infeas_eps = (mixed && o.infeas_tol > 0.0) ? std::max(o.infeas_tol, kFp32RayTol) : o.infeas_tol;
      ri.fold_every = o.ir_fold_checks;
      if (r == 0 && !w->tune[mixed ? 1 : 0].done) {
        launch_state_init(w->st, ri, w->scalars, s);
        launch_init_iterates<T>(a, 0, s);
        launch_adjoint<T>(a, w->grid_kt, s, 1);
        if ((rc = autotune<T>(w, a, s)) != PDHG_OK) return rc;
      }
      if (!o.host_loop && (rc = build_graph<T>(w)) != PDHG_OK) return rc;
      launch_state_init(w->st, ri, w->scalars, s);
      launch_init_iterates<T>(a, 0, s);
      run_adjoint<T>(w, a, s);
      launch_check<T>(a, w->grid_k, w->grid_kt, 1, s);
      launches += 4 + 1 + 2 + 1 + 3;
    }
    if (o.host_loop) {
      // Same kernels as the graph body, launched from the host; the done flag
      // is read after every check (one host wait per 64 attempts).
      for (;;) {
        for (int k = 0; k < kCheckEvery; ++k) {
          run_dual<T>(w, a, s);
          run_adjoint<T>(w, a, s);
        }
        launch_check<T>(a, w->grid_k, w->grid_kt, 0, s);
        CK(cudaMemcpyAsync(w->st_host, w->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (w->st_host->done) break;
      }
    } else {
      CK(cudaGraphLaunch(w->graph_exec[mixed ? 1 : 0], s));
    }
    launch_accumulate<T>(a, w->x_star, w->y_star, 0, s);
    CK(cudaMemcpyAsync(w->st_host, w->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    const DevState& h = *w->st_host;
    if (h.wait_timeout)
      return fail(PDHG_ERR_TIMEOUT, "a staged per-attempt kernel's bounded wait for its bulk copy gave up");
    k_done += h.k;
    accepted += h.accepted;
    restarts += h.restarts;
    checks += h.checks;
    launches += h.checks * (2 * kCheckEvery + 4) + 1;
    rounds = r;
    status = h.status;
    if (h.status != 0) break;  // optimal or a limit
    // Refinement fold: the round's current iterate is now part of x*, y*.
    // Delta_P / Delta_D grow by 1/rel_kkt relative to round 0, so their ratio
    // (and with it the meaning of the primal weight) stays the same.
    const double rel = (h.rel_kkt > 0.0 && std::isfinite(h.rel_kkt)) ? h.rel_kkt : 1e-300;
    const double scale = std::min(1.0 / rel, 1e12);
    fold = true;
    fold_f = dp0 * scale / dp;
    fold_rel = rel;
    dp = dp0 * scale;
    dd = dd0 * scale;
    if (r + 1 == max_rounds) status = PDHG_STATUS_ITER_LIMIT;
  }
  launch_output(w, x_out, y_out, s);
  CK(cudaEventRecord(w->ev[1], s));
  CK(cudaEventSynchronize(w->ev[1]));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, w->ev[0], w->ev[1]));
  const DevState& h = *w->st_host;
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->status = status;
    res->ir_rounds = mixed ? rounds : 0;
    res->iterations = k_done;
    res->accepted = accepted;
    res->restarts = restarts;
    res->checks = checks;
    res->rel_p = h.rel_p;
    res->rel_d = h.rel_d;
    res->rel_gap = h.rel_gap;
    res->rel_kkt = h.rel_kkt;
    res->primal_obj = h.pobj;
    res->dual_obj = h.dobj;
    res->solve_seconds = ms * 1e-3;
    for (int i = 0; i < 3; ++i) {
      res->time_to_tol[i] = h.t_tol[i];
      res->iters_to_tol[i] = h.k_tol[i];
    }
    res->eta = h.eta;
    res->omega = h.omega;
    res->kernel_launches = launches;
    res->returned_average = h.best_is_avg;
    res->launch_overlap = (w->opts.launch_overlap && !w->overlap_refused) ? 1 : 0;
  }
  w->solved = true;
  return h.numeric ? fail(PDHG_ERR_NUMERIC, "NaN/Inf met in a KKT evaluation") : PDHG_OK;
}

}  // namespace ucpdhg

using namespace ucpdhg;

extern "C" const char* pdhg_last_error(void) { return g_err.c_str(); }

extern "C" int pdhg_opts_default(pdhg_opts* o) {
  if (!o) return fail(PDHG_ERR_INVALID_ARG, "opts is NULL");
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-8;
  o->precision = PDHG_PREC_FP64;
  o->check_every = kCheckEvery;
  o->max_iters = 10000000;
  o->time_limit_s = 600.0;
  o->beta_sufficient = 0.2;
  o->beta_necessary = 0.8;
  o->beta_artificial = 0.36;
  o->omega_smoothing = 0.5;
  o->step_reduction_exp = 0.3;
  o->step_growth_exp = 0.6;
  o->ruiz_iters = 10;
  o->pock_chambolle = 1;
  o->ir_reduction = 0.5;
  o->ir_max_rounds = 100000;
  o->trace = 0;
  o->fixed_eta = 0.0;
  o->fixed_omega = 0.0;
  o->bound_obj_rescale = 0;
  o->artificial_total = 1;
  o->host_loop = 0;
  o->autotune = 1;
  o->cancel_flag = nullptr;
  o->kernel_variant = -1;
  o->kernel_grid = 0;
  o->infeas_tol = 1e-8;
  o->ir_fold_checks = 16;
  o->launch_overlap = 0;
  return PDHG_OK;
}

extern "C" int pdhg_workspace_create(const pdhg_problem* prob, const pdhg_opts* opts, void** out,
                                     void* stream) {
  g_err.clear();
  if (!out) return fail(PDHG_ERR_INVALID_ARG, "ws out-pointer is NULL");
  *out = nullptr;
  if (!prob) return fail(PDHG_ERR_INVALID_ARG, "problem is NULL");
  if (prob->n < 1 || prob->m < 1 || prob->m_eq < 0 || prob->m_eq > prob->m || prob->nnz < 0)
    return fail(PDHG_ERR_INVALID_ARG, "problem sizes: need n, m >= 1 and 0 <= m_eq <= m");
  if (prob->n >= ((int64_t)1 << 31) - 64 || prob->m >= ((int64_t)1 << 31) - 64 ||
      prob->nnz >= ((int64_t)1 << 31))
    return fail(PDHG_ERR_UNSUPPORTED, "problem sizes must stay below 2^31");
  if (!prob->row_ptr || !prob->c || !prob->l || !prob->u || !prob->q ||
      (prob->nnz > 0 && (!prob->col || !prob->val)))
    return fail(PDHG_ERR_INVALID_ARG, "problem has a NULL device pointer");
  pdhg_opts o;
  if (opts)
    o = *opts;
  else
    pdhg_opts_default(&o);
  int rc = validate_opts(&o);
  if (rc != PDHG_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w = new Workspace();
  w->prob = *prob;
  w->opts = o;
  w->n = prob->n;
  w->m = prob->m;
  w->m_eq = prob->m_eq;
  w->nnz = prob->nnz;
  auto bail = [&](int code) {
    release(w);
    delete w;
    return code;
  };
  if (cudaGetDevice(&w->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&w->num_sms, cudaDevAttrMultiProcessorCount, w->device) != cudaSuccess)
    return bail(fail(PDHG_ERR_CUDA, "no usable CUDA device"));
  // structure to the host
  std::vector<int64_t> rp(w->m + 1);
  std::vector<int32_t> col(w->nnz);
  if (cudaMemcpyAsync(rp.data(), prob->row_ptr, sizeof(int64_t) * (w->m + 1), cudaMemcpyDeviceToHost,
                      s) != cudaSuccess ||
      (w->nnz > 0 && cudaMemcpyAsync(col.data(), prob->col, sizeof(int32_t) * w->nnz,
                                     cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return bail(fail(PDHG_ERR_CUDA, "copying the CSR structure to the host failed"));
  if (rp[0] != 0 || rp[w->m] != w->nnz) return bail(fail(PDHG_ERR_INVALID_ARG, "row_ptr inconsistent"));
  for (int64_t i = 0; i < w->m; ++i)
    if (rp[i + 1] < rp[i]) return bail(fail(PDHG_ERR_INVALID_ARG, "row_ptr not monotone"));
  HostLayout L;
  std::string err;
  rc = build_layout(w->n, w->m, w->m_eq, rp, col, &L, &err);
  if (rc != PDHG_OK) return bail(fail(rc, err));
  auto up = [&](int32_t** dst, const std::vector<int32_t>& v) -> int {
    cudaError_t e = dalloc(w, dst, v.size() + 1);
    if (e != cudaSuccess) return PDHG_ERR_NOMEM;
    if (!v.empty() &&
        cudaMemcpy(*dst, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return PDHG_ERR_CUDA;
    return PDHG_OK;
  };
  w->K.nslices = (int32_t)(L.k_off.size() - 1);
  w->K.rows = (int32_t)w->m;
  w->K.nnz_pad = L.k_col.size();
  w->KT.nslices = (int32_t)(L.t_off.size() - 1);
  w->KT.rows = (int32_t)w->n;
  w->KT.nnz_pad = L.t_col.size();
  std::vector<int32_t> kch, tch;
  if (build_chunks(L.k_off, &kch, kStageEntries, 1 << 30) && build_chunks(L.t_off, &tch, kStageEntries, 1 << 30)) {
    w->K.nchunks = (int32_t)kch.size() - 1;
    w->KT.nchunks = (int32_t)tch.size() - 1;
    if (up(&w->K.chunks, kch) || up(&w->KT.chunks, tch))
      return bail(fail(PDHG_ERR_NOMEM, "device allocation/upload of the chunk tables failed"));
  }
  if (build_chunks(L.k_off, &kch, kRsEntries, kRsSlices) && build_chunks(L.t_off, &tch, kRsEntries, kRsSlices)) {
    w->K.nchunks2 = (int32_t)kch.size() - 1;
    w->KT.nchunks2 = (int32_t)tch.size() - 1;
    if (up(&w->K.chunks2, kch) || up(&w->KT.chunks2, tch))
      return bail(fail(PDHG_ERR_NOMEM, "device allocation/upload of the chunk tables failed"));
  }
  if (up(&w->perm_row, L.perm_row) || up(&w->perm_col, L.perm_col) || up(&w->K.off, L.k_off) ||
      up(&w->K.col, L.k_col) || up(&w->K.src, L.k_src) || up(&w->KT.off, L.t_off) ||
      up(&w->KT.col, L.t_col) || up(&w->KT.src, L.t_src))
    return bail(fail(PDHG_ERR_NOMEM, "device allocation/upload of the layout failed"));
  {
    int r2 = PDHG_OK;
    auto A = [&](auto** p, size_t cnt) {
      if (r2 == PDHG_OK && dalloc(w, p, cnt) != cudaSuccess) r2 = PDHG_ERR_NOMEM;
    };
    A(&w->K.val64, w->K.nnz_pad);
    A(&w->K.val32, w->K.nnz_pad);
    A(&w->KT.val64, w->KT.nnz_pad);
    A(&w->KT.val32, w->KT.nnz_pad);
    const int64_t n = w->n, m = w->m;
    A(&w->Dr, m);
    A(&w->Dc, n);
    A(&w->fac_r, m);
    A(&w->fac_c, n);
    A(&w->iDr, m);
    A(&w->iDc, n);
    A(&w->c_s, n);
    A(&w->l_s, n);
    A(&w->u_s, n);
    A(&w->q_s, m);
    A(&w->c_h, n);
    A(&w->l_h, n);
    A(&w->u_h, n);
    A(&w->q_h, m);
    A(&w->ylo_h, m);
    A(&w->c_f, n);
    A(&w->l_f, n);
    A(&w->u_f, n);
    A(&w->q_f, m);
    A(&w->ylo_f, m);
    A(&w->x_star, n);
    A(&w->y_star, m);
    A(&w->Kz_avg, m);
    A(&w->KTz_avg, n);
    A(&w->Kz_cur, m);
    A(&w->KTz_cur, n);
    A(&w->Kx_anc, m);
    A(&w->KTy_anc, n);
    A(&w->scr_m, m);
    A(&w->scr_n, n);
    A(&w->scalars, 16);
    A(&w->st, 1);
    A(&w->st_backup, 1);
    A(&w->partials, (size_t)3 * kMaxBlocks * kRegionStride);
    if (r2 != PDHG_OK) return bail(fail(r2, "device allocation failed"));
  }
  if (cudaMallocHost(&w->st_host, sizeof(DevState)) != cudaSuccess)
    return bail(fail(PDHG_ERR_NOMEM, "pinned allocation failed"));
  if (cudaMemset(w->st, 0, sizeof(DevState)) != cudaSuccess ||
      cudaMemset(w->scalars, 0, 16 * sizeof(double)) != cudaSuccess)
    return bail(fail(PDHG_ERR_CUDA, "memset failed"));
  if (cudaStreamCreateWithFlags(&w->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(PDHG_ERR_CUDA, "stream creation failed"));
  for (int i = 0; i < 4; ++i)
    if (cudaEventCreate(&w->ev[i]) != cudaSuccess) return bail(fail(PDHG_ERR_CUDA, "event creation failed"));
  w->grid_k = grid_for(w, blocks_per_sm_iter(), w->K.nslices);
  w->grid_kt = grid_for(w, blocks_per_sm_iter(), w->KT.nslices);
  w->grid_vec = w->num_sms * 8;
  if ((rc = ensure_trace(w)) != PDHG_OK) return bail(rc);
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(fail(PDHG_ERR_CUDA, "setup failed"));
  *out = w;
  return PDHG_OK;
}

static void drop_graphs(Workspace* w) {
  for (int i = 0; i < 2; ++i) {
    if (w->graph_exec[i]) cudaGraphExecDestroy(w->graph_exec[i]);
    if (w->graph[i]) cudaGraphDestroy(w->graph[i]);
    w->graph_exec[i] = nullptr;
    w->graph[i] = nullptr;
  }
}

extern "C" void pdhg_workspace_destroy(void* ws) {
  if (!ws) return;
  Workspace* w = (Workspace*)ws;
  release(w);
  delete w;
}

extern "C" int pdhg_set_opts(void* ws, const pdhg_opts* opts) {
  g_err.clear();
  if (!ws || !opts) return fail(PDHG_ERR_INVALID_ARG, "NULL argument");
  int rc = validate_opts(opts);
  if (rc != PDHG_OK) return rc;
  Workspace* w = (Workspace*)ws;
  w->opts = *opts;
  drop_graphs(w);  // graphs bake the cancel and trace pointers in
  release_batched(w);
  return ensure_trace(w);
}

extern "C" int pdhg_solve(void* ws, double* x_out, double* y_out, pdhg_result* res, void* stream) {
  g_err.clear();
  if (!ws) return fail(PDHG_ERR_INVALID_ARG, "workspace is NULL");
  Workspace* w = (Workspace*)ws;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != w->device)
    return fail(PDHG_ERR_INVALID_ARG, "current device differs from the workspace's device");
  cudaStream_t s = (cudaStream_t)stream;
  if (w->opts.precision == PDHG_PREC_MIXED) return solve_impl<float>(w, x_out, y_out, res, s);
  return solve_impl<double>(w, x_out, y_out, res, s);
}

extern "C" int pdhg_prepare(void* ws, void* stream) {
  g_err.clear();
  if (!ws) return fail(PDHG_ERR_INVALID_ARG, "workspace is NULL");
  Workspace* w = (Workspace*)ws;
  cudaStream_t s = (cudaStream_t)stream;
  launch_prepare(w, s);
  launch_to_f32(w->K.val64, w->K.val32, w->K.nnz_pad, s);
  launch_to_f32(w->KT.val64, w->KT.val32, w->KT.nnz_pad, s);
  w->values_f32 = true;
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  return PDHG_OK;
}

extern "C" int pdhg_get_scaling(void* ws, double* Dr, double* Dc, void* stream) {
  g_err.clear();
  if (!ws || !Dr || !Dc) return fail(PDHG_ERR_INVALID_ARG, "NULL argument");
  Workspace* w = (Workspace*)ws;
  cudaStream_t s = (cudaStream_t)stream;
  launch_scatter_perm(w->perm_row, w->Dr, Dr, w->m, s);
  launch_scatter_perm(w->perm_col, w->Dc, Dc, w->n, s);
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  return PDHG_OK;
}

extern "C" int pdhg_apply_K(void* ws, int32_t transpose, int32_t precision, const double* in,
                            double* out, void* stream) {
  g_err.clear();
  if (!ws || !in || !out) return fail(PDHG_ERR_INVALID_ARG, "NULL argument");
  if (precision != PDHG_PREC_FP64 && precision != PDHG_PREC_MIXED)
    return fail(PDHG_ERR_INVALID_ARG, "precision must be PDHG_PREC_FP64 or PDHG_PREC_MIXED");
  Workspace* w = (Workspace*)ws;
  cudaStream_t s = (cudaStream_t)stream;
  const bool tr = transpose != 0;
  const int32_t* perm_in = tr ? w->perm_row : w->perm_col;
  const int32_t* perm_out = tr ? w->perm_col : w->perm_row;
  const int64_t nin = tr ? w->m : w->n, nout = tr ? w->n : w->m;
  double* tin = tr ? w->scr_m : w->scr_n;
  double* tout = tr ? w->scr_n : w->scr_m;
  launch_gather_perm(perm_in, in, tin, nin, s);
  if (precision == PDHG_PREC_FP64) {
    launch_spmv64(tr ? w->KT.v64() : w->K.v64(), tin, tout, tr ? w->grid_kt : w->grid_k, s);
  } else {
    if (!w->values_f32) return fail(PDHG_ERR_INVALID_ARG, "FP32 values not prepared");
    float* fin = (float*)w->Kz_avg;  // scratch reuse: m doubles hold n or m floats
    float* fout = (float*)w->KTz_avg;
    if (tr) {
      fin = (float*)w->KTz_avg;
      fout = (float*)w->Kz_avg;
    }
    // Kz_avg has m doubles, KTz_avg n doubles: each holds 2x as many floats
    launch_to_f32(tin, tr ? (float*)w->Kz_avg : (float*)w->KTz_avg, nin, s);
    fin = tr ? (float*)w->Kz_avg : (float*)w->KTz_avg;
    fout = tr ? (float*)w->KTz_avg : (float*)w->Kz_avg;
    launch_spmv32(tr ? w->KT.v32() : w->K.v32(), fin, fout, tr ? w->grid_kt : w->grid_k, s);
    launch_to_f64(fout, tout, nout, s);
  }
  launch_scatter_perm(perm_out, tout, out, nout, s);
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  return PDHG_OK;
}

extern "C" int pdhg_get_trace(void* ws, double* attempts, int64_t cap_a, double* checks,
                              int64_t cap_c, int64_t* n_a, int64_t* n_c) {
  g_err.clear();
  if (!ws || !n_a || !n_c) return fail(PDHG_ERR_INVALID_ARG, "NULL argument");
  Workspace* w = (Workspace*)ws;
  if (!w->trace_a) return fail(PDHG_ERR_INVALID_ARG, "tracing was not enabled (opts.trace)");
  DevState h;
  CK(cudaMemcpy(&h, w->st, sizeof(DevState), cudaMemcpyDeviceToHost));
  *n_a = h.n_trace_a;
  *n_c = h.n_trace_c;
  int64_t ca = std::min(std::min(cap_a, h.n_trace_a), w->trace_cap_a);
  int64_t cc = std::min(std::min(cap_c, h.n_trace_c), w->trace_cap_c);
  if (attempts && ca > 0)
    CK(cudaMemcpy(attempts, w->trace_a, sizeof(double) * 5 * ca, cudaMemcpyDeviceToHost));
  if (checks && cc > 0)
    CK(cudaMemcpy(checks, w->trace_c, sizeof(double) * kTraceCheckCols * cc, cudaMemcpyDeviceToHost));
  return PDHG_OK;
}

extern "C" int pdhg_get_tuning(void* ws, int32_t* cfg) {
  g_err.clear();
  if (!ws || !cfg) return fail(PDHG_ERR_INVALID_ARG, "NULL argument");
  Workspace* w = (Workspace*)ws;
  for (int p = 0; p < 2; ++p) {
    const Tune& t = w->tune[p];
    cfg[4 * p + 0] = t.done ? t.unroll_dual : -1;
    cfg[4 * p + 1] = t.done ? t.grid_dual : 0;
    cfg[4 * p + 2] = t.done ? t.unroll_adj : -1;
    cfg[4 * p + 3] = t.done ? t.grid_adj : 0;
  }
  batched_tuning(w, cfg + 8);
  return PDHG_OK;
}

extern "C" int pdhg_time_kernels(void* ws, int32_t precision, int32_t reps, double* ms_dual,
                                 double* ms_adj, double* bytes_dual, double* bytes_adj,
                                 void* stream) {
  g_err.clear();
  if (!ws || reps < 1) return fail(PDHG_ERR_INVALID_ARG, "bad argument");
  Workspace* w = (Workspace*)ws;
  cudaStream_t s = (cudaStream_t)stream;
  const bool f32 = precision == PDHG_PREC_MIXED;
  if ((f32 && !w->b32.allocated) || (!f32 && !w->b64.allocated))
    return fail(PDHG_ERR_INVALID_ARG, "run a solve of this precision first");
  CK(cudaMemcpyAsync(w->st_backup, w->st, sizeof(DevState), cudaMemcpyDeviceToDevice, s));
  k_reopen_state<<<1, 1, 0, s>>>(w->st);
  float t_d = 0.f, t_a = 0.f;
  if (f32) {
    IterArgs<float> a = make_args<float>(w);
    run_dual<float>(w, a, s);
    run_adjoint<float>(w, a, s);
    CK(cudaEventRecord(w->ev[0], s));
    for (int r = 0; r < reps; ++r) run_dual<float>(w, a, s);
    CK(cudaEventRecord(w->ev[1], s));
    for (int r = 0; r < reps; ++r) run_adjoint<float>(w, a, s);
    CK(cudaEventRecord(w->ev[2], s));
  } else {
    IterArgs<double> a = make_args<double>(w);
    run_dual<double>(w, a, s);
    run_adjoint<double>(w, a, s);
    CK(cudaEventRecord(w->ev[0], s));
    for (int r = 0; r < reps; ++r) run_dual<double>(w, a, s);
    CK(cudaEventRecord(w->ev[1], s));
    for (int r = 0; r < reps; ++r) run_adjoint<double>(w, a, s);
    CK(cudaEventRecord(w->ev[2], s));
  }
  CK(cudaEventSynchronize(w->ev[2]));
  CK(cudaEventElapsedTime(&t_d, w->ev[0], w->ev[1]));
  CK(cudaEventElapsedTime(&t_a, w->ev[1], w->ev[2]));
  CK(cudaMemcpyAsync(w->st, w->st_backup, sizeof(DevState), cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  const double sz = f32 ? 4.0 : 8.0;
  const double n = (double)w->n, m = (double)w->m, nnz = (double)w->nnz;
  // algorithmic bytes: CSR-equivalent matrix stream (value + int32 column +
  // int32 row pointer), each gathered vector once, each streamed vector once.
  // dual, FP32: x' and x gathered; y, q, y_lo, ybar read; ybar, y' written
  // dual, FP64: x' gathered; y, q, ybar, K x read; ybar, y', K x' written
  // adjoint: y' gathered; x, xbar, c, l, u read; xbar, K^T y', x'' written
  if (ms_dual) *ms_dual = t_d / reps;
  if (ms_adj) *ms_adj = t_a / reps;
  if (bytes_dual)
    *bytes_dual = f32 ? nnz * (sz + 4.0) + 4.0 * m + 2.0 * sz * n + sz * m * 6.0
                      : nnz * (sz + 4.0) + 4.0 * m + sz * n + sz * m * 7.0;
  if (bytes_adj) *bytes_adj = nnz * (sz + 4.0) + 4.0 * n + sz * m + sz * n * 8.0;
  return PDHG_OK;
}

extern "C" int pdhg_solve_batched(void* ws, int32_t B, const double* l_b, const double* u_b,
                                  double* x_out, double* y_out, pdhg_result* res_b, void* stream);
extern "C" int pdhg_backward(void* ws, double g_cost, const double* g_x, double* grad_q,
                             double* grad_c, void* stream);
