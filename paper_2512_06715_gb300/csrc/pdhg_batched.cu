// Batched node LPs that share K, c and q and differ in their bounds (the
// branch-and-bound relaxations whose bounds the paper's PDHG provides,
// Sec. III.B), solved together: FP32 iterations, FP64 KKT checks and FP64
// iterative refinement, with per-instance step size, primal weight, restarts,
// refinement rounds and termination.
//
// Layout: every per-instance vector is interleaved, v[i * BP + b] (BP = 32 or
// 64 instance slots), so one sweep over K serves all instances: a warp owns a
// row, its lanes own instances, the row's column/value loads are broadcasts
// and the gather x[col * BP + b] is one contiguous 128/256 B access.
//
// Refinement rounds run inside the graph: when an instance's current iterate
// (x^, y^) halves the round's starting rel-KKT at a check without a restart,
// the next correction LP follows elementwise from the FP64 products the check
// already computed (K x^ and K^T y^):
//   q^' = f (q^ - K x^),  c^' = f (c^ - K^T y^),  [l^',u^'] = f ([l^,u^] - x^),
//   y_lo^' = f (y_lo^ - y^),  f = Delta'/Delta,  x* += x^/Delta,  y* += y^/Delta
// and the iteration state moves to the new coordinates v' = f (v - x^): the
// iterate becomes 0 (K x^ = K^T y^ = 0), anchors and averages shift with it,
// step size, primal weight and restart window carry over.  The whole batch is
// one CUDA graph whose while loop runs until every instance is done.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace ucpdhg {
namespace {

constexpr int kBWarps = 8;            // warps per block of the row/column sweeps
constexpr int kBThreads = kBWarps * 32;
constexpr int kKktWarps = 4;          // smaller blocks for the FP64 check sweeps
constexpr int kApplyRows = 4;         // rows per block of the elementwise kernels (x BP threads)
constexpr int kRowS = 7, kColS = 9;   // per-candidate sums (as in the single-instance check,
                                      // including the infeasibility-ray sums)
// Rows (columns) a warp sweeps together in kb_dual (kb_adjoint): R = 4, 2 or 1
// adjacent slots of a slice, read as int4/float4, int2/float2 or scalars; the
// batched autotuner picks R and the grid per matrix and batch width.
template <int R>
__device__ __forceinline__ void load_slots(const int32_t* __restrict__ c, const float* __restrict__ v,
                                           int (&cc)[R], float (&vv)[R]) {
  if constexpr (R == 4) {
    const int4 c4 = __ldg(reinterpret_cast<const int4*>(c));
    const float4 v4 = __ldg(reinterpret_cast<const float4*>(v));
    cc[0] = c4.x; cc[1] = c4.y; cc[2] = c4.z; cc[3] = c4.w;
    vv[0] = v4.x; vv[1] = v4.y; vv[2] = v4.z; vv[3] = v4.w;
  } else if constexpr (R == 2) {
    const int2 c2 = __ldg(reinterpret_cast<const int2*>(c));
    const float2 v2 = __ldg(reinterpret_cast<const float2*>(v));
    cc[0] = c2.x; cc[1] = c2.y;
    vv[0] = v2.x; vv[1] = v2.y;
  } else {
    cc[0] = __ldg(c);
    vv[0] = __ldg(v);
  }
}

// Per-instance state (array of B structs in device memory).
struct BInst {
  double eta, omega, dx2, w_last, pending_w, wsum, avg_div;
  int32_t par, accepted_last;
  int64_t k, k_total, since_restart, accepted, restarts, checks;
  double kkt0, kkt_prev;
  int32_t restart_now, restart_to_avg;
  int32_t done, status, rounds, act;  // act: takes part in the next attempts
  int32_t refine, finalize, cand_avg, round_checks;  // round_checks: checks this round
  double rel_p, rel_d, rel_gap, rel_kkt, pobj, dobj;
  double round_target;
  double round_rel0;      // rel_kkt of the current iterate at the round's start
  double dp, dd;          // Delta_P, Delta_D of the current round
  double next_scale;      // Delta' / Delta for the refinement step
  double const_p, const_d;
  double t_tol[3];
  int64_t k_tol[3];
  uint32_t pad2, pad3;
};

struct BGlobal {
  double tol, red;
  double beta_suff, beta_nec, beta_art, omega_smooth, red_exp, grow_exp;
  int64_t max_k;
  uint64_t t_start, t_limit_ns;
  double qnorm, cnorm;
  double infeas_eps;  // certificate tolerance of the infeasibility test (0: off)
  int32_t fold_every;  // a refinement round also ends after this many checks (0: off)
  int32_t n_real, all_done;
  uint32_t counter, counter2;
};

template <int BP>
struct BArgs {
  SellView<float> K, KT;      // FP32 values (iterations)
  SellView<double> K64, KT64; // FP64 values (checks)
  int32_t n, m, m_eq, B;
  // FP32 iterate data [len * BP]
  float *x[2], *y[2], *Kx[2], *KTy[2];
  float *xbar, *ybar, *xa, *ya;  // xbar, ybar: step-weighted sums since the last check
  double *xbar64, *ybar64;        // the sums since the last restart (FP64; the window's
                                  // FP32 sums are added in and cleared at every check,
                                  // so refinement folds re-express exact sums)
  float *cf, *lf, *uf, *qf, *ylf;
  // FP64 data [len * BP]
  double *xst, *yst;          // accumulated x*, y* (scaled space)
  double *ch, *lh, *uh;       // correction c^, l^, u^
  double *qh, *ylh;           // correction q^, y_lo^
  double *lo, *uo;            // instance bounds l~, u~ (scaled)
  double *Kzc, *Kza;          // K x^ of current / average (FP64)
  double *KTzc, *KTza;        // K^T y^ of current / average
  double *Kxa, *KTya;         // K x^, K^T y^ of the restart anchors (infeasibility rays)
  const double *c_obj, *q_obj, *iDr, *iDc, *Dr, *Dc;  // shared [len]
  BInst* inst;
  BGlobal* g;
  double* part;               // per-block partials
  volatile int32_t* cancel;
  unsigned long long cond;
  int32_t in_graph;
};

__device__ __forceinline__ double* preg(double* p, int r) { return p + (size_t)r * 8192 * 64 * 20; }

// Per-instance block reduction of NV values held by each lane for its
// instances b = lane + 32 h; result written to part[block][b][k] by threads
// b < BP.  smem: [warps][BP][NV].
template <int BP, int NV, int WARPS>
__device__ __forceinline__ void block_inst_sum(const double (&v)[BP / 32][NV], double* smem, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int h = 0; h < BP / 32; ++h)
#pragma unroll
    for (int k = 0; k < NV; ++k) smem[(wid * BP + lane + 32 * h) * NV + k] = v[h][k];
  __syncthreads();
  if (threadIdx.x < BP) {
    const int b = threadIdx.x;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int w = 0; w < WARPS; ++w) s += smem[(w * BP + b) * NV + k];
      out[((size_t)blockIdx.x * BP + b) * NV + k] = s;
    }
  }
  __syncthreads();
}

// Per-instance sums of NV partials over `nblocks` blocks (layout
// part[blk][BP][NV]) by ALL threads of the calling block: thread t sums the
// blocks t/BP, t/BP + C, ... (C = blockDim / BP chunks) for instance t % BP,
// then the chunks are combined in order.  Deterministic; result valid in
// threads t < BP.  smem: [C][BP][NV] doubles.
template <int BP, int NV>
__device__ __forceinline__ void inst_final_sum(const double* part, int nblocks, double* smem,
                                               double (&out)[NV]) {
  const int b = threadIdx.x % BP, c = threadIdx.x / BP, C = blockDim.x / BP;
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  if (c < C)
    for (int blk = c; blk < nblocks; blk += C)
#pragma unroll
      for (int k = 0; k < NV; ++k) v[k] += __ldcg(part + ((size_t)blk * BP + b) * NV + k);
#pragma unroll
  for (int k = 0; k < NV; ++k) smem[(c * BP + b) * NV + k] = v[k];
  __syncthreads();
  if (threadIdx.x < BP) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int cc = 0; cc < C; ++cc) s += smem[(cc * BP + b) * NV + k];
      out[k] = s;
    }
  }
  __syncthreads();
}

// Last-block detection shared by the kernels that finish with per-instance sums.
__device__ __forceinline__ bool last_block(uint32_t* counter) {
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  return last != 0;
}

// ---------------------------------------------------------------- attempt kernels

// K x' and the projected dual step for every active instance; the last block
// takes each instance's adaptive step decision.
template <int BP, int RW>
__global__ void __launch_bounds__(kBThreads) kb_dual(BArgs<BP> a) {
  BGlobal* g = a.g;
  if (g->all_done) return;
  constexpr int H = BP / 32;
  __shared__ float s_sigma[BP], s_pw[BP];
  __shared__ int s_par[BP], s_act[BP];
  if (threadIdx.x < BP) {
    const BInst& I = a.inst[threadIdx.x];
    s_sigma[threadIdx.x] = (float)(I.eta * I.omega);
    s_pw[threadIdx.x] = (float)I.pending_w;
    s_par[threadIdx.x] = I.par;
    s_act[threadIdx.x] = I.act;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * kBThreads + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kBThreads) >> 5;
  float a_dy2[H], a_int[H];
#pragma unroll
  for (int h = 0; h < H; ++h) a_dy2[h] = a_int[h] = 0.f;
  // gather base of each lane's instances (null: instance idle)
  const float* xg[H];
#pragma unroll
  for (int h = 0; h < H; ++h) {
    const int b = lane + 32 * h;
    xg[h] = s_act[b] ? a.x[1 - s_par[b]] + b : nullptr;
  }
  const int nq = (a.m + RW - 1) / RW;
  for (int qd = gw; qd < nq; qd += nw) {
    const int i0 = qd * RW;  // RW consecutive rows of one slice
    const int s = i0 >> 5;
    const int o_s = __ldg(a.K.off + s);
    const int base = o_s + (i0 & 31);
    const int w = (__ldg(a.K.off + s + 1) - o_s) >> 5;
    // row operands do not depend on the products: issue them first so their
    // latency overlaps the matrix stream and the gathers
    float ko[RW][H], yo[RW][H], qv[RW][H], lo[RW][H],
        yb[RW][H];
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const int b = lane + 32 * h, i = i0 + r;
        ko[r][h] = yo[r][h] = qv[r][h] = lo[r][h] = yb[r][h] = 0.f;
        if (i < a.m && xg[h]) {
          const size_t idx = (size_t)i * BP + b;
          const int p = s_par[b];
          ko[r][h] = a.Kx[p][idx];
          yo[r][h] = a.y[p][idx];
          qv[r][h] = a.qf[idx];
          if (i >= a.m_eq) lo[r][h] = a.ylf[idx];
          if (s_pw[b] != 0.f) yb[r][h] = a.ybar[idx];
        }
      }
    float acc[RW][H];
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
      for (int h = 0; h < H; ++h) acc[r][h] = 0.f;
    // entry k of the group's rows: RW adjacent slots (16 B aligned:
    // slice offsets are multiples of 32 and i0 of RW)
#pragma unroll 2
    for (int k = 0; k < w; ++k) {
      int c[RW];
      float v[RW];
      load_slots<RW>(a.K.col + base + k * kSlice, a.K.val + base + k * kSlice, c, v);
#pragma unroll
      for (int r = 0; r < RW; ++r)
#pragma unroll
        for (int h = 0; h < H; ++h)
          if (xg[h]) acc[r][h] += v[r] * __ldg(xg[h] + (size_t)c[r] * BP);
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      const int i = i0 + r;
      if (i >= a.m) continue;
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const int b = lane + 32 * h;
        if (!xg[h]) continue;
        const size_t idx = (size_t)i * BP + b;
        const int p = s_par[b];
        float t = qv[r][h] - 2.f * acc[r][h];
        t = t + ko[r][h];
        float v = yo[r][h] + s_sigma[b] * t;
        if (i >= a.m_eq) v = fmaxf(v, lo[r][h]);
        a.Kx[1 - p][idx] = acc[r][h];
        a.y[1 - p][idx] = v;
        if (s_pw[b] != 0.f) a.ybar[idx] = yb[r][h] + s_pw[b] * yo[r][h];
        const float dy = v - yo[r][h], dk = acc[r][h] - ko[r][h];
        a_dy2[h] += dy * dy;
        a_int[h] += dy * dk;
      }
    }
  }
  __shared__ double smem[kBWarps * BP * 2];
  double v[H][2];
#pragma unroll
  for (int h = 0; h < H; ++h) {
    v[h][0] = (double)a_dy2[h];
    v[h][1] = (double)a_int[h];
  }
  block_inst_sum<BP, 2, kBWarps>(v, smem, a.part);
  if (last_block(&g->counter)) {
    double tot[2];
    inst_final_sum<BP, 2>(a.part, gridDim.x, smem, tot);
    if (threadIdx.x < BP) {
      const int b = threadIdx.x;
      BInst& I = a.inst[b];
      if (I.act) {
        const double dy2 = tot[0], inter = tot[1];
        const double eta = I.eta, omega = I.omega;
        const double movement = omega * I.dx2 + dy2 / omega;
        const double interaction = 2.0 * fabs(inter);
        const double eta_max = interaction > 0.0 ? movement / interaction : INFINITY;
        I.k += 1;
        I.k_total += 1;
        // attempts of all rounds (a refinement round is a change of coordinates)
        const double eta_next = fmin((1.0 - step_power(I.k_total + 1, g->red_exp)) * eta_max,
                                     (1.0 + step_power(I.k_total + 1, g->grow_exp)) * eta);
        const int accept = eta <= eta_max;
        if (accept) {
          I.par = 1 - I.par;
          I.w_last = eta;
          I.pending_w = eta;
          I.wsum += eta;
          I.accepted += 1;
        } else {
          I.w_last = 0.0;
          I.pending_w = 0.0;
        }
        I.accepted_last = accept;
        I.since_restart += 1;
        I.eta = eta_next;
      }
    }
    if (threadIdx.x == 0) g->counter = 0;
  }
}

// K^T y' for instances whose step was accepted, the x-average update and the
// next primal step x'' = proj(x - tau (c - K^T y)).
template <int BP, int RW>
__global__ void __launch_bounds__(kBThreads) kb_adjoint(BArgs<BP> a) {
  BGlobal* g = a.g;
  if (g->all_done) return;
  constexpr int H = BP / 32;
  __shared__ float s_tau[BP], s_wl[BP];
  __shared__ int s_par[BP], s_act[BP], s_acc[BP];
  if (threadIdx.x < BP) {
    const BInst& I = a.inst[threadIdx.x];
    s_tau[threadIdx.x] = (float)(I.eta / I.omega);
    s_wl[threadIdx.x] = (float)I.w_last;
    s_par[threadIdx.x] = I.par;
    s_act[threadIdx.x] = I.act;
    s_acc[threadIdx.x] = I.act && I.accepted_last;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * kBThreads + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kBThreads) >> 5;
  float a_dx2[H];
#pragma unroll
  for (int h = 0; h < H; ++h) a_dx2[h] = 0.f;
  // gather base of each lane's instances (null: no new K^T y this attempt)
  const float* yg[H];
#pragma unroll
  for (int h = 0; h < H; ++h) {
    const int b = lane + 32 * h;
    yg[h] = s_acc[b] ? a.y[s_par[b]] + b : nullptr;
  }
  const int nq = (a.n + RW - 1) / RW;
  for (int qd = gw; qd < nq; qd += nw) {
    const int j0 = qd * RW;  // RW consecutive columns of one slice
    const int s = j0 >> 5;
    const int o_s = __ldg(a.KT.off + s);
    const int base = o_s + (j0 & 31);
    const int w = (__ldg(a.KT.off + s + 1) - o_s) >> 5;
    float x0[RW][H], cv[RW][H], lv[RW][H], uv[RW][H],
        xb[RW][H], go[RW][H];
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const int b = lane + 32 * h, j = j0 + r;
        x0[r][h] = cv[r][h] = lv[r][h] = uv[r][h] = xb[r][h] = go[r][h] = 0.f;
        if (j < a.n && s_act[b]) {
          const size_t idx = (size_t)j * BP + b;
          const int p = s_par[b];
          x0[r][h] = a.x[p][idx];
          cv[r][h] = a.cf[idx];
          lv[r][h] = a.lf[idx];
          uv[r][h] = a.uf[idx];
          if (!s_acc[b]) go[r][h] = a.KTy[p][idx];
          if (s_acc[b] && s_wl[b] != 0.f) xb[r][h] = a.xbar[idx];
        }
      }
    float acc[RW][H];
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
      for (int h = 0; h < H; ++h) acc[r][h] = 0.f;
#pragma unroll 2
    for (int k = 0; k < w; ++k) {
      int c[RW];
      float v[RW];
      load_slots<RW>(a.KT.col + base + k * kSlice, a.KT.val + base + k * kSlice, c, v);
#pragma unroll
      for (int r = 0; r < RW; ++r)
#pragma unroll
        for (int h = 0; h < H; ++h)
          if (yg[h]) acc[r][h] += v[r] * __ldg(yg[h] + (size_t)c[r] * BP);
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      const int j = j0 + r;
      if (j >= a.n) continue;
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const int b = lane + 32 * h;
        if (!s_act[b]) continue;
        const size_t idx = (size_t)j * BP + b;
        const int p = s_par[b];
        float gval;
        if (s_acc[b]) {
          gval = acc[r][h];
          a.KTy[p][idx] = gval;
          if (s_wl[b] != 0.f) a.xbar[idx] = xb[r][h] + s_wl[b] * x0[r][h];
        } else {
          gval = go[r][h];
        }
        float v = x0[r][h] - s_tau[b] * (cv[r][h] - gval);
        v = fminf(fmaxf(v, lv[r][h]), uv[r][h]);
        a.x[1 - p][idx] = v;
        const float d = v - x0[r][h];
        a_dx2[h] += d * d;
      }
    }
  }
  __shared__ double smem[kBWarps * BP];
  double v[H][1];
#pragma unroll
  for (int h = 0; h < H; ++h) v[h][0] = (double)a_dx2[h];
  block_inst_sum<BP, 1, kBWarps>(v, smem, a.part);
  if (last_block(&g->counter)) {
    double tot[1];
    inst_final_sum<BP, 1>(a.part, gridDim.x, smem, tot);
    if (threadIdx.x < BP) {
      const int b = threadIdx.x;
      if (a.inst[b].act) a.inst[b].dx2 = tot[0];
    }
    if (threadIdx.x == 0) g->counter = 0;
  }
}

// ---------------------------------------------------------------- checks (FP64)

// The infeasibility rays of each instance are the differences of its current
// and average iterates from its last restart anchor, tested as in the
// single-instance check (pdhg_kkt.cu): the anchors' FP64 products Kxa, KTya are
// seeded at the first check and moved at restarts and refinement folds.
template <int BP>
__global__ void __launch_bounds__(kKktWarps * 32) kb_kkt_row(BArgs<BP> a, int init) {
  BGlobal* g = a.g;
  if (g->all_done) return;
  constexpr int H = BP / 32;
  __shared__ double s_iw[BP], s_idp[BP], s_pw[BP];
  __shared__ int s_par[BP], s_act[BP];
  if (threadIdx.x < BP) {
    const BInst& I = a.inst[threadIdx.x];
    s_iw[threadIdx.x] = I.wsum > 0.0 ? 1.0 / I.wsum : 0.0;
    s_idp[threadIdx.x] = 1.0 / I.dp;
    s_pw[threadIdx.x] = I.pending_w;
    s_par[threadIdx.x] = I.par;
    s_act[threadIdx.x] = I.act;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  double acc[H][2 * kRowS];
#pragma unroll
  for (int h = 0; h < H; ++h)
#pragma unroll
    for (int k = 0; k < 2 * kRowS; ++k) acc[h][k] = 0.0;
  for (int i = gw; i < a.m; i += nw) {
    const int s = i >> 5, r = i & 31;
    const int o0 = __ldg(a.K64.off + s) + r;
    const int w = (__ldg(a.K64.off + s + 1) - __ldg(a.K64.off + s)) >> 5;
    double d0[H], d1[H];
#pragma unroll
    for (int h = 0; h < H; ++h) d0[h] = d1[h] = 0.0;
    for (int k = 0; k < w; ++k) {
      const int c = __ldg(a.K64.col + o0 + k * kSlice);
      const double v = __ldg(a.K64.val + o0 + k * kSlice);
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const int b = lane + 32 * h;
        if (!s_act[b]) continue;
        const size_t ci = (size_t)c * BP + b;
        d0[h] += v * (double)a.x[s_par[b]][ci];
        if (s_iw[b] > 0.0) d1[h] += v * ((double)a.xbar[ci] + a.xbar64[ci]);
      }
    }
    const double qo = a.q_obj[i], sr0 = a.iDr[i], dr0 = a.Dr[i];
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int b = lane + 32 * h;
      if (!s_act[b]) continue;
      const size_t idx = (size_t)i * BP + b;
      const bool has_avg = s_iw[b] > 0.0;
      const float yo = a.y[s_par[b]][idx];
      float yb = a.ybar[idx];
      if (s_pw[b] != 0.0) yb = yb + (float)s_pw[b] * yo;
      const double ybs = (double)yb + a.ybar64[idx];
      a.ybar64[idx] = ybs;
      a.ybar[idx] = 0.f;
      const double kx_avg = has_avg ? d1[h] * s_iw[b] : d0[h];
      a.Kzc[idx] = d0[h];
      a.Kza[idx] = kx_avg;
      if (init) a.Kxa[idx] = d0[h];
      const double kanc = init ? d0[h] : a.Kxa[idx];
      const double y_avg = has_avg ? ybs * s_iw[b] : (double)yo;
      const double qr = a.qh[idx], sr = s_idp[b] * sr0;
      const double yanc = (double)a.ya[idx];
      const bool ineq = i >= a.m_eq;
#pragma unroll
      for (int cnd = 0; cnd < 2; ++cnd) {
        const double kx = cnd ? kx_avg : d0[h];
        const double yv = cnd ? y_avg : (double)yo;
        double rr = qr - kx;
        if (ineq) rr = fmax(rr, 0.0);
        const double ru = rr * sr, dd = yv - yanc;
        const double kdx = (kx - kanc) * sr0;
        const double vr = ineq ? fmin(kdx, 0.0) : kdx;
        const double vs = ineq ? fmin(dd, 0.0) * dr0 : 0.0;
        acc[h][cnd * kRowS + 0] += rr * rr;
        acc[h][cnd * kRowS + 1] += ru * ru;
        acc[h][cnd * kRowS + 2] += qo * yv;
        acc[h][cnd * kRowS + 3] += dd * dd;
        acc[h][cnd * kRowS + 4] += vr * vr;
        acc[h][cnd * kRowS + 5] += vs * vs;
        acc[h][cnd * kRowS + 6] += qo * dd;
      }
    }
  }
  __shared__ double smem[kKktWarps * BP * 2 * kRowS];
  block_inst_sum<BP, 2 * kRowS, kKktWarps>(acc, smem, preg(a.part, 1));
}

template <int BP>
__global__ void __launch_bounds__(kKktWarps * 32) kb_kkt_col(BArgs<BP> a, int init) {
  BGlobal* g = a.g;
  if (g->all_done) return;
  constexpr int H = BP / 32;
  __shared__ double s_iw[BP], s_idd[BP];
  __shared__ int s_par[BP], s_act[BP];
  if (threadIdx.x < BP) {
    const BInst& I = a.inst[threadIdx.x];
    s_iw[threadIdx.x] = I.wsum > 0.0 ? 1.0 / I.wsum : 0.0;
    s_idd[threadIdx.x] = 1.0 / I.dd;
    s_par[threadIdx.x] = I.par;
    s_act[threadIdx.x] = I.act;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  double acc[H][2 * kColS];
#pragma unroll
  for (int h = 0; h < H; ++h)
#pragma unroll
    for (int k = 0; k < 2 * kColS; ++k) acc[h][k] = 0.0;
  for (int j = gw; j < a.n; j += nw) {
    const int s = j >> 5, r = j & 31;
    const int o0 = __ldg(a.KT64.off + s) + r;
    const int w = (__ldg(a.KT64.off + s + 1) - __ldg(a.KT64.off + s)) >> 5;
    double e0[H], e1[H];
#pragma unroll
    for (int h = 0; h < H; ++h) e0[h] = e1[h] = 0.0;
    for (int k = 0; k < w; ++k) {
      const int c = __ldg(a.KT64.col + o0 + k * kSlice);
      const double v = __ldg(a.KT64.val + o0 + k * kSlice);
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const int b = lane + 32 * h;
        if (!s_act[b]) continue;
        const size_t ci = (size_t)c * BP + b;
        e0[h] += v * (double)a.y[s_par[b]][ci];
        if (s_iw[b] > 0.0) e1[h] += v * ((double)a.ybar[ci] + a.ybar64[ci]);
      }
    }
    const double co = a.c_obj[j], sc0 = a.iDc[j], dc0 = a.Dc[j];
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int b = lane + 32 * h;
      if (!s_act[b]) continue;
      const size_t idx = (size_t)j * BP + b;
      const bool has_avg = s_iw[b] > 0.0;
      const double kty_avg = has_avg ? e1[h] * s_iw[b] : e0[h];
      a.KTzc[idx] = e0[h];
      a.KTza[idx] = kty_avg;
      if (init) a.KTya[idx] = e0[h];
      const double kanc = init ? e0[h] : a.KTya[idx];
      const double xc = (double)a.x[s_par[b]][idx];
      const double xbs = (double)a.xbar[idx] + a.xbar64[idx];
      a.xbar64[idx] = xbs;
      a.xbar[idx] = 0.f;
      const double x_avg = has_avg ? xbs * s_iw[b] : xc;
      const double lo = a.lo[idx], up = a.uo[idx];
      const bool lf = isfinite(lo), uf = isfinite(up);
      const double cr = a.ch[idx], sc = s_idd[b] * sc0, xanc = (double)a.xa[idx];
#pragma unroll
      for (int cnd = 0; cnd < 2; ++cnd) {
        const double kty = cnd ? kty_avg : e0[h];
        const double xv = cnd ? x_avg : xc;
        const double lam = cr - kty;
        const double proj = (lf ? fmax(lam, 0.0) : 0.0) + (uf ? fmin(lam, 0.0) : 0.0);
        const double rd = lam - proj, rdu = rd * sc, lp = proj * s_idd[b];
        const double bnd = (lf ? lo * fmax(lp, 0.0) : 0.0) - (uf ? up * fmax(-lp, 0.0) : 0.0);
        const double dx = xv - xanc;
        const double lr = kanc - kty, lru = lr * sc0;
        const double vl = (lf ? 0.0 : fmax(lru, 0.0)) + (uf ? 0.0 : fmin(lru, 0.0));
        const double bray = (lf ? lo * fmax(lr, 0.0) : 0.0) - (uf ? up * fmax(-lr, 0.0) : 0.0);
        const double dxu = dx * dc0;
        const double vb = (lf ? fmin(dxu, 0.0) : 0.0) + (uf ? fmax(dxu, 0.0) : 0.0);
        acc[h][cnd * kColS + 0] += rd * rd;
        acc[h][cnd * kColS + 1] += rdu * rdu;
        acc[h][cnd * kColS + 2] += co * xv;
        acc[h][cnd * kColS + 3] += bnd;
        acc[h][cnd * kColS + 4] += dx * dx;
        acc[h][cnd * kColS + 5] += vl * vl;
        acc[h][cnd * kColS + 6] += bray;
        acc[h][cnd * kColS + 7] += vb * vb;
        acc[h][cnd * kColS + 8] += co * dx;
      }
    }
  }
  __shared__ double smem[kKktWarps * BP * 2 * kColS];
  block_inst_sum<BP, 2 * kColS, kKktWarps>(acc, smem, preg(a.part, 2));
}

// One thread per instance: termination, restart, primal weight, end of a
// refinement round; the while condition clears when every instance is done.
template <int BP>
__global__ void __launch_bounds__(256) kb_control(BArgs<BP> a, int nb_row, int nb_col, int init) {
  BGlobal* g = a.g;
  __shared__ int s_running;
  __shared__ double smem[(256 / BP) * BP * 2 * kColS];
  if (threadIdx.x == 0) s_running = 0;
  __syncthreads();
  double rs[2 * kRowS], cs[2 * kColS];
  inst_final_sum<BP, 2 * kRowS>(preg(a.part, 1), nb_row, smem, rs);
  inst_final_sum<BP, 2 * kColS>(preg(a.part, 2), nb_col, smem, cs);
  const int b = threadIdx.x;
  if (b < BP && !g->all_done) {
    BInst& I = a.inst[b];
    I.restart_now = 0;
    I.refine = 0;
    I.finalize = 0;
    if (I.act) {
      const double omega = I.omega, idp = 1.0 / I.dp, idd = 1.0 / I.dd;
      double rel[2], relp[2], reld[2], relg[2], P[2], D[2], kw[2], rp2s[2], rd2s[2], gh[2], dxa[2],
          dya[2];
      bool finite = true;
      for (int c = 0; c < 2; ++c) {
        rp2s[c] = rs[c * kRowS + 0];
        const double rp2u = rs[c * kRowS + 1], qy = rs[c * kRowS + 2];
        dya[c] = rs[c * kRowS + 3];
        rd2s[c] = cs[c * kColS + 0];
        const double rd2u = cs[c * kColS + 1], cx = cs[c * kColS + 2], bnd = cs[c * kColS + 3];
        dxa[c] = cs[c * kColS + 4];
        for (int k = 0; k < kRowS; ++k) finite = finite && isfinite(rs[c * kRowS + k]);
        for (int k = 0; k < kColS; ++k) finite = finite && isfinite(cs[c * kColS + k]);
        P[c] = cx * idp + I.const_p;
        D[c] = qy * idd + I.const_d + bnd;
        relp[c] = sqrt(rp2u) / (1.0 + g->qnorm);
        reld[c] = sqrt(rd2u) / (1.0 + g->cnorm);
        relg[c] = fabs(P[c] - D[c]) / (1.0 + fabs(P[c]) + fabs(D[c]));
        rel[c] = fmax(relp[c], fmax(reld[c], relg[c]));
        // the correction LP's gap is Delta^2 times the LP's, its residuals
        // Delta times: weighting the gap by 1/Delta keeps the restart test
        // what it is for the same point in round 0 (up to a common factor)
        gh[c] = (P[c] - D[c]) * I.dp;
        kw[c] = sqrt(omega * rp2s[c] + rd2s[c] / omega + gh[c] * gh[c]);
      }
      const bool has_avg = I.wsum > 0.0;
      if (init) {
        I.kkt0 = I.kkt_prev = kw[0];
        I.round_target = fmax(g->tol, g->red * rel[0]);
        I.round_rel0 = rel[0];
      } else {
        I.checks += 1;
        I.round_checks += 1;
        I.pending_w = 0.0;
        const int best = (has_avg && rel[1] < rel[0]) ? 1 : 0;
        const uint64_t now = globaltimer_ns();
        const double thr[3] = {1e-4, 1e-6, 1e-8};
        for (int t = 0; t < 3; ++t)
          if (I.t_tol[t] < 0.0 && rel[best] <= thr[t]) {
            I.t_tol[t] = (double)(now - g->t_start) * 1e-9;
            I.k_tol[t] = I.k_total;
          }
        I.rel_p = relp[best];
        I.rel_d = reld[best];
        I.rel_gap = relg[best];
        I.rel_kkt = rel[best];
        I.pobj = P[best];
        I.dobj = D[best];
        int stop = 0;
        if (!finite) {
          stop = PDHG_STATUS_NUMERIC;
        } else if (rel[best] <= g->tol) {
          stop = PDHG_STATUS_OPTIMAL;
        } else if (I.k_total >= g->max_k) {
          stop = PDHG_STATUS_ITER_LIMIT;
        } else if (now - g->t_start >= g->t_limit_ns) {
          stop = PDHG_STATUS_TIME_LIMIT;
        } else if (a.cancel && *a.cancel) {
          stop = PDHG_STATUS_CANCELLED;
        } else if (g->infeas_eps > 0.0) {
          for (int c = 0; c < 2 && !stop; ++c) {
            const double d_obj = rs[c * kRowS + 6] + cs[c * kColS + 6];
            const double d_viol = sqrt(rs[c * kRowS + 5] + cs[c * kColS + 5]);
            const double p_obj = cs[c * kColS + 8];
            const double p_viol = sqrt(rs[c * kRowS + 4] + cs[c * kColS + 7]);
            if (d_obj > 0.0 && d_viol <= g->infeas_eps * d_obj)
              stop = PDHG_STATUS_PRIMAL_INFEASIBLE;
            else if (p_obj < 0.0 && p_viol <= g->infeas_eps * (-p_obj))
              stop = PDHG_STATUS_DUAL_INFEASIBLE;
          }
        }
        if (stop) {
          I.done = 1;
          I.act = 0;
          I.status = stop;
          I.finalize = 1;
          I.cand_avg = best;
        } else {
          int to_avg = (has_avg && kw[1] < kw[0]) ? 1 : 0;
          const double kc = kw[to_avg];
          int restart = (kc <= g->beta_suff * I.kkt0) ||
                        (kc <= g->beta_nec * I.kkt0 && kc > I.kkt_prev) ||
                        ((double)I.since_restart >= g->beta_art * (double)I.k_total);
          I.kkt_prev = kc;
          if (restart) {
            // distances in round-0 units (the correction coordinates are Delta
            // times larger): the "too small to update omega" test stays fixed
            const double Dx = sqrt(dxa[to_avg]) / I.dp, Dy = sqrt(dya[to_avg]) / I.dd;
            double om = omega;
            if (Dx > 1e-10 && Dy > 1e-10)
              om = exp(g->omega_smooth * log(Dy / Dx) + (1.0 - g->omega_smooth) * log(omega));
            I.omega = om;
            const double k0 = sqrt(om * rp2s[to_avg] + rd2s[to_avg] / om + gh[to_avg] * gh[to_avg]);
            I.restarts += 1;
            I.kkt0 = k0;
            I.kkt_prev = k0;
            I.avg_div = I.wsum;
            I.wsum = 0.0;
            I.since_restart = 0;
            I.restart_now = 1;
            I.restart_to_avg = to_avg;
          } else if (rel[0] <= I.round_target ||
                     (g->fold_every > 0 && I.round_checks >= g->fold_every &&
                      rel[0] <= I.round_rel0)) {
            // refinement fold (as pdhg_solve): the current iterate joins x*, y*
            // and kb_apply re-expresses the iteration state in the new
            // coordinates; step size, primal weight, averages and restart
            // window carry over
            const double relb = fmax(rel[0], 1e-300);
            const double scale = fmin(1.0 / relb, 1e12);
            const double f = scale / I.dp;  // Delta_P = Delta_D here
            I.refine = 1;
            I.round_checks = 0;
            I.cand_avg = 0;
            I.next_scale = f;
            I.round_target = fmax(g->tol, g->red * relb);
            I.round_rel0 = relb;
            I.rounds += 1;
            // KKT_w with the gap weighted back to round-0 units scales by f
            I.kkt0 *= f;
            I.kkt_prev *= f;
            I.rel_p = relp[0];
            I.rel_d = reld[0];
            I.rel_gap = relg[0];
            I.rel_kkt = rel[0];
            I.pobj = P[0];
            I.dobj = D[0];
          }
        }
      }
    }
    if (I.act) I.eta = fmin(I.eta, fp32_step_cap(I.omega));  // FP32 range (see fp32_step_cap)
    if (!I.done) atomicAdd(&s_running, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0 && !init) {
    const int all = (s_running == 0) || g->all_done;
    g->all_done = all;
    if (a.in_graph) cudaGraphSetConditional(a.cond, all ? 0u : 1u);
  }
}

// Elementwise, thread (r, b) = (threadIdx.x / BP, threadIdx.x % BP): restart
// moves, refinement steps and final accumulation per instance, plus the new
// pending primal step; per-instance sums of ||dx||^2, c~^T x*, q~^T y*.
template <int BP>
__global__ void __launch_bounds__(kApplyRows * BP) kb_apply(BArgs<BP> a) {
  BGlobal* g = a.g;
  const int b = threadIdx.x % BP, r0 = threadIdx.x / BP;
  const BInst& I = a.inst[b];
  const int restart = I.restart_now, refine = I.refine, fin = I.finalize;
  const int any = restart || refine || fin;
  const int p = I.par;
  const double f = I.next_scale;
  const double idp = 1.0 / I.dp, idd = 1.0 / I.dd;
  const double iw = I.wsum > 0.0 ? 1.0 / I.wsum : 0.0;
  const double wsum = I.wsum;
  const double div = I.avg_div;
  const int cand_avg = I.cand_avg;
  const float tau = (float)(I.eta / I.omega);
  double sdx = 0.0, scp = 0.0, scd = 0.0;
  if (any) {
    // rows
    for (int i = blockIdx.x * kApplyRows + r0; i < a.m; i += gridDim.x * kApplyRows) {
      const size_t idx = (size_t)i * BP + b;
      if (restart) {
        if (I.restart_to_avg) {
          a.y[p][idx] = (float)(((double)a.ybar[idx] + a.ybar64[idx]) / div);
          a.Kx[p][idx] = (float)a.Kza[idx];
        }
        a.ya[idx] = a.y[p][idx];
        a.ybar[idx] = 0.f;
        a.ybar64[idx] = 0.0;
        a.Kxa[idx] = I.restart_to_avg ? a.Kza[idx] : a.Kzc[idx];
      } else {
        const double yh = cand_avg ? ((double)a.ybar[idx] + a.ybar64[idx]) * iw : (double)a.y[p][idx];
        const double kz = cand_avg ? a.Kza[idx] : a.Kzc[idx];
        const double ys = a.yst[idx] + yh * idd;
        a.yst[idx] = ys;
        if (refine) {
          // fold at the current iterate (cand_avg = 0): new correction data,
          // then the state in the new coordinates v' = f (v - y^c)
          const double qn = f * (a.qh[idx] - kz);
          a.qh[idx] = qn;
          a.qf[idx] = (float)qn;
          if (i >= a.m_eq) {
            const double yl = f * (a.ylh[idx] - yh);
            a.ylh[idx] = yl;
            a.ylf[idx] = (float)yl;
          }
          a.ya[idx] = (float)(f * ((double)a.ya[idx] - yh));
          a.ybar64[idx] = f * ((double)a.ybar[idx] + a.ybar64[idx] - wsum * yh);
          a.ybar[idx] = 0.f;
          a.y[p][idx] = 0.f;
          a.Kx[p][idx] = 0.f;
          a.Kxa[idx] = f * (a.Kxa[idx] - kz);
        }
        scd += a.q_obj[i] * ys;
      }
    }
    // columns
    for (int j = blockIdx.x * kApplyRows + r0; j < a.n; j += gridDim.x * kApplyRows) {
      const size_t idx = (size_t)j * BP + b;
      if (restart) {
        a.KTya[idx] = I.restart_to_avg ? a.KTza[idx] : a.KTzc[idx];
        if (I.restart_to_avg) {
          a.x[p][idx] = (float)(((double)a.xbar[idx] + a.xbar64[idx]) / div);
          a.KTy[p][idx] = (float)a.KTza[idx];
        }
        const float x0 = a.x[p][idx];
        a.xa[idx] = x0;
        a.xbar[idx] = 0.f;
        a.xbar64[idx] = 0.0;
        float v = x0 - tau * (a.cf[idx] - a.KTy[p][idx]);
        v = fminf(fmaxf(v, a.lf[idx]), a.uf[idx]);
        a.x[1 - p][idx] = v;
        const double d = (double)(v - x0);
        sdx += d * d;
      } else {
        const double xh = cand_avg ? ((double)a.xbar[idx] + a.xbar64[idx]) * iw : (double)a.x[p][idx];
        const double kz = cand_avg ? a.KTza[idx] : a.KTzc[idx];
        const double xs = a.xst[idx] + xh * idp;
        a.xst[idx] = xs;
        if (refine) {
          const double cn = f * (a.ch[idx] - kz);
          // exact in FP64: the candidate may sit a rounding outside its bounds
          // (the FP32 iterate was projected onto FP32-rounded bounds, e.g. a
          // fixed variable); the new round corrects that, so no clamping here.
          // The round starts at x^ = y^ = 0 even if that is a rounding
          // outside [l^, u^]: the first projected step restores feasibility.
          const double ln = f * (a.lh[idx] - xh);
          const double un = f * (a.uh[idx] - xh);
          a.ch[idx] = cn;
          a.lh[idx] = ln;
          a.uh[idx] = un;
          a.cf[idx] = (float)cn;
          a.lf[idx] = (float)ln;
          a.uf[idx] = (float)un;
          a.xa[idx] = (float)(f * ((double)a.xa[idx] - xh));
          a.xbar64[idx] = f * ((double)a.xbar[idx] + a.xbar64[idx] - wsum * xh);
          a.xbar[idx] = 0.f;
          a.KTya[idx] = f * (a.KTya[idx] - kz);
          a.KTy[p][idx] = 0.f;
          a.x[p][idx] = 0.f;
          // the pending primal step from the new data (the same step in exact
          // arithmetic)
          float v = fminf(fmaxf(-tau * a.cf[idx], a.lf[idx]), a.uf[idx]);
          a.x[1 - p][idx] = v;
          sdx += (double)v * (double)v;
        }
        scp += a.c_obj[j] * xs;
      }
    }
  }
  __shared__ double smem[kApplyRows * BP * 3];
  smem[(r0 * BP + b) * 3 + 0] = sdx;
  smem[(r0 * BP + b) * 3 + 1] = scp;
  smem[(r0 * BP + b) * 3 + 2] = scd;
  __syncthreads();
  if (r0 == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int rr = 0; rr < kApplyRows; ++rr) {
      s0 += smem[(rr * BP + b) * 3 + 0];
      s1 += smem[(rr * BP + b) * 3 + 1];
      s2 += smem[(rr * BP + b) * 3 + 2];
    }
    double* out = a.part + ((size_t)blockIdx.x * BP + b) * 3;
    out[0] = s0;
    out[1] = s1;
    out[2] = s2;
  }
  if (last_block(&g->counter2)) {
    double tot[3];
    inst_final_sum<BP, 3>(a.part, gridDim.x, smem, tot);
    if (threadIdx.x < BP) {
      BInst& J = a.inst[threadIdx.x];
      if (J.restart_now || J.refine || J.finalize) {
        const double s0 = tot[0], s1 = tot[1], s2 = tot[2];
        if (J.restart_now) {
          J.dx2 = s0;
        } else {
          J.const_p = s1;
          J.const_d = s2;
        }
        if (J.refine) {
          // the same iteration in the new coordinates: only the scale and the
          // pending step's length change
          J.dx2 = s0;
          J.dp *= J.next_scale;
          J.dd = J.dp;
        }
      }
      J.restart_now = 0;
      J.refine = 0;
      J.finalize = 0;
    }
    if (threadIdx.x == 0) g->counter2 = 0;
  }
}

// ---------------------------------------------------------------- setup kernels

// Round-0 correction data per instance from the shared LP and the instance bounds.
template <int BP>
__global__ void kb_setup(BArgs<BP> a, const double* __restrict__ lb, const double* __restrict__ ub,
                         const int32_t* __restrict__ perm_col, const double* __restrict__ Dc,
                         const double* __restrict__ c_s, const double* __restrict__ q_s,
                         const double* __restrict__ l_s, const double* __restrict__ u_s) {
  const int64_t Nn = (int64_t)a.n * BP, Nm = (int64_t)a.m * BP;
  const int64_t N = Nn > Nm ? Nn : Nm;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t % BP);
    if (t < Nn) {
      const int j = (int)(t / BP);
      double lo = l_s[j], up = u_s[j];
      if (b < a.B) {
        const int o = perm_col[j];
        lo = lb[(size_t)b * a.n + o] / Dc[j];
        up = ub[(size_t)b * a.n + o] / Dc[j];
      }
      a.lo[t] = lo;
      a.uo[t] = up;
      a.lh[t] = lo;
      a.uh[t] = up;
      a.lf[t] = (float)lo;
      a.uf[t] = (float)up;
      a.ch[t] = c_s[j];
      a.cf[t] = (float)c_s[j];
      a.xst[t] = 0.0;
      const float x0 = fminf(fmaxf(0.f, (float)lo), (float)up);
      a.x[0][t] = x0;
      a.x[1][t] = x0;
      a.xa[t] = x0;
      a.xbar[t] = 0.f;
      a.xbar64[t] = 0.0;
      a.KTy[0][t] = a.KTy[1][t] = 0.f;
    }
    if (t < Nm) {
      const int i = (int)(t / BP);
      a.qh[t] = q_s[i];
      a.qf[t] = (float)q_s[i];
      const double yl = (i < a.m_eq) ? -INFINITY : 0.0;
      a.ylh[t] = yl;
      a.ylf[t] = (float)yl;
      a.yst[t] = 0.0;
      a.y[0][t] = a.y[1][t] = 0.f;
      a.ya[t] = a.ybar[t] = 0.f;
      a.ybar64[t] = 0.0;
    }
  }
}

// K x for every slot (initial point of round 0).
template <int BP>
__global__ void __launch_bounds__(kBThreads) kb_spmm(BArgs<BP> a) {
  constexpr int H = BP / 32;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * kBThreads + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kBThreads) >> 5;
  for (int i = gw; i < a.m; i += nw) {
    const int s = i >> 5, r = i & 31;
    const int o0 = __ldg(a.K.off + s) + r;
    const int w = (__ldg(a.K.off + s + 1) - __ldg(a.K.off + s)) >> 5;
    float acc[H];
#pragma unroll
    for (int h = 0; h < H; ++h) acc[h] = 0.f;
    for (int k = 0; k < w; ++k) {
      const int c = __ldg(a.K.col + o0 + k * kSlice);
      const float v = __ldg(a.K.val + o0 + k * kSlice);
#pragma unroll
      for (int h = 0; h < H; ++h) acc[h] += v * __ldg(a.x[0] + (size_t)c * BP + lane + 32 * h);
    }
#pragma unroll
    for (int h = 0; h < H; ++h) a.Kx[0][(size_t)i * BP + lane + 32 * h] = acc[h];
  }
}

// First pending primal step of round 0 (x' from x^0, K^T y = 0).
template <int BP>
__global__ void kb_first_primal(BArgs<BP> a) {
  const int64_t Nn = (int64_t)a.n * BP;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < Nn;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t % BP);
    const BInst& I = a.inst[b];
    const float tau = (float)(I.eta / I.omega);
    const float x0 = a.x[0][t];
    a.x[1][t] = fminf(fmaxf(x0 - tau * a.cf[t], a.lf[t]), a.uf[t]);
  }
}

// ||x' - x||^2 per instance, deterministic (one block per instance).
template <int BP>
__global__ void kb_dx2(BArgs<BP> a) {
  const int b = blockIdx.x;
  double s = 0.0;
  for (int j = threadIdx.x; j < a.n; j += blockDim.x) {
    const size_t idx = (size_t)j * BP + b;
    const double d = (double)a.x[1][idx] - (double)a.x[0][idx];
    s += d * d;
  }
  __shared__ double sm[kWarps];
  double v[1] = {s};
  block_sum<1>(v, sm);
  if (threadIdx.x == 0) a.inst[b].dx2 = v[0];
}

template <int BP>
__global__ void kb_output(BArgs<BP> a, const int32_t* __restrict__ perm_col,
                          const int32_t* __restrict__ perm_row, const double* __restrict__ Dc,
                          const double* __restrict__ Dr, double* x_out, double* y_out) {
  const int64_t Nn = (int64_t)a.n * a.B, Nm = (int64_t)a.m * a.B;
  const int64_t N = Nn > Nm ? Nn : Nm;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (x_out && t < Nn) {
      const int b = (int)(t / a.n), j = (int)(t % a.n);
      x_out[(size_t)b * a.n + perm_col[j]] = Dc[j] * a.xst[(size_t)j * BP + b];
    }
    if (y_out && t < Nm) {
      const int b = (int)(t / a.m), i = (int)(t % a.m);
      y_out[(size_t)b * a.m + perm_row[i]] = Dr[i] * a.yst[(size_t)i * BP + b];
    }
  }
}

__global__ void kb_init_state(BInst* inst, BGlobal* g, int B, int BP, const double* scalars,
                              BGlobal gin) {
  const int b = threadIdx.x;
  if (b == 0) {
    *g = gin;
    g->t_start = globaltimer_ns();
    g->qnorm = scalars[2];
    g->cnorm = scalars[3];
    g->all_done = 0;
    g->counter = g->counter2 = 0;
  }
  if (b < BP) {
    BInst I;
    memset(&I, 0, sizeof(I));
    I.eta = scalars[0];
    I.omega = scalars[1];
    I.act = b < B;
    I.done = b >= B;
    I.dp = I.dd = 1.0;
    I.next_scale = 1.0;
    I.rel_kkt = INFINITY;
    for (int t = 0; t < 3; ++t) {
      I.t_tol[t] = -1.0;
      I.k_tol[t] = -1;
    }
    inst[b] = I;
  }
}

struct Batched {
  int BP = 0, cap = 0;
  std::vector<void*> allocs;
  void* args = nullptr;  // BArgs<BP> host copy
  BInst* inst = nullptr;
  BInst* inst_host = nullptr;
  int32_t* done_host = nullptr;  // pinned copy of g->all_done (host-loop mode)
  BGlobal* g = nullptr;
  double* part = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int grid_rows = 0, grid_cols = 0, grid_kr = 0, grid_kc = 0, grid_apply = 0;
  int rw_dual = 4, rw_adj = 4;  // rows (columns) per warp of the sweeps
  bool tuned = false;
};

template <int BP>
void launch_sweep_dual(const BArgs<BP>& a, int rw, int grid, cudaStream_t s) {
  if (rw == 1)
    kb_dual<BP, 1><<<grid, kBThreads, 0, s>>>(a);
  else if (rw == 2)
    kb_dual<BP, 2><<<grid, kBThreads, 0, s>>>(a);
  else
    kb_dual<BP, 4><<<grid, kBThreads, 0, s>>>(a);
}

template <int BP>
void launch_sweep_adjoint(const BArgs<BP>& a, int rw, int grid, cudaStream_t s) {
  if (rw == 1)
    kb_adjoint<BP, 1><<<grid, kBThreads, 0, s>>>(a);
  else if (rw == 2)
    kb_adjoint<BP, 2><<<grid, kBThreads, 0, s>>>(a);
  else
    kb_adjoint<BP, 4><<<grid, kBThreads, 0, s>>>(a);
}

template <class P>
cudaError_t balloc(Batched* bt, P** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(P) + 16);
  if (e == cudaSuccess) {
    bt->allocs.push_back(q);
    *p = (P*)q;
  }
  return e;
}

template <int BP>
int setup_batched(Workspace* w, Batched* bt, BArgs<BP>* out) {
  BArgs<BP> a{};
  const size_t n = (size_t)w->n * BP, m = (size_t)w->m * BP;
  cudaError_t e = cudaSuccess;
  auto F = [&](float** p, size_t c) { if (e == cudaSuccess) e = balloc(bt, p, c); };
  auto D = [&](double** p, size_t c) { if (e == cudaSuccess) e = balloc(bt, p, c); };
  for (int i = 0; i < 2; ++i) {
    F(&a.x[i], n);
    F(&a.y[i], m);
    F(&a.Kx[i], m);
    F(&a.KTy[i], n);
  }
  F(&a.xbar, n); F(&a.ybar, m); F(&a.xa, n); F(&a.ya, m);
  F(&a.cf, n); F(&a.lf, n); F(&a.uf, n); F(&a.qf, m); F(&a.ylf, m);
  D(&a.xst, n); D(&a.yst, m); D(&a.ch, n); D(&a.lh, n); D(&a.uh, n); D(&a.qh, m); D(&a.ylh, m);
  D(&a.lo, n); D(&a.uo, n); D(&a.Kzc, m); D(&a.Kza, m); D(&a.KTzc, n); D(&a.KTza, n);
  D(&a.Kxa, m); D(&a.KTya, n); D(&a.xbar64, n); D(&a.ybar64, m);
  if (e == cudaSuccess) e = balloc(bt, &bt->inst, BP);
  if (e == cudaSuccess) e = balloc(bt, &bt->g, 1);
  if (e == cudaSuccess) e = balloc(bt, &bt->part, (size_t)3 * 8192 * 64 * 20);
  if (e != cudaSuccess) {
    g_err = std::string("batched allocation: ") + cudaGetErrorString(e);
    return PDHG_ERR_NOMEM;
  }
  if (cudaMallocHost(&bt->inst_host, sizeof(BInst) * BP) != cudaSuccess ||
      cudaMallocHost(&bt->done_host, sizeof(int32_t)) != cudaSuccess) {
    g_err = "batched pinned allocation failed";
    return PDHG_ERR_NOMEM;
  }
  a.K = w->K.v32();
  a.KT = w->KT.v32();
  a.K64 = w->K.v64();
  a.KT64 = w->KT.v64();
  a.n = (int32_t)w->n;
  a.m = (int32_t)w->m;
  a.m_eq = (int32_t)w->m_eq;
  a.c_obj = w->c_s;
  a.q_obj = w->q_s;
  a.iDr = w->iDr;
  a.iDc = w->iDc;
  a.Dr = w->Dr;
  a.Dc = w->Dc;
  a.inst = bt->inst;
  a.g = bt->g;
  a.part = bt->part;
  a.cancel = w->opts.cancel_flag;
  *out = a;
  const int sms = w->num_sms;
  // at least ~8 rows per warp, so the per-instance partials of small problems
  // stay few (their final sums sit on the critical path of every attempt)
  // the sweeps are grid-stride loops: one wave of resident blocks
  int occ_d = 0, occ_a = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_d, kb_dual<BP, 4>, kBThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_a, kb_adjoint<BP, 4>, kBThreads, 0);
  occ_d = std::max(occ_d, 1);
  occ_a = std::max(occ_a, 1);
  bt->grid_rows = std::max(1, std::min(sms * occ_d, (int)((w->m + 8 * kBWarps - 1) / (8 * kBWarps))));
  bt->grid_cols = std::max(1, std::min(sms * occ_a, (int)((w->n + 8 * kBWarps - 1) / (8 * kBWarps))));
  bt->grid_kr = std::max(1, std::min(sms * 8, (int)((w->m + 8 * kKktWarps - 1) / (8 * kKktWarps))));
  bt->grid_kc = std::max(1, std::min(sms * 8, (int)((w->n + 8 * kKktWarps - 1) / (8 * kKktWarps))));
  bt->grid_apply = std::max(
      1, std::min(sms * 8, (int)((std::max(w->n, w->m) + 16 * kApplyRows - 1) / (16 * kApplyRows))));
  bt->grid_rows = std::min(bt->grid_rows, 8192);
  bt->grid_cols = std::min(bt->grid_cols, 8192);
  bt->grid_kr = std::min(bt->grid_kr, 8192);
  bt->grid_kc = std::min(bt->grid_kc, 8192);
  bt->grid_apply = std::min(bt->grid_apply, 8192);
  return PDHG_OK;
}

template <int BP>
void launch_body(const BArgs<BP>& a, Batched* bt, cudaStream_t s, int init) {
  if (!init) {
    for (int k = 0; k < kCheckEvery; ++k) {
      launch_sweep_dual<BP>(a, bt->rw_dual, bt->grid_rows, s);
      launch_sweep_adjoint<BP>(a, bt->rw_adj, bt->grid_cols, s);
    }
  }
  kb_kkt_row<BP><<<bt->grid_kr, kKktWarps * 32, 0, s>>>(a, init);
  kb_kkt_col<BP><<<bt->grid_kc, kKktWarps * 32, 0, s>>>(a, init);
  kb_control<BP><<<1, 256, 0, s>>>(a, bt->grid_kr, bt->grid_kc, init);
  if (!init) kb_apply<BP><<<bt->grid_apply, kApplyRows * BP, 0, s>>>(a);
}

template <int BP>
int build_batched_graph(Workspace* w, Batched* bt, BArgs<BP> a) {
  if (bt->exec) return PDHG_OK;
  cudaGraph_t gph = nullptr;
  if (cudaGraphCreate(&gph, 0) != cudaSuccess) return PDHG_ERR_CUDA;
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, gph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
    return PDHG_ERR_CUDA;
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  std::memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(raw);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, gph, nullptr, nullptr, 0, &cp) != cudaSuccess) return PDHG_ERR_CUDA;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(w->cap_stream, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return PDHG_ERR_CUDA;
  a.in_graph = 1;
  a.cond = (unsigned long long)h;
  launch_body<BP>(a, bt, w->cap_stream, 0);
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(w->cap_stream, &captured);
  if (e != cudaSuccess) {
    g_err = std::string("batched graph capture: ") + cudaGetErrorString(e);
    return PDHG_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&bt->exec, gph, 0);
  if (e != cudaSuccess) {
    g_err = std::string("batched graph instantiate: ") + cudaGetErrorString(e);
    return PDHG_ERR_CUDA;
  }
  bt->graph = gph;
  return PDHG_OK;
}

// Device state, round-0 data, first primal step and initial KKT_w of every
// instance.
template <int BP>
void batched_start(Workspace* w, Batched* bt, const BArgs<BP>& a, int B, const double* l_b,
                   const double* u_b, cudaStream_t s) {
  const pdhg_opts& o = w->opts;
  BGlobal gin{};
  gin.tol = o.tol;
  gin.red = o.ir_reduction;
  gin.beta_suff = o.beta_sufficient;
  gin.beta_nec = o.beta_necessary;
  gin.beta_art = o.beta_artificial;
  gin.omega_smooth = o.omega_smoothing;
  gin.red_exp = o.step_reduction_exp;
  gin.grow_exp = o.step_growth_exp;
  gin.max_k = o.max_iters;
  gin.t_limit_ns = (uint64_t)(o.time_limit_s * 1e9);
  gin.infeas_eps = o.infeas_tol > 0.0 ? std::max(o.infeas_tol, kFp32RayTol) : 0.0;  // FP32 iterates
  gin.fold_every = o.ir_fold_checks;
  gin.n_real = B;
  kb_init_state<<<1, BP < 32 ? 32 : BP, 0, s>>>(bt->inst, bt->g, B, BP, w->scalars, gin);
  const int gv = std::min(w->num_sms * 8, 8192);
  kb_setup<BP><<<gv, 256, 0, s>>>(a, l_b, u_b, w->perm_col, w->Dc, w->c_s, w->q_s, w->l_s, w->u_s);
  kb_spmm<BP><<<bt->grid_rows, kBThreads, 0, s>>>(a);
  kb_first_primal<BP><<<gv, 256, 0, s>>>(a);
  kb_dx2<BP><<<BP, kBlock, 0, s>>>(a);
  launch_body<BP>(a, bt, s, 1);  // initial KKT_w of every instance
}

// The batched autotuner: rows (columns) per warp R in {1, 2, 4} and the grid
// (1 to 4 blocks per SM, capped by occupancy and by 8 rows per warp) of each
// sweep, timed with CUDA events on this matrix and batch width.  UCPDHG_TUNE_LOG=1
// prints the table to stderr.
template <int BP>
int autotune_batched(Workspace* w, Batched* bt, const BArgs<BP>& a, int B, const double* l_b,
                     const double* u_b, cudaStream_t s) {
  bt->tuned = true;
  if (!w->opts.autotune) {
    // fixed shape: kernel_variant 1, 2 or 4 sets R of both sweeps, kernel_grid
    // their blocks (both grid-stride loops; partials hold kMaxBlocks blocks)
    const int kv = w->opts.kernel_variant;
    if (kv == 1 || kv == 2 || kv == 4) bt->rw_dual = bt->rw_adj = kv;
    if (w->opts.kernel_grid > 0) bt->grid_rows = bt->grid_cols = std::min(w->opts.kernel_grid, kMaxBlocks);
    return PDHG_OK;
  }
  const char* log_env = std::getenv("UCPDHG_TUNE_LOG");
  const bool log = log_env && log_env[0] == '1';
  batched_start<BP>(w, bt, a, B, l_b, u_b, s);
  const int sms = w->num_sms;
  for (int which = 0; which < 2; ++which) {
    const int64_t len = which == 0 ? w->m : w->n;
    float best = 1e30f;
    int best_rw = 4, best_grid = which == 0 ? bt->grid_rows : bt->grid_cols;
    for (int rw : {4, 2, 1}) {
      int occ = 0;
      if (which == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, rw == 4 ? (const void*)kb_dual<BP, 4> : rw == 2 ? (const void*)kb_dual<BP, 2> : (const void*)kb_dual<BP, 1>,
            kBThreads, 0);
      else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, rw == 4 ? (const void*)kb_adjoint<BP, 4> : rw == 2 ? (const void*)kb_adjoint<BP, 2> : (const void*)kb_adjoint<BP, 1>,
            kBThreads, 0);
      occ = std::max(occ, 1);
      const int need = (int)std::max<int64_t>(1, (len + 8 * kBWarps - 1) / (8 * kBWarps));
      for (int bps = 1; bps <= std::min(occ, 8); ++bps) {
        const int g = std::min(std::min(sms * bps, need), 8192);
        auto run = [&]() {
          if (which == 0)
            launch_sweep_dual<BP>(a, rw, g, s);
          else
            launch_sweep_adjoint<BP>(a, rw, g, s);
        };
        run();
        cudaEventRecord(w->ev[2], s);
        for (int r = 0; r < 3; ++r) run();
        cudaEventRecord(w->ev[3], s);
        if (cudaEventSynchronize(w->ev[3]) != cudaSuccess) {
          g_err = std::string("batched autotune: ") + cudaGetErrorString(cudaGetLastError());
          return PDHG_ERR_CUDA;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, w->ev[2], w->ev[3]);
        if (log)
          std::fprintf(stderr, "autotune batched B=%d %s rows/warp %d grid %d: %.2f us\n", B,
                       which == 0 ? "dual" : "adjoint", rw, g, ms * 1000.f / 3.f);
        if (ms < best * 0.98f) {
          best = ms;
          best_rw = rw;
          best_grid = g;
        }
        if (g == need) break;
      }
    }
    if (which == 0) {
      bt->rw_dual = best_rw;
      bt->grid_rows = best_grid;
    } else {
      bt->rw_adj = best_rw;
      bt->grid_cols = best_grid;
    }
  }
  return cudaGetLastError() == cudaSuccess ? PDHG_OK : PDHG_ERR_CUDA;
}

template <int BP>
int solve_batched_impl(Workspace* w, int B, const double* l_b, const double* u_b, double* x_out,
                       double* y_out, pdhg_result* res, cudaStream_t s) {
  Batched* bt = (Batched*)w->batched;
  if (bt && bt->BP != BP) return -99;  // caller rebuilds
  if (!bt) {
    bt = new Batched();
    bt->BP = BP;
    w->batched = bt;
    BArgs<BP> a;
    int rc = setup_batched<BP>(w, bt, &a);
    if (rc != PDHG_OK) return rc;
    bt->args = new BArgs<BP>(a);
  }
  BArgs<BP> a = *(BArgs<BP>*)bt->args;
  a.B = B;
  a.in_graph = 0;
  const pdhg_opts& o = w->opts;
  if (!bt->tuned) {
    // time the sweeps' launch shapes on this batch (real attempts on scratch
    // state, re-initialised below), before the graph captures them
    launch_prepare(w, s);
    launch_to_f32(w->K.val64, w->K.val32, w->K.nnz_pad, s);
    launch_to_f32(w->KT.val64, w->KT.val32, w->KT.nnz_pad, s);
    int rc = autotune_batched<BP>(w, bt, a, B, l_b, u_b, s);
    if (rc != PDHG_OK) return rc;
  }
  if (!o.host_loop) {
    int rc = build_batched_graph<BP>(w, bt, a);
    if (rc != PDHG_OK) return rc;
  }
  cudaEventRecord(w->ev[0], s);
  launch_prepare(w, s);
  launch_to_f32(w->K.val64, w->K.val32, w->K.nnz_pad, s);
  launch_to_f32(w->KT.val64, w->KT.val32, w->KT.nnz_pad, s);
  w->values_f32 = true;
  batched_start<BP>(w, bt, a, B, l_b, u_b, s);
  if (o.host_loop) {
    // the graph body's kernels launched from the host (profilers cannot see
    // kernels inside a graph with conditional nodes); one wait per check
    for (;;) {
      launch_body<BP>(a, bt, s, 0);
      if (cudaMemcpyAsync(bt->done_host, &bt->g->all_done, sizeof(int32_t), cudaMemcpyDeviceToHost,
                          s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        g_err = std::string("batched host loop: ") + cudaGetErrorString(cudaGetLastError());
        return PDHG_ERR_CUDA;
      }
      if (*bt->done_host) break;
    }
  } else {
    cudaError_t e = cudaGraphLaunch(bt->exec, s);
    if (e != cudaSuccess) {
      g_err = std::string("batched graph launch: ") + cudaGetErrorString(e);
      return PDHG_ERR_CUDA;
    }
  }
  kb_output<BP><<<std::min(w->num_sms * 8, 8192), 256, 0, s>>>(a, w->perm_col, w->perm_row, w->Dc, w->Dr,
                                                               x_out, y_out);
  cudaEventRecord(w->ev[1], s);
  if (cudaMemcpyAsync(bt->inst_host, bt->inst, sizeof(BInst) * BP, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    g_err = std::string("batched solve: ") + cudaGetErrorString(cudaGetLastError());
    return PDHG_ERR_CUDA;
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, w->ev[0], w->ev[1]);
  int64_t checks_max = 0;
  for (int b = 0; b < B; ++b) checks_max = std::max(checks_max, bt->inst_host[b].checks);
  const int passes = o.ruiz_iters + (o.pock_chambolle ? 1 : 0);
  const int64_t launches = 8 + 4 * passes + 2 + 6 + 4 + (checks_max + 1) * (2 * kCheckEvery + 4) + 1;
  bool numeric = false;
  for (int b = 0; b < B; ++b) {
    const BInst& I = bt->inst_host[b];
    pdhg_result& r = res[b];
    std::memset(&r, 0, sizeof(r));
    r.status = I.status ? I.status : PDHG_STATUS_ITER_LIMIT;
    r.ir_rounds = I.rounds;
    r.iterations = I.k_total;
    r.accepted = I.accepted;
    r.restarts = I.restarts;
    r.checks = I.checks;
    r.rel_p = I.rel_p;
    r.rel_d = I.rel_d;
    r.rel_gap = I.rel_gap;
    r.rel_kkt = I.rel_kkt;
    r.primal_obj = I.pobj;
    r.dual_obj = I.dobj;
    r.solve_seconds = ms * 1e-3;
    for (int t = 0; t < 3; ++t) {
      r.time_to_tol[t] = I.t_tol[t];
      r.iters_to_tol[t] = I.k_tol[t];
    }
    r.eta = I.eta;
    r.omega = I.omega;
    r.kernel_launches = launches;
    numeric = numeric || I.status == PDHG_STATUS_NUMERIC;
  }
  if (numeric) {
    g_err = "NaN/Inf met in a batched KKT evaluation";
    return PDHG_ERR_NUMERIC;
  }
  return PDHG_OK;
}

}  // namespace

void batched_tuning(Workspace* w, int32_t* out) {
  const Batched* bt = (const Batched*)w->batched;
  const bool t = bt && bt->tuned;
  out[0] = t ? bt->rw_dual : -1;
  out[1] = t ? bt->grid_rows : 0;
  out[2] = t ? bt->rw_adj : -1;
  out[3] = t ? bt->grid_cols : 0;
}

void release_batched(Workspace* w) {
  Batched* bt = (Batched*)w->batched;
  if (!bt) return;
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  if (bt->inst_host) cudaFreeHost(bt->inst_host);
  if (bt->done_host) cudaFreeHost(bt->done_host);
  for (void* p : bt->allocs) cudaFree(p);
  if (bt->args) {
    if (bt->BP == 64)
      delete (BArgs<64>*)bt->args;
    else
      delete (BArgs<32>*)bt->args;
  }
  delete bt;
  w->batched = nullptr;
}

}  // namespace ucpdhg

using namespace ucpdhg;

extern "C" int pdhg_solve_batched(void* ws, int32_t B, const double* l_b, const double* u_b,
                                  double* x_out, double* y_out, pdhg_result* res_b, void* stream) {
  g_err.clear();
  if (!ws || !l_b || !u_b || !res_b) {
    g_err = "pdhg_solve_batched: NULL argument";
    return PDHG_ERR_INVALID_ARG;
  }
  if (B < 1 || B > 64) {
    g_err = "pdhg_solve_batched: B must be in 1..64";
    return PDHG_ERR_INVALID_ARG;
  }
  Workspace* w = (Workspace*)ws;
  cudaStream_t s = (cudaStream_t)stream;
  const int BP = B <= 32 ? 32 : 64;
  if (w->batched && ((Batched*)w->batched)->BP != BP) release_batched(w);
  int rc = BP == 32 ? solve_batched_impl<32>(w, B, l_b, u_b, x_out, y_out, res_b, s)
                    : solve_batched_impl<64>(w, B, l_b, u_b, x_out, y_out, res_b, s);
  return rc;
}
