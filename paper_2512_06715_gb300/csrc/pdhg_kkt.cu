// KKT / duality-gap evaluation, restart and termination control, iterative
// refinement and output (all reductions FP64, fixed order).
//
// A check runs every 64 attempts for two candidates, the current iterate and
// the step-weighted average since the last restart (Applegate et al., cited in
// Sec. II.E).  It evaluates, with the FP64 rescaled matrix,
//   outer (unscaled) measures of the original LP -> termination (rel_kkt)
//   KKT_w = sqrt(w ||r_p||^2 + ||r_d||^2 / w + gap^2) in the solver's own
//           (rescaled, refinement-scaled) space, the gap weighted back to
//           round-0 units                                 -> restart decision
// The iterate is the correction (x^, y^) of a refinement round: the implied
// point of the original LP is x~ = x* + x^/Delta_P, y~ = y* + y^/Delta_D, so
//   r_p(original) = (q^ - K~ x^) / Delta_P / Dr,  lambda = (c^ - K~^T y^)/Delta_D,
//   P = c~^T x^ / Delta_P + c~^T x*,  D = q~^T y^ / Delta_D + q~^T y* + bounds(lambda)
// A plain FP64 solve is the single round x* = y* = 0, Delta = 1.  In mixed
// precision a round ends at the first restart whose candidate reaches the
// round's target: the candidate joins x*, y* (FP64) and the next round starts
// from it at x^ = y^ = 0 with the same step size and primal weight, i.e. the
// same restart expressed in new coordinates.
#include "internal.cuh"

namespace ucpdhg {

__device__ __forceinline__ double* region(double* partials, int r) {
  return partials + (size_t)r * kMaxBlocks * kRegionStride;
}

// Infeasibility rays.  The differences since the last restart, dx = x - x_anchor
// and dy = y - y_anchor of each candidate, are tested as rays of the unscaled LP
// (x = Dc x~, y = Dr y~; K dx = (K~ dx~) / Dr, K^T dy = (K~^T dy~) / Dc).  The
// products K~ x~ of the anchors are kept (Kx_anc, KTy_anc: set at the first
// check, moved at restarts and refinement folds) so a ray needs no extra matrix
// pass: K~ dx~ = K~ x~ - Kx_anc.  A refinement round's coordinates scale every
// ray by a common factor, which the certificate ratios do not see.
//
// Row-side sums per candidate: 0 ||r_p~||^2, 1 ||r_p||^2 (unscaled), 2 q~^T y,
// 3 ||y - y_anchor||^2, 4 primal-ray row violations^2, 5 dual-ray sign
// violations^2 (dy < 0 on >= rows), 6 q~^T dy.
// Column-side: 0 ||r_d~||^2, 1 ||r_d||^2, 2 c~^T x, 3 bound term of D(y),
// 4 ||x - x_anchor||^2, 5 dual-ray lambda violations^2, 6 bound term of the
// dual ray, 7 primal-ray bound violations^2, 8 c~^T dx.
template <class T>
__global__ void __launch_bounds__(kBlock) k_kkt_row(IterArgs<T> a, int init) {
  DevState* st = a.st;
  if (st->done) return;
  const int p = st->par;
  const double wsum = st->wsum, pw = st->pending_w, inv_dp = st->inv_dp;
  const bool has_avg = wsum > 0.0;
  const double iw = has_avg ? 1.0 / wsum : 0.0;
  const T* __restrict__ xc = a.x[p];
  const T* __restrict__ xb = a.xbar;
  const T* __restrict__ yc = a.y[p];
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kBlock) >> 5;
  double acc[2 * kRowSums];
#pragma unroll
  for (int k = 0; k < 2 * kRowSums; ++k) acc[k] = 0.0;
  const SellView<double>& A = a.K64;
  for (int s = gw; s < A.nslices; s += nw) {
    const int o0 = A.off[s], w = (A.off[s + 1] - o0) >> 5;
    double d0 = 0.0, d1 = 0.0;
    for (int k = 0; k < w; ++k) {
      const int slot = o0 + k * kSlice + lane;
      const double v = __ldg(A.val + slot);
      const int c = __ldg(A.col + slot);
      d0 += v * (double)xc[c];
      if (has_avg) d1 += v * ((double)xb[c] + (a.xbar64 ? a.xbar64[c] : 0.0));
    }
    const int i = s * kSlice + lane;
    if (i < a.m) {
      const T yo = yc[i];
      T yb = a.ybar[i];
      if (pw != 0.0) {
        yb = yb + (T)pw * yo;
        a.ybar[i] = yb;
      }
      double ybs = (double)yb;  // the sum since the last restart
      if (a.ybar64) {
        ybs += a.ybar64[i];
        a.ybar64[i] = ybs;
        a.ybar[i] = 0;
      }
      const double kx_avg = has_avg ? d1 * iw : d0;
      if (has_avg) a.Kz_avg[i] = kx_avg;
      a.Kz_cur[i] = d0;
      if (init) a.Kx_anc[i] = d0;
      const double kanc = init ? d0 : a.Kx_anc[i];
      const double y_avg = has_avg ? ybs * iw : (double)yo;
      const double qr = a.q_res[i], qo = a.q_obj[i], idr = a.iDr[i], sr = inv_dp * idr;
      const double dr = a.Dr[i];
      const double yanc = (double)a.ya[i];
      const bool ineq = i >= a.m_eq;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const double kx = c ? kx_avg : d0;
        const double yv = c ? y_avg : (double)yo;
        double r = qr - kx;
        if (ineq) r = fmax(r, 0.0);
        const double ru = r * sr;
        const double dd = yv - yanc;
        const double kdx = (kx - kanc) * idr;                    // (K dx)_i, unscaled
        const double vr = ineq ? fmin(kdx, 0.0) : kdx;           // primal-ray row violation
        const double vs = ineq ? fmin(dd, 0.0) * dr : 0.0;       // dual-ray sign violation
        acc[c * kRowSums + 0] += r * r;
        acc[c * kRowSums + 1] += ru * ru;
        acc[c * kRowSums + 2] += qo * yv;
        acc[c * kRowSums + 3] += dd * dd;
        acc[c * kRowSums + 4] += vr * vr;
        acc[c * kRowSums + 5] += vs * vs;
        acc[c * kRowSums + 6] += qo * dd;
      }
    }
  }
  __shared__ double smem[kWarps * 2 * kRowSums];
  block_sum<2 * kRowSums>(acc, smem);
  if (threadIdx.x == 0) {
    double* out = region(a.partials, 1) + (size_t)blockIdx.x * 2 * kRowSums;
#pragma unroll
    for (int k = 0; k < 2 * kRowSums; ++k) out[k] = acc[k];
  }
}

template <class T>
__global__ void __launch_bounds__(kBlock) k_kkt_col(IterArgs<T> a, int init) {
  DevState* st = a.st;
  if (st->done) return;
  const int p = st->par;
  const double wsum = st->wsum, inv_dd = st->inv_dd;
  const bool has_avg = wsum > 0.0;
  const double iw = has_avg ? 1.0 / wsum : 0.0;
  const T* __restrict__ yc = a.y[p];
  const T* __restrict__ yb = a.ybar;
  const T* __restrict__ xc = a.x[p];
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kBlock) >> 5;
  double acc[2 * kColSums];
#pragma unroll
  for (int k = 0; k < 2 * kColSums; ++k) acc[k] = 0.0;
  const SellView<double>& A = a.KT64;
  for (int s = gw; s < A.nslices; s += nw) {
    const int o0 = A.off[s], w = (A.off[s + 1] - o0) >> 5;
    double e0 = 0.0, e1 = 0.0;
    for (int k = 0; k < w; ++k) {
      const int slot = o0 + k * kSlice + lane;
      const double v = __ldg(A.val + slot);
      const int c = __ldg(A.col + slot);
      e0 += v * (double)yc[c];
      // FP32 iterates: k_kkt_row has just flushed the window sums into ybar64
      // and zeroed ybar, so the FP64 sum alone is the y-average sum
      if (has_avg) e1 += v * (a.ybar64 ? a.ybar64[c] : (double)yb[c]);
    }
    const int j = s * kSlice + lane;
    if (j < a.n) {
      const double kty_avg = has_avg ? e1 * iw : e0;
      if (has_avg) a.KTz_avg[j] = kty_avg;
      a.KTz_cur[j] = e0;
      if (init) a.KTy_anc[j] = e0;
      const double kanc = init ? e0 : a.KTy_anc[j];
      double xbs = (double)a.xbar[j];  // the sum since the last restart
      if (a.xbar64) {
        xbs += a.xbar64[j];
        a.xbar64[j] = xbs;
        a.xbar[j] = 0;
      }
      const double x_avg = has_avg ? xbs * iw : (double)xc[j];
      const double lo = a.l_obj[j], up = a.u_obj[j];
      const bool lf = isfinite(lo), uf = isfinite(up);
      const double idc = a.iDc[j], dc = a.Dc[j];
      const double cr = a.c_res[j], co = a.c_obj[j], sc = inv_dd * idc;
      const double xanc = (double)a.xa[j];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const double kty = c ? kty_avg : e0;
        const double xv = c ? x_avg : (double)xc[j];
        const double lam = cr - kty;
        const double proj = (lf ? fmax(lam, 0.0) : 0.0) + (uf ? fmin(lam, 0.0) : 0.0);
        const double rd = lam - proj;
        const double rdu = rd * sc;
        const double lp = proj * inv_dd;
        const double bnd = (lf ? lo * fmax(lp, 0.0) : 0.0) - (uf ? up * fmax(-lp, 0.0) : 0.0);
        const double dx = xv - xanc;
        // dual ray: lambda~ = -K~^T dy~ (scaled; l~ lambda~ = l lambda), unscaled / Dc
        const double lr = kanc - kty;
        const double lru = lr * idc;
        const double vl = (lf ? 0.0 : fmax(lru, 0.0)) + (uf ? 0.0 : fmin(lru, 0.0));
        const double bray = (lf ? lo * fmax(lr, 0.0) : 0.0) - (uf ? up * fmax(-lr, 0.0) : 0.0);
        // primal ray: dx unscaled = Dc dx~
        const double dxu = dx * dc;
        const double vb = (lf ? fmin(dxu, 0.0) : 0.0) + (uf ? fmax(dxu, 0.0) : 0.0);
        acc[c * kColSums + 0] += rd * rd;
        acc[c * kColSums + 1] += rdu * rdu;
        acc[c * kColSums + 2] += co * xv;
        acc[c * kColSums + 3] += bnd;
        acc[c * kColSums + 4] += dx * dx;
        acc[c * kColSums + 5] += vl * vl;
        acc[c * kColSums + 6] += bray;
        acc[c * kColSums + 7] += vb * vb;
        acc[c * kColSums + 8] += co * dx;
      }
    }
  }
  __shared__ double smem[kWarps * 2 * kColSums];
  block_sum<2 * kColSums>(acc, smem);
  if (threadIdx.x == 0) {
    double* out = region(a.partials, 2) + (size_t)blockIdx.x * 2 * kColSums;
#pragma unroll
    for (int k = 0; k < 2 * kColSums; ++k) out[k] = acc[k];
  }
}

// One block: final reductions, termination, restart and primal-weight update.
template <class T>
__global__ void __launch_bounds__(kBlock) k_control(IterArgs<T> a, int nb_row, int nb_col, int init) {
  DevState* st = a.st;
  if (st->done) {
    if (a.in_graph && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0);
    return;
  }
  double rs[2 * kRowSums], cs[2 * kColSums];
  final_sum<2 * kRowSums>(region(a.partials, 1), nb_row, rs);
  final_sum<2 * kColSums>(region(a.partials, 2), nb_col, cs);
  if (threadIdx.x != 0) return;
  const double omega = st->omega;
  const double dp = 1.0 / st->inv_dp, dd = 1.0 / st->inv_dd;
  double rel[2], relp[2], reld[2], relg[2], P[2], D[2], kw[2], rp2s[2], rd2s[2], gh[2], dxa[2],
      dya[2];
  for (int c = 0; c < 2; ++c) {
    rp2s[c] = rs[c * kRowSums + 0];
    const double rp2u = rs[c * kRowSums + 1];
    const double qy = rs[c * kRowSums + 2];
    dya[c] = rs[c * kRowSums + 3];
    rd2s[c] = cs[c * kColSums + 0];
    const double rd2u = cs[c * kColSums + 1];
    const double cx = cs[c * kColSums + 2];
    const double bnd = cs[c * kColSums + 3];
    dxa[c] = cs[c * kColSums + 4];
    P[c] = cx * st->inv_dp + st->const_p;
    D[c] = qy * st->inv_dd + st->const_d + bnd;
    relp[c] = sqrt(rp2u) / (1.0 + st->qnorm);
    reld[c] = sqrt(rd2u) / (1.0 + st->cnorm);
    relg[c] = fabs(P[c] - D[c]) / (1.0 + fabs(P[c]) + fabs(D[c]));
    rel[c] = fmax(relp[c], fmax(reld[c], relg[c]));
    // Correction LP of a refinement round: residuals scale with Delta, the
    // gap with Delta^2.  Weighting the gap by Delta_0/Delta keeps KKT_w (and
    // with it the restart decisions) what it is for the same point in round 0,
    // up to a factor common to the whole round.
    gh[c] = (P[c] - D[c]) * dp * dd * st->gap_w;
    kw[c] = sqrt(omega * rp2s[c] + rd2s[c] / omega + gh[c] * gh[c]);
  }
  const bool has_avg = st->wsum > 0.0;
  if (init) {
    st->kkt0 = kw[0];
    st->kkt_prev = kw[0];
    st->best_is_avg = 0;
    // a refinement round ends at a restart whose candidate improves on the
    // round's starting point by the factor ir_red
    st->round_target = st->refine ? fmax(st->tol, st->ir_red * rel[0]) : st->tol;
    st->round_rel0 = rel[0];
    st->rel_p = relp[0];
    st->rel_d = reld[0];
    st->rel_gap = relg[0];
    st->rel_kkt = rel[0];
    st->pobj = P[0];
    st->dobj = D[0];
    return;
  }
  st->checks += 1;
  st->pending_w = 0.0;  // applied by k_kkt_row
  const int best = (has_avg && rel[1] < rel[0]) ? 1 : 0;
  st->best_is_avg = best;
  st->rel_p = relp[best];
  st->rel_d = reld[best];
  st->rel_gap = relg[best];
  st->rel_kkt = rel[best];
  st->pobj = P[best];
  st->dobj = D[best];
  const uint64_t now = globaltimer_ns();
  const double elapsed = (double)(now - st->t_start) * 1e-9;
  const double thr[3] = {1e-4, 1e-6, 1e-8};
  for (int i = 0; i < 3; ++i)
    if (st->t_tol[i] < 0.0 && rel[best] <= thr[i]) {
      st->t_tol[i] = elapsed;
      st->k_tol[i] = st->k_offset + st->k;
    }
  int done = 0, status = 0;
  // fmax/fmin (and the bound clamps of the iterations) drop NaNs, so test the
  // raw sums: any NaN/Inf in the data or the iterates shows up in one of them
  bool finite = true;
  for (int k = 0; k < 2 * kRowSums; ++k) finite = finite && isfinite(rs[k]);
  for (int k = 0; k < 2 * kColSums; ++k) finite = finite && isfinite(cs[k]);
  if (!finite || !isfinite(rel[0]) || !isfinite(rel[1])) {
    done = 1;
    status = PDHG_STATUS_NUMERIC;
    st->numeric = 1;
  } else if (rel[best] <= st->tol) {
    done = 1;
    status = PDHG_STATUS_OPTIMAL;
  } else if (st->k >= st->max_k || st->checks >= st->max_checks) {
    done = 1;
    status = PDHG_STATUS_ITER_LIMIT;
  } else if (now - st->t_start >= st->t_limit_ns) {
    done = 1;
    status = PDHG_STATUS_TIME_LIMIT;
  } else if (a.cancel && *a.cancel) {
    done = 1;
    status = PDHG_STATUS_CANCELLED;
  }
  if (!done && st->infeas_eps > 0.0 && !st->fixed) {
    // certificates from the candidates' rays (see the note above k_kkt_row)
    for (int c = 0; c < 2 && !done; ++c) {
      const double d_obj = rs[c * kRowSums + 6] + cs[c * kColSums + 6];
      const double d_viol = sqrt(rs[c * kRowSums + 5] + cs[c * kColSums + 5]);
      const double p_obj = cs[c * kColSums + 8];
      const double p_viol = sqrt(rs[c * kRowSums + 4] + cs[c * kColSums + 7]);
      if (d_obj > 0.0 && d_viol <= st->infeas_eps * d_obj) {
        done = 1;
        status = PDHG_STATUS_PRIMAL_INFEASIBLE;
      } else if (p_obj < 0.0 && p_viol <= st->infeas_eps * (-p_obj)) {
        done = 1;
        status = PDHG_STATUS_DUAL_INFEASIBLE;
      }
    }
  }
  int restart = 0, to_avg = 0;
  if (!done && !st->fixed) {
    to_avg = (has_avg && kw[1] < kw[0]) ? 1 : 0;
    const double kc = kw[to_avg];
    restart = (kc <= st->beta_suff * st->kkt0) ||
              (kc <= st->beta_nec * st->kkt0 && kc > st->kkt_prev) ||
              ((double)st->since_restart >=
               st->beta_art * (double)(st->art_total ? st->k_offset + st->k : st->k));
    st->kkt_prev = kc;
    if (restart) {
      // distances since the last restart, back in round-0 units: a correction
      // round's coordinates are Delta/Delta_0 times larger, and the
      // "distance too small to update omega" test must not loosen with them
      const double Dx = sqrt(dxa[to_avg]) * st->gap_w, Dy = sqrt(dya[to_avg]) * st->gap_w;
      double om = omega;
      if (Dx > 1e-10 && Dy > 1e-10) {
        const double th = st->omega_smooth;
        om = exp(th * log(Dy / Dx) + (1.0 - th) * log(omega));
      }
      st->omega = om;
      st->kkt0 = sqrt(om * rp2s[to_avg] + rd2s[to_avg] / om + gh[to_avg] * gh[to_avg]);
      st->kkt_prev = st->kkt0;
      st->restarts += 1;
      st->avg_div = st->wsum;
      st->wsum = 0.0;
      st->since_restart = 0;
    }
  }
  if (st->refine && !done && !restart && !st->fixed &&
      (rel[0] <= st->round_target ||
       (st->fold_every > 0 && st->checks >= st->fold_every && rel[0] <= st->round_rel0))) {
    // Refinement: the current iterate joins x*, y* in FP64 and the round ends
    // (at the round's target, or after fold_every checks: a long round lets
    // the FP32 iterate grow while its per-attempt changes shrink, until FP32
    // rounding eats them; folding re-centres it at 0);
    // the host re-expresses the whole iteration state (iterate, pending step,
    // averages, restart anchors) in the new coordinates (k_recenter), so the
    // method continues exactly where it was, with the FP32 values now
    // corrections of a smaller error.
    done = 1;
    status = 0;
    st->fold = 1;
    st->best_is_avg = 0;
    st->rel_p = relp[0];
    st->rel_d = reld[0];
    st->rel_gap = relg[0];
    st->rel_kkt = rel[0];
    st->pobj = P[0];
    st->dobj = D[0];
  }
  if (sizeof(T) == 4) st->eta = fmin(st->eta, fp32_step_cap(st->omega));
  st->restart_now = restart;
  st->restart_to_avg = to_avg;
  st->done = done;
  st->status = status;
  if (st->trace_on && a.trace_c) {
    int64_t t = st->n_trace_c;
    if (t < st->trace_cap_c) {
      double* r = a.trace_c + t * kTraceCheckCols;
      r[0] = (double)(st->k_offset + st->k);
      r[1] = (double)restart;
      r[2] = (double)to_avg;
      r[3] = st->omega;
      r[4] = kw[0];
      r[5] = kw[1];
      r[6] = rel[0];
      r[7] = rel[1];
      r[8] = relp[0];
      r[9] = reld[0];
      r[10] = relg[0];
      r[11] = st->eta;
    }
    st->n_trace_c = t + 1;
  }
  if (a.in_graph) cudaGraphSetConditional(a.cond, done ? 0u : 1u);
}

// Moves the iterate to the restart candidate, resets anchors and averages, and
// recomputes the pending primal step with the (possibly) new primal weight.
template <class T>
__global__ void __launch_bounds__(kBlock) k_restart_apply(IterArgs<T> a) {
  DevState* st = a.st;
  if (st->done || !st->restart_now) return;
  const int p = st->par;
  const int to_avg = st->restart_to_avg;
  const double div = st->avg_div;
  const T tau = (T)(st->eta / st->omega);
  T* x = a.x[p];
  T* y = a.y[p];
  double acc[1] = {0.0};
  const int64_t N = a.n > a.m ? a.n : a.m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < a.m) {
      if (to_avg) {
        y[t] = (T)(((double)a.ybar[t] + (a.ybar64 ? a.ybar64[t] : 0.0)) / div);
        if (StoresKx<T>::value) a.Kx[p][t] = (T)a.Kz_avg[t];
      }
      a.ya[t] = y[t];
      a.ybar[t] = 0;
      if (a.ybar64) a.ybar64[t] = 0.0;
      a.Kx_anc[t] = to_avg ? a.Kz_avg[t] : a.Kz_cur[t];
    }
    if (t < a.n) {
      a.KTy_anc[t] = to_avg ? a.KTz_avg[t] : a.KTz_cur[t];
      if (to_avg) {
        x[t] = (T)(((double)a.xbar[t] + (a.xbar64 ? a.xbar64[t] : 0.0)) / div);
        a.KTy[p][t] = (T)a.KTz_avg[t];
      }
      const T x0 = x[t];
      a.xa[t] = x0;
      a.xbar[t] = 0;
      if (a.xbar64) a.xbar64[t] = 0.0;
      T v = x0 - tau * (a.c[t] - a.KTy[p][t]);
      v = min(max(v, a.l[t]), a.u[t]);
      a.x[1 - p][t] = v;
      const double d = (double)v - (double)x0;
      acc[0] += d * d;
    }
  }
  if (publish_partials<1>(acc, a.partials, &st->counter)) {
    double tot[1];
    final_sum<1>(a.partials, gridDim.x, tot);
    if (threadIdx.x == 0) {
      st->dx2 = tot[0];
      st->restart_now = 0;
      st->counter = 0;
    }
  }
}

// x* += x^_best / Delta_P, y* += y^_best / Delta_D (FP64, scaled space).
template <class T>
__global__ void k_accumulate(IterArgs<T> a, double* x_star, double* y_star) {
  DevState* st = a.st;
  const int p = st->par;
  const int avg = st->best_is_avg;
  const double wsum = st->wsum, inv_dp = st->inv_dp, inv_dd = st->inv_dd;
  const int64_t N = a.n > a.m ? a.n : a.m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < a.n) {
      const double xv = avg ? ((double)a.xbar[t] + (a.xbar64 ? a.xbar64[t] : 0.0)) / wsum
                            : (double)a.x[p][t];
      x_star[t] = x_star[t] + xv * inv_dp;
    }
    if (t < a.m) {
      const double yv = avg ? ((double)a.ybar[t] + (a.ybar64 ? a.ybar64[t] : 0.0)) / wsum
                            : (double)a.y[p][t];
      y_star[t] = y_star[t] + yv * inv_dd;
    }
  }
}

// Refinement fold (mixed precision), after x* += x^_c / Delta and the new
// correction data for Delta' = f Delta: every FP32 vector of the iteration is
// re-expressed in the new coordinates v' = f (v - x^_c) (sums of eta-weighted
// iterates: f (sum - wsum x^_c)).  The iterate becomes 0, so K^T y^ = 0; the
// restart anchors and the averages move with it; the pending primal step is
// recomputed from the new data, which in exact arithmetic is the same step.
// Step size, primal weight, average weights and restart window are untouched,
// so the iteration continues where it was.
template <class T>
__global__ void __launch_bounds__(kBlock) k_recenter(IterArgs<T> a, double f) {
  DevState* st = a.st;
  const int p = st->par;
  const double wsum = st->wsum;
  const T tau = (T)(st->eta / st->omega);
  T* x = a.x[p];
  T* y = a.y[p];
  double acc[1] = {0.0};
  const int64_t N = a.n > a.m ? a.n : a.m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < a.m) {
      const double yc = (double)y[t];
      a.ya[t] = (T)(f * ((double)a.ya[t] - yc));
      if (a.ybar64) {  // FP64 sums (the FP32 window was flushed at the check)
        a.ybar64[t] = f * (a.ybar64[t] + (double)a.ybar[t] - wsum * yc);
        a.ybar[t] = 0;
      } else {
        a.ybar[t] = (T)(f * ((double)a.ybar[t] - wsum * yc));
      }
      y[t] = 0;
      if (StoresKx<T>::value) a.Kx[p][t] = 0;  // K x of the new iterate x = 0
      // the anchor moves with the coordinates: K x_a' = f (K x_a - K x_c)
      a.Kx_anc[t] = f * (a.Kx_anc[t] - a.Kz_cur[t]);
    }
    if (t < a.n) {
      a.KTy_anc[t] = f * (a.KTy_anc[t] - a.KTz_cur[t]);
      const double xc = (double)x[t];
      a.xa[t] = (T)(f * ((double)a.xa[t] - xc));
      if (a.xbar64) {
        a.xbar64[t] = f * (a.xbar64[t] + (double)a.xbar[t] - wsum * xc);
        a.xbar[t] = 0;
      } else {
        a.xbar[t] = (T)(f * ((double)a.xbar[t] - wsum * xc));
      }
      x[t] = 0;
      a.KTy[p][t] = 0;
      T v = -tau * a.c[t];
      v = min(max(v, a.l[t]), a.u[t]);
      a.x[1 - p][t] = v;
      acc[0] += (double)v * (double)v;
    }
  }
  if (publish_partials<1>(acc, a.partials, &st->counter)) {
    double tot[1];
    final_sum<1>(a.partials, gridDim.x, tot);
    if (threadIdx.x == 0) {
      st->dx2 = tot[0];
      st->counter = 0;
    }
  }
}

__global__ void k_state_continue(DevState* st, RoundContinue rc, const double* scalars) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->inv_dp = rc.inv_dp;
  st->inv_dd = rc.inv_dd;
  st->gap_w = rc.gap_w;
  st->const_p = scalars[6];
  st->const_d = scalars[7];
  // KKT_w with the gap weighted back to round-0 units scales by f as a whole
  st->kkt0 *= rc.f;
  st->kkt_prev *= rc.f;
  st->round_target = fmax(st->tol, st->ir_red * rc.rel);
  st->round_rel0 = rc.rel;
  st->k_offset = rc.k_offset;
  st->k = 0;
  st->max_k = rc.max_k;
  st->max_checks = rc.max_checks;
  st->accepted = 0;
  st->restarts = 0;
  st->checks = 0;
  st->restart_now = 0;
  st->done = 0;
  st->status = 0;
  st->fold = 0;
  st->counter = 0;
  st->counter2 = 0;
}

// Correction LP of a refinement round (Gleixner, Steffy and Wolter's
// iterative refinement for LP, with one scale factor per side):
//   q^ = dp (q~ - K~ x*),  c^ = dd (c~ - K~^T y*),  [l^, u^] = dp ([l~, u~] - x*),
//   y_lo^ = dd (0 - y*) on >= rows;  plus c~^T x* and q~^T y* as partials.
__global__ void k_ir_build(const double* __restrict__ q_s, const double* __restrict__ c_s,
                           const double* __restrict__ l_s, const double* __restrict__ u_s,
                           const double* __restrict__ x_star, const double* __restrict__ y_star,
                           const double* __restrict__ Kx, const double* __restrict__ KTy, double dp,
                           double dd, int64_t n, int64_t m, int64_t m_eq, double* q_h, double* c_h,
                           double* l_h, double* u_h, double* ylo_h, float* q_f, float* c_f,
                           float* l_f, float* u_f, float* ylo_f, double* partials) {
  double v[2] = {0.0, 0.0};
  const int64_t N = n > m ? n : m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < m) {
      const double qh = dp * (q_s[t] - Kx[t]);
      const double yl = (t < m_eq) ? -INFINITY : dd * (0.0 - y_star[t]);
      q_h[t] = qh;
      ylo_h[t] = yl;
      if (q_f) {
        q_f[t] = (float)qh;
        ylo_f[t] = (float)yl;
      }
      v[1] += q_s[t] * y_star[t];
    }
    if (t < n) {
      const double xs = x_star[t];
      const double ch = dd * (c_s[t] - KTy[t]);
      const double lh = dp * (l_s[t] - xs);
      const double uh = dp * (u_s[t] - xs);
      c_h[t] = ch;
      l_h[t] = lh;
      u_h[t] = uh;
      if (c_f) {
        c_f[t] = (float)ch;
        l_f[t] = (float)lh;
        u_f[t] = (float)uh;
      }
      v[0] += c_s[t] * xs;
    }
  }
  __shared__ double smem[kWarps * 2];
  block_sum<2>(v, smem);
  if (threadIdx.x == 0) {
    partials[blockIdx.x * 2 + 0] = v[0];
    partials[blockIdx.x * 2 + 1] = v[1];
  }
}

__global__ void k_ir_final(const double* partials, int nb, double* scalars) {
  double v[2];
  final_sum<2>(partials, nb, v);
  if (threadIdx.x == 0) {
    scalars[6] = v[0];
    scalars[7] = v[1];
  }
}

__global__ void k_output(const int32_t* __restrict__ perm_col, const int32_t* __restrict__ perm_row,
                         const double* __restrict__ Dc, const double* __restrict__ Dr,
                         const double* __restrict__ x_star, const double* __restrict__ y_star,
                         double* x_out, double* y_out, int64_t n, int64_t m) {
  const int64_t N = n > m ? n : m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (x_out && t < n) x_out[perm_col[t]] = Dc[t] * x_star[t];
    if (y_out && t < m) y_out[perm_row[t]] = Dr[t] * y_star[t];
  }
}

// ---------------------------------------------------------------------------

static int vgrid(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  if (g > 152 * 8) g = 152 * 8;
  return (int)(g < 1 ? 1 : g);
}

template <class T>
void launch_check(const IterArgs<T>& a, int grid_k, int grid_kt, int init, cudaStream_t s) {
  k_kkt_row<T><<<grid_k, kBlock, 0, s>>>(a, init);
  k_kkt_col<T><<<grid_kt, kBlock, 0, s>>>(a, init);
  k_control<T><<<1, kBlock, 0, s>>>(a, grid_k, grid_kt, init);
  if (!init) k_restart_apply<T><<<vgrid(a.n > a.m ? a.n : a.m), kBlock, 0, s>>>(a);
}

template <class T>
void launch_accumulate(const IterArgs<T>& a, double* x_star, double* y_star, int grid,
                       cudaStream_t s) {
  (void)grid;
  k_accumulate<T><<<vgrid(a.n > a.m ? a.n : a.m), kBlock, 0, s>>>(a, x_star, y_star);
}

template <class T>
void launch_recenter(const IterArgs<T>& a, double f, cudaStream_t s) {
  k_recenter<T><<<vgrid(a.n > a.m ? a.n : a.m), kBlock, 0, s>>>(a, f);
}

void launch_state_continue(DevState* st, const RoundContinue& rc, const double* scalars,
                           cudaStream_t s) {
  k_state_continue<<<1, 32, 0, s>>>(st, rc, scalars);
}

void launch_ir_build(Workspace* w, double dp, double dd, bool make_f32, cudaStream_t s) {
  launch_spmv64(w->K.v64(), w->x_star, w->scr_m, w->grid_k, s);
  launch_spmv64(w->KT.v64(), w->y_star, w->scr_n, w->grid_kt, s);
  const int g = vgrid(w->n > w->m ? w->n : w->m);
  k_ir_build<<<g, kBlock, 0, s>>>(w->q_s, w->c_s, w->l_s, w->u_s, w->x_star, w->y_star, w->scr_m,
                                  w->scr_n, dp, dd, w->n, w->m, w->m_eq, w->q_h, w->c_h, w->l_h,
                                  w->u_h, w->ylo_h, make_f32 ? w->q_f : nullptr,
                                  make_f32 ? w->c_f : nullptr, make_f32 ? w->l_f : nullptr,
                                  make_f32 ? w->u_f : nullptr, make_f32 ? w->ylo_f : nullptr,
                                  w->partials);
  k_ir_final<<<1, kBlock, 0, s>>>(w->partials, g, w->scalars);
}

void launch_output(Workspace* w, double* x_out, double* y_out, cudaStream_t s) {
  k_output<<<vgrid(w->n > w->m ? w->n : w->m), kBlock, 0, s>>>(
      w->perm_col, w->perm_row, w->Dc, w->Dr, w->x_star, w->y_star, x_out, y_out, w->n, w->m);
}

template void launch_check<double>(const IterArgs<double>&, int, int, int, cudaStream_t);
template void launch_check<float>(const IterArgs<float>&, int, int, int, cudaStream_t);
template void launch_accumulate<double>(const IterArgs<double>&, double*, double*, int,
                                        cudaStream_t);
template void launch_accumulate<float>(const IterArgs<float>&, double*, double*, int, cudaStream_t);
template void launch_recenter<double>(const IterArgs<double>&, double, cudaStream_t);
template void launch_recenter<float>(const IterArgs<float>&, double, cudaStream_t);

}  // namespace ucpdhg
