// The two kernels of one PDHG step attempt (Sec. II.E iteration, PDLP form):
//
//   k_dual    : K x' (sliced ELL, warp per 32-row slice) fused with the
//               projected dual step y' = max(y_lo, y + sigma (q - 2 K x' + K x));
//               FP32 recomputes K x in the same matrix pass (gathering x and
//               x'), FP64 reads the stored K x and writes K x' (StoresKx),
//               the lazy y-average update, and the FP64 partial sums ||dy||^2 and
//               dy^T K dx.  The block that finishes last reduces the partials in
//               fixed order and takes the adaptive step decision (accept/reject,
//               next eta) on the device.
//   k_adjoint : K^T y' for an accepted step (else the cached K^T y), the
//               x-average update, and -- fused -- the primal step of the NEXT
//               attempt x'' = proj_[l,u](x - tau (c - K^T y)) with ||dx||^2.
//
// Buffers are double-buffered by a parity bit in the device state: the
// current iterate is buf[par], the candidate buf[1-par]; accepting flips par.
#include "internal.cuh"

namespace ucpdhg {

// Row dot products of U consecutive slices (lane = row within each slice)
// with x.  Entries are consumed in predicated chunks of 4 per slice, so every
// column/value load of the U short rows (UC rows have 2-25 entries) is in
// flight before the dependent gathers of x.  U > 1 raises the bytes in flight
// per warp; the autotuner picks U per matrix.
// Slice offsets off[s0 .. s0+U] (clamped past the end, giving empty slices).
// The per-attempt kernels load the NEXT group's offsets one iteration ahead,
// so this L2 round trip is off the critical path.
template <class T, int U>
__device__ __forceinline__ void slice_offsets(const SellView<T>& A, int s0, int (&ob)[U + 1]) {
#pragma unroll
  for (int u = 0; u <= U; ++u) ob[u] = __ldg(A.off + min(s0 + u, A.nslices));
}

template <class T, int U>
__device__ __forceinline__ void sell_dot_pre(const SellView<T>& A, const int (&ob)[U + 1], int lane,
                                             const T* __restrict__ x, T (&acc)[U]) {
  int o0[U], w[U];
  int wmax = 0;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    o0[u] = ob[u] + lane;
    w[u] = (ob[u + 1] - ob[u]) >> 5;
    wmax = max(wmax, w[u]);
    acc[u] = 0;
  }
  for (int k0 = 0; k0 < wmax; k0 += 4) {
    int c[U][4];
    T v[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const bool ok = k0 + e < w[u];
        c[u][e] = ok ? __ldg(A.col + o0[u] + (k0 + e) * kSlice) : 0;
        v[u][e] = ok ? __ldg(A.val + o0[u] + (k0 + e) * kSlice) : (T)0;
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (k0 + e < w[u]) acc[u] += v[u][e] * __ldg(x + c[u][e]);
  }
}

// Two row products at once, K x1 and K x2, sharing the matrix stream (the
// second gather hits L2: the iterate vectors are a few MB).
template <class T, int U>
__device__ __forceinline__ void sell_dot2_pre(const SellView<T>& A, const int (&ob)[U + 1], int lane,
                                              const T* __restrict__ x1, const T* __restrict__ x2,
                                              T (&acc1)[U], T (&acc2)[U]) {
  int o0[U], w[U];
  int wmax = 0;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    o0[u] = ob[u] + lane;
    w[u] = (ob[u + 1] - ob[u]) >> 5;
    wmax = max(wmax, w[u]);
    acc1[u] = 0;
    acc2[u] = 0;
  }
  for (int k0 = 0; k0 < wmax; k0 += 4) {
    int c[U][4];
    T v[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const bool ok = k0 + e < w[u];
        c[u][e] = ok ? __ldg(A.col + o0[u] + (k0 + e) * kSlice) : 0;
        v[u][e] = ok ? __ldg(A.val + o0[u] + (k0 + e) * kSlice) : (T)0;
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (k0 + e < w[u]) {
          acc1[u] += v[u][e] * __ldg(x1 + c[u][e]);
          acc2[u] += v[u][e] * __ldg(x2 + c[u][e]);
        }
  }
}

template <class T, int U>
__device__ __forceinline__ void sell_dot_multi(const SellView<T>& A, int s0, int lane,
                                               const T* __restrict__ x, T (&acc)[U]) {
  int ob[U + 1];
  slice_offsets<T, U>(A, s0, ob);
  sell_dot_pre<T, U>(A, ob, lane, x, acc);
}

template <class T>
__device__ __forceinline__ T sell_dot(const SellView<T>& A, int s, int lane, const T* __restrict__ x) {
  T acc[1];
  sell_dot_multi<T, 1>(A, s, lane, x, acc);
  return acc[0];
}

template <class T, int U, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_dual(IterArgs<T> a) {
  grid_launch_dependents();
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kBlock) >> 5;
  int ob[U + 1];
  slice_offsets<T, U>(a.K, gw * U, ob);  // matrix only: before the previous kernel ends
  grid_wait_prior();
  DevState* st = a.st;
  __shared__ DualScalars<T> sc;
  if (threadIdx.x == 0) dual_scalars<T>(st, sc);
  __syncthreads();
  if (sc.done) return;
  const int p = sc.p;
  const bool has_pw = sc.has_pw;
  const T pwT = sc.pw;
  const T sigma = sc.sigma;
  const T* __restrict__ xn = a.x[1 - p];
  const T* __restrict__ xc = a.x[p];
  const T* __restrict__ yc = a.y[p];
  T* __restrict__ yn = a.y[1 - p];
  // partials in the iterate precision up to the block totals (FP64
  // throughput on this GPU is ~1/60 of FP32); the step rule is a heuristic
  T acc_dy2 = 0, acc_int = 0;
  for (int s0 = gw * U; s0 < a.K.nslices; s0 += nw * U) {
    int nb[U + 1];
    slice_offsets<T, U>(a.K, s0 + nw * U, nb);  // next group, one iteration ahead
    // row operands do not depend on the product: load them first so their
    // latency overlaps the matrix stream
    T yo[U], qi[U], lo[U], yb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = (s0 + u) * kSlice + lane;
      yo[u] = qi[u] = lo[u] = yb[u] = 0;
      if (i < a.m) {
        yo[u] = yc[i];
        qi[u] = a.q[i];
        if (i >= a.m_eq) lo[u] = dual_floor(a.ylo, i, a.m_eq);
        if (has_pw) yb[u] = a.ybar[i];
      }
    }
    // FP32: K x' and K x in one pass (K x recomputed: an L2 gather instead of
    // a stream read and write of m values).  FP64: K x' only, K x read.
    T kx[U], ko[U];
    if constexpr (StoresKx<T>::value) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = (s0 + u) * kSlice + lane;
        ko[u] = i < a.m ? a.Kx[p][i] : (T)0;
      }
      sell_dot_pre<T, U>(a.K, ob, lane, xn, kx);
    } else {
      sell_dot2_pre<T, U>(a.K, ob, lane, xn, xc, kx, ko);
    }
#pragma unroll
    for (int u = 0; u <= U; ++u) ob[u] = nb[u];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = (s0 + u) * kSlice + lane;
      if (i < a.m) {
        T t = qi[u] - (T)2 * kx[u];
        t = t + ko[u];
        T v = yo[u] + sigma * t;
        if (i >= a.m_eq) v = max(v, lo[u]);
        yn[i] = v;
        if constexpr (StoresKx<T>::value) a.Kx[1 - p][i] = kx[u];
        if (has_pw) a.ybar[i] = yb[u] + pwT * yo[u];
        const T dy = v - yo[u];
        const T dk = kx[u] - ko[u];
        acc_dy2 += dy * dy;
        acc_int += dy * dk;
      }
    }
  }
  T acc[2] = {acc_dy2, acc_int};
  if (publish_partials_t<2, T>(acc, a.partials, &st->counter)) {
    double tot[2];
    final_sum_t<2, T>(a.partials, gridDim.x, tot);
    if (threadIdx.x == 0) {
      decide_step(st, a, tot[0], tot[1]);
      st->counter = 0;
    }
  }
}

template <class T, int U, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_adjoint(IterArgs<T> a) {
  grid_launch_dependents();
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kBlock) >> 5;
  int ob[U + 1];
  slice_offsets<T, U>(a.KT, gw * U, ob);  // matrix only: before the previous kernel ends
  grid_wait_prior();
  DevState* st = a.st;
  __shared__ AdjScalars<T> sc;
  if (threadIdx.x == 0) adj_scalars<T>(st, sc);
  __syncthreads();
  if (sc.done) return;
  const int p = sc.p;
  const int acc_last = sc.acc_last;
  const bool upd_avg = sc.upd_avg;
  const T wlT = sc.wl;
  const T tau = sc.tau;
  const T* __restrict__ yc = a.y[p];
  const T* __restrict__ xc = a.x[p];
  T* __restrict__ kty = a.KTy[p];
  T* __restrict__ xn = a.x[1 - p];
  T acc_dx2 = 0;
  for (int s0 = gw * U; s0 < a.KT.nslices; s0 += nw * U) {
    int nb[U + 1];
    if (acc_last) slice_offsets<T, U>(a.KT, s0 + nw * U, nb);  // one iteration ahead
    T x0[U], cj[U], lj[U], uj[U], xb[U], g[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = (s0 + u) * kSlice + lane;
      x0[u] = cj[u] = lj[u] = uj[u] = xb[u] = g[u] = 0;
      if (j < a.n) {
        x0[u] = xc[j];
        cj[u] = a.c[j];
        lj[u] = a.l[j];
        uj[u] = a.u[j];
        if (upd_avg) xb[u] = a.xbar[j];
        if (!acc_last) g[u] = kty[j];
      }
    }
    if (acc_last) {
      sell_dot_pre<T, U>(a.KT, ob, lane, yc, g);
#pragma unroll
      for (int u = 0; u <= U; ++u) ob[u] = nb[u];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = (s0 + u) * kSlice + lane;
      if (j < a.n) {
        if (acc_last) kty[j] = g[u];
        if (upd_avg) a.xbar[j] = xb[u] + wlT * x0[u];
        T v = x0[u] - tau * (cj[u] - g[u]);
        v = min(max(v, lj[u]), uj[u]);
        xn[j] = v;
        const T d = v - x0[u];
        acc_dx2 += d * d;
      }
    }
  }
  T acc[1] = {acc_dx2};
  if (publish_partials_t<1, T>(acc, a.partials, &st->counter)) {
    double tot[1];
    final_sum_t<1, T>(a.partials, gridDim.x, tot);
    if (threadIdx.x == 0) {
      st->dx2 = tot[0];
      st->counter = 0;
    }
  }
}

// ---- software-pipelined variants (one slice per warp) -------------------------
//
// A warp sweeps its slices s, s + nw, s + 2 nw, ...  While the gathers of slice
// s are in flight, the first kStage entries (columns and values) and the row
// operands of slice s + nw are already loading, and the offsets of s + 2 nw
// before them: two dependent round trips per slice (matrix from HBM, gathered
// vector from L2) overlap instead of following each other.  Entries beyond
// kStage (the long minimum-up/down rows) are read after the gathers.

constexpr int kStage = 4;

template <class T>
struct SliceStage {
  int o0, w;          // first slot of this lane, entries per row
  int c[kStage];
  T v[kStage];
};

template <class T>
__device__ __forceinline__ void stage_slice(const SellView<T>& A, int ob, int oe, int lane,
                                            SliceStage<T>& g) {
  g.o0 = ob + lane;
  g.w = (oe - ob) >> 5;
#pragma unroll
  for (int e = 0; e < kStage; ++e) {
    const bool ok = e < g.w;
    g.c[e] = ok ? __ldg(A.col + g.o0 + e * kSlice) : 0;
    g.v[e] = ok ? __ldg(A.val + g.o0 + e * kSlice) : (T)0;
  }
}

// Row products of a staged slice with x1 and (if TWO) x2.
template <class T, bool TWO>
__device__ __forceinline__ void staged_dot(const SellView<T>& A, const SliceStage<T>& g,
                                           const T* __restrict__ x1, const T* __restrict__ x2,
                                           T& acc1, T& acc2) {
  acc1 = 0;
  acc2 = 0;
#pragma unroll
  for (int e = 0; e < kStage; ++e)
    if (e < g.w) {
      acc1 += g.v[e] * __ldg(x1 + g.c[e]);
      if (TWO) acc2 += g.v[e] * __ldg(x2 + g.c[e]);
    }
  for (int k0 = kStage; k0 < g.w; k0 += 4) {
    int c[4];
    T v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const bool ok = k0 + e < g.w;
      c[e] = ok ? __ldg(A.col + g.o0 + (k0 + e) * kSlice) : 0;
      v[e] = ok ? __ldg(A.val + g.o0 + (k0 + e) * kSlice) : (T)0;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (k0 + e < g.w) {
        acc1 += v[e] * __ldg(x1 + c[e]);
        if (TWO) acc2 += v[e] * __ldg(x2 + c[e]);
      }
  }
}

template <class T, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_dual_pipe(IterArgs<T> a) {
  grid_launch_dependents();
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kBlock) >> 5;
  const int ns = a.K.nslices;
  // matrix only before the previous kernel ends: the warp's first slice
  // (entries) and the offsets of its second
  SliceStage<T> cur;
  {
    const int s = min(gw, ns);
    stage_slice<T>(a.K, __ldg(a.K.off + s), __ldg(a.K.off + min(s + 1, ns)), lane, cur);
  }
  int nb0 = __ldg(a.K.off + min(gw + nw, ns)), nb1 = __ldg(a.K.off + min(gw + nw + 1, ns));
  grid_wait_prior();
  DevState* st = a.st;
  __shared__ DualScalars<T> sc;
  if (threadIdx.x == 0) dual_scalars<T>(st, sc);
  __syncthreads();
  if (sc.done) return;
  const int p = sc.p;
  const bool has_pw = sc.has_pw;
  const T pwT = sc.pw;
  const T sigma = sc.sigma;
  const T* __restrict__ xn = a.x[1 - p];
  const T* __restrict__ xc = a.x[p];
  const T* __restrict__ yc = a.y[p];
  T* __restrict__ yn = a.y[1 - p];
  T acc_dy2 = 0, acc_int = 0;
  constexpr bool kStored = StoresKx<T>::value;
  T yo, qi, lo, yb, kxo;
  auto row_ops = [&](int s, T& y0, T& q0, T& l0, T& b0, T& k0) {
    const int i = s * kSlice + lane;
    y0 = q0 = l0 = b0 = k0 = 0;
    if (s < ns && i < a.m) {
      y0 = yc[i];
      q0 = a.q[i];
      if (i >= a.m_eq) l0 = dual_floor(a.ylo, i, a.m_eq);
      if (has_pw) b0 = a.ybar[i];
      if (kStored) k0 = a.Kx[p][i];
    }
  };
  row_ops(gw, yo, qi, lo, yb, kxo);
  for (int s = gw; s < ns; s += nw) {
    // next slice: entries and row operands; offsets two slices ahead
    SliceStage<T> nxt;
    T yo2, qi2, lo2, yb2, kxo2;
    stage_slice<T>(a.K, nb0, nb1, lane, nxt);
    row_ops(s + nw, yo2, qi2, lo2, yb2, kxo2);
    nb0 = __ldg(a.K.off + min(s + 2 * nw, ns));
    nb1 = __ldg(a.K.off + min(s + 2 * nw + 1, ns));
    T kx, ko;
    if constexpr (kStored) {
      T unused;
      staged_dot<T, false>(a.K, cur, xn, xn, kx, unused);
      ko = kxo;
    } else {
      staged_dot<T, true>(a.K, cur, xn, xc, kx, ko);
    }
    const int i = s * kSlice + lane;
    if (i < a.m) {
      T t = qi - (T)2 * kx;
      t = t + ko;
      T v = yo + sigma * t;
      if (i >= a.m_eq) v = max(v, lo);
      yn[i] = v;
      if (kStored) a.Kx[1 - p][i] = kx;
      if (has_pw) a.ybar[i] = yb + pwT * yo;
      const T dy = v - yo;
      acc_dy2 += dy * dy;
      acc_int += dy * (kx - ko);
    }
    cur = nxt;
    yo = yo2;
    qi = qi2;
    lo = lo2;
    yb = yb2;
    kxo = kxo2;
  }
  T acc[2] = {acc_dy2, acc_int};
  if (publish_partials_t<2, T>(acc, a.partials, &st->counter)) {
    double tot[2];
    final_sum_t<2, T>(a.partials, gridDim.x, tot);
    if (threadIdx.x == 0) {
      decide_step(st, a, tot[0], tot[1]);
      st->counter = 0;
    }
  }
}

template <class T, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_adjoint_pipe(IterArgs<T> a) {
  grid_launch_dependents();
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kBlock) >> 5;
  const int ns = a.KT.nslices;
  // matrix only before the previous kernel ends (used only if the step it
  // decides is accepted)
  SliceStage<T> cur;
  {
    const int s = min(gw, ns);
    stage_slice<T>(a.KT, __ldg(a.KT.off + s), __ldg(a.KT.off + min(s + 1, ns)), lane, cur);
  }
  int nb0 = __ldg(a.KT.off + min(gw + nw, ns)), nb1 = __ldg(a.KT.off + min(gw + nw + 1, ns));
  grid_wait_prior();
  DevState* st = a.st;
  __shared__ AdjScalars<T> sc;
  if (threadIdx.x == 0) adj_scalars<T>(st, sc);
  __syncthreads();
  if (sc.done) return;
  const int p = sc.p;
  const int acc_last = sc.acc_last;
  const bool upd_avg = sc.upd_avg;
  const T wlT = sc.wl;
  const T tau = sc.tau;
  const T* __restrict__ yc = a.y[p];
  const T* __restrict__ xc = a.x[p];
  T* __restrict__ kty = a.KTy[p];
  T* __restrict__ xn = a.x[1 - p];
  T acc_dx2 = 0;
  auto col_ops = [&](int s, T& x0, T& c0, T& l0, T& u0, T& b0, T& g0) {
    const int j = s * kSlice + lane;
    x0 = c0 = l0 = u0 = b0 = g0 = 0;
    if (s < ns && j < a.n) {
      x0 = xc[j];
      c0 = a.c[j];
      l0 = a.l[j];
      u0 = a.u[j];
      if (upd_avg) b0 = a.xbar[j];
      if (!acc_last) g0 = kty[j];
    }
  };
  T x0, cj, lj, uj, xb, g;
  col_ops(gw, x0, cj, lj, uj, xb, g);
  for (int s = gw; s < ns; s += nw) {
    SliceStage<T> nxt;
    nxt.w = 0;
    T x2, c2, l2, u2, b2, g2;
    if (acc_last) {
      stage_slice<T>(a.KT, nb0, nb1, lane, nxt);
      nb0 = __ldg(a.KT.off + min(s + 2 * nw, ns));
      nb1 = __ldg(a.KT.off + min(s + 2 * nw + 1, ns));
    }
    col_ops(s + nw, x2, c2, l2, u2, b2, g2);
    if (acc_last) {
      T unused;
      staged_dot<T, false>(a.KT, cur, yc, yc, g, unused);
    }
    const int j = s * kSlice + lane;
    if (j < a.n) {
      if (acc_last) kty[j] = g;
      if (upd_avg) a.xbar[j] = xb + wlT * x0;
      T v = x0 - tau * (cj - g);
      v = min(max(v, lj), uj);
      xn[j] = v;
      const T d = v - x0;
      acc_dx2 += d * d;
    }
    cur = nxt;
    x0 = x2;
    cj = c2;
    lj = l2;
    uj = u2;
    xb = b2;
    g = g2;
  }
  T acc[1] = {acc_dx2};
  if (publish_partials_t<1, T>(acc, a.partials, &st->counter)) {
    double tot[1];
    final_sum_t<1, T>(a.partials, gridDim.x, tot);
    if (threadIdx.x == 0) {
      st->dx2 = tot[0];
      st->counter = 0;
    }
  }
}

// x = proj_[l,u](0), y = proj(0), averages and anchors reset; K^T y.
template <class T>
__global__ void k_init_vectors(IterArgs<T> a) {
  const int64_t N = a.n > a.m ? a.n : a.m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < a.n) {
      T v = min(max((T)0, a.l[t]), a.u[t]);
      a.x[0][t] = v;
      a.x[1][t] = v;
      a.xa[t] = v;
      a.xbar[t] = 0;
      if (a.xbar64) a.xbar64[t] = 0.0;
    }
    if (t < a.m) {
      T v = 0;
      if ((int)t >= a.m_eq) v = max(v, dual_floor(a.ylo, (int)t, a.m_eq));
      a.y[0][t] = v;
      a.y[1][t] = v;
      a.ya[t] = v;
      a.ybar[t] = 0;
      if (a.ybar64) a.ybar64[t] = 0.0;
    }
  }
}

template <class T>
__global__ void __launch_bounds__(kBlock) k_spmv_into(SellView<T> A, const T* __restrict__ x,
                                                      T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kBlock) >> 5;
  for (int s = gw; s < A.nslices; s += nw) {
    const T v = sell_dot(A, s, lane, x);
    const int r = s * kSlice + lane;
    if (r < A.rows) y[r] = v;
  }
}

__global__ void k_state_init(DevState* st, RoundInit r, const double* scalars) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (r.reset_steps) {
    st->eta = r.eta > 0.0 ? r.eta : scalars[0];
    st->omega = r.omega > 0.0 ? r.omega : scalars[1];
  }
  st->dx2 = 0.0;
  st->w_last = 0.0;
  st->pending_w = 0.0;
  st->wsum = 0.0;
  st->avg_div = 0.0;
  st->par = 0;
  st->accepted_last = 0;
  st->k = 0;
  st->since_restart = 0;
  st->accepted = 0;
  st->restarts = 0;
  st->checks = 0;
  st->kkt0 = 0.0;
  st->kkt_prev = 0.0;
  st->restart_now = 0;
  st->restart_to_avg = 0;
  st->done = 0;
  st->status = 0;
  st->best_is_avg = 0;
  st->numeric = 0;
  st->tol = r.tol;
  st->ir_red = r.ir_red;
  st->fold = 0;
  st->round_target = r.tol;
  st->max_k = r.max_k;
  st->max_checks = r.max_checks;
  st->k_offset = r.k_offset;
  st->t_limit_ns = r.t_limit_ns;
  if (r.first_round) {
    st->t_start = globaltimer_ns();
    for (int i = 0; i < 3; ++i) {
      st->t_tol[i] = -1.0;
      st->k_tol[i] = -1;
    }
    st->n_trace_a = 0;
    st->n_trace_c = 0;
  }
  st->beta_suff = r.beta_suff;
  st->beta_nec = r.beta_nec;
  st->beta_art = r.beta_art;
  st->omega_smooth = r.omega_smooth;
  st->red_exp = r.red_exp;
  st->grow_exp = r.grow_exp;
  st->infeas_eps = r.infeas_eps;
  st->fold_every = r.fold_every;
  st->wait_timeout = 0;
  st->fixed = r.fixed;
  st->art_total = r.art_total;
  st->trace_on = r.trace_on;
  st->trace_cap_a = r.trace_cap_a;
  st->trace_cap_c = r.trace_cap_c;
  st->qnorm = scalars[2];
  st->cnorm = scalars[3];
  st->inv_dp = r.inv_dp;
  st->inv_dd = r.inv_dd;
  st->gap_w = r.gap_w > 0.0 ? r.gap_w : 1.0;
  st->const_p = scalars[6];
  st->const_d = scalars[7];
  st->refine = r.refine;
  st->counter = 0;
  st->counter2 = 0;
}

// ---------------------------------------------------------------------------

static int vgrid(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  if (g > 152 * 8) g = 152 * 8;
  return (int)(g < 1 ? 1 : g);
}

template <class T>
void launch_init_iterates(const IterArgs<T>& a, int grid, cudaStream_t s) {
  (void)grid;
  k_init_vectors<T><<<vgrid(a.n > a.m ? a.n : a.m), kBlock, 0, s>>>(a);
  int gt = (a.KT.nslices + kWarps - 1) / kWarps;
  if (gt > kMaxBlocks) gt = kMaxBlocks;
  k_spmv_into<T><<<gt < 1 ? 1 : gt, kBlock, 0, s>>>(a.KT, a.y[0], a.KTy[0]);
  if (StoresKx<T>::value) {
    int gk = (a.K.nslices + kWarps - 1) / kWarps;
    if (gk > kMaxBlocks) gk = kMaxBlocks;
    k_spmv_into<T><<<gk < 1 ? 1 : gk, kBlock, 0, s>>>(a.K, a.x[0], a.Kx[0]);
  }
}

// Variants: 1, 2, 4 slices per warp; 0 software pipelined; 8 and 9 are the
// one-slice and the pipelined forms compiled for 8 resident blocks per SM
// (at most 32 registers, a few spilled to L1) -- more warps in flight against
// the HBM and L2 latency at the cost of the spills; 16 and 17 stage the matrix
// in shared memory with bulk copies (pdhg_staged.cu), one or two slices per
// warp at a time; 18 and 19 stage the row (column) operands with the matrix
// chunk (pdhg_rowstaged.cu); 20 and 21 keep two or three slices ahead in a
// per-warp shared-memory ring filled by cp.async (pdhg_ring.cu).
// Minimum resident blocks per SM that each variant is compiled for: the
// register budget that keeps the one-slice forms at 6 (FP32) or 5 (FP64)
// blocks per SM without spills (an unconstrained build takes ~58 registers and
// drops to 4 blocks per SM).
template <class T, int U>
struct MinBlocks {
  static constexpr int value = U == 1 ? (sizeof(T) == 4 ? 6 : 5) : (sizeof(T) == 4 ? 4 : 3);
};
template <class T>
struct MinBlocksPipe {
  static constexpr int value = sizeof(T) == 4 ? 5 : 3;
};

// One per-attempt kernel, with the programmatic-dependent-launch attribute when
// a.overlap is set (the kernel then overlaps its matrix prologue with the end
// of the previous kernel in the stream or graph).
template <class T>
static void launch_iter(void (*k)(IterArgs<T>), const IterArgs<T>& a, int grid, cudaStream_t s) {
  if (!a.overlap) {
    k<<<grid, kBlock, 0, s>>>(a);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, a);
}

template <class T>
void launch_dual(const IterArgs<T>& a, int grid, cudaStream_t s, int unroll) {
  switch (unroll) {
    case 0: launch_iter<T>(k_dual_pipe<T, MinBlocksPipe<T>::value>, a, grid, s); break;
    case 2: launch_iter<T>(k_dual<T, 2, MinBlocks<T, 2>::value>, a, grid, s); break;
    case 4: launch_iter<T>(k_dual<T, 4, MinBlocks<T, 4>::value>, a, grid, s); break;
    case 8: launch_iter<T>(k_dual<T, 1, 8>, a, grid, s); break;
    case 9: launch_iter<T>(k_dual_pipe<T, 8>, a, grid, s); break;
    case 16: launch_dual_staged<T>(a, grid, s, 1); break;
    case 17: launch_dual_staged<T>(a, grid, s, 2); break;
    case 18: launch_dual_rowstaged<T>(a, grid, s, 1); break;
    case 19: launch_dual_rowstaged<T>(a, grid, s, 2); break;
    case 20: launch_dual_ring<T>(a, grid, s, 3); break;
    case 21: launch_dual_ring<T>(a, grid, s, 4); break;
    default: launch_iter<T>(k_dual<T, 1, MinBlocks<T, 1>::value>, a, grid, s); break;
  }
}

template <class T>
void launch_adjoint(const IterArgs<T>& a, int grid, cudaStream_t s, int unroll) {
  switch (unroll) {
    case 0: launch_iter<T>(k_adjoint_pipe<T, MinBlocksPipe<T>::value>, a, grid, s); break;
    case 2: launch_iter<T>(k_adjoint<T, 2, MinBlocks<T, 2>::value>, a, grid, s); break;
    case 4: launch_iter<T>(k_adjoint<T, 4, MinBlocks<T, 4>::value>, a, grid, s); break;
    case 8: launch_iter<T>(k_adjoint<T, 1, 8>, a, grid, s); break;
    case 9: launch_iter<T>(k_adjoint_pipe<T, 8>, a, grid, s); break;
    case 16: launch_adjoint_staged<T>(a, grid, s, 1); break;
    case 17: launch_adjoint_staged<T>(a, grid, s, 2); break;
    case 18: launch_adjoint_rowstaged<T>(a, grid, s, 1); break;
    case 19: launch_adjoint_rowstaged<T>(a, grid, s, 2); break;
    case 20: launch_adjoint_ring<T>(a, grid, s, 3); break;
    case 21: launch_adjoint_ring<T>(a, grid, s, 4); break;
    default: launch_iter<T>(k_adjoint<T, 1, MinBlocks<T, 1>::value>, a, grid, s); break;
  }
}

void launch_state_init(DevState* st, const RoundInit& r, const double* scalars, cudaStream_t s) {
  k_state_init<<<1, 32, 0, s>>>(st, r, scalars);
}

int blocks_per_sm_iter() {
  int best = 1 << 30;
  const void* fns[4] = {(const void*)&k_dual<double, 1, MinBlocks<double, 1>::value>,
                        (const void*)&k_adjoint<double, 1, MinBlocks<double, 1>::value>,
                        (const void*)&k_dual<float, 1, MinBlocks<float, 1>::value>,
                        (const void*)&k_adjoint<float, 1, MinBlocks<float, 1>::value>};
  for (const void* f : fns) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, kBlock, 0) != cudaSuccess) b = 4;
    best = b < best ? b : best;
  }
  return best < 1 ? 1 : best;
}

template void launch_init_iterates<double>(const IterArgs<double>&, int, cudaStream_t);
template void launch_init_iterates<float>(const IterArgs<float>&, int, cudaStream_t);
template void launch_dual<double>(const IterArgs<double>&, int, cudaStream_t, int);
template void launch_dual<float>(const IterArgs<float>&, int, cudaStream_t, int);
template void launch_adjoint<double>(const IterArgs<double>&, int, cudaStream_t, int);
template void launch_adjoint<float>(const IterArgs<float>&, int, cudaStream_t, int);

}  // namespace ucpdhg
