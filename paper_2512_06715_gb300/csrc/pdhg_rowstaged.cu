// Per-attempt kernels with the matrix chunk AND the chunk's row (column)
// operands staged in shared memory by TMA bulk copies (variants 18, 19).
//
// The matrix-only staged kernels (pdhg_staged.cu) still load each slice's row
// operands (y, q, y_lo, y-average; x, c, l, u, x-average) with per-thread
// global loads after the chunk lands, so every slice waits one HBM latency for
// them before its gathers.  Here a chunk of at most kRsEntries entries and
// kRsSlices slices brings its 32 x slices rows of every operand vector along
// in the same barrier phase (contiguous in the internal order, 128-byte
// aligned, vectors allocated to a multiple of 32 entries), so a warp's slice
// only waits for its gathers from L2.  Same sums, same order per row as the
// other variants.
#include "staging.cuh"

namespace ucpdhg {
namespace {

using namespace staging;

constexpr int kRsRows = kRsSlices * kSlice;  // operand rows per chunk (kRsEntries, kRsSlices: common.cuh)

// Shared-memory layout: barriers, then per buffer the columns, values and NR
// operand vectors of kRsRows entries each.
template <class T, int NR>
struct RowStage {
  uint64_t* bar;
  unsigned char* base;
  static constexpr size_t kCol = (size_t)kRsEntries * sizeof(int32_t);
  static constexpr size_t kVal = (size_t)kRsEntries * sizeof(T);
  static constexpr size_t kRow = (size_t)kRsRows * sizeof(T);
  static constexpr size_t kBuf = kCol + kVal + NR * kRow;
  __device__ explicit RowStage(unsigned char* raw) : bar(reinterpret_cast<uint64_t*>(raw)), base(raw + 128) {}
  __device__ int32_t* col(int b) const { return reinterpret_cast<int32_t*>(base + b * kBuf); }
  __device__ T* val(int b) const { return reinterpret_cast<T*>(base + b * kBuf + kCol); }
  __device__ T* row(int b, int r) const { return reinterpret_cast<T*>(base + b * kBuf + kCol + kVal + r * kRow); }
};

template <class T, int NR>
constexpr size_t rowstage_bytes() {
  return 128 + 2 * RowStage<T, NR>::kBuf;
}

// Thread 0: copy chunk c of A (slices [s0, s1)) and the listed operand vectors'
// rows [32 s0, 32 s1) into buffer b; a null source is skipped.
template <class T, int NR>
__device__ __forceinline__ void issue_rows(const SellView<T>& A, const int32_t* chunks, int c,
                                          const RowStage<T, NR>& sm, int b, const T* const (&src)[NR]) {
  const int s0 = __ldg(chunks + c), s1 = __ldg(chunks + c + 1);
  const int e0 = __ldg(A.off + s0), e1 = __ldg(A.off + s1);
  const uint32_t ne = (uint32_t)(e1 - e0);
  const uint32_t rb = (uint32_t)((s1 - s0) * kSlice * sizeof(T));
  uint32_t bytes = ne * (uint32_t)(sizeof(int32_t) + sizeof(T));
#pragma unroll
  for (int r = 0; r < NR; ++r)
    if (src[r]) bytes += rb;
  mbar_expect_tx(&sm.bar[b], bytes);
  bulk_g2s(sm.col(b), A.col + e0, ne * (uint32_t)sizeof(int32_t), &sm.bar[b]);
  bulk_g2s(sm.val(b), A.val + e0, ne * (uint32_t)sizeof(T), &sm.bar[b]);
#pragma unroll
  for (int r = 0; r < NR; ++r)
    if (src[r]) bulk_g2s(sm.row(b, r), src[r] + (size_t)s0 * kSlice, rb, &sm.bar[b]);
}

}  // namespace

// Row operands staged: 0 y, 1 q, 2 y_lo (FP32) or K x (FP64), 3 y-average sum.
template <class T, int P>
__global__ void __launch_bounds__(kBlock) k_dual_rs(IterArgs<T> a) {
  DevState* st = a.st;
  __shared__ DualScalars<T> sc;
  if (threadIdx.x == 0) dual_scalars<T>(st, sc);
  __syncthreads();
  if (sc.done) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  RowStage<T, 4> sm(smem_raw);
  __shared__ int s_abort;
  const int p = sc.p;
  const bool has_pw = sc.has_pw;
  const T pwT = sc.pw;
  const T sigma = sc.sigma;
  const T* __restrict__ xn = a.x[1 - p];
  const T* __restrict__ xc = a.x[p];
  T* __restrict__ yn = a.y[1 - p];
  constexpr bool kStored = StoresKx<T>::value;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T* const src[4] = {a.y[p], a.q, kStored ? (const T*)a.Kx[p] : a.ylo, has_pw ? (const T*)a.ybar : nullptr};
  T acc_dy2 = 0, acc_int = 0;
  run_chunks(sm.bar, a.kchunks2_n, true, &s_abort, st,
             [&](int b, int c) { issue_rows<T, 4>(a.K, a.kchunks2, c, sm, b, src); }, [&](int b, int c) {
               const int s0 = __ldg(a.kchunks2 + c), s1 = __ldg(a.kchunks2 + c + 1);
               const int base = __ldg(a.K.off + s0);
               const T* ry = sm.row(b, 0);
               const T* rq = sm.row(b, 1);
               const T* r2 = sm.row(b, 2);
               const T* rb = sm.row(b, 3);
               for (int sg = s0 + warp; sg < s1; sg += kWarps * P) {
                 int o[P], w[P], row[P], loc[P];
#pragma unroll
                 for (int u = 0; u < P; ++u) {
                   const int s = sg + u * kWarps;
                   const bool in = s < s1;
                   const int ob = in ? __ldg(a.K.off + s) : base;
                   o[u] = ob - base + lane;
                   w[u] = in ? (__ldg(a.K.off + s + 1) - ob) >> 5 : 0;
                   row[u] = in ? s * kSlice + lane : a.m;
                   loc[u] = (s - s0) * kSlice + lane;
                 }
                 T kx[P], ko2[P];
                 staged_rows<T, P, !kStored>(sm.col(b), sm.val(b), o, w, xn, xc, kx, ko2);
#pragma unroll
                 for (int u = 0; u < P; ++u) {
                   const int i = row[u];
                   if (i >= a.m) continue;
                   const int li = loc[u];
                   const T yo = ry[li], qi = rq[li];
                   const T kxo = kStored ? r2[li] : ko2[u];
                   T t = qi - (T)2 * kx[u];
                   t = t + kxo;
                   T v = yo + sigma * t;
                   if (i >= a.m_eq) v = max(v, kStored ? dual_floor(a.ylo, i, a.m_eq) : r2[li]);
                   yn[i] = v;
                   if (kStored) a.Kx[1 - p][i] = kx[u];
                   if (has_pw) a.ybar[i] = rb[li] + pwT * yo;
                   const T dy = v - yo;
                   acc_dy2 += dy * dy;
                   acc_int += dy * (kx[u] - kxo);
                 }
               }
             });
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

// Column operands staged: 0 x, 1 c, 2 l, 3 u, 4 x-average sum.  A rejected step
// (no new K^T y) streams nothing and reads the cached K^T y from global memory.
template <class T, int P>
__global__ void __launch_bounds__(kBlock) k_adjoint_rs(IterArgs<T> a) {
  DevState* st = a.st;
  __shared__ AdjScalars<T> sc;
  if (threadIdx.x == 0) adj_scalars<T>(st, sc);
  __syncthreads();
  if (sc.done) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  RowStage<T, 5> sm(smem_raw);
  __shared__ int s_abort;
  const int p = sc.p;
  const int acc_last = sc.acc_last;
  const bool upd_avg = sc.upd_avg;
  const T wlT = sc.wl;
  const T tau = sc.tau;
  const T* __restrict__ yc = a.y[p];
  const T* __restrict__ xc = a.x[p];
  T* __restrict__ kty = a.KTy[p];
  T* __restrict__ xn = a.x[1 - p];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T* const src[5] = {xc, a.c, a.l, a.u, upd_avg ? (const T*)a.xbar : nullptr};
  T acc_dx2 = 0;
  run_chunks(sm.bar, a.tchunks2_n, acc_last != 0, &s_abort, st,
             [&](int b, int c) { issue_rows<T, 5>(a.KT, a.tchunks2, c, sm, b, src); }, [&](int b, int c) {
               const int s0 = __ldg(a.tchunks2 + c), s1 = __ldg(a.tchunks2 + c + 1);
               const int base = __ldg(a.KT.off + s0);
               for (int sg = s0 + warp; sg < s1; sg += kWarps * P) {
                 int o[P], w[P], col[P], loc[P];
                 T g[P];
#pragma unroll
                 for (int u = 0; u < P; ++u) {
                   const int s = sg + u * kWarps;
                   const bool in = s < s1;
                   const int ob = in ? __ldg(a.KT.off + s) : base;
                   o[u] = ob - base + lane;
                   w[u] = (in && acc_last) ? (__ldg(a.KT.off + s + 1) - ob) >> 5 : 0;
                   col[u] = in ? s * kSlice + lane : a.n;
                   loc[u] = (s - s0) * kSlice + lane;
                   g[u] = 0;
                 }
                 if (acc_last) {
                   T unused[P];
                   staged_rows<T, P, false>(sm.col(b), sm.val(b), o, w, yc, yc, g, unused);
                 }
#pragma unroll
                 for (int u = 0; u < P; ++u) {
                   const int j = col[u];
                   if (j >= a.n) continue;
                   const int lj = loc[u];
                   T x0, cj, lo, up, xb = 0;
                   if (acc_last) {
                     x0 = sm.row(b, 0)[lj];
                     cj = sm.row(b, 1)[lj];
                     lo = sm.row(b, 2)[lj];
                     up = sm.row(b, 3)[lj];
                     if (upd_avg) xb = sm.row(b, 4)[lj];
                   } else {
                     x0 = xc[j];
                     cj = a.c[j];
                     lo = a.l[j];
                     up = a.u[j];
                     g[u] = kty[j];
                   }
                   if (acc_last) kty[j] = g[u];
                   if (upd_avg) a.xbar[j] = xb + wlT * x0;
                   T v = x0 - tau * (cj - g[u]);
                   v = min(max(v, lo), up);
                   xn[j] = v;
                   const T d = v - x0;
                   acc_dx2 += d * d;
                 }
               }
             });
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

template <class T>
void launch_dual_rowstaged(const IterArgs<T>& a, int grid, cudaStream_t s, int pair) {
  if (pair == 2)
    k_dual_rs<T, 2><<<grid, kBlock, rowstage_bytes<T, 4>(), s>>>(a);
  else
    k_dual_rs<T, 1><<<grid, kBlock, rowstage_bytes<T, 4>(), s>>>(a);
}

template <class T>
void launch_adjoint_rowstaged(const IterArgs<T>& a, int grid, cudaStream_t s, int pair) {
  if (pair == 2)
    k_adjoint_rs<T, 2><<<grid, kBlock, rowstage_bytes<T, 5>(), s>>>(a);
  else
    k_adjoint_rs<T, 1><<<grid, kBlock, rowstage_bytes<T, 5>(), s>>>(a);
}

// Dynamic shared memory beyond 48 KB, allowed once per device per kernel.
int rowstaged_setup() {
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  if (done[dev]) return 0;
  struct F {
    const void* fn;
    size_t bytes;
  };
  const F fs[8] = {{(const void*)&k_dual_rs<float, 1>, rowstage_bytes<float, 4>()},
                   {(const void*)&k_dual_rs<float, 2>, rowstage_bytes<float, 4>()},
                   {(const void*)&k_adjoint_rs<float, 1>, rowstage_bytes<float, 5>()},
                   {(const void*)&k_adjoint_rs<float, 2>, rowstage_bytes<float, 5>()},
                   {(const void*)&k_dual_rs<double, 1>, rowstage_bytes<double, 4>()},
                   {(const void*)&k_dual_rs<double, 2>, rowstage_bytes<double, 4>()},
                   {(const void*)&k_adjoint_rs<double, 1>, rowstage_bytes<double, 5>()},
                   {(const void*)&k_adjoint_rs<double, 2>, rowstage_bytes<double, 5>()}};
  for (const F& f : fs)
    if (cudaFuncSetAttribute(f.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.bytes) != cudaSuccess)
      return -1;
  done[dev] = true;
  return 0;
}

template void launch_dual_rowstaged<float>(const IterArgs<float>&, int, cudaStream_t, int);
template void launch_dual_rowstaged<double>(const IterArgs<double>&, int, cudaStream_t, int);
template void launch_adjoint_rowstaged<float>(const IterArgs<float>&, int, cudaStream_t, int);
template void launch_adjoint_rowstaged<double>(const IterArgs<double>&, int, cudaStream_t, int);

}  // namespace ucpdhg
