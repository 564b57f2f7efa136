// Per-attempt kernels with the matrix stream staged in shared memory by the
// Tensor Memory Accelerator (variant 16 of the autotuner).
//
// The same two kernels as pdhg_kernels.cu (K x' with the projected dual step;
// K^T y' with the x-average update and the next primal step), computing the
// same sums in the same order per row, but the sliced-ELL columns and values
// reach the SM through 1-D bulk copies (cp.async.bulk ... mbarrier::complete_tx)
// instead of per-thread loads:
//
//   * the slices are cut into chunks of at most kStageEntries entries
//     (Chunks: contiguous slices; slice offsets are multiples of 32 entries, so
//     every chunk starts on a 128-byte boundary and spans a multiple of 128 B);
//   * each block owns chunks b, b + grid, b + 2 grid, ... and keeps two chunk
//     buffers: while its warps compute on one, the copy engine fills the other,
//     so each resident block keeps a whole chunk (16-24 KB) of HBM reads in
//     flight without spending registers or issue slots on them;
//   * a warp takes the chunk's slices in turn; its lanes read their rows'
//     columns from shared memory at once, so the dependent gathers of x (or y)
//     from L2 issue without waiting for HBM.
//
// Every wait on an mbarrier is bounded: on expiry the kernel records
// DevState::wait_timeout, skips the remaining work of the chunk (keeping the
// block's barriers), still drains the copies it issued (bounded again) and
// the host reports PDHG_ERR_TIMEOUT.
#include "staging.cuh"

namespace ucpdhg {
namespace {

using namespace staging;

// Shared-memory layout of a staged kernel: two barriers, then the two chunk
// buffers of columns and of values.
template <class T>
struct Stage {
  uint64_t* bar;
  int32_t* col0;  // buffer b: col0 + b * kStageEntries (no indexed pointer arrays: those
  T* val0;        // would live in local memory)
  __device__ explicit Stage(unsigned char* raw) {
    bar = reinterpret_cast<uint64_t*>(raw);
    col0 = reinterpret_cast<int32_t*>(raw + 128);
    val0 = reinterpret_cast<T*>(raw + 128 + 2 * kStageEntries * sizeof(int32_t));
  }
  __device__ int32_t* col(int b) const { return col0 + b * kStageEntries; }
  __device__ T* val(int b) const { return val0 + b * kStageEntries; }
};

template <class T>
constexpr size_t stage_bytes() {
  return 128 + 2 * (size_t)kStageEntries * (sizeof(int32_t) + sizeof(T));
}

// Thread 0: start the copy of chunk c of A into buffer b.
template <class T>
__device__ __forceinline__ void issue_chunk(const SellView<T>& A, const int32_t* chunks, int c,
                                           Stage<T>& sm, int b) {
  const int s0 = __ldg(chunks + c), s1 = __ldg(chunks + c + 1);
  const int e0 = __ldg(A.off + s0), e1 = __ldg(A.off + s1);
  const uint32_t ne = (uint32_t)(e1 - e0);
  mbar_expect_tx(&sm.bar[b], ne * (uint32_t)(sizeof(int32_t) + sizeof(T)));
  bulk_g2s(sm.col(b), A.col + e0, ne * (uint32_t)sizeof(int32_t), &sm.bar[b]);
  bulk_g2s(sm.val(b), A.val + e0, ne * (uint32_t)sizeof(T), &sm.bar[b]);
}

}  // namespace

template <class T, int P>
__global__ void __launch_bounds__(kBlock) k_dual_staged(IterArgs<T> a) {
  DevState* st = a.st;
  __shared__ DualScalars<T> sc;
  if (threadIdx.x == 0) dual_scalars<T>(st, sc);
  __syncthreads();
  if (sc.done) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Stage<T> sm(smem_raw);
  __shared__ int s_abort;
  const int p = sc.p;
  const bool has_pw = sc.has_pw;
  const T pwT = sc.pw;
  const T sigma = sc.sigma;
  const T* __restrict__ xn = a.x[1 - p];
  const T* __restrict__ xc = a.x[p];
  const T* __restrict__ yc = a.y[p];
  T* __restrict__ yn = a.y[1 - p];
  constexpr bool kStored = StoresKx<T>::value;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T acc_dy2 = 0, acc_int = 0;
  run_chunks(sm.bar, a.kchunks_n, true, &s_abort, st,
             [&](int b, int c) { issue_chunk<T>(a.K, a.kchunks, c, sm, b); }, [&](int b, int c) {
    const int s0 = __ldg(a.kchunks + c), s1 = __ldg(a.kchunks + c + 1);
    const int base = __ldg(a.K.off + s0);
    for (int sg = s0 + warp; sg < s1; sg += kWarps * P) {
      int o[P], w[P], row[P];
      T yo[P], qi[P], lo[P], yb[P], ko[P];
#pragma unroll
      for (int u = 0; u < P; ++u) {
        const int s = sg + u * kWarps;
        const bool in = s < s1;
        const int ob = in ? __ldg(a.K.off + s) : base;
        o[u] = ob - base + lane;
        w[u] = in ? (__ldg(a.K.off + s + 1) - ob) >> 5 : 0;
        row[u] = in ? s * kSlice + lane : a.m;
        const int i = row[u];
        yo[u] = qi[u] = lo[u] = yb[u] = ko[u] = 0;
        if (i < a.m) {
          yo[u] = yc[i];
          qi[u] = a.q[i];
          if (i >= a.m_eq) lo[u] = dual_floor(a.ylo, i, a.m_eq);
          if (has_pw) yb[u] = a.ybar[i];
          if (kStored) ko[u] = a.Kx[p][i];
        }
      }
      T kx[P], ko2[P];
      staged_rows<T, P, !kStored>(sm.col(b), sm.val(b), o, w, xn, xc, kx, ko2);
#pragma unroll
      for (int u = 0; u < P; ++u) {
        const int i = row[u];
        if (i >= a.m) continue;
        const T kxo = kStored ? ko[u] : ko2[u];
        T t = qi[u] - (T)2 * kx[u];
        t = t + kxo;
        T v = yo[u] + sigma * t;
        if (i >= a.m_eq) v = max(v, lo[u]);
        yn[i] = v;
        if (kStored) a.Kx[1 - p][i] = kx[u];
        if (has_pw) a.ybar[i] = yb[u] + pwT * yo[u];
        const T dy = v - yo[u];
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

template <class T, int P>
__global__ void __launch_bounds__(kBlock) k_adjoint_staged(IterArgs<T> a) {
  DevState* st = a.st;
  __shared__ AdjScalars<T> sc;
  if (threadIdx.x == 0) adj_scalars<T>(st, sc);
  __syncthreads();
  if (sc.done) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Stage<T> sm(smem_raw);
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
  T acc_dx2 = 0;
  // a rejected step reuses the cached K^T y: no matrix stream at all
  run_chunks(sm.bar, a.tchunks_n, acc_last != 0, &s_abort, st,
             [&](int b, int c) { issue_chunk<T>(a.KT, a.tchunks, c, sm, b); }, [&](int b, int c) {
    const int s0 = __ldg(a.tchunks + c), s1 = __ldg(a.tchunks + c + 1);
    const int base = __ldg(a.KT.off + s0);
    for (int sg = s0 + warp; sg < s1; sg += kWarps * P) {
      int o[P], w[P], col[P];
      T x0[P], cj[P], lj[P], uj[P], xb[P], g[P];
#pragma unroll
      for (int u = 0; u < P; ++u) {
        const int s = sg + u * kWarps;
        const bool in = s < s1;
        const int ob = in ? __ldg(a.KT.off + s) : base;
        o[u] = ob - base + lane;
        w[u] = (in && acc_last) ? (__ldg(a.KT.off + s + 1) - ob) >> 5 : 0;
        col[u] = in ? s * kSlice + lane : a.n;
        const int j = col[u];
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
        T unused[P];
        staged_rows<T, P, false>(sm.col(b), sm.val(b), o, w, yc, yc, g, unused);
      }
#pragma unroll
      for (int u = 0; u < P; ++u) {
        const int j = col[u];
        if (j >= a.n) continue;
        if (acc_last) kty[j] = g[u];
        if (upd_avg) a.xbar[j] = xb[u] + wlT * x0[u];
        T v = x0[u] - tau * (cj[u] - g[u]);
        v = min(max(v, lj[u]), uj[u]);
        xn[j] = v;
        const T d = v - x0[u];
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

// pair: slices a warp processes at once (1 or 2)
template <class T>
void launch_dual_staged(const IterArgs<T>& a, int grid, cudaStream_t s, int pair) {
  if (pair == 2)
    k_dual_staged<T, 2><<<grid, kBlock, stage_bytes<T>(), s>>>(a);
  else
    k_dual_staged<T, 1><<<grid, kBlock, stage_bytes<T>(), s>>>(a);
}

template <class T>
void launch_adjoint_staged(const IterArgs<T>& a, int grid, cudaStream_t s, int pair) {
  if (pair == 2)
    k_adjoint_staged<T, 2><<<grid, kBlock, stage_bytes<T>(), s>>>(a);
  else
    k_adjoint_staged<T, 1><<<grid, kBlock, stage_bytes<T>(), s>>>(a);
}

// Dynamic shared memory above the default 48 KB must be allowed once per
// kernel before its first launch.
int staged_setup() {
  static bool done[64] = {false};  // per device: function attributes belong to a device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  if (done[dev]) return 0;
  const void* f32[4] = {(const void*)&k_dual_staged<float, 1>, (const void*)&k_dual_staged<float, 2>,
                        (const void*)&k_adjoint_staged<float, 1>, (const void*)&k_adjoint_staged<float, 2>};
  const void* f64[4] = {(const void*)&k_dual_staged<double, 1>, (const void*)&k_dual_staged<double, 2>,
                        (const void*)&k_adjoint_staged<double, 1>, (const void*)&k_adjoint_staged<double, 2>};
  for (int i = 0; i < 4; ++i) {
    if (cudaFuncSetAttribute(f32[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_bytes<float>()) !=
            cudaSuccess ||
        cudaFuncSetAttribute(f64[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_bytes<double>()) !=
            cudaSuccess)
      return -1;
  }
  done[dev] = true;
  return 0;
}

template void launch_dual_staged<float>(const IterArgs<float>&, int, cudaStream_t, int);
template void launch_dual_staged<double>(const IterArgs<double>&, int, cudaStream_t, int);
template void launch_adjoint_staged<float>(const IterArgs<float>&, int, cudaStream_t, int);
template void launch_adjoint_staged<double>(const IterArgs<double>&, int, cudaStream_t, int);

}  // namespace ucpdhg
