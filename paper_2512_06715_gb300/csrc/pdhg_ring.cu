// Per-attempt kernels with a per-warp ring of asynchronous copies (variants 20
// and 21 of the two sweeps of one PDHG step attempt, Sec. II.E).
//
// The sliced-ELL sweeps are latency-bound: a warp's slice waits for its matrix
// entries and row operands from HBM, then for the gathered iterate from L2, and
// the register-pipelined variants keep only the next slice in flight.  Here
// every warp owns R shared-memory slots and, with cp.async (LDGSTS, no
// registers held while the copy is in flight), fills the slot of the slice R-1
// sweeps ahead with that slice's first kRingE entries per row (columns and
// values) and its row operands, before it computes the current slice from its
// own slot.  The copies are 16-byte pieces spread over the warp and cached in
// L2 only; the ring needs no block barrier, only the warp's wait for the copy
// group of the slice it consumes.  Entries beyond kRingE (the long rows) are
// read directly.
// Products are summed in the same order as the other variants.
#include "internal.cuh"

namespace ucpdhg {
namespace {

constexpr int kRingE = 4;  // entries per row copied with the slice

__device__ __forceinline__ uint32_t ring_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16 bytes global -> shared, cached in L2 only (the streamed matrix and
// operands do not displace the gathered iterate from L1); both addresses
// 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(ring_u32(dst)), "l"(src) : "memory");
}

// The copies of one slice, spread over the warp in 16-byte pieces: kRingE
// entry rows of columns and of values (128 B each for int32/FP32, 256 B for
// FP64 values) and NR operand rows.  Every slice offset is a multiple of 32
// entries and every vector a whole number of 32-row slices long, so each piece
// is aligned and inside its array.  src(v) is operand row v's first element,
// or nullptr if the row is not needed.
template <class T, int NR, class Slot, class Src>
__device__ __forceinline__ void issue_slice(Slot& sl, const int* col, const T* val, int ob, int w, int lane,
                                            Src src) {
  constexpr int EP = 16 / (int)sizeof(T);  // elements of T per piece
  constexpr int PP = kSlice / EP;          // pieces per 32-element row of T
#pragma unroll
  for (int t = lane; t < kRingE * 8; t += 32) {  // columns: 8 pieces per entry row
    const int e = t >> 3, pc = t & 7;
    if (e < w) cp_async16(&sl.col[e][pc * 4], col + ob + e * kSlice + pc * 4);
  }
#pragma unroll
  for (int t = lane; t < kRingE * PP; t += 32) {
    const int e = t / PP, pc = t % PP;
    if (e < w) cp_async16(&sl.val[e][pc * EP], val + ob + e * kSlice + pc * EP);
  }
#pragma unroll
  for (int t = lane; t < NR * PP; t += 32) {
    const int v = t / PP, pc = t % PP;
    const T* p = src(v);
    if (p) cp_async16(&sl.row[v][pc * EP], p + pc * EP);
  }
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One slot: a slice's first kRingE entries of each of its 32 rows, NR row
// operands, and the slice's first offset and width (written by lane 0).
template <class T, int NR>
struct RingSlot {
  int col[kRingE][kSlice];
  T val[kRingE][kSlice];
  T row[NR][kSlice];
  int hdr[4];
};

template <class T>
constexpr int dual_ops() {
  return StoresKx<T>::value ? 5 : 4;  // y, q, y_lo, y-average sum (+ K x in FP64)
}
constexpr int kAdjOps = 6;  // x, c, l, u, x-average sum, cached K^T y

template <class T, int NR, int R>
constexpr size_t ring_bytes() {
  return sizeof(RingSlot<T, NR>) * R * kWarps;
}

template <class T, int R>
__global__ void __launch_bounds__(kBlock) k_dual_ring(IterArgs<T> a) {
  DevState* st = a.st;
  __shared__ DualScalars<T> sc;
  if (threadIdx.x == 0) dual_scalars<T>(st, sc);
  __syncthreads();
  if (sc.done) return;
  constexpr int NR = dual_ops<T>();
  using Slot = RingSlot<T, NR>;
  constexpr bool kStored = StoresKx<T>::value;
  extern __shared__ __align__(16) unsigned char ring_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Slot* ring = reinterpret_cast<Slot*>(ring_raw) + warp * R;
  const int p = sc.p;
  const bool has_pw = sc.has_pw;
  const T pwT = sc.pw;
  const T sigma = sc.sigma;
  const T* __restrict__ xn = a.x[1 - p];
  const T* __restrict__ xc = a.x[p];
  const T* __restrict__ yc = a.y[p];
  T* __restrict__ yn = a.y[1 - p];
  const T* __restrict__ kxc = kStored ? a.Kx[p] : nullptr;
  const int gw = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kBlock) >> 5;
  const int ns = a.K.nslices;
  // copies of slice s (entries [ob, oe)) into sl; one copy group per call,
  // empty past the last slice
  auto issue = [&](int s, int ob, int oe, Slot& sl) {
    if (s < ns) {
      const int w = (oe - ob) >> 5;
      if (lane == 0) {
        sl.hdr[0] = ob;
        sl.hdr[1] = w;
      }
      const int r0 = s * kSlice;
      issue_slice<T, NR>(sl, a.K.col, a.K.val, ob, w, lane, [&](int v) -> const T* {
        switch (v) {
          case 0: return yc + r0;
          case 1: return a.q + r0;
          case 2: return a.ylo ? a.ylo + r0 : nullptr;
          case 3: return has_pw ? a.ybar + r0 : nullptr;
          default: return kStored ? kxc + r0 : nullptr;
        }
      });
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 0; k < R - 1; ++k) {
    const int s = min(gw + k * nw, ns);
    issue(gw + k * nw, __ldg(a.K.off + s), __ldg(a.K.off + min(s + 1, ns)), ring[k]);
  }
  int s_next = gw + (R - 1) * nw;
  int nb0 = __ldg(a.K.off + min(s_next, ns)), nb1 = __ldg(a.K.off + min(s_next + 1, ns));
  T acc_dy2 = 0, acc_int = 0;
  int k = 0;
  for (int s = gw; s < ns; s += nw) {
    int kn = k + R - 1;
    if (kn >= R) kn -= R;
    issue(s_next, nb0, nb1, ring[kn]);
    s_next += nw;
    nb0 = __ldg(a.K.off + min(s_next, ns));
    nb1 = __ldg(a.K.off + min(s_next + 1, ns));
    cp_async_wait<R - 1>();  // this lane's copies of slice s have landed
    __syncwarp();            // and every other lane's, and lane 0's header
    const Slot& sl = ring[k];
    const int o0 = sl.hdr[0] + lane, w = sl.hdr[1];
    T kx = 0, ko = 0;
#pragma unroll
    for (int e = 0; e < kRingE; ++e)
      if (e < w) {
        const int c = sl.col[e][lane];
        const T v = sl.val[e][lane];
        kx += v * __ldg(xn + c);
        if constexpr (!kStored) ko += v * __ldg(xc + c);
      }
    for (int k0 = kRingE; k0 < w; k0 += 4) {
      int c[4];
      T v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const bool ok = k0 + e < w;
        c[e] = ok ? __ldg(a.K.col + o0 + (k0 + e) * kSlice) : 0;
        v[e] = ok ? __ldg(a.K.val + o0 + (k0 + e) * kSlice) : (T)0;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (k0 + e < w) {
          kx += v[e] * __ldg(xn + c[e]);
          if constexpr (!kStored) ko += v[e] * __ldg(xc + c[e]);
        }
    }
    const int i = s * kSlice + lane;
    if (i < a.m) {
      const T yo = sl.row[0][lane], qi = sl.row[1][lane];
      if constexpr (kStored) ko = sl.row[NR - 1][lane];
      T t = qi - (T)2 * kx;
      t = t + ko;
      T v = yo + sigma * t;
      if (i >= a.m_eq) v = max(v, a.ylo ? sl.row[2][lane] : (T)0);
      yn[i] = v;
      if constexpr (kStored) a.Kx[1 - p][i] = kx;
      if (has_pw) a.ybar[i] = sl.row[3][lane] + pwT * yo;
      const T dy = v - yo;
      acc_dy2 += dy * dy;
      acc_int += dy * (kx - ko);
    }
    __syncwarp();  // every lane has read the slot before lane 0 rewrites a header
    k = (k + 1 == R) ? 0 : k + 1;
  }
  cp_async_wait<0>();
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

template <class T, int R>
__global__ void __launch_bounds__(kBlock) k_adjoint_ring(IterArgs<T> a) {
  DevState* st = a.st;
  __shared__ AdjScalars<T> sc;
  if (threadIdx.x == 0) adj_scalars<T>(st, sc);
  __syncthreads();
  if (sc.done) return;
  using Slot = RingSlot<T, kAdjOps>;
  extern __shared__ __align__(16) unsigned char ring_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Slot* ring = reinterpret_cast<Slot*>(ring_raw) + warp * R;
  const int p = sc.p;
  const int acc_last = sc.acc_last;
  const bool upd_avg = sc.upd_avg;
  const T wlT = sc.wl;
  const T tau = sc.tau;
  const T* __restrict__ yc = a.y[p];
  const T* __restrict__ xc = a.x[p];
  T* __restrict__ kty = a.KTy[p];
  T* __restrict__ xn = a.x[1 - p];
  const int gw = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nw = (gridDim.x * kBlock) >> 5;
  const int ns = a.KT.nslices;
  // a rejected step reuses the cached K^T y: no matrix entries are copied
  auto issue = [&](int s, int ob, int oe, Slot& sl) {
    if (s < ns) {
      const int w = acc_last ? (oe - ob) >> 5 : 0;
      if (lane == 0) {
        sl.hdr[0] = ob;
        sl.hdr[1] = w;
      }
      const int r0 = s * kSlice;
      issue_slice<T, kAdjOps>(sl, a.KT.col, a.KT.val, ob, w, lane, [&](int v) -> const T* {
        switch (v) {
          case 0: return xc + r0;
          case 1: return a.c + r0;
          case 2: return a.l + r0;
          case 3: return a.u + r0;
          case 4: return upd_avg ? a.xbar + r0 : nullptr;
          default: return acc_last ? nullptr : kty + r0;
        }
      });
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 0; k < R - 1; ++k) {
    const int s = min(gw + k * nw, ns);
    issue(gw + k * nw, __ldg(a.KT.off + s), __ldg(a.KT.off + min(s + 1, ns)), ring[k]);
  }
  int s_next = gw + (R - 1) * nw;
  int nb0 = __ldg(a.KT.off + min(s_next, ns)), nb1 = __ldg(a.KT.off + min(s_next + 1, ns));
  T acc_dx2 = 0;
  int k = 0;
  for (int s = gw; s < ns; s += nw) {
    int kn = k + R - 1;
    if (kn >= R) kn -= R;
    issue(s_next, nb0, nb1, ring[kn]);
    s_next += nw;
    nb0 = __ldg(a.KT.off + min(s_next, ns));
    nb1 = __ldg(a.KT.off + min(s_next + 1, ns));
    cp_async_wait<R - 1>();
    __syncwarp();
    const Slot& sl = ring[k];
    const int o0 = sl.hdr[0] + lane, w = sl.hdr[1];
    const int j = s * kSlice + lane;
    T g = 0;
    if (acc_last) {
#pragma unroll
      for (int e = 0; e < kRingE; ++e)
        if (e < w) g += sl.val[e][lane] * __ldg(yc + sl.col[e][lane]);
      for (int k0 = kRingE; k0 < w; k0 += 4) {
        int c[4];
        T v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const bool ok = k0 + e < w;
          c[e] = ok ? __ldg(a.KT.col + o0 + (k0 + e) * kSlice) : 0;
          v[e] = ok ? __ldg(a.KT.val + o0 + (k0 + e) * kSlice) : (T)0;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (k0 + e < w) g += v[e] * __ldg(yc + c[e]);
      }
    } else if (j < a.n) {
      g = sl.row[5][lane];
    }
    if (j < a.n) {
      const T x0 = sl.row[0][lane], cj = sl.row[1][lane];
      if (acc_last) kty[j] = g;
      if (upd_avg) a.xbar[j] = sl.row[4][lane] + wlT * x0;
      T v = x0 - tau * (cj - g);
      v = min(max(v, sl.row[2][lane]), sl.row[3][lane]);
      xn[j] = v;
      const T d = v - x0;
      acc_dx2 += d * d;
    }
    __syncwarp();
    k = (k + 1 == R) ? 0 : k + 1;
  }
  cp_async_wait<0>();
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

}  // namespace

// Variant 20: a ring of 3 slots per warp (two slices ahead), 21: 4 slots.
template <class T>
void launch_dual_ring(const IterArgs<T>& a, int grid, cudaStream_t s, int slots) {
  constexpr int NR = dual_ops<T>();
  if (slots == 4)
    k_dual_ring<T, 4><<<grid, kBlock, ring_bytes<T, NR, 4>(), s>>>(a);
  else
    k_dual_ring<T, 3><<<grid, kBlock, ring_bytes<T, NR, 3>(), s>>>(a);
}

template <class T>
void launch_adjoint_ring(const IterArgs<T>& a, int grid, cudaStream_t s, int slots) {
  if (slots == 4)
    k_adjoint_ring<T, 4><<<grid, kBlock, ring_bytes<T, kAdjOps, 4>(), s>>>(a);
  else
    k_adjoint_ring<T, 3><<<grid, kBlock, ring_bytes<T, kAdjOps, 3>(), s>>>(a);
}

// Dynamic shared memory beyond 48 KB, allowed once per device per kernel.
int ring_setup() {
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  if (done[dev]) return 0;
  struct F {
    const void* fn;
    size_t bytes;
  };
  const F fs[8] = {
      {(const void*)&k_dual_ring<float, 3>, ring_bytes<float, dual_ops<float>(), 3>()},
      {(const void*)&k_dual_ring<float, 4>, ring_bytes<float, dual_ops<float>(), 4>()},
      {(const void*)&k_adjoint_ring<float, 3>, ring_bytes<float, kAdjOps, 3>()},
      {(const void*)&k_adjoint_ring<float, 4>, ring_bytes<float, kAdjOps, 4>()},
      {(const void*)&k_dual_ring<double, 3>, ring_bytes<double, dual_ops<double>(), 3>()},
      {(const void*)&k_dual_ring<double, 4>, ring_bytes<double, dual_ops<double>(), 4>()},
      {(const void*)&k_adjoint_ring<double, 3>, ring_bytes<double, kAdjOps, 3>()},
      {(const void*)&k_adjoint_ring<double, 4>, ring_bytes<double, kAdjOps, 4>()}};
  for (const F& f : fs)
    if (cudaFuncSetAttribute(f.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.bytes) != cudaSuccess)
      return -1;
  done[dev] = true;
  return 0;
}

template void launch_dual_ring<float>(const IterArgs<float>&, int, cudaStream_t, int);
template void launch_dual_ring<double>(const IterArgs<double>&, int, cudaStream_t, int);
template void launch_adjoint_ring<float>(const IterArgs<float>&, int, cudaStream_t, int);
template void launch_adjoint_ring<double>(const IterArgs<double>&, int, cudaStream_t, int);

}  // namespace ucpdhg
