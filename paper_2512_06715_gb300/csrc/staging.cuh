// Building blocks of the kernels that stage operands in shared memory with
// 1-D bulk copies of the Tensor Memory Accelerator (cp.async.bulk completing on
// an mbarrier): barrier and copy wrappers, the row products from a staged
// chunk, and the two-buffer chunk pipeline with bounded waits.
#pragma once

#include "internal.cuh"

namespace ucpdhg {
namespace staging {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bounded wait for the phase with the given parity; false if it never completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (int it = 0; it < (1 << 20); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// 1-D bulk copy global -> shared, completing `bytes` on the barrier.  Both
// addresses 16-byte aligned, bytes a multiple of 16 (chunk boundaries are
// slice boundaries: multiples of 32 entries).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Row products of P slices of the staged chunk at once (lane = row of each),
// entries in predicated groups of 4 per slice, so the gathers of all P slices
// of a group issue together before the first is consumed.
template <class T, int P, bool TWO>
__device__ __forceinline__ void staged_rows(const int32_t* __restrict__ scol, const T* __restrict__ sval,
                                            const int (&o)[P], const int (&w)[P], const T* __restrict__ x1,
                                            const T* __restrict__ x2, T (&acc1)[P], T (&acc2)[P]) {
  int wmax = 0;
#pragma unroll
  for (int u = 0; u < P; ++u) {
    acc1[u] = 0;
    acc2[u] = 0;
    wmax = max(wmax, w[u]);
  }
  for (int k0 = 0; k0 < wmax; k0 += 4) {
    int c[P][4];
    T v[P][4];
#pragma unroll
    for (int u = 0; u < P; ++u)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const bool ok = k0 + e < w[u];
        c[u][e] = ok ? scol[o[u] + (k0 + e) * kSlice] : 0;
        v[u][e] = ok ? sval[o[u] + (k0 + e) * kSlice] : (T)0;
      }
#pragma unroll
    for (int u = 0; u < P; ++u)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (k0 + e < w[u]) {
          acc1[u] += v[u][e] * __ldg(x1 + c[u][e]);
          if (TWO) acc2[u] += v[u][e] * __ldg(x2 + c[u][e]);
        }
  }
}

// Chunk pipeline: thread 0 keeps two copies in flight (issue(buffer, chunk)
// starts one and arms the buffer's barrier); work(buffer, chunk) runs when a
// chunk has landed.  Bounded waits: a timeout marks the block aborted (it
// keeps its barriers, starts no copies, skips the work) and thread 0 drains
// the copies it issued (bounded again); DevState::wait_timeout tells the host.
template <class Issue, class Work>
__device__ __forceinline__ void run_chunks(uint64_t* bar, int nch, bool stream, int* s_abort, DevState* st,
                                           Issue&& issue, Work&& work) {
  const int G = gridDim.x;
  const int nmine = (int)blockIdx.x < nch ? (nch - 1 - (int)blockIdx.x) / G + 1 : 0;
  int issued = 0;  // thread 0: chunks whose copy was started
  if (threadIdx.x == 0) {
    *s_abort = 0;
    if (stream) {
      mbar_init(&bar[0], 1);
      mbar_init(&bar[1], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && stream)
    for (; issued < 2 && issued < nmine; ++issued) issue(issued, blockIdx.x + issued * G);
  int first_pending = nmine;
  for (int i = 0; i < nmine; ++i) {
    const int b = i & 1;
    bool ok = *s_abort == 0;
    if (ok && stream) ok = mbar_wait(&bar[b], (uint32_t)((i >> 1) & 1));
    if (!ok) {
      *s_abort = 1;
      if (first_pending > i) first_pending = i;
    }
    if (ok) work(b, blockIdx.x + i * G);
    __syncthreads();  // every warp is done with buffer b
    if (threadIdx.x == 0 && stream && *s_abort == 0 && issued < nmine) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(b, blockIdx.x + issued * G);
      ++issued;
    }
  }
  if (threadIdx.x == 0 && *s_abort) {
    st->wait_timeout = 1;
    for (int k = first_pending; k < issued; ++k) mbar_wait(&bar[k & 1], (uint32_t)((k >> 1) & 1));
  }
}

}  // namespace staging
}  // namespace ucpdhg
