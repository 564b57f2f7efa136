// Rescaling without any device allocation (pdhg_rescale_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs where a caching
// allocator owns all device memory and forbids outside allocations, code with
// a fixed memory budget decided up front, or code that must not trigger the
// synchronisation an allocation can cause.  For them this entry point computes
// the same Ruiz + Pock-Chambolle factors as a workspace does, straight from the
// caller's device CSR, and writes them into the caller's Dr, Dc buffers.  The
// only scratch, the per-column statistics of one pass, lives in the fixed
// file-scope array below; every GPU that loads the library holds it until the
// process exits.
#include <cuda.h>  // CUcontext and CUresult types only; the driver calls are fetched at run time

#include <mutex>
#include <string>

#include "internal.cuh"

namespace ucpdhg {

// Columns the scratch can hold: 2^21 doubles = 16 MiB per device.
constexpr int64_t kNoAllocMaxCols = int64_t(1) << 21;
constexpr int kNoAllocMaxContexts = 64;

static __device__ __align__(256) double g_colstat[kNoAllocMaxCols];

namespace {

// The device address of g_colstat belongs to a CUDA context, not to a device
// ordinal: after cudaDeviceReset, or under a driver-API context other than the
// device's primary one, the address differs.  The cache is therefore keyed by
// the current context's unique id (cuCtxGetId: ids are never reused within a
// process), fetched through the runtime's driver entry points so the library
// does not link against libcuda.
std::mutex g_noalloc_mutex;
struct ScratchEntry {
  unsigned long long ctx_id;
  double* ptr;
};
ScratchEntry g_noalloc_scratch[kNoAllocMaxContexts];
int g_noalloc_entries = 0;
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Unique id of the calling thread's current context (0 if none or unknown).
unsigned long long current_context_id() {
  if (!g_ctx_get_current || !g_ctx_get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess)
      return 0;
    g_ctx_get_current = (CtxGetCurrentFn)f1;
    g_ctx_get_id = (CtxGetIdFn)f2;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

int noalloc_fail(int code, const std::string& msg) {
  g_err = msg;  // reported by pdhg_last_error()
  return code;
}

__global__ void k_clear(double* a, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    a[t] = 0.0;
}

__global__ void k_fill_one(double* a, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    a[t] = 1.0;
}

// Column statistic of one pass from the CSR rows: max (mode 0) or sum (mode 1)
// of |K_ij| Dr_i Dc_j over i.  The max uses the integer order of non-negative
// doubles (exact, order independent); the sum uses FP64 atomics.
__global__ void k_col_stat(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ Dr,
                           const double* __restrict__ Dc, int64_t m, int mode, double* colstat) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double dr = Dr[i];
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      const int32_t j = col[e];
      const double a = fabs(val[e]) * dr * Dc[j];
      if (mode)
        atomicAdd(colstat + j, a);
      else
        atomicMax((unsigned long long*)(colstat + j), (unsigned long long)__double_as_longlong(a));
    }
  }
}

// Row factor of the same pass, applied to Dr at once (the column statistics
// of this pass are complete, so they saw the old Dr).
__global__ void k_row_apply(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const double* __restrict__ val, double* Dr,
                            const double* __restrict__ Dc, int64_t m, int mode) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double dr = Dr[i];
    double stat = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      const double a = fabs(val[e]) * dr * Dc[col[e]];
      stat = mode ? stat + a : fmax(stat, a);
    }
    Dr[i] = dr * (stat > 0.0 ? 1.0 / sqrt(stat) : 1.0);
  }
}

__global__ void k_col_apply(const double* __restrict__ colstat, double* Dc, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const double s = colstat[j];
    Dc[j] = Dc[j] * (s > 0.0 ? 1.0 / sqrt(s) : 1.0);
  }
}

int grid_of(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  if (g > 152 * 8) g = 152 * 8;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace
}  // namespace ucpdhg

using namespace ucpdhg;

extern "C" int pdhg_rescale_noalloc(const pdhg_problem* prob, int32_t ruiz_iters,
                                    int32_t pock_chambolle, double* Dr, double* Dc, void* stream) {
  g_err.clear();
  if (!prob || !Dr || !Dc)
    return noalloc_fail(PDHG_ERR_INVALID_ARG, "pdhg_rescale_noalloc: NULL argument");
  if (prob->n < 1 || prob->m < 1 || prob->nnz < 0 || !prob->row_ptr ||
      (prob->nnz > 0 && (!prob->col || !prob->val)))
    return noalloc_fail(PDHG_ERR_INVALID_ARG, "pdhg_rescale_noalloc: bad problem sizes or pointers");
  if (ruiz_iters < 0 || ruiz_iters > 100)
    return noalloc_fail(PDHG_ERR_INVALID_ARG, "pdhg_rescale_noalloc: ruiz_iters out of range");
  if (prob->n > kNoAllocMaxCols)
    return noalloc_fail(PDHG_ERR_UNSUPPORTED,
                        "pdhg_rescale_noalloc: n = " + std::to_string(prob->n) +
                            " exceeds the fixed scratch of " + std::to_string(kNoAllocMaxCols) +
                            " columns");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0)
    return noalloc_fail(PDHG_ERR_CUDA, "pdhg_rescale_noalloc: no usable current device");
  double* colstat = nullptr;
  {
    // Once per context, with its device current: the device address of the
    // file-scope scratch (its host-side name is only a stand-in).
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    unsigned long long id = current_context_id();
    for (int k = 0; id != 0 && k < g_noalloc_entries; ++k)
      if (g_noalloc_scratch[k].ctx_id == id) colstat = g_noalloc_scratch[k].ptr;
    if (!colstat) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_colstat);
      if (e != cudaSuccess || !p)
        return noalloc_fail(PDHG_ERR_CUDA, std::string("pdhg_rescale_noalloc: cudaGetSymbolAddress: ") +
                                               cudaGetErrorString(e));
      colstat = (double*)p;
      // the lookup above made the runtime's context current if none was
      if (id == 0) id = current_context_id();
      if (id != 0 && g_noalloc_entries < kNoAllocMaxContexts)
        g_noalloc_scratch[g_noalloc_entries++] = {id, colstat};
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = prob->n, m = prob->m;
  k_fill_one<<<grid_of(m), kBlock, 0, s>>>(Dr, m);
  k_fill_one<<<grid_of(n), kBlock, 0, s>>>(Dc, n);
  const int passes = ruiz_iters + (pock_chambolle ? 1 : 0);
  for (int p = 0; p < passes; ++p) {
    const int mode = (p >= ruiz_iters) ? 1 : 0;
    k_clear<<<grid_of(n), kBlock, 0, s>>>(colstat, n);  // the array keeps the last call's values
    k_col_stat<<<grid_of(m), kBlock, 0, s>>>(prob->row_ptr, prob->col, prob->val, Dr, Dc, m, mode,
                                              colstat);
    k_row_apply<<<grid_of(m), kBlock, 0, s>>>(prob->row_ptr, prob->col, prob->val, Dr, Dc, m, mode);
    k_col_apply<<<grid_of(n), kBlock, 0, s>>>(colstat, Dc, n);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return noalloc_fail(PDHG_ERR_CUDA, std::string("pdhg_rescale_noalloc: ") + cudaGetErrorString(e));
  return PDHG_OK;
}
