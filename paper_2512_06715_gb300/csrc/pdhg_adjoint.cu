// Active-set linear algebra at the last solve: the vector-Jacobian product of
// the LP solution map (pdhg_backward) and the active-set polish of the solution
// to a basic one (pdhg_polish, a crossover-lite: the paper's pipeline hands the
// PDHG point to a crossover, Sec. III.B).
//
// At a nondegenerate optimum the active set -- equality rows, >= rows with
// positive dual, variables held at a bound by their reduced cost -- is a
// square nonsingular system: with A the active rows and F the variables not at
// a bound, S = K_{A,F} is square.  Then
//   d cost / d q = y*,  d cost / d c = x*                   (envelope theorem)
//   d (g_x^T x*) / d q_A = lambda_A  with  S^T lambda_A = g_F,  d (g_x^T x*) / d c = 0
//   polish:  S x_F = q_A - K_{A,B} x_B  (x_B at its bounds),  S^T y_A = c_F
// In the rescaled space K~ = Dr K Dc these are systems with S~ = K~_{A,F}, solved
// by conjugate gradients on the normal equations S~ S~^T z = rhs (Jacobi
// preconditioned: diag(S~ S~^T)_i = sum over free j of K~_ij^2) with the FP64
// sliced-ELL products of the workspace under row/column masks:
//   mode 0 (S~^T z = r):  S~ S~^T z = S~ r, converged when ||S~^T z - r|| <= tol ||r||
//   mode 1 (S~ x = b):    S~ S~^T z = b, x = S~^T z, converged when ||S~ S~^T z - b|| <= tol ||b||
// The whole CG loop runs on the device as one CUDA graph with a conditional
// WHILE node (16 iterations and one true-residual check per body); its scalars
// (alpha, beta, residuals) live in device memory, so the host waits once per
// solve instead of once per dot product.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace ucpdhg {
namespace {

constexpr int kCgPerBody = 16;  // CG iterations per graph body (then a true-residual check)

int vg(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  if (g > 152 * 8) g = 152 * 8;
  return (int)(g < 1 ? 1 : g);
}

// Device-resident CG scalars.
struct CGState {
  double rr, rr0, alpha, beta, target, resid, rhs2;  // rr: preconditioned r^T M^-1 r
  int64_t it, max_it;
  int32_t mode, done, converged, pad;
  uint32_t counter, counter2;
};

// Active-set masks in the rescaled space from x~*, y~*, s~ = K~x~* - q~ and
// lambda~ = c~ - K~^T y~*: a >= row is active iff y~_i > s~_i; a variable is at
// a bound iff its reduced cost outweighs its distance to that bound (or l = u).
// xfix: the bound a non-free variable sits at (its value otherwise).
__global__ void k_classify(const double* __restrict__ x, const double* __restrict__ y,
                           const double* __restrict__ Kx, const double* __restrict__ KTy,
                           const double* __restrict__ q, const double* __restrict__ c,
                           const double* __restrict__ l, const double* __restrict__ u, int64_t n,
                           int64_t m, int64_t m_eq, double* rowA, double* colF, double* xfix,
                           double* partials) {
  double cnt[2] = {0.0, 0.0};
  const int64_t N = n > m ? n : m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < m) {
      double a = 1.0;
      if (t >= m_eq) {
        const double s = Kx[t] - q[t];
        a = (y[t] > s) ? 1.0 : 0.0;
      }
      rowA[t] = a;
      cnt[0] += a;
    }
    if (t < n) {
      const double lam = c[t] - KTy[t];
      const double lo = l[t], up = u[t];
      double at = x[t];
      bool fixed = false;
      if (isfinite(lo) && isfinite(up) && lo == up) {
        fixed = true;
        at = lo;
      } else if (isfinite(lo) && lam > 0.0 && lam > x[t] - lo) {
        fixed = true;
        at = lo;
      } else if (isfinite(up) && lam < 0.0 && -lam > up - x[t]) {
        fixed = true;
        at = up;
      }
      const double f = fixed ? 0.0 : 1.0;
      colF[t] = f;
      xfix[t] = at;
      cnt[1] += f;
    }
  }
  __shared__ double sm[kWarps * 2];
  block_sum<2>(cnt, sm);
  if (threadIdx.x == 0) {
    partials[blockIdx.x * 2 + 0] = cnt[0];
    partials[blockIdx.x * 2 + 1] = cnt[1];
  }
}

__global__ void k_final2(const double* partials, int nb, double* out) {
  double v[2];
  final_sum<2>(partials, nb, v);
  if (threadIdx.x == 0) {
    out[0] = v[0];
    out[1] = v[1];
  }
}

// out = outmask .* (A (inmask .* in)), masks optional.  Skipped when the CG is
// done, or when only_mode >= 0 and the CG runs in another mode.
__global__ void __launch_bounds__(kBlock) k_mspmv(SellView<double> A, const double* __restrict__ in,
                                                  const double* __restrict__ inmask,
                                                  const double* __restrict__ outmask,
                                                  double* __restrict__ out, const CGState* cg,
                                                  int only_mode) {
  if (cg && (cg->done || (only_mode >= 0 && cg->mode != only_mode))) return;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int s = gw; s < A.nslices; s += nw) {
    const int o0 = A.off[s], w = (A.off[s + 1] - o0) >> 5;
    double acc = 0.0;
    for (int k = 0; k < w; ++k) {
      const int slot = o0 + k * kSlice + lane;
      const int c = __ldg(A.col + slot);
      double v = __ldg(in + c);
      if (inmask) v *= __ldg(inmask + c);
      acc += __ldg(A.val + slot) * v;
    }
    const int r = s * kSlice + lane;
    if (r < A.rows) out[r] = outmask ? acc * outmask[r] : acc;
  }
}

// Jacobi preconditioner of S~ S~^T: dinv_i = 1 / sum_{j free} K~_ij^2 on active
// rows (1 elsewhere, where the residual is 0 anyway).
__global__ void __launch_bounds__(kBlock) k_jacobi(SellView<double> A, const double* __restrict__ colF,
                                                   const double* __restrict__ rowA, double* dinv) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int s = gw; s < A.nslices; s += nw) {
    const int o0 = A.off[s], w = (A.off[s + 1] - o0) >> 5;
    double d = 0.0;
    for (int k = 0; k < w; ++k) {
      const int slot = o0 + k * kSlice + lane;
      const double v = __ldg(A.val + slot);
      d += v * v * __ldg(colF + __ldg(A.col + slot));
    }
    const int r = s * kSlice + lane;
    if (r < A.rows) dinv[r] = (rowA[r] > 0.0 && d > 0.0) ? 1.0 / d : 1.0;
  }
}

__global__ void k_cg_init(CGState* cg, int mode, double tol2, int64_t max_it) {
  cg->mode = mode;
  cg->target = tol2;  // scaled by ||rhs||^2 in k_cg_start
  cg->max_it = max_it;
  cg->it = 0;
  cg->done = 0;
  cg->converged = 0;
  cg->resid = 0.0;
  cg->counter = cg->counter2 = 0;
}

// z = 0, P = M^-1 R; rr = R^T M^-1 R, and ||rhs||^2 (r.r over n in mode 0,
// R.R in mode 1).
__global__ void __launch_bounds__(kBlock) k_cg_start(double* z, double* P, const double* __restrict__ R,
                                                     const double* __restrict__ dinv,
                                                     const double* __restrict__ r, int64_t m, int64_t n,
                                                     CGState* cg, double* partials) {
  const int mode = cg->mode;
  double v[3] = {0.0, 0.0, 0.0};
  const int64_t N = n > m ? n : m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < m) {
      z[t] = 0.0;
      const double zt = dinv[t] * R[t];
      P[t] = zt;
      v[0] += R[t] * zt;
      v[2] += R[t] * R[t];
    }
    if (mode == 0 && t < n) v[1] += r[t] * r[t];
  }
  if (publish_partials<3>(v, partials, &cg->counter)) {
    double tot[3];
    final_sum<3>(partials, gridDim.x, tot);
    if (threadIdx.x == 0) {
      const double gg = mode == 0 ? tot[1] : tot[2];
      cg->rr = tot[0];
      cg->rr0 = tot[0];
      cg->rhs2 = gg;
      cg->target *= (gg > 0.0 ? gg : 1.0);
      if (!(tot[2] > 0.0)) {
        cg->done = 1;
        cg->converged = 1;
      }
      cg->counter = 0;
    }
  }
}

// alpha = rr / (P.Q)
__global__ void __launch_bounds__(kBlock) k_cg_pq(const double* __restrict__ P, const double* __restrict__ Q,
                                                  int64_t m, CGState* cg, double* partials) {
  if (cg->done) return;
  double v[1] = {0.0};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x)
    v[0] += P[t] * Q[t];
  if (publish_partials<1>(v, partials, &cg->counter)) {
    double tot[1];
    final_sum<1>(partials, gridDim.x, tot);
    if (threadIdx.x == 0) {
      if (tot[0] > 0.0)
        cg->alpha = cg->rr / tot[0];
      else
        cg->done = 1;  // breakdown: not positive definite on this subspace
      cg->counter = 0;
    }
  }
}

// z += alpha P, R -= alpha Q, Zp = M^-1 R; beta = R^T Zp / rr, rr = R^T Zp
__global__ void __launch_bounds__(kBlock) k_cg_update(double* z, const double* __restrict__ P, double* R,
                                                      const double* __restrict__ Q,
                                                      const double* __restrict__ dinv, double* Zp,
                                                      int64_t m, CGState* cg, double* partials) {
  if (cg->done) return;
  const double alpha = cg->alpha;
  double v[1] = {0.0};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    z[t] += alpha * P[t];
    const double rn = R[t] - alpha * Q[t];
    R[t] = rn;
    const double zn = dinv[t] * rn;
    Zp[t] = zn;
    v[0] += rn * zn;
  }
  if (publish_partials<1>(v, partials, &cg->counter)) {
    double tot[1];
    final_sum<1>(partials, gridDim.x, tot);
    if (threadIdx.x == 0) {
      cg->beta = tot[0] / cg->rr;
      cg->rr = tot[0];
      cg->it += 1;
      if (cg->it >= cg->max_it) cg->done = 1;
      cg->counter = 0;
    }
  }
}

// P = Zp + beta P  (Zp = M^-1 R)
__global__ void k_cg_dir(double* P, const double* __restrict__ Zp, int64_t m, const CGState* cg) {
  if (cg->done) return;
  const double beta = cg->beta;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x)
    P[t] = Zp[t] + beta * P[t];
}

// True residual: mode 0 ||T - r||^2 over n (T = S^T z), mode 1 ||Q2 - b||^2 over m
// (Q2 = S S^T z); converged when it reaches the target.
__global__ void __launch_bounds__(kBlock) k_cg_resid(const double* __restrict__ T,
                                                     const double* __restrict__ r,
                                                     const double* __restrict__ Q2,
                                                     const double* __restrict__ b, int64_t m, int64_t n,
                                                     CGState* cg, double* partials) {
  if (cg->done) return;
  const int mode = cg->mode;
  const double* u = mode == 0 ? T : Q2;
  const double* w = mode == 0 ? r : b;
  const int64_t len = mode == 0 ? n : m;
  double v[1] = {0.0};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < len;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double d = u[t] - w[t];
    v[0] += d * d;
  }
  if (publish_partials<1>(v, partials, &cg->counter2)) {
    double tot[1];
    final_sum<1>(partials, gridDim.x, tot);
    if (threadIdx.x == 0) {
      cg->resid = tot[0];
      if (tot[0] <= cg->target) {
        cg->done = 1;
        cg->converged = 1;
      }
      cg->counter2 = 0;
    }
  }
}

__global__ void k_cg_cond(const CGState* cg, unsigned long long handle) {
  if (threadIdx.x == 0) cudaGraphSetConditional((cudaGraphConditionalHandle)handle, cg->done ? 0u : 1u);
}

__global__ void k_mask_mul(const double* __restrict__ a, const double* __restrict__ mask, double* out,
                           int64_t n, const double* __restrict__ scale) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    double v = a[t] * mask[t];
    if (scale) v *= scale[t];
    out[t] = v;
  }
}

// b = rowA .* (q~ - K~ x_B)  (Kb holds K~ x_B)
__global__ void k_polish_rhs(const double* __restrict__ q, const double* __restrict__ Kb,
                             const double* __restrict__ rowA, double* b, int64_t m) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x)
    b[t] = rowA[t] * (q[t] - Kb[t]);
}

// out = (1 - F) .* xfix: the variables held at a bound, the free ones 0
__global__ void k_fixed_part(const double* __restrict__ xfix, const double* __restrict__ colF, double* out,
                             int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = colF[t] > 0.0 ? 0.0 : xfix[t];
}

// x = F .* T + (1 - F) .* xfix
__global__ void k_polish_x(const double* __restrict__ T, const double* __restrict__ colF,
                           const double* __restrict__ xfix, double* x, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    x[t] = colF[t] > 0.0 ? T[t] : xfix[t];
}

// Optimality measures of a point (x~, y~) of the rescaled LP, unscaled (the
// definitions of pdhg.h): sums 0 ||r_p||^2, 1 ||r_d||^2, 2 c~^T x~, 3 q~^T y~,
// 4 bound term of D, 5 bound violations^2 of x, 6 sign violations^2 of y.
constexpr int kPolishSums = 7;
__global__ void __launch_bounds__(kBlock) k_polish_kkt(
    const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ Kx,
    const double* __restrict__ KTy, const double* __restrict__ q, const double* __restrict__ c,
    const double* __restrict__ l, const double* __restrict__ u, const double* __restrict__ Dr,
    const double* __restrict__ Dc, const double* __restrict__ iDr, const double* __restrict__ iDc,
    int64_t n, int64_t m, int64_t m_eq, double* partials) {
  double v[kPolishSums];
#pragma unroll
  for (int k = 0; k < kPolishSums; ++k) v[k] = 0.0;
  const int64_t N = n > m ? n : m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < m) {
      double r = q[t] - Kx[t];
      if (t >= m_eq) r = fmax(r, 0.0);
      r *= iDr[t];
      v[0] += r * r;
      v[3] += q[t] * y[t];
      if (t >= m_eq) {
        const double sv = fmin(y[t], 0.0) * Dr[t];
        v[6] += sv * sv;
      }
    }
    if (t < n) {
      const double lo = l[t], up = u[t];
      const bool lf = isfinite(lo), uf = isfinite(up);
      const double lam = c[t] - KTy[t];
      const double proj = (lf ? fmax(lam, 0.0) : 0.0) + (uf ? fmin(lam, 0.0) : 0.0);
      const double rd = (lam - proj) * iDc[t];
      v[1] += rd * rd;
      v[2] += c[t] * x[t];
      v[4] += (lf ? lo * fmax(proj, 0.0) : 0.0) - (uf ? up * fmax(-proj, 0.0) : 0.0);
      const double bv = ((lf ? fmax(lo - x[t], 0.0) : 0.0) + (uf ? fmax(x[t] - up, 0.0) : 0.0)) * Dc[t];
      v[5] += bv * bv;
    }
  }
  __shared__ double sm[kWarps * kPolishSums];
  block_sum<kPolishSums>(v, sm);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < kPolishSums; ++k) partials[blockIdx.x * kPolishSums + k] = v[k];
}

__global__ void k_polish_final(const double* partials, int nb, double* out) {
  double v[kPolishSums];
  final_sum<kPolishSums>(partials, nb, v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < kPolishSums; ++k) out[k] = v[k];
}

__global__ void k_backward_out(const int32_t* __restrict__ perm_row, const int32_t* __restrict__ perm_col,
                               const double* __restrict__ Dr, const double* __restrict__ Dc,
                               const double* __restrict__ ys, const double* __restrict__ xs,
                               const double* __restrict__ mu, const double* __restrict__ rowA,
                               double g_cost, int has_gx, double* grad_q, double* grad_c, int64_t n,
                               int64_t m) {
  const int64_t N = n > m ? n : m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < m) {
      double gq = g_cost * Dr[t] * ys[t];
      if (has_gx) gq += rowA[t] * Dr[t] * mu[t];
      grad_q[perm_row[t]] = gq;
    }
    if (t < n) grad_c[perm_col[t]] = g_cost * Dc[t] * xs[t];
  }
}

// unscaled output in original order: out[perm[t]] = D[t] v[t]
__global__ void k_unscale_out(const int32_t* __restrict__ perm, const double* __restrict__ D,
                              const double* __restrict__ v, double* out, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    out[perm[t]] = D[t] * v[t];
}

}  // namespace

// FP64 scratch of the active-set solves, allocated at the first call.
struct AdjBufs {
  double *Kx = nullptr, *KTy = nullptr, *rowA = nullptr, *colF = nullptr, *xfix = nullptr;
  double *z = nullptr, *R = nullptr, *P = nullptr, *Q = nullptr, *Q2 = nullptr, *b = nullptr;
  double *T = nullptr, *r = nullptr, *xp = nullptr, *yp = nullptr, *dinv = nullptr, *Zp = nullptr;
  CGState* cg = nullptr;
  CGState* cg_host = nullptr;  // pinned
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void*> allocs;
};

void release_adjoint(Workspace* w) {
  AdjBufs* ab = (AdjBufs*)w->adjoint;
  if (!ab) return;
  if (ab->exec) cudaGraphExecDestroy(ab->exec);
  if (ab->graph) cudaGraphDestroy(ab->graph);
  if (ab->cg_host) cudaFreeHost(ab->cg_host);
  for (void* p : ab->allocs) cudaFree(p);
  delete ab;
  w->adjoint = nullptr;
}

static int adj_bufs(Workspace* w, AdjBufs** out) {
  if (w->adjoint) {
    *out = (AdjBufs*)w->adjoint;
    return PDHG_OK;
  }
  AdjBufs* ab = new AdjBufs();
  const int64_t n = w->n, m = w->m;
  double** vm[] = {&ab->Kx, &ab->rowA, &ab->z, &ab->R, &ab->P, &ab->Q, &ab->Q2, &ab->b, &ab->yp,
                   &ab->dinv, &ab->Zp};
  double** vn[] = {&ab->KTy, &ab->colF, &ab->xfix, &ab->T, &ab->r, &ab->xp};
  bool ok = true;
  for (double** p : vm) {
    void* q = nullptr;
    ok = ok && cudaMalloc(&q, sizeof(double) * (m + 2)) == cudaSuccess;
    if (ok) ab->allocs.push_back(q), *p = (double*)q;
  }
  for (double** p : vn) {
    void* q = nullptr;
    ok = ok && cudaMalloc(&q, sizeof(double) * (n + 2)) == cudaSuccess;
    if (ok) ab->allocs.push_back(q), *p = (double*)q;
  }
  void* q = nullptr;
  ok = ok && cudaMalloc(&q, sizeof(CGState)) == cudaSuccess;
  if (ok) ab->allocs.push_back(q), ab->cg = (CGState*)q;
  ok = ok && cudaMallocHost(&ab->cg_host, sizeof(CGState)) == cudaSuccess;
  if (!ok) {
    w->adjoint = ab;
    release_adjoint(w);
    g_err = "active-set solve: device allocation failed";
    return PDHG_ERR_NOMEM;
  }
  w->adjoint = ab;
  *out = ab;
  return PDHG_OK;
}

// One CG iteration and the periodic residual check, enqueued on s (the graph
// body; every kernel returns at once when the CG is done).
static void cg_body(Workspace* w, AdjBufs* ab, cudaStream_t s, unsigned long long handle) {
  const int64_t n = w->n, m = w->m;
  double* part = w->partials;
  for (int it = 0; it < kCgPerBody; ++it) {
    k_mspmv<<<w->grid_kt, kBlock, 0, s>>>(w->KT.v64(), ab->P, ab->rowA, ab->colF, ab->T, ab->cg, -1);
    k_mspmv<<<w->grid_k, kBlock, 0, s>>>(w->K.v64(), ab->T, ab->colF, ab->rowA, ab->Q, ab->cg, -1);
    k_cg_pq<<<vg(m), kBlock, 0, s>>>(ab->P, ab->Q, m, ab->cg, part);
    k_cg_update<<<vg(m), kBlock, 0, s>>>(ab->z, ab->P, ab->R, ab->Q, ab->dinv, ab->Zp, m, ab->cg, part);
    k_cg_dir<<<vg(m), kBlock, 0, s>>>(ab->P, ab->Zp, m, ab->cg);
  }
  k_mspmv<<<w->grid_kt, kBlock, 0, s>>>(w->KT.v64(), ab->z, ab->rowA, ab->colF, ab->T, ab->cg, -1);
  k_mspmv<<<w->grid_k, kBlock, 0, s>>>(w->K.v64(), ab->T, ab->colF, ab->rowA, ab->Q2, ab->cg, 1);
  k_cg_resid<<<vg(n > m ? n : m), kBlock, 0, s>>>(ab->T, ab->r, ab->Q2, ab->b, m, n, ab->cg, part);
  k_cg_cond<<<1, 32, 0, s>>>(ab->cg, handle);
}

static int build_cg_graph(Workspace* w, AdjBufs* ab) {
  if (ab->exec) return PDHG_OK;
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return PDHG_ERR_CUDA;
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
    cudaGraphDestroy(g);
    return PDHG_ERR_CUDA;
  }
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  std::memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(raw);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess) {
    cudaGraphDestroy(g);
    return PDHG_ERR_CUDA;
  }
  if (cudaStreamBeginCaptureToGraph(w->cap_stream, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGraphDestroy(g);
    return PDHG_ERR_CUDA;
  }
  cg_body(w, ab, w->cap_stream, (unsigned long long)h);
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(w->cap_stream, &captured);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ab->exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    g_err = std::string("active-set CG graph: ") + cudaGetErrorString(e);
    return PDHG_ERR_CUDA;
  }
  ab->graph = g;
  return PDHG_OK;
}

// Solves S~ S~^T z = rhs on the device (mode 0: rhs = S~ r with r in ab->r;
// mode 1: rhs = ab->b) and copies the final CG scalars to *out.  One host wait.
static int cg_run(Workspace* w, AdjBufs* ab, int mode, double tol, int64_t max_it, cudaStream_t s,
                  CGState* out) {
  int rc = build_cg_graph(w, ab);
  if (rc != PDHG_OK) return rc;
  const int64_t n = w->n, m = w->m;
  k_cg_init<<<1, 1, 0, s>>>(ab->cg, mode, tol * tol, max_it);
  if (mode == 0)
    k_mspmv<<<w->grid_k, kBlock, 0, s>>>(w->K.v64(), ab->r, ab->colF, ab->rowA, ab->R, nullptr, -1);
  else
    cudaMemcpyAsync(ab->R, ab->b, sizeof(double) * m, cudaMemcpyDeviceToDevice, s);
  k_cg_start<<<vg(n > m ? n : m), kBlock, 0, s>>>(ab->z, ab->P, ab->R, ab->dinv, ab->r, m, n, ab->cg,
                                                   w->partials);
  cudaError_t e = cudaGraphLaunch(ab->exec, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ab->cg_host, ab->cg, sizeof(CGState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_err = std::string("active-set CG: ") + cudaGetErrorString(e);
    return PDHG_ERR_CUDA;
  }
  *out = *ab->cg_host;
  return PDHG_OK;
}

// Active set of the last solve: masks, fixed values, counts (one host wait).
static int classify(Workspace* w, AdjBufs* ab, cudaStream_t s, int64_t* nA, int64_t* nF) {
  const int64_t n = w->n, m = w->m;
  launch_spmv64(w->K.v64(), w->x_star, ab->Kx, w->grid_k, s);
  launch_spmv64(w->KT.v64(), w->y_star, ab->KTy, w->grid_kt, s);
  const int gN = vg(n > m ? n : m);
  double* scal = w->scalars + 8;  // [8..15] scratch scalars
  k_classify<<<gN, kBlock, 0, s>>>(w->x_star, w->y_star, ab->Kx, ab->KTy, w->q_s, w->c_s, w->l_s, w->u_s,
                                   n, m, w->m_eq, ab->rowA, ab->colF, ab->xfix, w->partials);
  k_final2<<<1, kBlock, 0, s>>>(w->partials, gN, scal);
  k_jacobi<<<w->grid_k, kBlock, 0, s>>>(w->K.v64(), ab->colF, ab->rowA, ab->dinv);
  double hs[2];
  if (cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    g_err = std::string("active set: ") + cudaGetErrorString(cudaGetLastError());
    return PDHG_ERR_CUDA;
  }
  *nA = (int64_t)llround(hs[0]);
  *nF = (int64_t)llround(hs[1]);
  return PDHG_OK;
}

static int64_t cg_max_it(int64_t nA) { return std::min<int64_t>(20 * (nA + 10), 200000); }

// A polish is accepted when both systems reach this relative residual (the CG
// aims at 1e-13; the normal equations square the active set's condition number,
// which can stop FP64 CG short of that).
constexpr double kPolishAccept = 1e-9;

}  // namespace ucpdhg

using namespace ucpdhg;

extern "C" int pdhg_backward(void* ws, double g_cost, const double* g_x, double* grad_q,
                             double* grad_c, void* stream) {
  g_err.clear();
  if (!ws || !grad_q || !grad_c) {
    g_err = "pdhg_backward: NULL argument";
    return PDHG_ERR_INVALID_ARG;
  }
  Workspace* w = (Workspace*)ws;
  if (!w->solved) {
    g_err = "pdhg_backward: no solution in this workspace (call pdhg_solve first)";
    return PDHG_ERR_INVALID_ARG;
  }
  AdjBufs* ab = nullptr;
  int rc = adj_bufs(w, &ab);
  if (rc != PDHG_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = w->n, m = w->m;
  int64_t nA = 0, nF = 0;
  if ((rc = classify(w, ab, s, &nA, &nF)) != PDHG_OK) return rc;
  const bool has_gx = g_x != nullptr;
  if (has_gx && nA != nF) {
    g_err = "pdhg_backward: the active set is not square (" + std::to_string(nA) + " active rows, " +
            std::to_string(nF) + " free variables): the LP is degenerate at this solution";
    return PDHG_ERR_NUMERIC;
  }
  if (has_gx) {
    // r = Dc g_F (internal order); S~^T mu = r
    launch_gather_perm(w->perm_col, g_x, ab->T, n, s);
    k_mask_mul<<<vg(n), kBlock, 0, s>>>(ab->T, ab->colF, ab->r, n, w->Dc);
    CGState st;
    if ((rc = cg_run(w, ab, 0, 1e-13, cg_max_it(nA), s, &st)) != PDHG_OK) return rc;
    // converged to 1e-13, or at least to a relative residual of 1e-8
    if (!st.converged && !(st.resid <= 1e10 * st.target)) {
      g_err = "pdhg_backward: CG on the active set did not converge (" + std::to_string(st.it) +
              " iterations)";
      return PDHG_ERR_NUMERIC;
    }
  }
  k_backward_out<<<vg(n > m ? n : m), kBlock, 0, s>>>(w->perm_row, w->perm_col, w->Dr, w->Dc, w->y_star,
                                                      w->x_star, ab->z, ab->rowA, g_cost,
                                                      has_gx ? 1 : 0, grad_q, grad_c, n, m);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_err = std::string("pdhg_backward: ") + cudaGetErrorString(e);
    return PDHG_ERR_CUDA;
  }
  return PDHG_OK;
}

extern "C" int pdhg_polish(void* ws, double* x_out, double* y_out, pdhg_polish_result* res, void* stream) {
  g_err.clear();
  if (!ws || !res) {
    g_err = "pdhg_polish: NULL argument";
    return PDHG_ERR_INVALID_ARG;
  }
  Workspace* w = (Workspace*)ws;
  if (!w->solved) {
    g_err = "pdhg_polish: no solution in this workspace (call pdhg_solve first)";
    return PDHG_ERR_INVALID_ARG;
  }
  std::memset(res, 0, sizeof(*res));
  AdjBufs* ab = nullptr;
  int rc = adj_bufs(w, &ab);
  if (rc != PDHG_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = w->n, m = w->m;
  int64_t nA = 0, nF = 0;
  if ((rc = classify(w, ab, s, &nA, &nF)) != PDHG_OK) return rc;
  res->active_rows = nA;
  res->free_vars = nF;
  if (nA != nF) {
    res->status = PDHG_POLISH_NOT_SQUARE;
    return PDHG_OK;
  }
  // primal: x_B at its bounds, S~ x_F = rowA .* (q~ - K~ x_B), x_F = S~^T z
  k_fixed_part<<<vg(n), kBlock, 0, s>>>(ab->xfix, ab->colF, ab->xp, n);
  launch_spmv64(w->K.v64(), ab->xp, ab->Kx, w->grid_k, s);
  k_polish_rhs<<<vg(m), kBlock, 0, s>>>(w->q_s, ab->Kx, ab->rowA, ab->b, m);
  CGState sp, sd;
  if ((rc = cg_run(w, ab, 1, 1e-13, cg_max_it(nA), s, &sp)) != PDHG_OK) return rc;
  k_mspmv<<<w->grid_kt, kBlock, 0, s>>>(w->KT.v64(), ab->z, ab->rowA, ab->colF, ab->T, nullptr, -1);
  k_polish_x<<<vg(n), kBlock, 0, s>>>(ab->T, ab->colF, ab->xfix, ab->xp, n);
  // dual: S~^T y_A = c~_F, y = 0 off the active rows
  k_mask_mul<<<vg(n), kBlock, 0, s>>>(w->c_s, ab->colF, ab->r, n, nullptr);
  if ((rc = cg_run(w, ab, 0, 1e-13, cg_max_it(nA), s, &sd)) != PDHG_OK) return rc;
  k_mask_mul<<<vg(m), kBlock, 0, s>>>(ab->z, ab->rowA, ab->yp, m, nullptr);
  // optimality measures of the polished point (unscaled LP)
  launch_spmv64(w->K.v64(), ab->xp, ab->Kx, w->grid_k, s);
  launch_spmv64(w->KT.v64(), ab->yp, ab->KTy, w->grid_kt, s);
  const int gN = vg(n > m ? n : m);
  k_polish_kkt<<<gN, kBlock, 0, s>>>(ab->xp, ab->yp, ab->Kx, ab->KTy, w->q_s, w->c_s, w->l_s, w->u_s,
                                     w->Dr, w->Dc, w->iDr, w->iDc, n, m, w->m_eq, w->partials);
  double* sums = ab->Q2;  // scratch: kPolishSums doubles
  k_polish_final<<<1, kBlock, 0, s>>>(w->partials, gN, sums);
  if (x_out) k_unscale_out<<<vg(n), kBlock, 0, s>>>(w->perm_col, w->Dc, ab->xp, x_out, n);
  if (y_out) k_unscale_out<<<vg(m), kBlock, 0, s>>>(w->perm_row, w->Dr, ab->yp, y_out, m);
  double h[kPolishSums + 4];
  cudaError_t e = cudaMemcpyAsync(h, sums, sizeof(double) * kPolishSums, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h + kPolishSums, w->scalars, sizeof(double) * 4,
                                            cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_err = std::string("pdhg_polish: ") + cudaGetErrorString(e);
    return PDHG_ERR_CUDA;
  }
  const double qnorm = h[kPolishSums + 2], cnorm = h[kPolishSums + 3];
  const double P = h[2], D = h[3] + h[4];
  res->rel_p = std::sqrt(h[0]) / (1.0 + qnorm);
  res->rel_d = std::sqrt(h[1]) / (1.0 + cnorm);
  res->rel_gap = std::fabs(P - D) / (1.0 + std::fabs(P) + std::fabs(D));
  res->rel_kkt = std::max(res->rel_p, std::max(res->rel_d, res->rel_gap));
  res->primal_obj = P;
  res->dual_obj = D;
  res->bound_violation = std::sqrt(h[5]);
  res->dual_sign_violation = std::sqrt(h[6]);
  res->cg_iterations_primal = (int32_t)sp.it;
  res->cg_iterations_dual = (int32_t)sd.it;
  // relative residuals of the two systems at their last true-residual check
  res->cg_residual_primal = sp.converged && sp.resid == 0.0 ? 0.0 : std::sqrt(sp.resid / std::max(sp.rhs2, 1e-300));
  res->cg_residual_dual = sd.converged && sd.resid == 0.0 ? 0.0 : std::sqrt(sd.resid / std::max(sd.rhs2, 1e-300));
  res->status = (std::max(res->cg_residual_primal, res->cg_residual_dual) <= kPolishAccept)
                    ? PDHG_POLISH_OK
                    : PDHG_POLISH_NO_CONVERGENCE;
  return PDHG_OK;
}
