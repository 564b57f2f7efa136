// Vector-Jacobian product of the LP solution map at the last solve (the
// relaxed UC's optimal cost and dispatch as functions of the right-hand side,
// which holds the load on the balance rows, and of the cost vector).
//
// At a nondegenerate optimum the active set -- equality rows, >= rows with
// positive dual, variables held at a bound by their reduced cost -- is a
// square nonsingular system M x = rhs, M = [K_A; E_B].  Hence
//   d cost / d q = y*,  d cost / d c = x*                   (envelope theorem)
//   d (g_x^T x*) / d q_A = lambda_A,  M^T lambda = g_x,  d (g_x^T x*) / d c = 0
// and on the variables F not at a bound M^T lambda = g_x reduces to the square
// system K_{A,F}^T lambda_A = g_F.  In the rescaled space K~ = Dr K Dc this is
// K~_{A,F}^T mu = Dc g_F with lambda = Dr mu, solved by conjugate gradients on
// the normal equations (K~_{A,F} K~_{A,F}^T) mu = K~_{A,F} Dc g_F with the
// FP64 sliced-ELL products of the workspace and masks for A and F.
#include <cmath>
#include <string>
#include <vector>

#include "internal.cuh"

namespace ucpdhg {
namespace {

int vg(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  if (g > 152 * 8) g = 152 * 8;
  return (int)(g < 1 ? 1 : g);
}

// Active-set masks in the rescaled space from x~*, y~*, s~ = K~x~* - q~ and
// lambda~ = c~ - K~^T y~*: a >= row is active iff y~_i > s~_i; a variable is at
// a bound iff its reduced cost outweighs its distance to that bound (or l = u).
__global__ void k_classify(const double* __restrict__ x, const double* __restrict__ y,
                           const double* __restrict__ Kx, const double* __restrict__ KTy,
                           const double* __restrict__ q, const double* __restrict__ c,
                           const double* __restrict__ l, const double* __restrict__ u, int64_t n,
                           int64_t m, int64_t m_eq, double* rowA, double* colF, double* partials) {
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
      bool fixed = false;
      if (isfinite(lo) && isfinite(up) && lo == up) fixed = true;
      if (isfinite(lo) && lam > 0.0 && lam > x[t] - lo) fixed = true;
      if (isfinite(up) && lam < 0.0 && -lam > up - x[t]) fixed = true;
      const double f = fixed ? 0.0 : 1.0;
      colF[t] = f;
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

__global__ void k_mask_mul(const double* __restrict__ a, const double* __restrict__ mask, double* out,
                           int64_t n, double scale_if_nonnull, const double* __restrict__ scale) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    double v = a[t] * mask[t];
    if (scale) v *= scale[t];
    out[t] = v * scale_if_nonnull;
  }
}

// z = alpha * a + beta * b (elementwise)
__global__ void k_axpby(double alpha, const double* __restrict__ a, double beta,
                        const double* __restrict__ b, double* z, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    z[t] = alpha * a[t] + beta * b[t];
}

// deterministic dot products: per-block partials of a.b (and optionally c.d)
__global__ void k_dot2(const double* __restrict__ a, const double* __restrict__ b,
                       const double* __restrict__ c, const double* __restrict__ d, int64_t n,
                       double* partials) {
  double v[2] = {0.0, 0.0};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    v[0] += a[t] * b[t];
    if (c) v[1] += c[t] * d[t];
  }
  __shared__ double sm[kWarps * 2];
  block_sum<2>(v, sm);
  if (threadIdx.x == 0) {
    partials[blockIdx.x * 2 + 0] = v[0];
    partials[blockIdx.x * 2 + 1] = v[1];
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

}  // namespace
}  // namespace ucpdhg

using namespace ucpdhg;

namespace ucpdhg {

// FP64 scratch of the adjoint, allocated at the first pdhg_backward call.
struct AdjBufs {
  double *Kx = nullptr, *KTy = nullptr, *rowA = nullptr, *colF = nullptr, *mu = nullptr;
  double *R = nullptr, *P = nullptr, *Q = nullptr, *T = nullptr, *r = nullptr, *tn = nullptr,
         *tm = nullptr;
  std::vector<void*> allocs;
};

void release_adjoint(Workspace* w) {
  AdjBufs* ab = (AdjBufs*)w->adjoint;
  if (!ab) return;
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
  double** vm[] = {&ab->Kx, &ab->rowA, &ab->mu, &ab->R, &ab->P, &ab->Q, &ab->tm};
  double** vn[] = {&ab->KTy, &ab->colF, &ab->T, &ab->r, &ab->tn};
  for (double** p : vm) {
    void* q = nullptr;
    if (cudaMalloc(&q, sizeof(double) * (m + 2)) != cudaSuccess) {
      for (void* a : ab->allocs) cudaFree(a);
      delete ab;
      g_err = "pdhg_backward: device allocation failed";
      return PDHG_ERR_NOMEM;
    }
    ab->allocs.push_back(q);
    *p = (double*)q;
  }
  for (double** p : vn) {
    void* q = nullptr;
    if (cudaMalloc(&q, sizeof(double) * (n + 2)) != cudaSuccess) {
      for (void* a : ab->allocs) cudaFree(a);
      delete ab;
      g_err = "pdhg_backward: device allocation failed";
      return PDHG_ERR_NOMEM;
    }
    ab->allocs.push_back(q);
    *p = (double*)q;
  }
  w->adjoint = ab;
  *out = ab;
  return PDHG_OK;
}

}  // namespace ucpdhg

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
  launch_spmv64(w->K.v64(), w->x_star, ab->Kx, w->grid_k, s);
  launch_spmv64(w->KT.v64(), w->y_star, ab->KTy, w->grid_kt, s);
  const int64_t N = n > m ? n : m;
  const int gN = vg(N);
  double* part = w->partials;
  double* scal = w->scalars + 8;  // [8..15] scratch scalars
  k_classify<<<gN, kBlock, 0, s>>>(w->x_star, w->y_star, ab->Kx, ab->KTy, w->q_s, w->c_s, w->l_s,
                                   w->u_s, n, m, w->m_eq, ab->rowA, ab->colF, part);
  k_final2<<<1, kBlock, 0, s>>>(part, gN, scal);
  double hs[2];
  if (cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    g_err = std::string("pdhg_backward: ") + cudaGetErrorString(cudaGetLastError());
    return PDHG_ERR_CUDA;
  }
  const int64_t nA = (int64_t)llround(hs[0]), nF = (int64_t)llround(hs[1]);
  const bool has_gx = g_x != nullptr;
  if (has_gx && nA != nF) {
    g_err = "pdhg_backward: the active set is not square (" + std::to_string(nA) + " active rows, " +
            std::to_string(nF) + " free variables): the LP is degenerate at this solution";
    return PDHG_ERR_NUMERIC;
  }
  double* mu = ab->mu;
  if (has_gx) {
    double *R = ab->R, *P = ab->P, *Q = ab->Q, *T = ab->T, *r = ab->r, *tn = ab->tn, *tm = ab->tm;
    const double *rowA = ab->rowA, *colF = ab->colF;
    // r = Dc g_F (internal order)
    launch_gather_perm(w->perm_col, g_x, r, n, s);
    k_mask_mul<<<vg(n), kBlock, 0, s>>>(r, colF, r, n, 1.0, w->Dc);
    auto applyS = [&](const double* in_n, double* out_m) {  // A .* (K~ (F .* in))
      k_mask_mul<<<vg(n), kBlock, 0, s>>>(in_n, colF, tn, n, 1.0, nullptr);
      launch_spmv64(w->K.v64(), tn, out_m, w->grid_k, s);
      k_mask_mul<<<vg(m), kBlock, 0, s>>>(out_m, rowA, out_m, m, 1.0, nullptr);
    };
    auto applyST = [&](const double* in_m, double* out_n) {  // F .* (K~^T (A .* in))
      k_mask_mul<<<vg(m), kBlock, 0, s>>>(in_m, rowA, tm, m, 1.0, nullptr);
      launch_spmv64(w->KT.v64(), tm, out_n, w->grid_kt, s);
      k_mask_mul<<<vg(n), kBlock, 0, s>>>(out_n, colF, out_n, n, 1.0, nullptr);
    };
    auto dot = [&](const double* a, const double* bb, int64_t len, double* outh) -> int {
      const int g = vg(len);
      k_dot2<<<g, kBlock, 0, s>>>(a, bb, nullptr, nullptr, len, part);
      k_final2<<<1, kBlock, 0, s>>>(part, g, scal);
      double v[2];
      if (cudaMemcpyAsync(v, scal, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return PDHG_ERR_CUDA;
      *outh = v[0];
      return PDHG_OK;
    };
    // CG on (S S^T) mu = S r, S = K~_{A,F}
    cudaMemsetAsync(mu, 0, sizeof(double) * m, s);
    applyS(r, R);
    cudaMemcpyAsync(P, R, sizeof(double) * m, cudaMemcpyDeviceToDevice, s);
    double rr = 0.0, gg = 0.0;
    if ((rc = dot(R, R, m, &rr)) != PDHG_OK) return rc;
    if ((rc = dot(r, r, n, &gg)) != PDHG_OK) return rc;
    const double rr0 = rr;
    const double target = 1e-26 * (gg > 0.0 ? gg : 1.0);  // ||S^T mu - r|| <= 1e-13 ||r||
    const int64_t max_it = std::min<int64_t>(20 * (nA + 10), 200000);
    for (int64_t it = 0; it < max_it && rr > 0.0; ++it) {
      applyST(P, T);
      applyS(T, Q);
      double pq = 0.0;
      if ((rc = dot(P, Q, m, &pq)) != PDHG_OK) return rc;
      if (!(pq > 0.0)) break;
      const double alpha = rr / pq;
      k_axpby<<<vg(m), kBlock, 0, s>>>(1.0, mu, alpha, P, mu, m);
      k_axpby<<<vg(m), kBlock, 0, s>>>(1.0, R, -alpha, Q, R, m);
      double rr_new = 0.0;
      if ((rc = dot(R, R, m, &rr_new)) != PDHG_OK) return rc;
      if ((it & 15) == 15 || rr_new <= 1e-32 * rr0) {
        applyST(mu, T);
        k_axpby<<<vg(n), kBlock, 0, s>>>(1.0, T, -1.0, r, T, n);
        double e = 0.0;
        if ((rc = dot(T, T, n, &e)) != PDHG_OK) return rc;
        if (e <= target) break;
      }
      const double beta = rr_new / rr;
      rr = rr_new;
      k_axpby<<<vg(m), kBlock, 0, s>>>(1.0, R, beta, P, P, m);
    }
  }
  k_backward_out<<<gN, kBlock, 0, s>>>(w->perm_row, w->perm_col, w->Dr, w->Dc, w->y_star, w->x_star,
                                       mu, ab->rowA, g_cost, has_gx ? 1 : 0, grad_q, grad_c, n, m);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_err = std::string("pdhg_backward: ") + cudaGetErrorString(e);
    return PDHG_ERR_CUDA;
  }
  return PDHG_OK;
}
