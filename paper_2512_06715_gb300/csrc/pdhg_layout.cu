// Internal layout (length-sorted orderings, sliced ELL) and the rescaling pass.
//
// Rows of K are reordered by decreasing length inside the equality block and
// inside the inequality block (stable), columns by decreasing column count, so
// that each 32-row slice holds rows of (nearly) equal length and padding stays
// negligible on the UC sparsity (rows of 2 to ~25 entries).  K and K^T are both
// kept in this layout; every vector the iterations touch lives in the internal
// order, so no permutation is applied inside the PDHG loop.
//
// Rescaling (the PDLP preconditioning of Applegate et al., cited in Sec. II.E):
// Ruiz l_inf passes r_i = 1/sqrt(max_j |K~_ij|), s_j = 1/sqrt(max_i |K~_ij|),
// then one Pock-Chambolle alpha = 1 pass with l_1 sums, both factors of a pass
// taken from the same K~.  The factors accumulate in Dr, Dc and the matrix is
// formed once at the end as K~_ij = K_ij (Dr_i Dc_j).
#include <algorithm>
#include <numeric>

#include "internal.cuh"

namespace ucpdhg {

int build_layout(int64_t n, int64_t m, int64_t m_eq, const std::vector<int64_t>& rp,
                 const std::vector<int32_t>& col, HostLayout* L, std::string* err) {
  std::vector<int32_t> rlen(m), clen(n, 0);
  for (int64_t i = 0; i < m; ++i) rlen[i] = (int32_t)(rp[i + 1] - rp[i]);
  for (size_t e = 0; e < col.size(); ++e) {
    if (col[e] < 0 || col[e] >= n) {
      *err = "column index out of range in CSR";
      return PDHG_ERR_INVALID_ARG;
    }
    clen[col[e]]++;
  }
  L->perm_row.resize(m);
  std::iota(L->perm_row.begin(), L->perm_row.end(), 0);
  auto by_rlen = [&](int32_t a, int32_t b) { return rlen[a] > rlen[b]; };
  std::stable_sort(L->perm_row.begin(), L->perm_row.begin() + m_eq, by_rlen);
  std::stable_sort(L->perm_row.begin() + m_eq, L->perm_row.end(), by_rlen);
  L->perm_col.resize(n);
  std::iota(L->perm_col.begin(), L->perm_col.end(), 0);
  std::stable_sort(L->perm_col.begin(), L->perm_col.end(),
                   [&](int32_t a, int32_t b) { return clen[a] > clen[b]; });
  std::vector<int32_t> inv_row(m), inv_col(n);
  for (int64_t i = 0; i < m; ++i) inv_row[L->perm_row[i]] = (int32_t)i;
  for (int64_t j = 0; j < n; ++j) inv_col[L->perm_col[j]] = (int32_t)j;

  // ---- K in sliced ELL over internal rows ----
  const int64_t ks = (m + kSlice - 1) / kSlice;
  L->k_off.assign(ks + 1, 0);
  int64_t tot = 0;
  for (int64_t s = 0; s < ks; ++s) {
    int32_t w = 0;
    for (int lane = 0; lane < kSlice; ++lane) {
      int64_t i = s * kSlice + lane;
      if (i < m) w = std::max(w, rlen[L->perm_row[i]]);
    }
    tot += (int64_t)w * kSlice;
    if (tot >= (int64_t)1 << 31) {
      *err = "padded nnz of K exceeds 2^31";
      return PDHG_ERR_UNSUPPORTED;
    }
    L->k_off[s + 1] = (int32_t)tot;
  }
  L->k_col.assign(tot, 0);
  L->k_src.assign(tot, -1);
  for (int64_t s = 0; s < ks; ++s) {
    for (int lane = 0; lane < kSlice; ++lane) {
      int64_t i = s * kSlice + lane;
      if (i >= m) continue;
      int32_t o = L->perm_row[i];
      for (int32_t k = 0; k < rlen[o]; ++k) {
        int64_t e = rp[o] + k;
        int64_t slot = L->k_off[s] + (int64_t)k * kSlice + lane;
        L->k_col[slot] = inv_col[col[e]];
        L->k_src[slot] = (int32_t)e;
      }
    }
  }

  // ---- K^T in sliced ELL over internal columns (entries by ascending row) ----
  std::vector<int64_t> cptr(n + 1, 0);
  for (int64_t j = 0; j < n; ++j) cptr[j + 1] = cptr[j] + clen[j];
  std::vector<int32_t> crow(col.size()), csrc(col.size());
  {
    std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
    for (int64_t i = 0; i < m; ++i)
      for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        int64_t pos = fill[col[e]]++;
        crow[pos] = (int32_t)i;
        csrc[pos] = (int32_t)e;
      }
  }
  const int64_t ts = (n + kSlice - 1) / kSlice;
  L->t_off.assign(ts + 1, 0);
  tot = 0;
  for (int64_t s = 0; s < ts; ++s) {
    int32_t w = 0;
    for (int lane = 0; lane < kSlice; ++lane) {
      int64_t j = s * kSlice + lane;
      if (j < n) w = std::max(w, clen[L->perm_col[j]]);
    }
    tot += (int64_t)w * kSlice;
    if (tot >= (int64_t)1 << 31) {
      *err = "padded nnz of K^T exceeds 2^31";
      return PDHG_ERR_UNSUPPORTED;
    }
    L->t_off[s + 1] = (int32_t)tot;
  }
  L->t_col.assign(tot, 0);
  L->t_src.assign(tot, -1);
  for (int64_t s = 0; s < ts; ++s) {
    for (int lane = 0; lane < kSlice; ++lane) {
      int64_t j = s * kSlice + lane;
      if (j >= n) continue;
      int32_t o = L->perm_col[j];
      for (int64_t k = 0; k < clen[o]; ++k) {
        int64_t slot = L->t_off[s] + k * kSlice + lane;
        L->t_col[slot] = inv_row[crow[cptr[o] + k]];
        L->t_src[slot] = csrc[cptr[o] + k];
      }
    }
  }
  return PDHG_OK;
}

bool build_chunks(const std::vector<int32_t>& off, std::vector<int32_t>* chunks, int max_entries,
                  int max_slices) {
  chunks->clear();
  const int32_t ns = (int32_t)off.size() - 1;
  chunks->push_back(0);
  int32_t s0 = 0;
  for (int32_t s = 0; s < ns; ++s) {
    if (off[s + 1] - off[s] > max_entries) {
      chunks->clear();
      return false;
    }
    if (off[s + 1] - off[s0] > max_entries || s + 1 - s0 > max_slices) {
      chunks->push_back(s);
      s0 = s;
    }
  }
  if (ns > 0) chunks->push_back(ns);
  return true;
}

// ---------------------------------------------------------------------------
// kernels of the preparation pass

__global__ void k_load_vals(const int32_t* __restrict__ src, const double* __restrict__ csr,
                            double* __restrict__ out, int64_t nnz_pad) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz_pad;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t e = src[t];
    out[t] = (e >= 0) ? csr[e] : 0.0;
  }
}

__global__ void k_load_vecs(const int32_t* __restrict__ perm_col, const int32_t* __restrict__ perm_row,
                            const double* c, const double* l, const double* u, const double* q,
                            double* c_s, double* l_s, double* u_s, double* q_s, double* Dr,
                            double* Dc, int64_t n, int64_t m) {
  int64_t N = n > m ? n : m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < n) {
      int32_t o = perm_col[t];
      c_s[t] = c[o];
      l_s[t] = l[o];
      u_s[t] = u[o];
      Dc[t] = 1.0;
    }
    if (t < m) {
      q_s[t] = q[perm_row[t]];
      Dr[t] = 1.0;
    }
  }
}

// Per internal row of A: max (mode 0) or sum (mode 1) of |A_ij| drow_i dcol_j,
// turned into the factor 1/sqrt(stat) (1 for an empty row).
__global__ void k_row_factor(SellView<double> A, const double* __restrict__ drow,
                             const double* __restrict__ dcol, int mode, double* __restrict__ fac) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int s = gw; s < A.nslices; s += nw) {
    const int o0 = A.off[s], w = (A.off[s + 1] - o0) >> 5;
    const int r = s * kSlice + lane;
    if (r >= A.rows) continue;
    const double dr = drow[r];
    double stat = 0.0;
    for (int k = 0; k < w; ++k) {
      int slot = o0 + k * kSlice + lane;
      double a = fabs(A.val[slot]) * dr * dcol[A.col[slot]];
      stat = mode ? stat + a : fmax(stat, a);
    }
    fac[r] = stat > 0.0 ? 1.0 / sqrt(stat) : 1.0;
  }
}

__global__ void k_mul_inplace(double* a, const double* f, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    a[t] *= f[t];
}

// K~ = K (drow_i dcol_j); the product of the two factors is formed first so that
// K and K^T get bit-identical values.
__global__ void k_scale_vals(SellView<double> A, double* val, const double* __restrict__ drow,
                             const double* __restrict__ dcol) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int s = gw; s < A.nslices; s += nw) {
    const int o0 = A.off[s], w = (A.off[s + 1] - o0) >> 5;
    const int r = s * kSlice + lane;
    if (r >= A.rows) continue;
    const double dr = drow[r];
    for (int k = 0; k < w; ++k) {
      int slot = o0 + k * kSlice + lane;
      val[slot] = val[slot] * (dr * dcol[A.col[slot]]);
    }
  }
}

// Scaled vectors plus the norms ||c||, ||q|| (unscaled) and ||c~||, ||q~||, and
// max |K~| as per-block partials (deterministic final pass in k_prepare_final).
__global__ void k_scale_vecs(double* c_s, double* l_s, double* u_s, double* q_s,
                             const double* __restrict__ Dr, const double* __restrict__ Dc, int64_t n,
                             int64_t m, double* partials, double* iDr, double* iDc) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  int64_t N = n > m ? n : m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < n) {
      double c = c_s[t], d = Dc[t];
      v[0] += c * c;
      double cs = d * c;
      c_s[t] = cs;
      v[2] += cs * cs;
      iDc[t] = 1.0 / d;
      l_s[t] = l_s[t] / d;
      u_s[t] = u_s[t] / d;
    }
    if (t < m) {
      double q = q_s[t];
      v[1] += q * q;
      iDr[t] = 1.0 / Dr[t];
      double qs = Dr[t] * q;
      q_s[t] = qs;
      v[3] += qs * qs;
    }
  }
  __shared__ double smem[kWarps * 4];
  block_sum<4>(v, smem);
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) partials[blockIdx.x * 4 + k] = v[k];
}

__global__ void k_absmax_partial(const double* __restrict__ val, int64_t nnz_pad, double* partials) {
  double mx = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz_pad;
       t += (int64_t)gridDim.x * blockDim.x)
    mx = fmax(mx, fabs(val[t]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  __shared__ double sm[kWarps];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < kWarps; ++w) r = fmax(r, sm[w]);
    partials[blockIdx.x] = r;
  }
}

// scalars[0] = eta0 = 1/max|K~|, [1] = omega0, [2] = ||q||, [3] = ||c||,
// [4] = ||c~||, [5] = ||q~||.
__global__ void k_prepare_final(const double* vec_partials, int nb_vec, const double* max_partials,
                                int nb_max, double* scalars) {
  double v[4];
  final_sum<4>(vec_partials, nb_vec, v);
  __shared__ double mx_s[kBlock];
  double mx = 0.0;
  for (int b = threadIdx.x; b < nb_max; b += blockDim.x) mx = fmax(mx, max_partials[b]);
  mx_s[threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) r = fmax(r, mx_s[t]);
    double cn = sqrt(v[2]), qn = sqrt(v[3]);
    scalars[0] = r > 0.0 ? 1.0 / r : 1.0;
    scalars[1] = (cn > 1e-10 && qn > 1e-10) ? cn / qn : 1.0;
    scalars[2] = sqrt(v[1]);
    scalars[3] = sqrt(v[0]);
    scalars[4] = cn;
    scalars[5] = qn;
  }
}

__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (float)in[t];
}

__global__ void k_to_f64(const float* __restrict__ in, double* __restrict__ out, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (double)in[t];
}

template <class T>
__global__ void __launch_bounds__(kBlock) k_spmv(SellView<T> A, const T* __restrict__ x,
                                                 T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int s = gw; s < A.nslices; s += nw) {
    const int o0 = A.off[s], w = (A.off[s + 1] - o0) >> 5;
    const int32_t* cp = A.col + o0 + lane;
    const T* vp = A.val + o0 + lane;
    T acc = 0;
    for (int k = 0; k < w; ++k) acc += __ldg(vp + k * kSlice) * __ldg(x + __ldg(cp + k * kSlice));
    const int r = s * kSlice + lane;
    if (r < A.rows) y[r] = acc;
  }
}

__global__ void k_gather_perm(const int32_t* __restrict__ perm, const double* __restrict__ in,
                              double* __restrict__ out, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = in[perm[t]];
}

__global__ void k_scatter_perm(const int32_t* __restrict__ perm, const double* __restrict__ in,
                               double* __restrict__ out, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    out[perm[t]] = in[t];
}

// ---------------------------------------------------------------------------
// launchers

static int vec_grid(int64_t n, int sms) {
  int64_t g = (n + kBlock - 1) / kBlock;
  int64_t cap = (int64_t)sms * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

void launch_spmv64(const SellView<double>& A, const double* x, double* y, int grid, cudaStream_t s) {
  k_spmv<double><<<grid, kBlock, 0, s>>>(A, x, y);
}
void launch_spmv32(const SellView<float>& A, const float* x, float* y, int grid, cudaStream_t s) {
  k_spmv<float><<<grid, kBlock, 0, s>>>(A, x, y);
}
void launch_gather_perm(const int32_t* perm, const double* in, double* out, int64_t n,
                        cudaStream_t s) {
  k_gather_perm<<<vec_grid(n, 152), kBlock, 0, s>>>(perm, in, out, n);
}
void launch_scatter_perm(const int32_t* perm, const double* in, double* out, int64_t n,
                         cudaStream_t s) {
  k_scatter_perm<<<vec_grid(n, 152), kBlock, 0, s>>>(perm, in, out, n);
}
void launch_to_f32(const double* in, float* out, int64_t n, cudaStream_t s) {
  k_to_f32<<<vec_grid(n, 152), kBlock, 0, s>>>(in, out, n);
}
void launch_to_f64(const float* in, double* out, int64_t n, cudaStream_t s) {
  k_to_f64<<<vec_grid(n, 152), kBlock, 0, s>>>(in, out, n);
}

void launch_prepare(Workspace* w, cudaStream_t s) {
  const int sms = w->num_sms;
  k_load_vals<<<vec_grid(w->K.nnz_pad, sms), kBlock, 0, s>>>(w->K.src, w->prob.val, w->K.val64,
                                                              w->K.nnz_pad);
  k_load_vals<<<vec_grid(w->KT.nnz_pad, sms), kBlock, 0, s>>>(w->KT.src, w->prob.val, w->KT.val64,
                                                               w->KT.nnz_pad);
  const int64_t N = w->n > w->m ? w->n : w->m;
  k_load_vecs<<<vec_grid(N, sms), kBlock, 0, s>>>(w->perm_col, w->perm_row, w->prob.c, w->prob.l,
                                                  w->prob.u, w->prob.q, w->c_s, w->l_s, w->u_s,
                                                  w->q_s, w->Dr, w->Dc, w->n, w->m);
  const int passes = w->opts.ruiz_iters + (w->opts.pock_chambolle ? 1 : 0);
  for (int p = 0; p < passes; ++p) {
    const int mode = (p >= w->opts.ruiz_iters) ? 1 : 0;
    k_row_factor<<<w->grid_k, kBlock, 0, s>>>(w->K.v64(), w->Dr, w->Dc, mode, w->fac_r);
    k_row_factor<<<w->grid_kt, kBlock, 0, s>>>(w->KT.v64(), w->Dc, w->Dr, mode, w->fac_c);
    k_mul_inplace<<<vec_grid(w->m, sms), kBlock, 0, s>>>(w->Dr, w->fac_r, w->m);
    k_mul_inplace<<<vec_grid(w->n, sms), kBlock, 0, s>>>(w->Dc, w->fac_c, w->n);
  }
  k_scale_vals<<<w->grid_k, kBlock, 0, s>>>(w->K.v64(), w->K.val64, w->Dr, w->Dc);
  k_scale_vals<<<w->grid_kt, kBlock, 0, s>>>(w->KT.v64(), w->KT.val64, w->Dc, w->Dr);
  const int gv = vec_grid(N, sms);
  double* part_vec = w->partials;
  double* part_max = w->partials + (size_t)kMaxBlocks * kRegionStride;
  k_scale_vecs<<<gv, kBlock, 0, s>>>(w->c_s, w->l_s, w->u_s, w->q_s, w->Dr, w->Dc, w->n, w->m,
                                     part_vec, w->iDr, w->iDc);
  const int gm = vec_grid(w->K.nnz_pad, sms);
  k_absmax_partial<<<gm, kBlock, 0, s>>>(w->K.val64, w->K.nnz_pad, part_max);
  k_prepare_final<<<1, kBlock, 0, s>>>(part_vec, gv, part_max, gm, w->scalars);
  w->values_f32 = false;
}

}  // namespace ucpdhg
