// Synthetic DC unit-commitment LP relaxation generator (host only, no solver
// arithmetic).  The paper's UC model (Sec. II.A) is the GO-Challenge-3
// formulation whose document and data are not available; this builds a seeded
// DC-UC relaxation with the paper's network sizes (Sec. II.B, Table I) and the
// row families the paper lists for its UC module: nodal balance, DC line
// limits, output limits tied to commitment, ramping, start-up/shut-down logic
// and minimum up/down times.
//
// Random streams: SplitMix64 (Steele, Lea, Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014), one stream per component,
// started at seed ^ (component * golden-gamma).  Uniforms take the top 53 bits.
#include "../../include/uc_lp.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_set>
#include <vector>

namespace {

thread_local std::string g_err;

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

struct SplitMix64 {
  uint64_t s;
  SplitMix64(uint64_t seed, uint64_t component) : s(seed ^ (component * kGamma)) {}
  uint64_t next() {
    uint64_t z = (s += kGamma);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
  double uniform(double a, double b) { return a + (b - a) * uniform(); }
  // Box-Muller, one normal per call (the second is discarded).
  double normal() {
    double u1 = uniform();
    double u2 = uniform();
    if (u1 < 1e-300) u1 = 1e-300;
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
  int64_t below(int64_t n) { return (int64_t)(uniform() * (double)n); }
};

enum Stream : uint64_t {
  kStreamChords = 1,
  kStreamReactance = 2,
  kStreamLineLimit = 3,
  kStreamGenBus = 4,
  kStreamGenParams = 5,
  kStreamLoadWeight = 6,
};

// Conjugate gradient with Jacobi preconditioning on the Laplacian of the
// network grounded at bus 0 (row and column 0 removed).  Returns theta with
// theta[0] = 0.  The Laplacian is symmetric positive definite once grounded on
// a connected network.
std::vector<double> grounded_laplacian_solve(int N, const std::vector<int>& from,
                                             const std::vector<int>& to,
                                             const std::vector<double>& b_line,
                                             const std::vector<double>& inj) {
  std::vector<double> theta(N, 0.0);
  if (N <= 1) return theta;
  std::vector<double> diag(N, 0.0);
  for (size_t l = 0; l < from.size(); ++l) {
    diag[from[l]] += b_line[l];
    diag[to[l]] += b_line[l];
  }
  auto apply = [&](const std::vector<double>& v, std::vector<double>& out) {
    std::fill(out.begin(), out.end(), 0.0);
    for (size_t l = 0; l < from.size(); ++l) {
      double f = b_line[l] * (v[from[l]] - v[to[l]]);
      out[from[l]] += f;
      out[to[l]] -= f;
    }
    out[0] = 0.0;  // grounded row
  };
  std::vector<double> r(inj), z(N), p(N), Ap(N);
  r[0] = 0.0;
  double rnorm0 = 0.0;
  for (int i = 0; i < N; ++i) rnorm0 += r[i] * r[i];
  rnorm0 = std::sqrt(rnorm0);
  if (rnorm0 == 0.0) return theta;
  for (int i = 0; i < N; ++i) z[i] = (i == 0) ? 0.0 : r[i] / diag[i];
  p = z;
  double rz = 0.0;
  for (int i = 0; i < N; ++i) rz += r[i] * z[i];
  const int max_it = 50 * N + 1000;
  for (int it = 0; it < max_it; ++it) {
    apply(p, Ap);
    double pAp = 0.0;
    for (int i = 0; i < N; ++i) pAp += p[i] * Ap[i];
    if (!(pAp > 0.0)) break;
    double alpha = rz / pAp;
    double rn = 0.0;
    for (int i = 1; i < N; ++i) {
      theta[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
      rn += r[i] * r[i];
    }
    if (std::sqrt(rn) <= 1e-14 * rnorm0) break;
    for (int i = 1; i < N; ++i) z[i] = r[i] / diag[i];
    double rz_new = 0.0;
    for (int i = 1; i < N; ++i) rz_new += r[i] * z[i];
    double beta = rz_new / rz;
    rz = rz_new;
    for (int i = 1; i < N; ++i) p[i] = z[i] + beta * p[i];
    p[0] = 0.0;
  }
  theta[0] = 0.0;
  return theta;
}

struct Builder {
  // COO rows, assembled row by row; each row merged and sorted on close.
  std::vector<int64_t> row_ptr{0};
  std::vector<int32_t> col;
  std::vector<double> val;
  std::vector<double> q;
  std::vector<int32_t> row_kind;
  std::vector<std::pair<int32_t, double>> cur;

  void add(int64_t j, double a) { cur.emplace_back((int32_t)j, a); }
  void close(double rhs, int kind) {
    std::sort(cur.begin(), cur.end(),
              [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
                return a.first < b.first;
              });
    size_t k = 0;
    while (k < cur.size()) {
      int32_t j = cur[k].first;
      double a = 0.0;
      while (k < cur.size() && cur[k].first == j) a += cur[k++].second;
      if (a != 0.0) {
        col.push_back(j);
        val.push_back(a);
      }
    }
    cur.clear();
    row_ptr.push_back((int64_t)col.size());
    q.push_back(rhs);
    row_kind.push_back(kind);
  }
};

template <class T>
T* dup(const std::vector<T>& v) {
  T* p = (T*)std::malloc(sizeof(T) * (v.empty() ? 1 : v.size()));
  if (p && !v.empty()) std::memcpy(p, v.data(), sizeof(T) * v.size());
  return p;
}

}  // namespace

extern "C" const char* uc_lp_last_error(void) { return g_err.c_str(); }

extern "C" void uc_lp_free(uc_lp* lp) {
  if (!lp) return;
  void* ptrs[] = {lp->row_ptr, lp->col, lp->val, lp->c, lp->l, lp->u, lp->q, lp->var_kind,
                  lp->row_kind, lp->idx_p, lp->idx_u, lp->idx_v, lp->idx_w, lp->idx_theta,
                  lp->row_balance, lp->load, lp->gen_bus, lp->line_from, lp->line_to,
                  lp->gen_pmax, lp->gen_cost, lp->gen_noload, lp->gen_min_up, lp->gen_min_dn};
  for (void* p : ptrs) std::free(p);
  std::free(lp);
}

extern "C" int uc_lp_build(const uc_params* prm, uc_lp** out) {
  g_err.clear();
  if (!out) {
    g_err = "uc_lp_build: out is NULL";
    return UC_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (!prm) {
    g_err = "uc_lp_build: params is NULL";
    return UC_ERR_INVALID_ARG;
  }
  const int N = prm->n_bus, L = prm->n_line, G = prm->n_gen, T = prm->n_periods;
  if (N < 1 || G < 1 || T < 1 || L < 0) {
    g_err = "uc_lp_build: n_bus, n_gen, n_periods must be >= 1 and n_line >= 0";
    return UC_ERR_INVALID_ARG;
  }
  if ((N == 1 && L != 0) || (N == 2 && L != 1) || (N >= 3 && L < N)) {
    g_err = "uc_lp_build: n_line must be 0 for 1 bus, 1 for 2 buses, >= n_bus otherwise";
    return UC_ERR_INVALID_ARG;
  }
  if (N >= 3 && (int64_t)L > (int64_t)N * (N - 1) / 2) {
    g_err = "uc_lp_build: more lines than bus pairs";
    return UC_ERR_INVALID_ARG;
  }
  if (!(prm->horizon_hours > 0.0) || !(prm->s_base > 0.0) || !(prm->peak_frac > 0.0)) {
    g_err = "uc_lp_build: horizon_hours, s_base, peak_frac must be > 0";
    return UC_ERR_INVALID_ARG;
  }
  const uint64_t seed = prm->seed;
  const double S = prm->s_base;
  const double dt = prm->horizon_hours / T;
  const bool slack = prm->with_slack != 0;

  // ---- network: ring + distinct random chords -------------------------------
  std::vector<int> from, to;
  std::unordered_set<uint64_t> edges;
  auto key = [](int a, int b) {
    if (a > b) std::swap(a, b);
    return ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
  };
  if (N == 2) {
    from.push_back(0);
    to.push_back(1);
  } else if (N >= 3) {
    for (int i = 0; i < N; ++i) {
      from.push_back(i);
      to.push_back((i + 1) % N);
      edges.insert(key(i, (i + 1) % N));
    }
    SplitMix64 rc(seed, kStreamChords);
    while ((int)from.size() < L) {
      int a = (int)rc.below(N), b = (int)rc.below(N);
      if (a == b || edges.count(key(a, b))) continue;
      edges.insert(key(a, b));
      from.push_back(a);
      to.push_back(b);
    }
  }
  std::vector<double> x_line(L), b_line(L);
  {
    SplitMix64 rx(seed, kStreamReactance);
    for (int l = 0; l < L; ++l) {
      x_line[l] = rx.uniform(0.01, 0.1);
      b_line[l] = S / x_line[l];
    }
  }

  // ---- generators ------------------------------------------------------------
  std::vector<int32_t> gen_bus(G), ut(G), dtn(G);
  std::vector<double> cost(G), noload(G), su(G), pmax(G), pmin(G), ramp(G), sur(G);
  {
    SplitMix64 rb(seed, kStreamGenBus);
    for (int g = 0; g < G; ++g) gen_bus[g] = (int32_t)rb.below(N);
    SplitMix64 rg(seed, kStreamGenParams);
    for (int g = 0; g < G; ++g) {
      cost[g] = rg.uniform(10.0, 80.0);
      noload[g] = rg.uniform(100.0, 1000.0);
      su[g] = rg.uniform(500.0, 5000.0);
      pmax[g] = rg.uniform(20.0, 400.0);
      int h_up = 2 + (int)rg.below(5);
      int h_dn = 2 + (int)rg.below(5);
      pmin[g] = 0.3 * pmax[g];
      ramp[g] = 0.5 * pmax[g] * dt;
      sur[g] = std::max(pmin[g], ramp[g]);
      ut[g] = std::max(1, (int)std::ceil(h_up / dt - 1e-9));
      dtn[g] = std::max(1, (int)std::ceil(h_dn / dt - 1e-9));
    }
  }
  double sum_pmax = 0.0;
  for (int g = 0; g < G; ++g) sum_pmax += pmax[g];

  // ---- loads -----------------------------------------------------------------
  std::vector<double> wbus(N);
  {
    SplitMix64 rw(seed, kStreamLoadWeight);
    for (int b = 0; b < N; ++b) wbus[b] = std::exp(0.5 * rw.normal());
  }
  double sum_w = 0.0;
  for (int b = 0; b < N; ++b) sum_w += wbus[b];
  std::vector<double> shape(T), Dt(T);
  double smax = 0.0;
  for (int t = 0; t < T; ++t) {
    double h = std::fmod((t + 0.5) * dt, 24.0);
    shape[t] = 0.6 + 0.25 * std::exp(-(h - 9.0) * (h - 9.0) / 4.5) +
               0.4 * std::exp(-(h - 19.0) * (h - 19.0) / 8.0);
    smax = std::max(smax, shape[t]);
  }
  double d_peak = 0.0, d_sum = 0.0;
  for (int t = 0; t < T; ++t) {
    Dt[t] = prm->peak_frac * sum_pmax * shape[t] / smax;
    d_peak = std::max(d_peak, Dt[t]);
    d_sum += Dt[t];
  }
  std::vector<double> load((size_t)T * N);
  for (int t = 0; t < T; ++t)
    for (int b = 0; b < N; ++b) load[(size_t)t * N + b] = Dt[t] * wbus[b] / sum_w;
  const double d_mean = d_sum / ((double)T * N);

  // ---- line limits with a DC-flow floor ---------------------------------------
  // Injection of the proportional all-on dispatch per unit of system load.
  std::vector<double> inj(N, 0.0);
  for (int g = 0; g < G; ++g) inj[gen_bus[g]] += pmax[g] / sum_pmax;
  for (int b = 0; b < N; ++b) inj[b] -= wbus[b] / sum_w;
  std::vector<double> theta_hat = grounded_laplacian_solve(N, from, to, b_line, inj);
  std::vector<double> flim(L);
  {
    SplitMix64 rf(seed, kStreamLineLimit);
    for (int l = 0; l < L; ++l) {
      double fhat = b_line[l] * (theta_hat[from[l]] - theta_hat[to[l]]);
      flim[l] = std::max(rf.uniform(1.0, 3.0) * d_mean, 1.05 * d_peak * std::fabs(fhat));
    }
  }

  // ---- variables (period-major blocks) ------------------------------------------
  std::vector<int> gen_buses;  // buses with at least one generator, ascending
  {
    std::vector<char> has(N, 0);
    for (int g = 0; g < G; ++g) has[gen_bus[g]] = 1;
    for (int b = 0; b < N; ++b)
      if (has[b]) gen_buses.push_back(b);
  }
  std::vector<int> spill_slot(N, -1);
  for (size_t k = 0; k < gen_buses.size(); ++k) spill_slot[gen_buses[k]] = (int)k;
  const int64_t nb = 4LL * G + N + (slack ? (int64_t)N + (int64_t)gen_buses.size() : 0);
  const int64_t n = nb * T;
  auto vp = [&](int t, int g) { return (int64_t)t * nb + g; };
  auto vu = [&](int t, int g) { return (int64_t)t * nb + G + g; };
  auto vv = [&](int t, int g) { return (int64_t)t * nb + 2LL * G + g; };
  auto vw = [&](int t, int g) { return (int64_t)t * nb + 3LL * G + g; };
  auto vth = [&](int t, int b) { return (int64_t)t * nb + 4LL * G + b; };
  auto vshed = [&](int t, int b) { return (int64_t)t * nb + 4LL * G + N + b; };
  auto vspill = [&](int t, int k) { return (int64_t)t * nb + 4LL * G + 2LL * N + k; };

  std::vector<double> c(n, 0.0), lo(n, 0.0), up(n, 0.0);
  std::vector<int32_t> vkind(n, 0);
  const double inf = INFINITY;
  for (int t = 0; t < T; ++t) {
    for (int g = 0; g < G; ++g) {
      c[vp(t, g)] = dt * cost[g];
      lo[vp(t, g)] = 0.0;
      up[vp(t, g)] = pmax[g];
      vkind[vp(t, g)] = UC_VAR_P;
      c[vu(t, g)] = dt * noload[g];
      lo[vu(t, g)] = 0.0;
      up[vu(t, g)] = 1.0;
      vkind[vu(t, g)] = UC_VAR_U;
      c[vv(t, g)] = su[g];
      lo[vv(t, g)] = 0.0;
      up[vv(t, g)] = (t == 0) ? 0.0 : 1.0;
      vkind[vv(t, g)] = UC_VAR_V;
      c[vw(t, g)] = 0.0;
      lo[vw(t, g)] = 0.0;
      up[vw(t, g)] = (t == 0) ? 0.0 : 1.0;
      vkind[vw(t, g)] = UC_VAR_W;
    }
    for (int b = 0; b < N; ++b) {
      lo[vth(t, b)] = (b == 0) ? 0.0 : -inf;
      up[vth(t, b)] = (b == 0) ? 0.0 : inf;
      vkind[vth(t, b)] = UC_VAR_THETA;
      if (slack) {
        c[vshed(t, b)] = dt * 1000.0;
        lo[vshed(t, b)] = 0.0;
        up[vshed(t, b)] = load[(size_t)t * N + b];
        vkind[vshed(t, b)] = UC_VAR_SHED;
      }
    }
    if (slack) {
      for (size_t k = 0; k < gen_buses.size(); ++k) {
        c[vspill(t, (int)k)] = dt * 1000.0;
        lo[vspill(t, (int)k)] = 0.0;
        up[vspill(t, (int)k)] = inf;
        vkind[vspill(t, (int)k)] = UC_VAR_SPILL;
      }
    }
  }

  // ---- rows: equalities first -----------------------------------------------------
  std::vector<std::vector<int>> gens_at(N), lines_at(N);
  for (int g = 0; g < G; ++g) gens_at[gen_bus[g]].push_back(g);
  for (int l = 0; l < L; ++l) {
    lines_at[from[l]].push_back(l);
    lines_at[to[l]].push_back(l);
  }
  Builder B;
  std::vector<int64_t> row_bal((size_t)T * N);
  for (int t = 0; t < T; ++t) {
    for (int b = 0; b < N; ++b) {
      for (int g : gens_at[b]) B.add(vp(t, g), 1.0);
      for (int l : lines_at[b]) {
        // flow f_l = B_l (th_from - th_to) leaves 'from' and enters 'to'
        double sgn = (from[l] == b) ? -1.0 : 1.0;
        B.add(vth(t, from[l]), sgn * b_line[l]);
        B.add(vth(t, to[l]), -sgn * b_line[l]);
      }
      if (slack) {
        B.add(vshed(t, b), 1.0);
        if (spill_slot[b] >= 0) B.add(vspill(t, spill_slot[b]), -1.0);
      }
      row_bal[(size_t)t * N + b] = (int64_t)B.q.size();
      B.close(load[(size_t)t * N + b], UC_ROW_BALANCE);
    }
  }
  for (int t = 1; t < T; ++t)
    for (int g = 0; g < G; ++g) {
      B.add(vu(t, g), 1.0);
      B.add(vu(t - 1, g), -1.0);
      B.add(vv(t, g), -1.0);
      B.add(vw(t, g), 1.0);
      B.close(0.0, UC_ROW_LOGIC);
    }
  const int64_t m_eq = (int64_t)B.q.size();
  for (int s = 0; s < 2; ++s) {
    double sgn = (s == 0) ? 1.0 : -1.0;
    for (int t = 0; t < T; ++t)
      for (int l = 0; l < L; ++l) {
        B.add(vth(t, from[l]), sgn * b_line[l]);
        B.add(vth(t, to[l]), -sgn * b_line[l]);
        B.close(-flim[l], s == 0 ? UC_ROW_FLOW_POS : UC_ROW_FLOW_NEG);
      }
  }
  for (int t = 0; t < T; ++t)
    for (int g = 0; g < G; ++g) {
      B.add(vp(t, g), 1.0);
      B.add(vu(t, g), -pmin[g]);
      B.close(0.0, UC_ROW_PMIN);
    }
  for (int t = 0; t < T; ++t)
    for (int g = 0; g < G; ++g) {
      B.add(vu(t, g), pmax[g]);
      B.add(vp(t, g), -1.0);
      B.close(0.0, UC_ROW_PMAX);
    }
  for (int t = 1; t < T; ++t)
    for (int g = 0; g < G; ++g) {
      B.add(vp(t - 1, g), 1.0);
      B.add(vp(t, g), -1.0);
      B.add(vu(t - 1, g), ramp[g]);
      B.add(vv(t, g), sur[g]);
      B.close(0.0, UC_ROW_RAMP_UP);
    }
  for (int t = 1; t < T; ++t)
    for (int g = 0; g < G; ++g) {
      B.add(vp(t, g), 1.0);
      B.add(vp(t - 1, g), -1.0);
      B.add(vu(t, g), ramp[g]);
      B.add(vw(t, g), sur[g]);
      B.close(0.0, UC_ROW_RAMP_DN);
    }
  for (int t = 1; t < T; ++t)
    for (int g = 0; g < G; ++g) {
      B.add(vu(t, g), 1.0);
      for (int tau = std::max(1, t - ut[g] + 1); tau <= t; ++tau) B.add(vv(tau, g), -1.0);
      B.close(0.0, UC_ROW_MIN_UP);
    }
  for (int t = 1; t < T; ++t)
    for (int g = 0; g < G; ++g) {
      B.add(vu(t, g), -1.0);
      for (int tau = std::max(1, t - dtn[g] + 1); tau <= t; ++tau) B.add(vw(tau, g), -1.0);
      B.close(-1.0, UC_ROW_MIN_DN);
    }

  // ---- pack -------------------------------------------------------------------------
  uc_lp* lp = (uc_lp*)std::calloc(1, sizeof(uc_lp));
  if (!lp) {
    g_err = "uc_lp_build: out of host memory";
    return UC_ERR_NOMEM;
  }
  lp->n = n;
  lp->m = (int64_t)B.q.size();
  lp->m_eq = m_eq;
  lp->nnz = (int64_t)B.col.size();
  lp->row_ptr = dup(B.row_ptr);
  lp->col = dup(B.col);
  lp->val = dup(B.val);
  lp->c = dup(c);
  lp->l = dup(lo);
  lp->u = dup(up);
  lp->q = dup(B.q);
  lp->var_kind = dup(vkind);
  lp->row_kind = dup(B.row_kind);
  lp->n_gen = G;
  lp->n_bus = N;
  lp->n_line = L;
  lp->n_periods = T;
  std::vector<int64_t> ip((size_t)T * G), iu((size_t)T * G), iv((size_t)T * G), iw((size_t)T * G),
      ith((size_t)T * N);
  for (int t = 0; t < T; ++t) {
    for (int g = 0; g < G; ++g) {
      ip[(size_t)t * G + g] = vp(t, g);
      iu[(size_t)t * G + g] = vu(t, g);
      iv[(size_t)t * G + g] = vv(t, g);
      iw[(size_t)t * G + g] = vw(t, g);
    }
    for (int b = 0; b < N; ++b) ith[(size_t)t * N + b] = vth(t, b);
  }
  lp->idx_p = dup(ip);
  lp->idx_u = dup(iu);
  lp->idx_v = dup(iv);
  lp->idx_w = dup(iw);
  lp->idx_theta = dup(ith);
  lp->row_balance = dup(row_bal);
  lp->load = dup(load);
  lp->gen_bus = dup(gen_bus);
  std::vector<int32_t> f32(from.begin(), from.end()), t32(to.begin(), to.end());
  lp->line_from = dup(f32);
  lp->line_to = dup(t32);
  lp->gen_pmax = dup(pmax);
  lp->gen_cost = dup(cost);
  lp->gen_noload = dup(noload);
  lp->gen_min_up = dup(ut);
  lp->gen_min_dn = dup(dtn);
  lp->dt_hours = dt;
  void* chk[] = {lp->row_ptr, lp->col, lp->val, lp->c, lp->l, lp->u, lp->q, lp->var_kind,
                 lp->row_kind, lp->idx_p, lp->idx_u, lp->idx_v, lp->idx_w, lp->idx_theta,
                 lp->row_balance, lp->load, lp->gen_bus, lp->line_from, lp->line_to,
                 lp->gen_pmax, lp->gen_cost, lp->gen_noload, lp->gen_min_up, lp->gen_min_dn};
  for (void* p : chk)
    if (!p) {
      uc_lp_free(lp);
      g_err = "uc_lp_build: out of host memory";
      return UC_ERR_NOMEM;
    }
  *out = lp;
  return UC_OK;
}
