// Learning stage on the GPU for CNF formulas: loopy belief propagation on the surrogate
// Hamiltonian (Sec. "4-SAT Problems Near Computational Phase Transitions"; App. "Loopy Belief
// propagation for k-local Hamiltonians over conjugate normal form"), connected backbone growth
// (Sec. "Generating backbones of rigid variables") and the two-chain schedule of Algorithm 1.
//
// Messages live on the edges e = a * kmax + q of the clause slots (literal id 2v + neg, padding
// literal 2n) for S seeds at once, seed-fastest ([e][S]), so the threads of a warp handle the
// same edge of 32 seeds and every load is coalesced. One LBP iteration = a variable pass (the
// cavity fields h_{i->a} of every edge of a variable from its total field) then a clause pass
// (u_{a->i} of every literal of a clause from the other literals' h). Double precision.
//
// Frames: spin r = 2x - 1; literal i of clause a is satisfied by sigma_ai (+1 positive, -1
// negated). h_{i->a} = sigma_ai (lambda eps_i s*_i + sum_{b != a} sigma_bi u_{b->i});
// u_{a->i} = -1/2 ln[1 - (1 - e^{-2 beta}) prod_{j != i} (1 - tanh h_{j->a}) / 2].
#include <math.h>

#include "nmc_internal.h"

namespace nmc {

namespace {

constexpr int kLbpBlock = 256;
enum : int { kRunning = 0, kWaiting = 1, kFinished = 2 };

__device__ __forceinline__ double lit_sigma(int l) { return (l & 1) ? -1.0 : 1.0; }

// h of every edge at the first lambda: sigma lambda eps s*.
__global__ void lbp_init_h_kernel(const int32_t *__restrict__ clits, long long n_edges, int32_t n,
                                  int32_t S, const double *__restrict__ bias, double *h) {
  const long long total = n_edges * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long e = i / S;
    const int s = (int)(i % S);
    const int l = clits[e];
    h[i] = l >= 2 * n ? 0.0 : lit_sigma(l) * bias[(size_t)(l >> 1) * S + s];
  }
}

// bias[v][s] = lambda eps_v s*_{v,s} (eps and x_star in new variable order).
__global__ void lbp_bias_kernel(const double *__restrict__ eps, const uint8_t *__restrict__ xs,
                                int32_t n, int32_t S, double lambda, double *bias) {
  const long long total = (long long)n * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(i / S);
    bias[i] = lambda * eps[v] * (2.0 * (double)xs[i] - 1.0);
  }
}

// Clause pass: u of every literal of clause a for seed s; the largest change per seed goes to
// dmax (non-negative doubles order like their bit patterns).
__global__ void lbp_clause_kernel(const int32_t *__restrict__ clits, int32_t m, int32_t kmax,
                                  int32_t n, int32_t S, const double *__restrict__ h, double *u,
                                  double c, const int32_t *__restrict__ status,
                                  unsigned long long *dmax, int track) {
  const long long total = (long long)m * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long a = i / S;
    const int s = (int)(i % S);
    if (status && status[s] != kRunning) continue;
    double f[8];
    int k = 0;
    for (int q = 0; q < kmax; ++q) {
      const long long e = a * kmax + q;
      f[q] = 1.0;
      if (clits[e] < 2 * n) {
        f[q] = 1.0 / (1.0 + exp(2.0 * h[e * S + s]));  // (1 - tanh h) / 2, one exp
        ++k;
      }
    }
    double dm = 0.0;
    for (int q = 0; q < kmax; ++q) {
      const long long e = a * kmax + q;
      if (clits[e] >= 2 * n) continue;
      double prod = 1.0;
      for (int j = 0; j < kmax; ++j)
        if (j != q) prod *= f[j];  // padding slots hold 1.0
      const double un = -0.5 * log1p(-c * prod);
      const double d = fabs(un - u[e * S + s]);
      if (d > dm) dm = d;
      u[e * S + s] = un;
    }
    (void)k;
    if (track && dm > 0.0) atomicMax(&dmax[s], (unsigned long long)__double_as_longlong(dm));
  }
}

// Variable pass: total field of v for seed s, then the cavity field of each of its edges.
__global__ void lbp_var_kernel(const int32_t *__restrict__ vptr, const int32_t *__restrict__ vedge,
                               const int32_t *__restrict__ clits, int32_t n, int32_t S,
                               const double *__restrict__ bias, const double *__restrict__ u,
                               double *h, const int32_t *__restrict__ status) {
  const long long total = (long long)n * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(i / S), s = (int)(i % S);
    if (status[s] != kRunning) continue;
    double field = bias[i];
    const int p0 = vptr[v], p1 = vptr[v + 1];
    for (int p = p0; p < p1; ++p) {
      const long long e = vedge[p];
      field += lit_sigma(clits[e]) * u[e * S + s];
    }
    for (int p = p0; p < p1; ++p) {
      const long long e = vedge[p];
      const double sg = lit_sigma(clits[e]);
      h[e * S + s] = sg * (field - sg * u[e * S + s]);
    }
  }
}

// Per seed after an iteration at lambda index k: count, convergence, failure, bookkeeping.
__global__ void lbp_control_kernel(int32_t S, int32_t k, int32_t n_lambda, double tol,
                                   int32_t max_iter, int32_t *status, int32_t *iters,
                                   double *deltas, int32_t *n_done, int32_t *lam_idx,
                                   int32_t *copy_flag, unsigned long long *dmax, int32_t *running) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S || status[s] != kRunning) return;
  const double d = __longlong_as_double((long long)dmax[s]);
  dmax[s] = 0ull;
  const int it = ++iters[(size_t)s * n_lambda + k];
  deltas[(size_t)s * n_lambda + k] = d;
  if (d < tol) {
    n_done[s] = k + 1;
    lam_idx[s] = k;
    copy_flag[s] = 1;  // work -> good
    status[s] = kWaiting;
  } else if (it >= max_iter) {
    if (n_done[s] > 0) copy_flag[s] = 2;  // good -> work (fall back)
    else lam_idx[s] = k;
    status[s] = kFinished;
  } else {
    atomicAdd(running, 1);
  }
}

__global__ void lbp_copy_kernel(long long n_edges, int32_t S, int32_t *copy_flag, double *h,
                                double *u, double *hg, double *ug) {
  const long long total = n_edges * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int f = copy_flag[i % S];
    if (f == 1) {
      hg[i] = h[i];
      ug[i] = u[i];
    } else if (f == 2) {
      h[i] = hg[i];
      u[i] = ug[i];
    }
  }
}

__global__ void lbp_clear_flags_kernel(int32_t S, int32_t *copy_flag) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S) copy_flag[s] = 0;
}

// Start of lambda index k: waiting seeds run again (k < n_lambda) or finish.
__global__ void lbp_advance_kernel(int32_t S, int32_t k, int32_t n_lambda, int32_t *status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S && status[s] == kWaiting) status[s] = k < n_lambda ? kRunning : kFinished;
}

// Marginals <r_v> (new order -> original order) with each seed's own lambda, and (p, q1) per
// seed in a fixed summation order (one block per seed).
__global__ void lbp_marg_kernel(const int32_t *__restrict__ vptr, const int32_t *__restrict__ vedge,
                                const int32_t *__restrict__ clits, const int32_t *__restrict__ orig,
                                int32_t n, int32_t S, const double *__restrict__ eps,
                                const uint8_t *__restrict__ xs, const double *__restrict__ lambdas,
                                const int32_t *__restrict__ lam_idx, const double *__restrict__ u,
                                double *marg, double *overlap) {
  const int s = blockIdx.x;
  const double lam = lambdas[lam_idx[s]];
  __shared__ double sp[kLbpBlock], sq[kLbpBlock];
  double p = 0.0, q = 0.0;
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    const double sv = 2.0 * (double)xs[(size_t)v * S + s] - 1.0;
    double field = lam * eps[v] * sv;
    for (int k = vptr[v]; k < vptr[v + 1]; ++k) {
      const long long e = vedge[k];
      field += lit_sigma(clits[e]) * u[e * S + s];
    }
    const double mv = tanh(field);
    marg[(size_t)s * n + orig[v]] = mv;
    p += sv * mv;
    q += mv * mv;
  }
  sp[threadIdx.x] = p;
  sq[threadIdx.x] = q;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sp[threadIdx.x] += sp[threadIdx.x + o];
      sq[threadIdx.x] += sq[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    overlap[2 * s] = sp[0] / n;
    overlap[2 * s + 1] = sq[0] / n;
  }
}

// <prod_{i in a} r_i> = [prod_i sigma_i t_i - c prod_i (-sigma_i) (1 - t_i)/2] / z_a,
// z_a = 1 - c prod_i (1 - t_i)/2, t_i = tanh h_{i->a} (the clause's configurations summed in
// closed form: the violating configuration r_i = -sigma_i carries weight e^{-2 beta}).
__global__ void lbp_corr_kernel(const int32_t *__restrict__ clits, int32_t m, int32_t kmax,
                                int32_t n, int32_t S, const double *__restrict__ h, double c,
                                double *corr) {
  const long long total = (long long)m * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long a = i / S;
    const int s = (int)(i % S);
    double free_prod = 1.0, viol_prod = 1.0, sign = 1.0;
    int k = 0;
    for (int q = 0; q < kmax; ++q) {
      const long long e = a * kmax + q;
      const int l = clits[e];
      if (l >= 2 * n) continue;
      const double sg = lit_sigma(l), t = tanh(h[e * S + s]);
      free_prod *= sg * t;
      viol_prod *= (1.0 - t) / 2.0;
      sign *= -sg;
      ++k;
    }
    const double z = 1.0 - c * viol_prod;
    corr[(size_t)s * m + a] = k > 0 ? (free_prod - c * sign * viol_prod) / z : 0.0;
  }
}

unsigned blocks_for(long long work) {
  long long g = (work + kLbpBlock - 1) / kLbpBlock;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

// xs[v][s] = x_in[s][orig v] (0/1), eps[v] = eps_in[orig v] or, without eps_in, the number of
// clauses of v.
static __global__ void lbp_prepare_kernel(const uint8_t *__restrict__ x_in, const double *__restrict__ eps_in,
                                   const int32_t *__restrict__ orig, const int32_t *__restrict__ vptr,
                                   int32_t n, int32_t S, uint8_t *xs, double *eps) {
  const long long total = (long long)n * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(i / S), s = (int)(i % S);
    xs[i] = x_in[(size_t)s * n + orig[v]];
    if (s == 0) eps[v] = eps_in ? eps_in[orig[v]] : (double)(vptr[v + 1] - vptr[v]);
  }
}

size_t lbp_scratch_bytes(int32_t n, int32_t m, int32_t kmax, int32_t S, int32_t n_lambda) {
  auto up = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
  const size_t E = (size_t)m * kmax;
  return 4 * up(sizeof(double) * E * S) + up(sizeof(double) * (size_t)n * S) +
         up(sizeof(unsigned long long) * S) + 3 * up(sizeof(int32_t) * S) + up(sizeof(int32_t)) +
         up(sizeof(double) * n_lambda);
}

cudaError_t lbp_prepare(const uint8_t *x_in, const double *eps_in, const int32_t *orig,
                        const int32_t *vptr, int32_t n, int32_t S, uint8_t *xs, double *eps,
                        cudaStream_t st) {
  lbp_prepare_kernel<<<blocks_for((long long)n * S), kLbpBlock, 0, st>>>(x_in, eps_in, orig, vptr, n,
                                                                      S, xs, eps);
  return cudaGetLastError();
}

int lbp_run(const LbpArgs &A, cudaStream_t st) {
  auto up = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
  const int32_t S = A.S, n = A.n, m = A.m, kmax = A.kmax, L = A.n_lambda;
  const long long E = (long long)m * kmax;
  char *p = static_cast<char *>(A.scratch);
  double *h = reinterpret_cast<double *>(p); p += up(sizeof(double) * E * S);
  double *u = reinterpret_cast<double *>(p); p += up(sizeof(double) * E * S);
  double *hg = reinterpret_cast<double *>(p); p += up(sizeof(double) * E * S);
  double *ug = reinterpret_cast<double *>(p); p += up(sizeof(double) * E * S);
  double *bias = reinterpret_cast<double *>(p); p += up(sizeof(double) * (size_t)n * S);
  unsigned long long *dmax = reinterpret_cast<unsigned long long *>(p); p += up(sizeof(unsigned long long) * S);
  int32_t *status = reinterpret_cast<int32_t *>(p); p += up(sizeof(int32_t) * S);
  int32_t *lam_idx = reinterpret_cast<int32_t *>(p); p += up(sizeof(int32_t) * S);
  int32_t *copy_flag = reinterpret_cast<int32_t *>(p); p += up(sizeof(int32_t) * S);
  int32_t *running = reinterpret_cast<int32_t *>(p); p += up(sizeof(int32_t));
  double *lam_dev = reinterpret_cast<double *>(p);
  const double c = -expm1(-2.0 * A.beta);
  cudaError_t e;
#define LBP_CHECK(x)                 \
  do {                               \
    if ((e = (x)) != cudaSuccess) return (int)e; \
  } while (0)
  LBP_CHECK(cudaMemsetAsync(dmax, 0, sizeof(unsigned long long) * S, st));
  LBP_CHECK(cudaMemsetAsync(status, 0, sizeof(int32_t) * S, st));  // kRunning
  LBP_CHECK(cudaMemsetAsync(lam_idx, 0, sizeof(int32_t) * S, st));
  LBP_CHECK(cudaMemsetAsync(copy_flag, 0, sizeof(int32_t) * S, st));
  LBP_CHECK(cudaMemsetAsync(A.iters, 0, sizeof(int32_t) * S * L, st));
  LBP_CHECK(cudaMemsetAsync(A.deltas, 0, sizeof(double) * S * L, st));
  LBP_CHECK(cudaMemsetAsync(A.n_done, 0, sizeof(int32_t) * S, st));
  LBP_CHECK(cudaMemsetAsync(u, 0, sizeof(double) * E * S, st));
  LBP_CHECK(cudaMemcpyAsync(lam_dev, A.lambdas, sizeof(double) * L, cudaMemcpyHostToDevice, st));
  const unsigned gS = (unsigned)((S + kLbpBlock - 1) / kLbpBlock);
  // initial messages at lambda_0: h from the bias, u from those h
  lbp_bias_kernel<<<blocks_for((long long)n * S), kLbpBlock, 0, st>>>(A.eps, A.xs, n, S, A.lambdas[0], bias);
  lbp_init_h_kernel<<<blocks_for(E * S), kLbpBlock, 0, st>>>(A.clits, E, n, S, bias, h);
  lbp_clause_kernel<<<blocks_for((long long)m * S), kLbpBlock, 0, st>>>(A.clits, m, kmax, n, S, h, u, c,
                                                                     nullptr, dmax, 0);
  LBP_CHECK(cudaGetLastError());
  for (int32_t k = 0; k < L; ++k) {
    if (k > 0) {
      lbp_advance_kernel<<<gS, kLbpBlock, 0, st>>>(S, k, L, status);
      lbp_bias_kernel<<<blocks_for((long long)n * S), kLbpBlock, 0, st>>>(A.eps, A.xs, n, S, A.lambdas[k], bias);
    }
    for (int32_t it = 0; it < A.max_iter; ++it) {
      lbp_var_kernel<<<blocks_for((long long)n * S), kLbpBlock, 0, st>>>(A.vptr, A.vedge, A.clits, n, S,
                                                                       bias, u, h, status);
      lbp_clause_kernel<<<blocks_for((long long)m * S), kLbpBlock, 0, st>>>(A.clits, m, kmax, n, S, h, u,
                                                                         c, status, dmax, 1);
      LBP_CHECK(cudaMemsetAsync(running, 0, sizeof(int32_t), st));
      lbp_control_kernel<<<gS, kLbpBlock, 0, st>>>(S, k, L, A.tol, A.max_iter, status, A.iters,
                                                   A.deltas, A.n_done, lam_idx, copy_flag, dmax,
                                                   running);
      lbp_copy_kernel<<<blocks_for(E * S), kLbpBlock, 0, st>>>(E, S, copy_flag, h, u, hg, ug);
      lbp_clear_flags_kernel<<<gS, kLbpBlock, 0, st>>>(S, copy_flag);
      LBP_CHECK(cudaGetLastError());
      int32_t run_h = 0;
      LBP_CHECK(cudaMemcpyAsync(&run_h, running, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      LBP_CHECK(cudaStreamSynchronize(st));
      if (run_h == 0) break;
    }
  }
  lbp_advance_kernel<<<gS, kLbpBlock, 0, st>>>(S, L, L, status);
  lbp_marg_kernel<<<S, kLbpBlock, 0, st>>>(A.vptr, A.vedge, A.clits, A.orig, n, S, A.eps, A.xs,
                                          lam_dev, lam_idx, u, A.marg, A.overlap);
  lbp_corr_kernel<<<blocks_for((long long)m * S), kLbpBlock, 0, st>>>(A.clits, m, kmax, n, S, h, c,
                                                                   A.corr);
  LBP_CHECK(cudaGetLastError());
#undef LBP_CHECK
  return 0;
}

// ---- backbones ------------------------------------------------------------------------------
//
// J~_a = atanh|<prod r>| / beta. Factors with J~ above the cutoff or the seed threshold link
// their variables; components under the linking factors are found by label propagation (min
// original id, with pointer jumping); a component is a backbone when it holds a seed factor
// (J~ above the seed threshold). Labels: the component's smallest original variable id, -1
// outside every backbone. S problems (seeds) side by side: labels [S][n] in new order.
namespace {

constexpr int32_t kNoLabel = 0x7FFFFFFF;

__global__ void bb_init_kernel(const int32_t *__restrict__ clits, int32_t m, int32_t kmax,
                               int32_t n, int32_t S, const double *__restrict__ corr, double beta,
                               double seed_thr, double cutoff, const int32_t *__restrict__ orig,
                               uint8_t *link, int32_t *label) {
  const long long total = (long long)m * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / m);
    const long long a = i % m;
    const double jt = atanh(fabs(corr[(size_t)s * m + a])) / beta;
    const uint8_t f = (uint8_t)((jt > cutoff || jt > seed_thr) ? 1 : 0) | (uint8_t)(jt > seed_thr ? 2 : 0);
    link[i] = f;
    if (f)
      for (int q = 0; q < kmax; ++q) {
        const int l = clits[a * kmax + q];
        if (l < 2 * n) label[(size_t)s * n + (l >> 1)] = orig[l >> 1];  // same value from every writer
      }
  }
}

__global__ void bb_fill_kernel(int32_t n, int32_t S, int32_t *label) {
  const long long total = (long long)n * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    label[i] = kNoLabel;
}

__global__ void bb_propagate_kernel(const int32_t *__restrict__ clits, int32_t m, int32_t kmax,
                                    int32_t n, int32_t S, const uint8_t *__restrict__ link,
                                    int32_t *label, int32_t *changed) {
  const long long total = (long long)m * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    if (!link[i]) continue;
    const int s = (int)(i / m);
    const long long a = i % m;
    int32_t *ls = label + (size_t)s * n;
    int mn = kNoLabel;
    for (int q = 0; q < kmax; ++q) {
      const int l = clits[a * kmax + q];
      if (l < 2 * n) mn = min(mn, ls[l >> 1]);
    }
    for (int q = 0; q < kmax; ++q) {
      const int l = clits[a * kmax + q];
      if (l < 2 * n && atomicMin(&ls[l >> 1], mn) > mn) *changed = 1;
    }
  }
}

// Pointer jumping: a label is the original id of a variable whose own label may be smaller.
__global__ void bb_jump_kernel(int32_t n, int32_t S, const int32_t *__restrict__ newid,
                               int32_t *label, int32_t *changed) {
  const long long total = (long long)n * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / n);
    const int l = label[i];
    if (l == kNoLabel) continue;
    const int l2 = label[(size_t)s * n + newid[l]];
    if (l2 < l && atomicMin(&label[i], l2) > l2) *changed = 1;
  }
}

__global__ void bb_seed_kernel(const int32_t *__restrict__ clits, int32_t m, int32_t kmax,
                               int32_t n, int32_t S, const uint8_t *__restrict__ link,
                               const int32_t *__restrict__ label, const int32_t *__restrict__ newid,
                               uint8_t *seeded) {
  const long long total = (long long)m * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    if (!(link[i] & 2)) continue;
    const int s = (int)(i / m);
    const long long a = i % m;
    for (int q = 0; q < kmax; ++q) {
      const int l = clits[a * kmax + q];
      if (l < 2 * n) {
        seeded[(size_t)s * n + newid[label[(size_t)s * n + (l >> 1)]]] = 1;
        break;
      }
    }
  }
}

__global__ void bb_final_kernel(int32_t n, int32_t S, const int32_t *__restrict__ orig,
                                const int32_t *__restrict__ newid, const int32_t *__restrict__ label,
                                const uint8_t *__restrict__ seeded, int32_t *out, int32_t *n_clusters) {
  const long long total = (long long)n * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / n), v = (int)(i % n);
    const int l = label[i];
    int r = -1;
    if (l != kNoLabel && seeded[(size_t)s * n + newid[l]]) {
      r = l;
      if (orig[v] == l) atomicAdd(&n_clusters[s], 1);
    }
    out[(size_t)s * n + orig[v]] = r;
  }
}

// The two-chain schedule of Algorithm 1 in Q16, step-major: per cycle t_hot steps with the
// backbone at base / heat and the rest held, t_cold steps with the backbone held and the rest at
// base, t_unlearn steps with every variable at base.
__global__ void bb_schedule_kernel(const int32_t *__restrict__ lab, const int32_t *__restrict__ orig,
                                   int32_t n, int32_t n_steps,
                                   float base, float heat, int32_t t_hot, int32_t t_cold,
                                   int32_t t_unlearn, uint32_t *bq) {
  const long long total = (long long)n * n_steps;
  const uint32_t qb = __float2uint_rn(base * 65536.0f);
  const uint32_t qh = __float2uint_rn(__fdiv_rn(base, heat) * 65536.0f);
  const int cyc = t_hot + t_cold + t_unlearn;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i / n), v = (int)(i % n);
    const int pos = t % cyc;
    const bool bb = lab[orig[v]] >= 0;
    uint32_t q;
    if (pos < t_hot) q = bb ? qh : kFrozenQ16;
    else if (pos < t_hot + t_cold) q = bb ? kFrozenQ16 : qb;
    else q = qb;
    bq[i] = q;
  }
}

}  // namespace

size_t backbone_scratch_bytes(int32_t n, int32_t m, int32_t S) {
  auto up = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
  return up((size_t)m * S) + up(sizeof(int32_t) * (size_t)n * S) + up((size_t)n * S) +
         2 * up(sizeof(int32_t) * S) + up(sizeof(int32_t));
}

int backbone_run(const BackboneArgs &A, cudaStream_t st) {
  auto up = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
  const int32_t n = A.n, m = A.m, S = A.S;
  char *p = static_cast<char *>(A.scratch);
  uint8_t *link = reinterpret_cast<uint8_t *>(p); p += up((size_t)m * S);
  int32_t *label = reinterpret_cast<int32_t *>(p); p += up(sizeof(int32_t) * (size_t)n * S);
  uint8_t *seeded = reinterpret_cast<uint8_t *>(p); p += up((size_t)n * S);
  p += 2 * up(sizeof(int32_t) * S);
  int32_t *changed = reinterpret_cast<int32_t *>(p);
  cudaError_t e;
  if ((e = cudaMemsetAsync(seeded, 0, (size_t)n * S, st)) != cudaSuccess) return (int)e;
  if ((e = cudaMemsetAsync(A.n_clusters, 0, sizeof(int32_t) * S, st)) != cudaSuccess) return (int)e;
  bb_fill_kernel<<<blocks_for((long long)n * S), kLbpBlock, 0, st>>>(n, S, label);
  bb_init_kernel<<<blocks_for((long long)m * S), kLbpBlock, 0, st>>>(A.clits, m, A.kmax, n, S, A.corr,
                                                                  A.beta, A.seed_thr, A.cutoff,
                                                                  A.orig, link, label);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  // every round lowers some label or stops; n rounds bound any component's propagation
  for (int32_t round = 0; round <= n + 1; ++round) {
    if ((e = cudaMemsetAsync(changed, 0, sizeof(int32_t), st)) != cudaSuccess) return (int)e;
    bb_propagate_kernel<<<blocks_for((long long)m * S), kLbpBlock, 0, st>>>(A.clits, m, A.kmax, n, S,
                                                                         link, label, changed);
    bb_jump_kernel<<<blocks_for((long long)n * S), kLbpBlock, 0, st>>>(n, S, A.newid, label, changed);
    if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    int32_t ch = 0;
    if ((e = cudaMemcpyAsync(&ch, changed, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return (int)e;
    if (!ch) break;
  }
  bb_seed_kernel<<<blocks_for((long long)m * S), kLbpBlock, 0, st>>>(A.clits, m, A.kmax, n, S, link,
                                                                  label, A.newid, seeded);
  bb_final_kernel<<<blocks_for((long long)n * S), kLbpBlock, 0, st>>>(n, S, A.orig, A.newid, label,
                                                                   seeded, A.labels, A.n_clusters);
  return (int)cudaGetLastError();
}

cudaError_t backbone_schedule(const int32_t *lab, const int32_t *orig, int32_t n, int32_t n_steps,
                              float base, float heat, int32_t t_hot, int32_t t_cold,
                              int32_t t_unlearn, uint32_t *bq, cudaStream_t st) {
  bb_schedule_kernel<<<blocks_for((long long)n * n_steps), kLbpBlock, 0, st>>>(
      lab, orig, n, n_steps, base, heat, t_hot, t_cold, t_unlearn, bq);
  return cudaGetLastError();
}

}  // namespace nmc
