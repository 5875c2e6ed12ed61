/*
 * lbp_oracle.c -- plain, slow CPU oracle for the learning stage of Nonequilibrium Monte Carlo
 * over a CNF formula (Mohseni et al., arXiv:2111.13628): loopy belief propagation on the
 * surrogate Hamiltonian, effective factor couplings and connected backbone growth.
 *
 * TEST INFRASTRUCTURE ONLY (loaded by the tests, the smoke check and the bench's CPU leg). It
 * shares no code with the CUDA library. Double precision throughout.
 *
 * Definitions (Sec. "4-SAT Problems Near Computational Phase Transitions"; App. "Loopy Belief
 * propagation for k-local Hamiltonians over conjugate normal form"; Sec. "Generating backbones
 * of rigid variables"), with the readings this file fixes:
 *  Spins r_i = 2 x_i - 1. Literal i of clause a is satisfied by the spin sigma_ai (+1 for a
 *    positive literal, -1 for a negated one); its violating value is J_i^a = -sigma_ai. Clause
 *    weight omega_a = exp(-2 beta) on its single violating configuration, 1 otherwise.
 *  Variable -> clause message, in the clause's frame (positive = towards satisfying a):
 *    h_{i->a} = sigma_ai (lambda eps_i s*_i + sum_{b in di \ a} sigma_bi u_{b->i}).
 *    (The paper writes the agreeing clauses with +, the disagreeing ones with -: the same sum.
 *    It leaves the bias term without the frame sign; it is read in the variable's frame.)
 *  Clause -> variable message:
 *    u_{a->i} = -1/2 ln[1 - (1 - exp(-2 beta)) prod_{j in da \ i} (1 - tanh h_{j->a}) / 2].
 *  Schedule: messages start from h = sigma lambda_0 eps s*, u from those h (the paper's
 *    initialisation). An iteration recomputes every h from the previous u, then every u from
 *    the new h (parallel updates). Converged when max |u_new - u_old| < tol. lambda continues
 *    through the given list without re-initialising; when a lambda fails to converge within
 *    max_iter iterations the messages of the previous (converged) lambda are restored and the
 *    continuation stops.
 *  Marginal: <r_i> = tanh(lambda eps_i s*_i + sum_{a in di} sigma_ai u_{a->i}).
 *  Clause correlation: <prod_{i in da} r_i> = sum over the 2^k configurations of mu_a(r) prod r,
 *    mu_a(r) = omega_a(r) prod_i (1 - J_i r_i tanh h_{i->a}) / 2 / z_a (the defining sum; the
 *    paper's closed form drops the term prod_i (-J_i tanh h_{i->a}) of that sum).
 *  Overlaps: p = (1/N) sum_i s*_i <r_i>, q1 = (1/N) sum_i <r_i>^2.
 *  Effective factor coupling J~_a = beta^-1 artanh |<prod r>| (the magnitude measures rigidity).
 *  Backbones: factors with J~ > seed threshold are nuclei; from each nucleus (in clause order)
 *    a cluster grows through every factor with J~ above the cutoff (or above the seed
 *    threshold) that touches it, until nothing can be added; each cluster is labelled by its
 *    smallest variable id; variables in no cluster get -1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t n, m, kmax;
  const int32_t *lits;
  int32_t *vptr; /* n+1: incident edges of each variable */
  int32_t *vedge; /* edge ids e = a*kmax + q */
} lbp_graph;

static int lbp_var(int32_t l) { return (l > 0 ? l : -l) - 1; }
static double lbp_sigma(int32_t l) { return l > 0 ? 1.0 : -1.0; }

static void lbp_graph_build(lbp_graph *g, int32_t n, int32_t m, int32_t kmax, const int32_t *lits) {
  g->n = n;
  g->m = m;
  g->kmax = kmax;
  g->lits = lits;
  g->vptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
  for (int64_t e = 0; e < (int64_t)m * kmax; ++e)
    if (lits[e] != 0) g->vptr[lbp_var(lits[e]) + 1]++;
  for (int32_t v = 0; v < n; ++v) g->vptr[v + 1] += g->vptr[v];
  g->vedge = (int32_t *)malloc(sizeof(int32_t) * ((size_t)g->vptr[n] + 1));
  int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  memcpy(fill, g->vptr, sizeof(int32_t) * (size_t)n);
  for (int64_t e = 0; e < (int64_t)m * kmax; ++e)
    if (lits[e] != 0) g->vedge[fill[lbp_var(lits[e])]++] = (int32_t)e;
  free(fill);
}

static void lbp_graph_free(lbp_graph *g) {
  free(g->vptr);
  free(g->vedge);
}

/* u of edge e = (a, q) from the h of the other literals of clause a. */
static double lbp_u(const lbp_graph *g, const double *h, int64_t e, double c) {
  const int64_t a = e / g->kmax;
  double prod = 1.0;
  for (int q = 0; q < g->kmax; ++q) {
    const int64_t f = a * g->kmax + q;
    if (f == e || g->lits[f] == 0) continue;
    prod *= (1.0 - tanh(h[f])) / 2.0;
  }
  return -0.5 * log1p(-c * prod);
}

/* h of edge e = (a, i): sigma_ai (lambda eps_i s_i + sum over the other clauses of i). */
static double lbp_h(const lbp_graph *g, const double *u, int64_t e, double bias_i) {
  const int32_t i = lbp_var(g->lits[e]);
  double field = bias_i;
  for (int32_t p = g->vptr[i]; p < g->vptr[i + 1]; ++p) {
    const int32_t f = g->vedge[p];
    if (f == e) continue;
    field += lbp_sigma(g->lits[f]) * u[f];
  }
  return lbp_sigma(g->lits[e]) * field;
}

/*
 * One seed. x_star: n uint8 0/1 (s* = 2x - 1). eps: n doubles. lambdas: n_lambda values used in
 * order. Outputs: marg[n], corr[m], iters[n_lambda] (iterations run at each lambda, 0 if not
 * reached), deltas[n_lambda] (last max |du|), *n_done = lambdas that converged, overlap[2] =
 * (p, q1), lambda_out = the lambda of the returned messages. Returns 0, or -1 on bad arguments.
 */
int orc_cnf_lbp(int32_t n, int32_t m, int32_t kmax, const int32_t *lits, const uint8_t *x_star,
                const double *eps, double beta, int32_t n_lambda, const double *lambdas,
                double tol, int32_t max_iter, double *marg, double *corr, int32_t *iters,
                double *deltas, int32_t *n_done, double *overlap, double *lambda_out) {
  if (n <= 0 || m < 0 || kmax <= 0 || n_lambda <= 0 || max_iter < 1) return -1;
  lbp_graph g;
  lbp_graph_build(&g, n, m, kmax, lits);
  const int64_t E = (int64_t)m * kmax;
  const double c = -expm1(-2.0 * beta); /* 1 - exp(-2 beta) */
  double *h = (double *)calloc((size_t)E + 1, sizeof(double));
  double *u = (double *)calloc((size_t)E + 1, sizeof(double));
  double *un = (double *)calloc((size_t)E + 1, sizeof(double));
  double *hg = (double *)calloc((size_t)E + 1, sizeof(double));
  double *ug = (double *)calloc((size_t)E + 1, sizeof(double));
  double *bias = (double *)malloc(sizeof(double) * (size_t)n);
  for (int32_t k = 0; k < n_lambda; ++k) {
    iters[k] = 0;
    deltas[k] = 0.0;
  }
  /* initial messages at lambda_0 */
  for (int32_t i = 0; i < n; ++i) bias[i] = lambdas[0] * eps[i] * (2.0 * x_star[i] - 1.0);
  for (int64_t e = 0; e < E; ++e)
    if (lits[e] != 0) h[e] = lbp_sigma(lits[e]) * bias[lbp_var(lits[e])];
  for (int64_t e = 0; e < E; ++e)
    if (lits[e] != 0) u[e] = lbp_u(&g, h, e, c);
  int32_t done = 0;
  double lam_ret = lambdas[0];
  for (int32_t k = 0; k < n_lambda; ++k) {
    for (int32_t i = 0; i < n; ++i) bias[i] = lambdas[k] * eps[i] * (2.0 * x_star[i] - 1.0);
    int conv = 0;
    for (int32_t it = 1; it <= max_iter; ++it) {
      for (int64_t e = 0; e < E; ++e)
        if (lits[e] != 0) h[e] = lbp_h(&g, u, e, bias[lbp_var(lits[e])]);
      double dmax = 0.0;
      for (int64_t e = 0; e < E; ++e) {
        if (lits[e] == 0) continue;
        un[e] = lbp_u(&g, h, e, c);
        const double d = fabs(un[e] - u[e]);
        if (d > dmax) dmax = d;
      }
      memcpy(u, un, sizeof(double) * (size_t)E);
      iters[k] = it;
      deltas[k] = dmax;
      if (dmax < tol) {
        conv = 1;
        break;
      }
    }
    if (conv) {
      done = k + 1;
      lam_ret = lambdas[k];
      memcpy(hg, h, sizeof(double) * (size_t)E);
      memcpy(ug, u, sizeof(double) * (size_t)E);
    } else {
      if (done > 0) { /* fall back to the last converged lambda */
        memcpy(h, hg, sizeof(double) * (size_t)E);
        memcpy(u, ug, sizeof(double) * (size_t)E);
      } else {
        lam_ret = lambdas[k];
      }
      break;
    }
  }
  for (int32_t i = 0; i < n; ++i) bias[i] = lam_ret * eps[i] * (2.0 * x_star[i] - 1.0);
  double p = 0.0, q1 = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    double field = bias[i];
    for (int32_t q = g.vptr[i]; q < g.vptr[i + 1]; ++q) {
      const int32_t f = g.vedge[q];
      field += lbp_sigma(lits[f]) * u[f];
    }
    marg[i] = tanh(field);
    p += (2.0 * x_star[i] - 1.0) * marg[i];
    q1 += marg[i] * marg[i];
  }
  overlap[0] = p / n;
  overlap[1] = q1 / n;
  /* clause correlations by the defining sum over the 2^k configurations of the clause */
  for (int64_t a = 0; a < m; ++a) {
    int32_t idx[8];
    int k = 0;
    for (int q = 0; q < kmax && k < 8; ++q)
      if (lits[a * kmax + q] != 0) idx[k++] = q;
    double zsum = 0.0, rsum = 0.0;
    for (int cfg = 0; cfg < (1 << k); ++cfg) {
      double w = 1.0, prod_r = 1.0;
      int violating = 1;
      for (int j = 0; j < k; ++j) {
        const int64_t f = a * kmax + idx[j];
        const double r = ((cfg >> j) & 1) ? 1.0 : -1.0;
        const double J = -lbp_sigma(lits[f]);
        w *= (1.0 - J * r * tanh(h[f])) / 2.0;
        prod_r *= r;
        if (r != J) violating = 0;
      }
      if (violating) w *= exp(-2.0 * beta);
      zsum += w;
      rsum += w * prod_r;
    }
    corr[a] = k > 0 ? rsum / zsum : 0.0;
  }
  *n_done = done;
  *lambda_out = lam_ret;
  free(h);
  free(u);
  free(un);
  free(hg);
  free(ug);
  free(bias);
  lbp_graph_free(&g);
  return 0;
}

/* Backbone labels from clause correlations (see the header). Returns the number of clusters. */
int32_t orc_cnf_backbone(int32_t n, int32_t m, int32_t kmax, const int32_t *lits,
                         const double *corr, double beta, double seed_thr, double cutoff,
                         int32_t *label) {
  lbp_graph g;
  lbp_graph_build(&g, n, m, kmax, lits);
  double *jt = (double *)malloc(sizeof(double) * ((size_t)m + 1));
  for (int64_t a = 0; a < m; ++a) jt[a] = atanh(fabs(corr[a])) / beta;
  for (int32_t v = 0; v < n; ++v) label[v] = -1;
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  int32_t *member = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  char *in = (char *)calloc((size_t)n + 1, 1);
  int32_t clusters = 0;
  for (int64_t a = 0; a < m; ++a) {
    if (!(jt[a] > seed_thr)) continue;
    int fresh = 0;
    for (int q = 0; q < kmax; ++q) {
      const int32_t l = lits[a * kmax + q];
      if (l != 0 && label[lbp_var(l)] < 0) fresh = 1;
    }
    if (!fresh) continue;
    int32_t qh = 0, qt = 0, nm = 0;
    for (int q = 0; q < kmax; ++q) {
      const int32_t l = lits[a * kmax + q];
      if (l == 0) continue;
      const int32_t v = lbp_var(l);
      if (!in[v]) {
        in[v] = 1;
        queue[qt++] = v;
        member[nm++] = v;
      }
    }
    while (qh < qt) {
      const int32_t v = queue[qh++];
      for (int32_t p = g.vptr[v]; p < g.vptr[v + 1]; ++p) {
        const int64_t b = g.vedge[p] / kmax;
        if (!(jt[b] > cutoff || jt[b] > seed_thr)) continue;
        for (int q = 0; q < kmax; ++q) {
          const int32_t l = lits[b * kmax + q];
          if (l == 0) continue;
          const int32_t w = lbp_var(l);
          if (!in[w]) {
            in[w] = 1;
            queue[qt++] = w;
            member[nm++] = w;
          }
        }
      }
    }
    int32_t lab = n;
    for (int32_t j = 0; j < nm; ++j)
      if (member[j] < lab) lab = member[j];
    for (int32_t j = 0; j < nm; ++j) label[member[j]] = lab;
    ++clusters;
  }
  free(jt);
  free(queue);
  free(member);
  free(in);
  lbp_graph_free(&g);
  return clusters;
}
