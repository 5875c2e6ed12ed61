/*
 * nmc_oracle.c -- plain, slow CPU oracle for the inhomogeneous Metropolis sweep of
 * Nonequilibrium Monte Carlo (Mohseni et al., arXiv:2111.13628).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's CPU-baseline
 * leg load this file. It shares no code, header, table or constant generator with the
 * CUDA library; both sides are written from the same prose definition of the dynamics.
 *
 * What it computes (the paper fixes the energy, the single-variable Metropolis move and a
 * per-variable inverse temperature; every other choice is a stated reading):
 *
 *  k-SAT energy (Sec. "4-SAT Problems Near Computational Phase Transitions": the cost is the
 *    number of violated clauses of a CNF formula): E(x) = #clauses with no true literal.
 *    Literal +(v+1) is true iff x_v = 1, literal -(v+1) iff x_v = 0.
 *  Move (Metropolis-Hastings local update, Introduction; a different temperature per region
 *    of the system, Sec. "Nonequilibrium Nonlocal Monte Carlo"; two chains with the backbone
 *    heated 2-10x, Sec. "Nonequilibrium inhomogeneous sampling over subgraphs"): flip one
 *    variable v with its own beta_v[t]; accept with probability min(1, exp(-beta_v[t] dE)).
 *  Sweep order (the paper leaves a "sweep" undefined): a DSatur colouring of the
 *    variable-interaction graph (Brelaz, CACM 1979: repeatedly colour the uncoloured variable
 *    whose coloured neighbours show the most distinct colours, here ties broken by more clause
 *    occurrences, then by the smaller id, giving it the smallest colour none of its neighbours
 *    holds), colours visited in ascending order, each colour class (an independent set) updated
 *    against the state left by earlier colours. Within a class, ascending id (any order gives
 *    the same result).
 *  Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = seed, counter
 *    (v, t, r>>2, TAG_KSAT_SWEEP), output word r&3 for replica r's attempt on v at sweep t.
 *  Acceptance: dE <= 0 accepts with no draw. Otherwise bq = Q16 beta (round half even),
 *    idx = (bq*dE) >> 8, accept iff idx < L and u < Tab[idx], with
 *    Tab[j] = min(2^32-1, floor(2^32 exp(-j/256))) and L the first j with Tab[j] = 0.
 *  Best-so-far: starts at the initial state, replaced after a full sweep on strictly lower E.
 *  Replica exchange (App. "Adaptive Parallel Tempering": swap probability
 *    min{1, exp[(beta_i - beta_j)(E_i - E_j)]} for replicas at adjacent temperatures): G ladders
 *    of L slots, replica g*L + i in ladder g; replica r sits at slot s(r) of its ladder, with Q16
 *    temperature lq[s]; its moves use min(2^32-1, (lq[s(r)] * bq_v[t]) >> 16). After every S
 *    sweeps (sweep t with (t+1) % S == 0, round q = (t+1)/S - 1) the pairs of adjacent slots
 *    (k, k+1) with k = q mod 2, k+2, ... of every ladder try to exchange their replicas a (at k)
 *    and b (at k+1): d = (lq[k] - lq[k+1]) (E_a - E_b) accepts when d >= 0, else iff
 *    ((-d) >> 8) < L and u < Tab[(-d) >> 8] for u = word 0 of the Philox block for counter
 *    (k, q, g, TAG_PT_SWAP). The QAP chain takes the same ladder on its pair temperature
 *    (bq_r + bq_s) >> 1, with the exchange product formed exactly in 128 bits.
 *  Frozen units (the two chains of Algorithm 1 sample one subset with the other held fixed,
 *    Fig. 2 caption): beta_v[t] = +infinity holds unit v fixed at step t. A frozen k-SAT variable
 *    is not attempted; a QAP swap that involves a frozen facility is rejected (its Philox block is
 *    still drawn, so nothing else shifts).
 *  Collective move (the nonlocal backbone flip of Fig. 1(c)): replica r proposes x' = x xor m_r
 *    and accepts when dE = E(x') - E(x) <= 0, else iff ((bq dE) >> 8) < L and u < Tab[...] with
 *    bq = Q16(beta_r) and u = word r&3 of the Philox block for counter
 *    (move_id, 0, r>>2, TAG_CLUSTER); the best-so-far follows on strictly lower E.
 *  Whitening (Sec. "Whitening procedure for low energy states"): see orc_ksat_whitening.
 *  Energy statistics (the adaptive ladder of the same appendix measures the energy variance at
 *    each temperature): sums of E and E^2 of every replica over the end-of-sweep energies of
 *    the sweeps t >= stats_t0.
 *  QAP (Sec. "Quadratic Assignment Problems", Koopmans-Beckmann form without the placement
 *    term): C(p) = sum_ij F_ij D_{p(i)p(j)}, F and D symmetric with zero diagonal. One step is
 *    n swap attempts; attempt a of step t draws Philox counter (a, t, r, TAG_QAP_STEP):
 *    u0 -> r = (u0 n)>>32, u1 -> s' = (u1 (n-1))>>32, s = s' + (s' >= r), u2 -> acceptance
 *    at bq = (bq_r[t] + bq_s[t]) >> 1.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TAG_KSAT_INIT 0x4B494E49u  /* "KINI" */
#define ORC_TAG_KSAT_SWEEP 0x4B535750u /* "KSWP" */
#define ORC_TAG_QAP_INIT 0x51494E49u   /* "QINI" */
#define ORC_TAG_QAP_STEP 0x51535450u   /* "QSTP" */
#define ORC_TAG_PT_SWAP 0x50545357u    /* "PTSW" */
#define ORC_TAG_CLUSTER 0x434C5354u    /* "CLST" */
#define ORC_FROZEN 0xFFFFFFFFu         /* Q16 value of beta = +infinity: the unit is held */
#define ORC_TAB_CAP 8192

/* ---------------------------------------------------------------------------------------
 * Philox4x32-10, from the published definition: ten rounds; each round multiplies counter
 * words 0 and 2 by 0xD2511F53 and 0xCD9E8D57 (64-bit products split into hi/lo), the new
 * words are (hi(c2*M1) ^ c1 ^ k0, lo(c2*M1), hi(c0*M0) ^ c3 ^ k1, lo(c0*M0)), and the key is
 * bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85 between rounds.
 * ------------------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

static uint32_t philox_word(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed,
                            int word) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[word];
}

/* ---------------------------------------------------------------------------------------
 * Acceptance thresholds and beta quantisation (the integer form of min(1, exp(-beta dE))).
 * ------------------------------------------------------------------------------------- */

/* Fills tab[0..cap) and returns L = the first j with floor(2^32 exp(-j/256)) = 0
 * (all entries from L on are zero), or -1 if cap is too small. */
int orc_threshold_table(uint32_t *tab, int cap) {
  for (int j = 0; j < cap; ++j) {
    double v = ldexp(exp(-(double)j / 256.0), 32);
    uint32_t t;
    if (v >= 4294967295.0)
      t = 0xFFFFFFFFu;
    else
      t = (uint32_t)floor(v);
    tab[j] = t;
    if (t == 0) {
      for (int q = j; q < cap; ++q) tab[q] = 0;
      return j;
    }
  }
  return -1;
}

/* beta in Q16: nearest integer to beta * 65536, ties to even. beta must be +infinity (frozen:
 * ORC_FROZEN), or finite, >= 0 and <= 65535 (the library rejects anything else). */
uint32_t orc_quantize_beta(float beta) {
  if (isinf(beta) && beta > 0) return ORC_FROZEN;
  double v = (double)beta * 65536.0;
  return (uint32_t)nearbyint(v);
}

typedef struct {
  uint32_t tab[ORC_TAB_CAP];
  int len;
} orc_table;

static void table_init(orc_table *t) { t->len = orc_threshold_table(t->tab, ORC_TAB_CAP); }

/* Returns 1 if an uphill move (dE > 0) with quantised beta bq is accepted by draw u. */
static int accept_uphill(const orc_table *t, uint32_t bq, int64_t dE, uint32_t u) {
  uint64_t idx = ((uint64_t)bq * (uint64_t)dE) >> 8;
  if (idx >= (uint64_t)t->len) return 0;
  return u < t->tab[idx];
}

/* The threshold the oracle compares a draw against, for tests of the acceptance rule. */
uint32_t orc_uphill_threshold(uint32_t bq, int64_t dE) {
  static orc_table tb;
  static int ready = 0;
  if (!ready) {
    table_init(&tb);
    ready = 1;
  }
  uint64_t idx = ((uint64_t)bq * (uint64_t)dE) >> 8;
  if (idx >= (uint64_t)tb.len) return 0;
  return tb.tab[idx];
}

/* ---------------------------------------------------------------------------------------
 * k-SAT: the formula, its energy, the single-flip energy change and the colouring.
 * ------------------------------------------------------------------------------------- */
typedef struct {
  int32_t n, m, kmax;
  const int32_t *lits; /* m*kmax DIMACS literals, 0 = unused slot */
  int32_t *inc_ptr;    /* n+1: clauses containing each variable */
  int32_t *inc;        /* clause ids */
} orc_cnf;

static int lit_var(int32_t l) { return (l > 0 ? l : -l) - 1; }
static int lit_true(int32_t l, const uint8_t *x) { return l > 0 ? x[lit_var(l)] : !x[lit_var(l)]; }

static void cnf_build(orc_cnf *f, int32_t n, int32_t m, int32_t kmax, const int32_t *lits) {
  f->n = n;
  f->m = m;
  f->kmax = kmax;
  f->lits = lits;
  f->inc_ptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
  for (int64_t a = 0; a < m; ++a)
    for (int q = 0; q < kmax; ++q) {
      int32_t l = lits[a * kmax + q];
      if (l != 0) f->inc_ptr[lit_var(l) + 1]++;
    }
  for (int v = 0; v < n; ++v) f->inc_ptr[v + 1] += f->inc_ptr[v];
  f->inc = (int32_t *)malloc(sizeof(int32_t) * ((size_t)f->inc_ptr[n] + 1));
  int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  memcpy(fill, f->inc_ptr, sizeof(int32_t) * (size_t)n);
  for (int64_t a = 0; a < m; ++a)
    for (int q = 0; q < kmax; ++q) {
      int32_t l = lits[a * kmax + q];
      if (l != 0) f->inc[fill[lit_var(l)]++] = (int32_t)a;
    }
  free(fill);
}

static void cnf_free(orc_cnf *f) {
  free(f->inc_ptr);
  free(f->inc);
}

static int clause_true_count(const orc_cnf *f, int64_t a, const uint8_t *x) {
  int c = 0;
  for (int q = 0; q < f->kmax; ++q) {
    int32_t l = f->lits[a * f->kmax + q];
    if (l != 0 && lit_true(l, x)) ++c;
  }
  return c;
}

/* E(x): the number of clauses with no true literal. */
int64_t orc_ksat_energy(int32_t n, int32_t m, int32_t kmax, const int32_t *lits,
                        const uint8_t *x) {
  (void)n;
  int64_t e = 0;
  for (int64_t a = 0; a < m; ++a) {
    int sat = 0;
    for (int q = 0; q < kmax; ++q) {
      int32_t l = lits[a * kmax + q];
      if (l != 0 && lit_true(l, x)) sat = 1;
    }
    if (!sat) ++e;
  }
  return e;
}

/* E of each of S assignments (rows of X, S x n uint8) into e[S]: orc_ksat_energy row by row. */
void orc_ksat_energies(int32_t n, int32_t m, int32_t kmax, const int32_t *lits, int64_t S,
                       const uint8_t *X, int64_t *e) {
  for (int64_t s = 0; s < S; ++s) e[s] = orc_ksat_energy(n, m, kmax, lits, X + s * n);
}

/* dE of flipping v, from the clauses that contain v: a clause whose only true literal is v's
 * becomes violated (+1); a violated clause becomes satisfied (-1). */
static int64_t cnf_delta(const orc_cnf *f, const uint8_t *x, int v) {
  int64_t d = 0;
  for (int32_t e = f->inc_ptr[v]; e < f->inc_ptr[v + 1]; ++e) {
    int64_t a = f->inc[e];
    int cnt = clause_true_count(f, a, x);
    int own = 0;
    for (int q = 0; q < f->kmax; ++q) {
      int32_t l = f->lits[a * f->kmax + q];
      if (l != 0 && lit_var(l) == v) own = lit_true(l, x);
    }
    if (own && cnt == 1) d += 1;
    if (cnt == 0) d -= 1;
  }
  return d;
}

int64_t orc_ksat_delta(int32_t n, int32_t m, int32_t kmax, const int32_t *lits,
                       const uint8_t *x, int32_t v) {
  orc_cnf f;
  cnf_build(&f, n, m, kmax, lits);
  int64_t d = cnf_delta(&f, x, v);
  cnf_free(&f);
  return d;
}

/* DSatur colouring. Neighbours of v: the variables sharing a clause with v. Saturation of an
 * uncoloured v: the number of distinct colours among its coloured neighbours. Each step picks
 * the uncoloured variable of largest saturation, then of most clause occurrences, then of
 * smallest id, and gives it the smallest colour held by none of its neighbours. The candidate
 * is found with a binary max-heap of (saturation, occurrences, -id) entries; an entry whose
 * saturation is out of date (the variable's saturation rose after it was pushed) or whose
 * variable is coloured is dropped when it surfaces, so the top valid entry is always the
 * variable the rule picks. Returns the number of colours. */
typedef struct {
  int32_t sat, deg, v;
} col_entry;

static int col_before(col_entry a, col_entry b) { /* a is picked before b */
  if (a.sat != b.sat) return a.sat > b.sat;
  if (a.deg != b.deg) return a.deg > b.deg;
  return a.v < b.v;
}

static void heap_push(col_entry *h, int64_t *len, col_entry e) {
  int64_t i = (*len)++;
  h[i] = e;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (!col_before(h[i], h[p])) break;
    col_entry t = h[i];
    h[i] = h[p];
    h[p] = t;
    i = p;
  }
}

static col_entry heap_pop(col_entry *h, int64_t *len) {
  col_entry top = h[0];
  h[0] = h[--(*len)];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, b = i;
    if (l < *len && col_before(h[l], h[b])) b = l;
    if (r < *len && col_before(h[r], h[b])) b = r;
    if (b == i) break;
    col_entry t = h[i];
    h[i] = h[b];
    h[b] = t;
    i = b;
  }
  return top;
}

static int32_t cnf_colour(const orc_cnf *f, int32_t *colour) {
  const int32_t n = f->n;
  /* a colour never exceeds a variable's count of neighbour slots, so `bound` colours suffice */
  int64_t slots_max = 0, slots_all = 0;
  for (int v = 0; v < n; ++v) {
    int64_t s = 0;
    for (int32_t e = f->inc_ptr[v]; e < f->inc_ptr[v + 1]; ++e) {
      int64_t a = f->inc[e];
      for (int q = 0; q < f->kmax; ++q)
        if (f->lits[a * f->kmax + q] != 0) ++s;
      --s; /* v itself */
    }
    if (s > slots_max) slots_max = s;
    slots_all += s;
  }
  const int64_t bound = slots_max + 1, words = (bound + 63) / 64;
  uint64_t *seen = (uint64_t *)calloc((size_t)n * (size_t)words, sizeof(uint64_t)); /* colours next to v */
  int32_t *sat = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
  col_entry *heap = (col_entry *)malloc(sizeof(col_entry) * (size_t)(n + slots_all + 1));
  int64_t len = 0;
  int32_t ncol = 0;
  for (int v = 0; v < n; ++v) {
    colour[v] = -1;
    col_entry e = {0, f->inc_ptr[v + 1] - f->inc_ptr[v], v};
    heap_push(heap, &len, e);
  }
  while (len > 0) {
    col_entry e = heap_pop(heap, &len);
    const int v = e.v;
    if (colour[v] >= 0 || e.sat != sat[v]) continue; /* coloured, or an out-of-date entry */
    int32_t c = 0;
    while (seen[(size_t)v * words + c / 64] >> (c % 64) & 1u) ++c;
    colour[v] = c;
    if (c + 1 > ncol) ncol = c + 1;
    for (int32_t i = f->inc_ptr[v]; i < f->inc_ptr[v + 1]; ++i) {
      int64_t a = f->inc[i];
      for (int q = 0; q < f->kmax; ++q) {
        int32_t l = f->lits[a * f->kmax + q];
        if (l == 0) continue;
        int u = lit_var(l);
        if (u == v || colour[u] >= 0) continue;
        uint64_t *w = &seen[(size_t)u * words + c / 64];
        if (*w >> (c % 64) & 1u) continue;
        *w |= (uint64_t)1 << (c % 64);
        col_entry g = {++sat[u], f->inc_ptr[u + 1] - f->inc_ptr[u], u};
        heap_push(heap, &len, g);
      }
    }
  }
  free(seen);
  free(sat);
  free(heap);
  return ncol;
}

int32_t orc_ksat_colour(int32_t n, int32_t m, int32_t kmax, const int32_t *lits,
                        int32_t *colour) {
  orc_cnf f;
  cnf_build(&f, n, m, kmax, lits);
  int32_t c = cnf_colour(&f, colour);
  cnf_free(&f);
  return c;
}

/* ---------------------------------------------------------------------------------------
 * k-SAT anneal: replicas are independent chains; host threads split replicas only.
 * ------------------------------------------------------------------------------------- */
typedef struct {
  const orc_cnf *f;
  const orc_table *tab;
  const int32_t *order; /* variables in sweep order: colour-major, id-minor */
  const uint32_t *bq;   /* n * n_steps, Q16 */
  int32_t n_steps, t0, t1;
  uint64_t seed;
  const int32_t *rep_ids; /* nr replica ids */
  int32_t nr;
  const uint8_t *init;      /* nr*n or NULL */
  const uint8_t *init_best; /* nr*n or NULL (continue a chain: best so far) */
  const int64_t *init_best_e;
  uint8_t *final_states;
  int64_t *energies, *best_energies;
  uint8_t *best_states;
  int32_t stats_t0;
  int64_t *e_sum, *e_sq; /* nr each or NULL */
  int32_t j_begin, j_end;
} ksat_job;

static void ksat_one_replica(const ksat_job *J, int32_t j) {
  const orc_cnf *f = J->f;
  int32_t n = f->n;
  uint32_t r = (uint32_t)J->rep_ids[j];
  uint8_t *x = (uint8_t *)malloc((size_t)n + 1);
  uint8_t *best = (uint8_t *)malloc((size_t)n + 1);
  if (J->init) {
    memcpy(x, J->init + (size_t)j * n, (size_t)n);
  } else {
    for (int v = 0; v < n; ++v)
      x[v] = (uint8_t)(philox_word((uint32_t)v, 0u, r >> 2, ORC_TAG_KSAT_INIT, J->seed, r & 3) & 1u);
  }
  int64_t e = orc_ksat_energy(n, f->m, f->kmax, f->lits, x);
  int64_t best_e;
  if (J->init_best) {
    memcpy(best, J->init_best + (size_t)j * n, (size_t)n);
    best_e = J->init_best_e[j];
  } else {
    memcpy(best, x, (size_t)n);
    best_e = e;
  }
  for (int32_t t = J->t0; t < J->t1; ++t) {
    for (int32_t p = 0; p < n; ++p) {
      int v = J->order[p];
      const uint32_t bqv = J->bq[(size_t)v * J->n_steps + t];
      if (bqv == ORC_FROZEN) continue;
      int64_t d = cnf_delta(f, x, v);
      int acc;
      if (d <= 0) {
        acc = 1;
      } else {
        uint32_t u = philox_word((uint32_t)v, (uint32_t)t, r >> 2, ORC_TAG_KSAT_SWEEP, J->seed, r & 3);
        acc = accept_uphill(J->tab, bqv, d, u);
      }
      if (acc) {
        x[v] ^= 1u;
        e += d;
      }
    }
    if (e < best_e) {
      best_e = e;
      memcpy(best, x, (size_t)n);
    }
    if (J->e_sum && t >= J->stats_t0) {
      J->e_sum[j] += e;
      J->e_sq[j] += e * e;
    }
  }
  if (J->final_states) memcpy(J->final_states + (size_t)j * n, x, (size_t)n);
  if (J->energies) J->energies[j] = e;
  if (J->best_energies) J->best_energies[j] = best_e;
  if (J->best_states) memcpy(J->best_states + (size_t)j * n, best, (size_t)n);
  free(x);
  free(best);
}

static void *ksat_worker(void *arg) {
  const ksat_job *J = (const ksat_job *)arg;
  for (int32_t j = J->j_begin; j < J->j_end; ++j) ksat_one_replica(J, j);
  return NULL;
}

/*
 * Runs sweeps t0..t1-1 for nr replicas (ids rep_ids, or 0..nr-1 if NULL).
 * beta: n * n_steps float32, row v = schedule of variable v. init: nr*n uint8 (NULL = Philox
 * initial state). init_best/init_best_e continue a chain's best-so-far (both NULL = fresh).
 * e_sum/e_sq (nr each, zeroed here, or NULL): energy statistics of sweeps t >= stats_t0.
 * Outputs may be NULL. Returns 0, or -1 on a bad argument.
 */
int orc_ksat_anneal(int32_t n, int32_t m, int32_t kmax, const int32_t *lits, int32_t n_steps,
                    const float *beta, int32_t nr, const int32_t *rep_ids, int32_t t0, int32_t t1,
                    uint64_t seed, const uint8_t *init, const uint8_t *init_best,
                    const int64_t *init_best_e, int32_t n_threads, uint8_t *final_states,
                    int64_t *energies, int64_t *best_energies, uint8_t *best_states,
                    int32_t stats_t0, int64_t *e_sum, int64_t *e_sq) {
  if (n <= 0 || m < 0 || kmax <= 0 || t0 < 0 || t1 < t0 || t1 > n_steps || nr < 0) return -1;
  orc_cnf f;
  cnf_build(&f, n, m, kmax, lits);
  orc_table tab;
  table_init(&tab);
  int32_t *colour = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t ncol = cnf_colour(&f, colour);
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t p = 0;
  for (int32_t c = 0; c < ncol; ++c)
    for (int32_t v = 0; v < n; ++v)
      if (colour[v] == c) order[p++] = v;
  uint32_t *bq = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n * (size_t)n_steps);
  for (size_t i = 0; i < (size_t)n * (size_t)n_steps; ++i) bq[i] = orc_quantize_beta(beta[i]);
  int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nr + 1));
  for (int32_t j = 0; j < nr; ++j) ids[j] = rep_ids ? rep_ids[j] : j;

  if (n_threads < 1) n_threads = 1;
  if (n_threads > nr) n_threads = nr > 0 ? nr : 1;
  if (e_sum && e_sq) {
    memset(e_sum, 0, sizeof(int64_t) * (size_t)nr);
    memset(e_sq, 0, sizeof(int64_t) * (size_t)nr);
  } else {
    e_sum = e_sq = NULL;
  }
  ksat_job *jobs = (ksat_job *)calloc((size_t)n_threads, sizeof(ksat_job));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  for (int w = 0; w < n_threads; ++w) {
    ksat_job *J = &jobs[w];
    J->f = &f;
    J->tab = &tab;
    J->order = order;
    J->bq = bq;
    J->n_steps = n_steps;
    J->t0 = t0;
    J->t1 = t1;
    J->seed = seed;
    J->rep_ids = ids;
    J->nr = nr;
    J->init = init;
    J->init_best = init_best;
    J->init_best_e = init_best_e;
    J->final_states = final_states;
    J->energies = energies;
    J->best_energies = best_energies;
    J->best_states = best_states;
    J->stats_t0 = stats_t0;
    J->e_sum = e_sum;
    J->e_sq = e_sq;
    J->j_begin = (int32_t)((int64_t)nr * w / n_threads);
    J->j_end = (int32_t)((int64_t)nr * (w + 1) / n_threads);
  }
  for (int w = 1; w < n_threads; ++w) pthread_create(&th[w], NULL, ksat_worker, &jobs[w]);
  ksat_worker(&jobs[0]);
  for (int w = 1; w < n_threads; ++w) pthread_join(th[w], NULL);
  free(jobs);
  free(th);
  free(ids);
  free(bq);
  free(order);
  free(colour);
  cnf_free(&f);
  return 0;
}


/* ---------------------------------------------------------------------------------------
 * k-SAT with replica exchange (single-threaded: the exchange rounds couple the replicas).
 * ------------------------------------------------------------------------------------- */
/*
 * Runs sweeps t0..t1-1 of R = G * L replicas with exchange rounds every S sweeps. ladder: L
 * floats (slot temperatures, multiplied into the per-variable schedule). slots: R int32 in/out
 * (the slot of each replica within its ladder; a permutation of 0..L-1 per ladder).
 * init/init_best/init_best_e as orc_ksat_anneal (init NULL = Philox initial states). Returns 0
 * or -1 on a bad argument.
 */
int orc_ksat_pt_anneal(int32_t n, int32_t m, int32_t kmax, const int32_t *lits, int32_t n_steps,
                       const float *beta, int32_t R, int32_t L, const float *ladder,
                       int32_t *slots, int32_t t0, int32_t t1, int32_t S, uint64_t seed,
                       const uint8_t *init, const uint8_t *init_best, const int64_t *init_best_e,
                       uint8_t *final_states, int64_t *energies, int64_t *best_energies,
                       uint8_t *best_states) {
  if (n <= 0 || m < 0 || kmax <= 0 || t0 < 0 || t1 < t0 || t1 > n_steps || R <= 0 || S <= 0 ||
      L <= 0 || R % L != 0)
    return -1;
  const int32_t G = R / L;
  orc_cnf f;
  cnf_build(&f, n, m, kmax, lits);
  orc_table tab;
  table_init(&tab);
  int32_t *colour = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t ncol = cnf_colour(&f, colour);
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t p = 0;
  for (int32_t c = 0; c < ncol; ++c)
    for (int32_t v = 0; v < n; ++v)
      if (colour[v] == c) order[p++] = v;
  uint32_t *bq = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n * (size_t)n_steps);
  for (size_t i = 0; i < (size_t)n * (size_t)n_steps; ++i) bq[i] = orc_quantize_beta(beta[i]);
  uint32_t *lq = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)L);
  for (int32_t k = 0; k < L; ++k) lq[k] = orc_quantize_beta(ladder[k]);
  int32_t *at = (int32_t *)malloc(sizeof(int32_t) * (size_t)R); /* at[g*L + k]: replica at slot k */
  for (int32_t r = 0; r < R; ++r) at[(r / L) * L + slots[r]] = r;
  uint8_t *x = (uint8_t *)malloc((size_t)R * n);
  uint8_t *best = (uint8_t *)malloc((size_t)R * n);
  int64_t *e = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);
  int64_t *be = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);
  for (int32_t r = 0; r < R; ++r) {
    uint8_t *xr = x + (size_t)r * n;
    if (init)
      memcpy(xr, init + (size_t)r * n, (size_t)n);
    else
      for (int v = 0; v < n; ++v)
        xr[v] = (uint8_t)(philox_word((uint32_t)v, 0u, (uint32_t)r >> 2, ORC_TAG_KSAT_INIT, seed, r & 3) & 1u);
    e[r] = orc_ksat_energy(n, m, kmax, lits, xr);
    if (init_best) {
      memcpy(best + (size_t)r * n, init_best + (size_t)r * n, (size_t)n);
      be[r] = init_best_e[r];
    } else {
      memcpy(best + (size_t)r * n, xr, (size_t)n);
      be[r] = e[r];
    }
  }
  for (int32_t t = t0; t < t1; ++t) {
    for (int32_t r = 0; r < R; ++r) {
      uint8_t *xr = x + (size_t)r * n;
      const uint64_t mult = lq[slots[r]];
      for (int32_t q = 0; q < n; ++q) {
        const int v = order[q];
        if (bq[(size_t)v * n_steps + t] == ORC_FROZEN) continue;
        const int64_t d = cnf_delta(&f, xr, v);
        int acc;
        if (d <= 0) {
          acc = 1;
        } else {
          uint64_t b = (mult * (uint64_t)bq[(size_t)v * n_steps + t]) >> 16;
          if (b > 0xFFFFFFFFull) b = 0xFFFFFFFFull;
          const uint32_t u = philox_word((uint32_t)v, (uint32_t)t, (uint32_t)r >> 2, ORC_TAG_KSAT_SWEEP, seed, r & 3);
          acc = accept_uphill(&tab, (uint32_t)b, d, u);
        }
        if (acc) {
          xr[v] ^= 1u;
          e[r] += d;
        }
      }
      if (e[r] < be[r]) {
        be[r] = e[r];
        memcpy(best + (size_t)r * n, xr, (size_t)n);
      }
    }
    if ((t + 1) % S == 0) {
      const uint32_t round = (uint32_t)((t + 1) / S - 1);
      for (int32_t g = 0; g < G; ++g) {
        int32_t *atg = at + (size_t)g * L;
        for (int32_t k = (int32_t)(round & 1u); k + 1 < L; k += 2) {
          const int32_t a = atg[k], b = atg[k + 1];
          const int64_t d = ((int64_t)lq[k] - (int64_t)lq[k + 1]) * (e[a] - e[b]);
          int acc = 1;
          if (d < 0) {
            const uint64_t idx = ((uint64_t)(-d)) >> 8;
            const uint32_t u = philox_word((uint32_t)k, round, (uint32_t)g, ORC_TAG_PT_SWAP, seed, 0);
            acc = idx < (uint64_t)tab.len && u < tab.tab[idx];
          }
          if (acc) {
            atg[k] = b;
            atg[k + 1] = a;
            slots[a] = k + 1;
            slots[b] = k;
          }
        }
      }
    }
  }
  if (final_states) memcpy(final_states, x, (size_t)R * n);
  if (best_states) memcpy(best_states, best, (size_t)R * n);
  for (int32_t r = 0; r < R; ++r) {
    if (energies) energies[r] = e[r];
    if (best_energies) best_energies[r] = be[r];
  }
  free(x);
  free(best);
  free(e);
  free(be);
  free(at);
  free(lq);
  free(bq);
  free(order);
  free(colour);
  cnf_free(&f);
  return 0;
}

/* ---------------------------------------------------------------------------------------
 * QAP (Koopmans-Beckmann, symmetric F and D with zero diagonal).
 * ------------------------------------------------------------------------------------- */

/* C(p) = sum_{i,j} F_ij D_{p(i) p(j)} */
int64_t orc_qap_cost(int32_t n, const int32_t *F, const int32_t *D, const int16_t *p) {
  int64_t c = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) c += (int64_t)F[i * n + j] * (int64_t)D[p[i] * n + p[j]];
  return c;
}

/* Change of C when facilities r and s exchange locations (r != s). With F, D symmetric and
 * zero-diagonal only the rows r and s change: 2 sum_{k != r,s} (F_rk - F_sk)(D_{p(s)p(k)} -
 * D_{p(r)p(k)}). */
int64_t orc_qap_swap_delta(int32_t n, const int32_t *F, const int32_t *D, const int16_t *p,
                           int32_t r, int32_t s) {
  int64_t acc = 0;
  for (int k = 0; k < n; ++k) {
    if (k == r || k == s) continue;
    int64_t df = (int64_t)F[r * n + k] - (int64_t)F[s * n + k];
    int64_t dd = (int64_t)D[p[s] * n + p[k]] - (int64_t)D[p[r] * n + p[k]];
    acc += df * dd;
  }
  return 2 * acc;
}

typedef struct {
  int32_t n;
  const int32_t *F, *D;
  const orc_table *tab;
  const uint32_t *bq;
  int32_t n_steps, t0, t1;
  uint64_t seed;
  const int32_t *rep_ids;
  const int16_t *init, *init_best;
  const int64_t *init_best_e;
  int16_t *final_perms, *best_perms;
  int64_t *energies, *best_energies;
  int32_t stats_t0;
  double *e_sum, *e_sq; /* nr each or NULL: sums of E and E^2 (double, step order) */
  int32_t j_begin, j_end;
} qap_job;

static void qap_one_replica(const qap_job *J, int32_t j) {
  int32_t n = J->n;
  uint32_t r = (uint32_t)J->rep_ids[j];
  int16_t *p = (int16_t *)malloc(sizeof(int16_t) * ((size_t)n + 1));
  int16_t *best = (int16_t *)malloc(sizeof(int16_t) * ((size_t)n + 1));
  if (J->init) {
    memcpy(p, J->init + (size_t)j * n, sizeof(int16_t) * (size_t)n);
  } else {
    /* Fisher-Yates from the identity: for q = n-1..1 exchange q with (u (q+1)) >> 32. */
    for (int q = 0; q < n; ++q) p[q] = (int16_t)q;
    for (int q = n - 1; q >= 1; --q) {
      uint32_t u = philox_word((uint32_t)q, 0u, r, ORC_TAG_QAP_INIT, J->seed, 0);
      int kk = (int)(((uint64_t)u * (uint64_t)(q + 1)) >> 32);
      int16_t tmp = p[q];
      p[q] = p[kk];
      p[kk] = tmp;
    }
  }
  int64_t e = orc_qap_cost(n, J->F, J->D, p);
  int64_t best_e;
  if (J->init_best) {
    memcpy(best, J->init_best + (size_t)j * n, sizeof(int16_t) * (size_t)n);
    best_e = J->init_best_e[j];
  } else {
    memcpy(best, p, sizeof(int16_t) * (size_t)n);
    best_e = e;
  }
  for (int32_t t = J->t0; t < J->t1; ++t) {
    if (n >= 2) {
      for (int32_t a = 0; a < n; ++a) {
        uint32_t ctr[4] = {(uint32_t)a, (uint32_t)t, r, ORC_TAG_QAP_STEP};
        uint32_t key[2] = {(uint32_t)J->seed, (uint32_t)(J->seed >> 32)};
        uint32_t u[4];
        orc_philox4x32_10(ctr, key, u);
        int32_t fr = (int32_t)(((uint64_t)u[0] * (uint64_t)n) >> 32);
        int32_t fs = (int32_t)(((uint64_t)u[1] * (uint64_t)(n - 1)) >> 32);
        if (fs >= fr) fs += 1;
        if (J->bq[(size_t)fr * J->n_steps + t] == ORC_FROZEN ||
            J->bq[(size_t)fs * J->n_steps + t] == ORC_FROZEN)
          continue;
        int64_t d = orc_qap_swap_delta(n, J->F, J->D, p, fr, fs);
        int acc;
        if (d <= 0) {
          acc = 1;
        } else {
          uint32_t bq = (uint32_t)(((uint64_t)J->bq[(size_t)fr * J->n_steps + t] +
                                    (uint64_t)J->bq[(size_t)fs * J->n_steps + t]) >> 1);
          acc = accept_uphill(J->tab, bq, d, u[2]);
        }
        if (acc) {
          int16_t tmp = p[fr];
          p[fr] = p[fs];
          p[fs] = tmp;
          e += d;
        }
      }
    }
    if (e < best_e) {
      best_e = e;
      memcpy(best, p, sizeof(int16_t) * (size_t)n);
    }
    if (J->e_sum && t >= J->stats_t0) {
      J->e_sum[j] += (double)e;
      J->e_sq[j] += (double)e * (double)e;
    }
  }
  if (J->final_perms) memcpy(J->final_perms + (size_t)j * n, p, sizeof(int16_t) * (size_t)n);
  if (J->energies) J->energies[j] = e;
  if (J->best_energies) J->best_energies[j] = best_e;
  if (J->best_perms) memcpy(J->best_perms + (size_t)j * n, best, sizeof(int16_t) * (size_t)n);
  free(p);
  free(best);
}

static void *qap_worker(void *arg) {
  const qap_job *J = (const qap_job *)arg;
  for (int32_t j = J->j_begin; j < J->j_end; ++j) qap_one_replica(J, j);
  return NULL;
}

/* Runs steps t0..t1-1 of the QAP swap chain for nr replicas; arguments as orc_ksat_anneal,
 * with int16 permutations p[facility] = location. e_sum / e_sq (nr doubles each, or NULL):
 * per replica, the end-of-step costs of steps t >= stats_t0 added in step order in double
 * (costs reach 2^33, their squares 2^66). */
int orc_qap_anneal(int32_t n, const int32_t *F, const int32_t *D, int32_t n_steps,
                   const float *beta, int32_t nr, const int32_t *rep_ids, int32_t t0, int32_t t1,
                   uint64_t seed, const int16_t *init, const int16_t *init_best,
                   const int64_t *init_best_e, int32_t n_threads, int16_t *final_perms,
                   int64_t *energies, int64_t *best_energies, int16_t *best_perms,
                   int32_t stats_t0, double *e_sum, double *e_sq) {
  if (n <= 0 || t0 < 0 || t1 < t0 || t1 > n_steps || nr < 0) return -1;
  if (e_sum && e_sq) {
    for (int32_t j = 0; j < nr; ++j) e_sum[j] = e_sq[j] = 0.0;
  } else {
    e_sum = e_sq = NULL;
  }
  orc_table tab;
  table_init(&tab);
  uint32_t *bq = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n * (size_t)n_steps);
  for (size_t i = 0; i < (size_t)n * (size_t)n_steps; ++i) bq[i] = orc_quantize_beta(beta[i]);
  int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nr + 1));
  for (int32_t j = 0; j < nr; ++j) ids[j] = rep_ids ? rep_ids[j] : j;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > nr) n_threads = nr > 0 ? nr : 1;
  qap_job *jobs = (qap_job *)calloc((size_t)n_threads, sizeof(qap_job));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  for (int w = 0; w < n_threads; ++w) {
    qap_job *J = &jobs[w];
    J->n = n;
    J->F = F;
    J->D = D;
    J->tab = &tab;
    J->bq = bq;
    J->n_steps = n_steps;
    J->t0 = t0;
    J->t1 = t1;
    J->seed = seed;
    J->rep_ids = ids;
    J->init = init;
    J->init_best = init_best;
    J->init_best_e = init_best_e;
    J->final_perms = final_perms;
    J->best_perms = best_perms;
    J->energies = energies;
    J->best_energies = best_energies;
    J->stats_t0 = stats_t0;
    J->e_sum = e_sum;
    J->e_sq = e_sq;
    J->j_begin = (int32_t)((int64_t)nr * w / n_threads);
    J->j_end = (int32_t)((int64_t)nr * (w + 1) / n_threads);
  }
  for (int w = 1; w < n_threads; ++w) pthread_create(&th[w], NULL, qap_worker, &jobs[w]);
  qap_worker(&jobs[0]);
  for (int w = 1; w < n_threads; ++w) pthread_join(th[w], NULL);
  free(jobs);
  free(th);
  free(ids);
  free(bq);
  return 0;
}

/* ---------------------------------------------------------------------------------------
 * Collective (cluster) move on R k-SAT replicas.
 * ------------------------------------------------------------------------------------- */
/*
 * states: R*n uint8 in/out; energies, best_energies: R int64 in/out; best_states: R*n in/out.
 * mask: mask_rows*n uint8 (mask_rows 1: one mask for all replicas, or R). beta: R floats.
 * accepted: R uint8 out (nullable). rep_ids: the replica id of each row, which picks its Philox
 * stream (NULL = 0..R-1). Row r of a per-replica mask belongs to row r of the states, like beta[r],
 * whatever its id. Returns 0 or -1 on a bad argument.
 */
int orc_ksat_cluster_flip(int32_t n, int32_t m, int32_t kmax, const int32_t *lits, int32_t R,
                          uint8_t *states, int64_t *energies, uint8_t *best_states,
                          int64_t *best_energies, int32_t mask_rows, const uint8_t *mask,
                          const float *beta, uint32_t move_id, uint64_t seed, uint8_t *accepted,
                          const int32_t *rep_ids) {
  if (n <= 0 || m < 0 || kmax <= 0 || R <= 0 || (mask_rows != 1 && mask_rows != R)) return -1;
  orc_table tab;
  table_init(&tab);
  uint8_t *y = (uint8_t *)malloc((size_t)n);
  for (int32_t r = 0; r < R; ++r) {
    const uint32_t id = rep_ids ? (uint32_t)rep_ids[r] : (uint32_t)r;
    uint8_t *x = states + (size_t)r * n;
    const uint8_t *mr = mask + (size_t)(mask_rows == 1 ? 0 : r) * n;
    for (int32_t v = 0; v < n; ++v) y[v] = (uint8_t)(x[v] ^ (mr[v] & 1u));
    const int64_t e0 = orc_ksat_energy(n, m, kmax, lits, x);
    const int64_t e1 = orc_ksat_energy(n, m, kmax, lits, y);
    const int64_t d = e1 - e0;
    int acc = 1;
    if (d > 0) {
      const uint32_t u = philox_word(move_id, 0u, id >> 2, ORC_TAG_CLUSTER, seed, (int)(id & 3u));
      acc = accept_uphill(&tab, orc_quantize_beta(beta[r]), d, u);
    }
    if (acc) {
      memcpy(x, y, (size_t)n);
      energies[r] = e1;
      if (e1 < best_energies[r]) {
        best_energies[r] = e1;
        memcpy(best_states + (size_t)r * n, x, (size_t)n);
      }
    } else {
      energies[r] = e0;
    }
    if (accepted) accepted[r] = (uint8_t)acc;
  }
  free(y);
  return 0;
}

/* ---------------------------------------------------------------------------------------
 * Whitening (Sec. "Whitening procedure for low energy states").
 * ------------------------------------------------------------------------------------- */
/*
 * Variables are inspected one at a time, in id order, repeatedly until a whole pass marks
 * nothing new. Variable v becomes white (star) when no clause containing it blocks it. A clause
 * blocks v when it is neither satisfied by another of its variables nor holds another white
 * variable; with `generalized` (the paper's extension to low-energy states) a clause only blocks v
 * when it is moreover satisfied by v itself, so violated clauses never report a frozen variable.
 * frozen: n uint8 out (1 = not white at the fixed point). Returns the number of frozen variables.
 */
int32_t orc_ksat_whitening(int32_t n, int32_t m, int32_t kmax, const int32_t *lits,
                           const uint8_t *x, int32_t generalized, uint8_t *frozen) {
  orc_cnf f;
  cnf_build(&f, n, m, kmax, lits);
  uint8_t *star = (uint8_t *)calloc((size_t)n + 1, 1);
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int32_t v = 0; v < n; ++v) {
      if (star[v]) continue;
      int blocked = 0;
      for (int32_t e = f.inc_ptr[v]; e < f.inc_ptr[v + 1] && !blocked; ++e) {
        const int64_t a = f.inc[e];
        int other_true = 0, other_star = 0, own_true = 0;
        for (int q = 0; q < kmax; ++q) {
          const int32_t l = lits[a * kmax + q];
          if (l == 0) continue;
          const int u = lit_var(l);
          if (u == v) {
            own_true = lit_true(l, x);
          } else {
            if (lit_true(l, x)) other_true = 1;
            if (star[u]) other_star = 1;
          }
        }
        if (!other_true && !other_star && (own_true || !generalized)) blocked = 1;
      }
      if (!blocked) {
        star[v] = 1;
        changed = 1;
      }
    }
  }
  int32_t cnt = 0;
  for (int32_t v = 0; v < n; ++v) {
    frozen[v] = (uint8_t)(star[v] ? 0 : 1);
    cnt += frozen[v];
  }
  free(star);
  cnf_free(&f);
  return cnt;
}

/* ---------------------------------------------------------------------------------------
 * QAP with replica exchange (single-threaded: the exchange rounds couple the replicas).
 * ------------------------------------------------------------------------------------- */
/*
 * As orc_ksat_pt_anneal for the QAP swap chain: R = G * L replicas, replica g*L + i in ladder
 * g, slot s(r) with Q16 temperature lq[s]; an uphill swap of replica r is tested at
 * min(2^32-1, (lq[s(r)] * ((bq_r[t] + bq_s[t]) >> 1)) >> 16). Exchange rounds as for k-SAT, with
 * the product (lq[k] - lq[k+1]) (E_a - E_b) formed exactly in 128 bits (QAP costs reach 2^33).
 */
int orc_qap_pt_anneal(int32_t n, const int32_t *F, const int32_t *D, int32_t n_steps,
                      const float *beta, int32_t R, int32_t L, const float *ladder,
                      int32_t *slots, int32_t t0, int32_t t1, int32_t S, uint64_t seed,
                      const int16_t *init, const int16_t *init_best, const int64_t *init_best_e,
                      int16_t *final_perms, int64_t *energies, int64_t *best_energies,
                      int16_t *best_perms) {
  if (n <= 0 || t0 < 0 || t1 < t0 || t1 > n_steps || R <= 0 || S <= 0 || L <= 0 || R % L != 0)
    return -1;
  const int32_t G = R / L;
  orc_table tab;
  table_init(&tab);
  uint32_t *bq = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n * (size_t)n_steps);
  for (size_t i = 0; i < (size_t)n * (size_t)n_steps; ++i) bq[i] = orc_quantize_beta(beta[i]);
  uint32_t *lq = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)L);
  for (int32_t k = 0; k < L; ++k) lq[k] = orc_quantize_beta(ladder[k]);
  int32_t *at = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
  for (int32_t r = 0; r < R; ++r) at[(r / L) * L + slots[r]] = r;
  int16_t *p = (int16_t *)malloc(sizeof(int16_t) * (size_t)R * n);
  int16_t *best = (int16_t *)malloc(sizeof(int16_t) * (size_t)R * n);
  int64_t *e = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);
  int64_t *be = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int32_t r = 0; r < R; ++r) {
    int16_t *pr = p + (size_t)r * n;
    if (init) {
      memcpy(pr, init + (size_t)r * n, sizeof(int16_t) * (size_t)n);
    } else {
      for (int q = 0; q < n; ++q) pr[q] = (int16_t)q;
      for (int q = n - 1; q >= 1; --q) {
        const uint32_t u = philox_word((uint32_t)q, 0u, (uint32_t)r, ORC_TAG_QAP_INIT, seed, 0);
        const int kk = (int)(((uint64_t)u * (uint64_t)(q + 1)) >> 32);
        const int16_t tmp = pr[q];
        pr[q] = pr[kk];
        pr[kk] = tmp;
      }
    }
    e[r] = orc_qap_cost(n, F, D, pr);
    if (init_best) {
      memcpy(best + (size_t)r * n, init_best + (size_t)r * n, sizeof(int16_t) * (size_t)n);
      be[r] = init_best_e[r];
    } else {
      memcpy(best + (size_t)r * n, pr, sizeof(int16_t) * (size_t)n);
      be[r] = e[r];
    }
  }
  for (int32_t t = t0; t < t1; ++t) {
    for (int32_t r = 0; r < R && n >= 2; ++r) {
      int16_t *pr = p + (size_t)r * n;
      const uint64_t mult = lq[slots[r]];
      for (int32_t a = 0; a < n; ++a) {
        const uint32_t ctr[4] = {(uint32_t)a, (uint32_t)t, (uint32_t)r, ORC_TAG_QAP_STEP};
        uint32_t u[4];
        orc_philox4x32_10(ctr, key, u);
        const int32_t fr = (int32_t)(((uint64_t)u[0] * (uint64_t)n) >> 32);
        int32_t fs = (int32_t)(((uint64_t)u[1] * (uint64_t)(n - 1)) >> 32);
        if (fs >= fr) fs += 1;
        const uint32_t br = bq[(size_t)fr * n_steps + t], bs = bq[(size_t)fs * n_steps + t];
        if (br == ORC_FROZEN || bs == ORC_FROZEN) continue;
        const int64_t d = orc_qap_swap_delta(n, F, D, pr, fr, fs);
        int acc = 1;
        if (d > 0) {
          uint64_t b = (mult * (((uint64_t)br + (uint64_t)bs) >> 1)) >> 16;
          if (b > 0xFFFFFFFFull) b = 0xFFFFFFFFull;
          acc = accept_uphill(&tab, (uint32_t)b, d, u[2]);
        }
        if (acc) {
          const int16_t tmp = pr[fr];
          pr[fr] = pr[fs];
          pr[fs] = tmp;
          e[r] += d;
        }
      }
      if (e[r] < be[r]) {
        be[r] = e[r];
        memcpy(best + (size_t)r * n, pr, sizeof(int16_t) * (size_t)n);
      }
    }
    if ((t + 1) % S == 0) {
      const uint32_t round = (uint32_t)((t + 1) / S - 1);
      for (int32_t g = 0; g < G; ++g) {
        int32_t *atg = at + (size_t)g * L;
        for (int32_t k = (int32_t)(round & 1u); k + 1 < L; k += 2) {
          const int32_t a = atg[k], b = atg[k + 1];
          const __int128 dd = (__int128)((int64_t)lq[k] - (int64_t)lq[k + 1]) * (__int128)(e[a] - e[b]);
          int acc = 1;
          if (dd < 0) {
            const __int128 idx = (-dd) >> 8;
            const uint32_t u = philox_word((uint32_t)k, round, (uint32_t)g, ORC_TAG_PT_SWAP, seed, 0);
            acc = idx < (__int128)tab.len && u < tab.tab[(size_t)idx];
          }
          if (acc) {
            atg[k] = b;
            atg[k + 1] = a;
            slots[a] = k + 1;
            slots[b] = k;
          }
        }
      }
    }
  }
  if (final_perms) memcpy(final_perms, p, sizeof(int16_t) * (size_t)R * n);
  if (best_perms) memcpy(best_perms, best, sizeof(int16_t) * (size_t)R * n);
  for (int32_t r = 0; r < R; ++r) {
    if (energies) energies[r] = e[r];
    if (best_energies) best_energies[r] = be[r];
  }
  free(p);
  free(best);
  free(e);
  free(be);
  free(at);
  free(lq);
  free(bq);
  return 0;
}
