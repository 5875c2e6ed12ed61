// Internal declarations shared by the translation units of libnmc (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <new>
#include <string>
#include <utility>
#include <vector>

struct nmc_ctx;

namespace nmc {

// Philox counter tags (word 3 of the counter) that separate the streams of the chain.
constexpr uint32_t kTagKsatInit = 0x4B494E49u;
constexpr uint32_t kTagKsatSweep = 0x4B535750u;
constexpr uint32_t kTagQapInit = 0x51494E49u;
constexpr uint32_t kTagQapStep = 0x51535450u;
constexpr uint32_t kTagPtSwap = 0x50545357u;
constexpr uint32_t kTagCluster = 0x434C5354u;
// Q16 schedule entry of beta = +infinity: the unit is held fixed at that step (a frozen
// variable is not attempted; a QAP swap involving a frozen facility is rejected).
constexpr uint32_t kFrozenQ16 = 0xFFFFFFFFu;

constexpr int kTabCap = 8192;    // capacity of the acceptance-threshold table
constexpr int kMaxReplicas = 4096;
constexpr int kMaxDegree = 1023; // occurrences of one variable (10-bit sliced counters)
constexpr int kMaxQapN = 256;

// Barrier shared by all CTAs of a cooperative launch: every CTA publishes the number of
// barriers it has passed in its own flag and waits until all flags reach it.
constexpr int kMaxGridCtas = 1024;
struct GridBarrier {
  int sticky;  // set when a wait expired; kept across launches until the host reads it
  int error;   // set when a wait expired; the launch stops early (cleared every launch)
  unsigned int flags[kMaxGridCtas];
};
// Bytes of GridBarrier cleared before every launch (everything but sticky).
constexpr size_t kBarrierResetOffset = sizeof(int);
constexpr size_t kBarrierResetBytes = sizeof(GridBarrier) - sizeof(int);

// Device-resident k-SAT instance after the host build (variables renumbered so that every
// colour class is a contiguous id range; "new" ids below).
struct KsatDevice {
  int32_t n, m, kmax, n_colours, kq;  // kq = int4 words per occurrence (1: k<=4, 2: k<=8)
  int32_t nb;                         // bits of the sliced counters (covers the max degree)
  int32_t n_occ;                      // occurrences incl. padding (multiple of 4 per variable)
  int32_t n_groups;                   // groups of 32 variables of the interleaved lists
  int4 *occ;                          // n_occ * kq: {own sign mask, other literal ids...}
  int32_t *occ_ptr;                   // n+1
  int32_t *col_ptr;                   // n_colours+1 (device copy)
  int32_t *orig;                      // n: new id -> original id
  int32_t *newid;                     // n: original id -> new id
  int32_t *clits;                     // m * kmax literal ids (2*new+neg), pad = 2n (false)
  int4 *occ_t;                        // occurrence lists interleaved per 32-variable group
  int32_t *grp_base;                  // groups+1: start of each group in occ_t (int4 units)
  int32_t *cgrp;                      // n_colours+1: first group of each colour class
};

// Replica state of one k-SAT replica set: W = ceil(R/32) words per literal row.
struct KsatReplicas {
  int32_t R, W;
  uint32_t *S;        // (2n+2) * W: row 2v = x_v bits, row 2v+1 = not x_v, rows 2n/2n+1 dummy
  uint32_t *best;     // n * W ([var][word]), then n * W of word-major staging for the batched kernel
  int32_t *energy;    // 32W
  int32_t *best_energy;
  uint32_t *imp;      // W: replicas whose best improved at the last sweep end (pending copy)
  GridBarrier *bar;
};

struct QapDevice {
  int32_t n;
  uint8_t *F, *D;  // n*n, entries 0..255
};

struct QapReplicas {
  int32_t R;
  int16_t *perm;       // R * n
  int16_t *best_perm;  // R * n
  int64_t *energy, *best_energy;
};

// One work item of the batched kernel: one word (32 replicas) of one replica set, sweeps
// [t0, t1), with pointers into the instance, its schedule and the replica set.
struct BatchItem {
  const int4 *occ_t;
  const int32_t *grp_base;
  const int32_t *cgrp;
  const int32_t *col_ptr;
  const int32_t *orig;
  const uint32_t *bq;
  uint32_t *S;
  uint32_t *best;
  int32_t *energy;
  int32_t *best_energy;
  int32_t n, n_colours, W, w, t0, t1;
  uint32_t k0, k1;
  // Replica exchange and energy statistics (kernels instantiated for them only):
  const uint32_t *mult;  // 32W Q16 temperature multipliers of the replicas, or null
  long long *stats;      // 64W: per-replica sums of E (first 32W) and E^2 (next 32W), or null
  int32_t stats_t0;      // sweeps t >= stats_t0 add their end-of-sweep energies to stats
  int32_t n_groups;      // groups of 32 variables; grp_base[n_groups + 1 + g]: g's sign regions
};

// ---- k-SAT launchers (ksat.cu); all asynchronous on `st` -------------------------------
// Initial states (Philox, or init_dev [R][n] 0/1 bytes) and, with set_best, best = state.
cudaError_t ksat_init_states(const KsatDevice &I, KsatReplicas &Rp, uint64_t seed,
                             const uint8_t *init_dev, cudaStream_t st, bool set_best = true);
// Energies from scratch and, with set_best, best energies = energies.
cudaError_t ksat_energies(const KsatDevice &I, KsatReplicas &Rp, cudaStream_t st,
                          bool set_best = true);
cudaError_t ksat_sweeps(const KsatDevice &I, KsatReplicas &Rp, const uint32_t *bq,
                        const uint32_t *tab, int32_t tab_len, int32_t t0, int32_t t1,
                        uint64_t seed, int device, cudaStream_t st);
cudaError_t ksat_unpack(const KsatDevice &I, const KsatReplicas &Rp, uint8_t *states,
                        uint8_t *best_states, int64_t *energies, int64_t *best_energies,
                        cudaStream_t st);
// Shape of the sweep kernel for W % 32 == 0: warps per variable (1, 2 or 4; 0 selects the
// general kernel).
void set_sweep_shape(int warps_per_variable);
cudaError_t wait_selftest(GridBarrier *gb, unsigned long long limit_ns, cudaStream_t st);
cudaError_t quantize_schedule_factored(const float *base, const float *factor, int32_t n_units,
                                       int32_t n_steps, const int32_t *orig, uint32_t *bq,
                                       int32_t *bad, cudaStream_t st);
cudaError_t quantize_schedule(const float *beta, int32_t n_units, int32_t n_steps,
                              const int32_t *orig, uint32_t *bq, int32_t *bad,
                              cudaStream_t st);

// ---- batched k-SAT (batch.cu) -----------------------------------------------------------
// Largest n whose word vector fits the batched kernel's shared memory on `device`.
size_t batch_max_vars(int tab_len, int device);
// Runs n_items items (all of one occurrence width kq) in one launch with cs CTAs (1, 2, 4, 8)
// per item; next_item is a device int. With pt, every item carries temperature multipliers
// (mult) and may carry energy statistics. lanes: lanes per variable (1, 4, 8; 0 = the built-in
// choice from cs and max_n).
// Estimated GPU time, in microseconds, of one sweep of one 32-replica word of a k-SAT instance
// with n variables in n_colours classes on one CTA (the shape of a launch with many items): per
// class a latency floor plus the variables' share of a 512-thread round, rounds beyond 512
// variables in full (from measured sweeps: ~2.4k cycles per class of a few variables, ~16k per
// full round). Used to order work items and to size serving slices by time, not for results.
double ksat_sweep_us(int32_t n, int32_t n_colours);
// The same for one swap step (n attempts) of one 32-replica block of a QAP instance.
double qap_step_us(int32_t n);

cudaError_t ksat_batch(const BatchItem *items_dev, int n_items, int kq, int cs, int max_n,
                       int *next_item, const uint32_t *tab, int tab_len, int device,
                       cudaStream_t st, bool pt = false, int lanes = 0);

// A validated batched launch, ready to be placed into device memory: the work items in launch
// order (occurrence width 1 first, then 2), with their counts, shapes and the context's
// stream, table and device. Filled by batch_plan (api.cu).
struct BatchPlan {
  std::vector<BatchItem> items;
  size_t off[2];
  int cnt[2];
  int max_n[2];
  int cs[2];
  int lanes[2];  // 0 = built-in choice
  int device;
  cudaStream_t stream;
  const uint32_t *tab;
  int tab_len;
};
// Validates a batch as nmc_batch_run does and fills `plan`; returns NMC_OK or an error code
// (recorded on the context).
int batch_plan(nmc_ctx *ctx, int32_t n_sets, const int32_t *rs, const int32_t *t0,
               const int32_t *t1, BatchPlan *plan);
// Records an error message on the context; returns `code`.
int set_ctx_error(nmc_ctx *ctx, int code, const char *msg);

// Allocator whose elements start uninitialised: the large host arrays of an instance are
// written element by element by several threads, so a serial zero fill first is wasted work.
// Every element of a vector using it must be written before it is read.
template <typename T>
struct UninitAlloc : std::allocator<T> {
  template <typename U>
  struct rebind {
    using other = UninitAlloc<U>;
  };
  UninitAlloc() = default;
  template <typename U>
  UninitAlloc(const UninitAlloc<U> &) noexcept {}
  template <typename U>
  void construct(U *p) noexcept {
    ::new (static_cast<void *>(p)) U;
  }
  template <typename U, typename... A>
  void construct(U *p, A &&...a) {
    ::new (static_cast<void *>(p)) U(std::forward<A>(a)...);
  }
};
using HostVec = std::vector<int32_t, UninitAlloc<int32_t>>;

// A k-SAT instance prepared on the host (checks, colouring, renumbering, occurrence lists),
// ready to upload. prepare_ksat needs no context or device, so callers can run it on any
// thread; upload_ksat makes it resident on the context's device (nmc_load_ksat = both).
struct HostKsat {
  int code = 0;
  std::string err;
  int32_t n = 0, m = 0, K = 0, n_colours = 0, kq = 1, nb = 2, n_occ = 0;
  HostVec occ, clits, occ_t;
  std::vector<int32_t> occ_ptr, col_ptr, orig, newid, grp_base, cgrp, colour;
};
int prepare_ksat(int32_t n_vars, int32_t n_clauses, int32_t k_max, const int32_t *lits,
                 HostKsat *out);
int upload_ksat(nmc_ctx *ctx, HostKsat &h, int32_t *inst_out);

// ---- replica exchange and the adaptive ladder (pt.cu) ----------------------------------
// One exchange round q of G ladders of L slots (replica g*L + i belongs to ladder g): the
// pairs of slots (k, k+1), k = q mod 2, k+2, ..., of every ladder exchange their replicas on
// the Metropolis test of (lq[k] - lq[k+1]) (E_a - E_b); slot, at and mult follow the swaps.
cudaError_t pt_exchange(const uint32_t *lq, int32_t L, int32_t G, const int32_t *energy,
                        int32_t *slot, int32_t *at, uint32_t *mult, const uint32_t *tab,
                        int32_t tab_len, uint32_t round, uint32_t k0, uint32_t k1,
                        cudaStream_t st);
// The same round for 64-bit energies (QAP costs); the product is tested exactly in 128 bits.
cudaError_t pt_exchange64(const uint32_t *lq, int32_t L, int32_t G, const long long *energy,
                          int32_t *slot, int32_t *at, uint32_t *mult, const uint32_t *tab,
                          int32_t tab_len, uint32_t round, uint32_t k0, uint32_t k1,
                          cudaStream_t st);
// bq[i] = Q16(float(beta)) for i < count (a constant schedule).
cudaError_t fill_schedule(uint32_t *bq, size_t count, double beta, int32_t *bad, cudaStream_t st);
// From per-replica energy sums over `samples` sweeps of R replicas: sigma = sqrt(<E^2> - <E>^2)
// (IEEE double, no contraction); out[0] = sigma, out[1] = beta + alpha / sigma.
cudaError_t ladder_step(const long long *stats, int32_t R, int32_t W, long long samples,
                        double beta, double alpha, double *out, cudaStream_t st);
// The same from per-replica double sums stats[2][R] (QAP costs), added over r = 0..R-1 in order.
cudaError_t ladder_step_f64(const double *stats, int32_t R, long long samples, double beta,
                            double alpha, double *out, cudaStream_t st);

// ---- collective move (cluster.cu) --------------------------------------------------------
// Device scratch one ksat_cluster_flip needs for an instance of n variables and W words.
size_t cluster_scratch_bytes(int32_t n, int32_t W);
// Replica r proposes flipping the variables of its mask (mask_dev: uint8 [rows][n], original
// order, rows 1 or R) and accepts by the Metropolis rule at beta_dev[r] (validated, R floats);
// energies, best energies, states and best states follow. acc_dev (nullable): R bytes out.
cudaError_t ksat_cluster_flip(const KsatDevice &I, KsatReplicas &Rp, const uint8_t *mask_dev,
                              int32_t rows, const float *beta_dev, uint32_t move_id,
                              uint64_t seed, const uint32_t *tab, int32_t tab_len, void *scratch,
                              uint8_t *acc_dev, cudaStream_t st);

// ---- learning stage: CNF LBP, backbones, two-chain schedule (lbp.cu) ----------------------
struct LbpArgs {
  const int32_t *clits, *vptr, *vedge, *orig;  // device: clause literal ids, var -> edge CSR
  int32_t n, m, kmax, S, n_lambda, max_iter;
  const double *eps;      // device [n], new order
  const uint8_t *xs;      // device [n][S] seeds (0/1), new order, seed fastest
  const double *lambdas;  // host [n_lambda]
  double beta, tol;
  void *scratch;          // lbp_scratch_bytes
  double *marg;           // device out [S][n], original order
  double *corr;           // device out [S][m]
  int32_t *iters;         // device out [S][n_lambda]
  double *deltas;         // device out [S][n_lambda]
  int32_t *n_done;        // device out [S]
  double *overlap;        // device out [S][2]: p, q1
};
size_t lbp_scratch_bytes(int32_t n, int32_t m, int32_t kmax, int32_t S, int32_t n_lambda);
cudaError_t lbp_prepare(const uint8_t *x_in, const double *eps_in, const int32_t *orig,
                        const int32_t *vptr, int32_t n, int32_t S, uint8_t *xs, double *eps,
                        cudaStream_t st);
// Runs the continuation; returns 0 or a cudaError_t value. Synchronises the stream once per
// iteration (to see whether any seed is still iterating).
int lbp_run(const LbpArgs &A, cudaStream_t st);

struct BackboneArgs {
  const int32_t *clits, *orig, *newid;
  int32_t n, m, kmax, S;
  const double *corr;  // device [S][m]
  double beta, seed_thr, cutoff;
  void *scratch;       // backbone_scratch_bytes
  int32_t *labels;     // device out [S][n], original order
  int32_t *n_clusters; // device out [S]
};
size_t backbone_scratch_bytes(int32_t n, int32_t m, int32_t S);
int backbone_run(const BackboneArgs &A, cudaStream_t st);
// lab: device [n] labels in original order (-1 = not in a backbone); bq [n_steps][n] new order.
cudaError_t backbone_schedule(const int32_t *lab, const int32_t *orig, int32_t n, int32_t n_steps,
                              float base, float heat, int32_t t_hot, int32_t t_cold,
                              int32_t t_unlearn, uint32_t *bq, cudaStream_t st);

// ---- whitening (whitening.cu) ------------------------------------------------------------
size_t whitening_scratch_bytes(int32_t n, int32_t W);
// X: state words, variable u's word w at X[u * xrows2 * W + w] (S with xrows2 = 2, best with 1).
// count: device [R]; frozen: device [R][n] original order (nullable); *rounds: rounds run.
// Returns 0 or a cudaError_t value; synchronises once per round.
int whitening_run(const KsatDevice &I, const uint32_t *X, int32_t xrows2, int32_t R, int32_t W,
                  int generalized, void *scratch, int32_t *count, uint8_t *frozen, int32_t *rounds,
                  cudaStream_t st);

// ---- QAP launchers (qap.cu) ------------------------------------------------------------
// Arguments of one QAP launch (or, in a batched launch, of one CTA: one block of 32 replicas).
struct QapArgs {
  const uint8_t *F, *D;
  int16_t *perm, *best_perm;
  long long *energy, *best_energy;
  const uint32_t *bq;
  const uint32_t *tab;
  int32_t tab_len, n, R, t0, t1;
  uint32_t k0, k1;
  int init_mode;  // 0: run steps; 1: draw initial states (Fisher-Yates); 2: states given
  int block;      // batched launches: replica block (32 replicas) this CTA runs; else -1
  const uint32_t *mult;  // replica exchange: Q16 temperature multiplier of each replica, or null
  double *stats;         // energy statistics [2][R] (running sums of E and E^2), or null
  int32_t stats_t0;      // first step whose end-of-step cost enters stats
};

QapArgs qap_block_args(const QapDevice &I, QapReplicas &Rp, const uint32_t *bq, const uint32_t *tab,
                       int32_t tab_len, int32_t t0, int32_t t1, uint64_t seed, int block);
// Launch shape of the QAP kernels for an instance of n facilities: 0..kQapShapes-1 (lanes per
// replica and facilities per lane); a batched launch takes items of one shape.
constexpr int kQapShapes = 12;
int qap_shape(int n);
// The batched QAP launches of these sets (as nmc_qap_batch_run does them), each launch shape on
// an auxiliary stream forked from the context's stream after the work-list upload; *joins gets
// the streams to join. qap_batch_join makes the context's stream wait for them; call it also
// after an error, so that nothing launched is left unjoined.
int qap_batch_enqueue(nmc_ctx *ctx, int32_t n_sets, const int32_t *rs, const int32_t *t0,
                      const int32_t *t1, uint32_t *joins);
int qap_batch_join(nmc_ctx *ctx, uint32_t joins);
// Runs n_blocks QAP replica blocks (items_dev[b] for CTA b) in one launch; every item has
// qap_shape(n) == shape, and max_n (the largest n) sizes the shared memory.
cudaError_t qap_batch(const QapArgs *items_dev, int n_blocks, int shape, int max_n, int tab_len,
                      cudaStream_t st);
// (older single-set launchers below) ------------------------------------------------------------
// Initial permutations (Fisher-Yates from Philox, or init_dev [R][n]) with their costs; with
// set_best the best-so-far is set to them too.
cudaError_t qap_init_states(const QapDevice &I, QapReplicas &Rp, uint64_t seed,
                            const int16_t *init_dev, cudaStream_t st, bool set_best = true);
cudaError_t qap_steps(const QapDevice &I, QapReplicas &Rp, const uint32_t *bq,
                      const uint32_t *tab, int32_t tab_len, int32_t t0, int32_t t1,
                      uint64_t seed, cudaStream_t st);
cudaError_t qap_unpack(const QapDevice &I, const QapReplicas &Rp, int16_t *perms,
                       int16_t *best_perms, int64_t *energies, int64_t *best_energies,
                       cudaStream_t st);

}  // namespace nmc
