/*
 * nmc.h -- C ABI of the GB300 engine for the inhomogeneous Metropolis sweep of Nonequilibrium
 * Monte Carlo (NMC; Mohseni et al., arXiv:2111.13628).
 *
 * The engine runs the sampling stage of NMC (Algorithm 1, "nonlocal exploration", "local
 * exploitation" and "unlearning" steps): single-variable Metropolis updates with a separate
 * inverse temperature beta_v[t] for every variable v at every sweep t (Sec. "Nonequilibrium
 * inhomogeneous sampling over subgraphs"), over many independent replicas of a random k-SAT
 * formula (energy = number of violated clauses, Sec. "4-SAT Problems Near Computational Phase
 * Transitions") or of a Koopmans-Beckmann QAP (swap moves on a permutation, Sec. "Quadratic
 * Assignment Problems"). A homogeneous profile is the unlearning phase; a short schedule is one
 * of the learning stage's exploratory runs.
 *
 * Dynamics (fixed here so that every result is reproducible bit for bit):
 *   - sweep order: DSatur colouring of the variable-interaction graph (the uncoloured variable
 *     whose coloured neighbours show the most distinct colours, then the one in more clauses,
 *     then the smaller id, takes the smallest colour its neighbours leave free); one sweep
 *     visits colours in ascending order, every colour class (an independent set) updated
 *     against the state left by the earlier colours;
 *   - random numbers: Philox4x32-10 keyed by the 64-bit seed; replica r's attempt on variable
 *     v at sweep t uses word r&3 of the block for counter (v, t, r>>2, 0x4B535750);
 *   - acceptance: dE <= 0 always; otherwise with bq = round_half_even(beta * 2^16) and
 *     j = (bq * dE) >> 8, accept iff u < floor(2^32 exp(-j/256)) (capped at 2^32-1);
 *   - best-so-far: the initial state, then replaced after any sweep that ends strictly lower.
 * The QAP chain is defined in nmc_load_qap.
 *
 * Conventions: every function returns NMC_OK (0) or a negative NMC_E* code and never aborts;
 * nmc_last_error() describes the last failure on that context. Host pointers are read during
 * the call only (the caller keeps ownership); results go to caller-owned buffers. Device
 * state (instances, schedules, replica sets) is owned by the context and stays resident
 * until it is released or the context is destroyed. Work is issued on the context's stream;
 * calls that return host data synchronise that stream. A context is not thread-safe: use one
 * per host thread, or serialise calls.
 */
#ifndef NMC_H_
#define NMC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NMC_OK 0
#define NMC_EINVAL (-1)   /* bad argument: ids, sizes, literals, beta outside [0, 65535] */
#define NMC_ENOMEM (-2)   /* device allocation failed */
#define NMC_ECUDA (-3)    /* a CUDA call failed (message from the runtime) */
#define NMC_ETIMEOUT (-4) /* a bounded device-side wait expired; the result is not valid */
#define NMC_ESTATE (-5)   /* call out of order (no schedule, schedule too short, wrong kind) */

#define NMC_KIND_KSAT 1
#define NMC_KIND_QAP 2

typedef struct nmc_ctx nmc_ctx;

/* Outputs of a replica set, all caller-owned (host or device, as the call states); any field
 * may be NULL to skip it. k-SAT states are uint8 [R][N] (0/1, original variable order); QAP
 * states are int16 [R][n] with p[facility] = location. Energies are int64 [R]. */
typedef struct nmc_result {
  void *states;
  int64_t *energies;
  int64_t *best_energies;
  void *best_states;
} nmc_result;

/* Creates a context on CUDA device `device`. `cuda_stream` is a cudaStream_t to issue work on
 * (NULL: the context creates and owns a non-blocking stream). */
int nmc_create(nmc_ctx **out, int device, void *cuda_stream);
/* Synchronises and frees everything the context owns. NULL is ignored. */
void nmc_destroy(nmc_ctx *ctx);
/* Message for the last failed call on ctx (static string when ctx is NULL). */
const char *nmc_last_error(nmc_ctx *ctx);
/* Waits for all work issued on the context's stream. */
int nmc_sync(nmc_ctx *ctx);

/*
 * Loads a CNF formula (the factor graph of Sec. "k-local factor-graph"; clauses a, variables
 * i, literals in DIMACS form). lits: n_clauses * k_max int32, clause a in row a, literal
 * +(v+1) / -(v+1) for x_v / not x_v, 0 for an unused slot. Requirements (else NMC_EINVAL):
 * 1 <= n_vars < 2^28, 0 <= n_clauses < 2^31, 1 <= k_max <= 8, every |literal| <= n_vars,
 * at least one literal per clause, no variable twice in one clause, every variable in at most
 * 1023 clauses (a rejected formula names the first clause at fault). Builds, on the host, the
 * colouring and the occurrence lists (with up to 16 short-lived host threads; the colouring
 * itself is sequential), and uploads them. *inst_out receives the instance id.
 */
int nmc_load_ksat(nmc_ctx *ctx, int32_t n_vars, int32_t n_clauses, int32_t k_max,
                  const int32_t *lits, int32_t *inst_out);

/*
 * Loads a Koopmans-Beckmann QAP (Sec. "Quadratic Assignment Problems", without the placement
 * term): cost C(p) = sum_ij F[i][j] D[p(i)][p(j)]. F (flows) and D (distances) are n*n int32,
 * row-major, symmetric, zero diagonal, entries in [0, 255]; 1 <= n <= 256 (else NMC_EINVAL).
 * One schedule step is n swap attempts; attempt a of step t of replica r draws the Philox block
 * for counter (a, t, r, 0x51535450): facility r_ = (u0 n) >> 32, s' = (u1 (n-1)) >> 32,
 * s = s' + (s' >= r_), and u2 decides an uphill swap at bq = (bq_r_[t] + bq_s[t]) >> 1.
 */
int nmc_load_qap(nmc_ctx *ctx, int32_t n, const int32_t *F, const int32_t *D, int32_t *inst_out);

/* Releases an instance, its schedule and nothing else (replica sets of it must be released
 * first, else NMC_ESTATE). */
int nmc_unload(nmc_ctx *ctx, int32_t inst);

/* Number of colours and, if colour_out != NULL, the colour of every variable (int32 [N]) of a
 * k-SAT instance. */
int nmc_ksat_colouring(nmc_ctx *ctx, int32_t inst, int32_t *colour_out, int32_t *n_colours);

/* The same colouring (the sweep order) of a formula given as for nmc_load_ksat, computed on the
 * host alone: no context and no device. colour_out (nullable): int32 [n_vars]; n_colours
 * (required). NMC_EINVAL for a formula nmc_load_ksat rejects. */
int nmc_ksat_colour_host(int32_t n_vars, int32_t n_clauses, int32_t k_max, const int32_t *lits,
                         int32_t *colour_out, int32_t *n_colours);

/*
 * Sets the inverse-temperature profile beta[unit][step] of an instance (units = variables or
 * facilities): n_units * n_steps float32, row-major (row = one unit's schedule), host memory.
 * Every value must be in [0, 65535] or +infinity (checked on the device; else NMC_EINVAL). The
 * profile is quantised to Q16 and stored step-major on the device. Replaces any earlier one.
 * beta = +infinity holds the unit fixed at that step (the two chains of Algorithm 1 each sample
 * one subset with the other fixed, Fig. 2 caption): a held k-SAT variable is not attempted, a
 * QAP swap that involves a held facility is rejected; no other draw or unit is affected.
 */
int nmc_set_schedule(nmc_ctx *ctx, int32_t inst, int32_t n_steps, const float *beta);
/* As nmc_set_schedule, with beta in device memory (read on the context's stream). */
int nmc_set_schedule_device(nmc_ctx *ctx, int32_t inst, int32_t n_steps, const float *beta_dev);
/* As nmc_set_schedule for the rank-one profile beta[u][t] = base[t] * factor[u] (the product
 * rounded to float32, round to nearest even): a global anneal scaled per unit, the shape of
 * the sampling stage's heated-backbone profiles. base: n_steps floats, factor: n_units floats,
 * host memory. */
int nmc_set_schedule_factored(nmc_ctx *ctx, int32_t inst, int32_t n_steps, const float *base,
                              const float *factor);

/*
 * Creates a resident replica set of `replicas` chains (1..4096) of an instance, seeded by
 * `seed`. init_states (host, nullable): k-SAT uint8 [R][N] 0/1, QAP int16 [R][n] permutations;
 * NULL draws the initial states from Philox (k-SAT: bit 0 of word r&3 for counter
 * (v, 0, r>>2, 0x4B494E49); QAP: Fisher-Yates from the identity, position q (n-1 down to 1)
 * exchanged with (u (q+1)) >> 32 for u word 0 of counter (q, 0, r, 0x51494E49)). Computes the
 * energies; best-so-far = initial. *rs_out receives the replica-set id.
 */
int nmc_replicas_create(nmc_ctx *ctx, int32_t inst, int32_t replicas, uint64_t seed,
                        const void *init_states, int32_t *rs_out);
/* Re-initialises an existing replica set in place (no allocation): new seed, new initial
 * states (init_states as in nmc_replicas_create), energies recomputed, best-so-far reset. */
int nmc_replicas_reset(nmc_ctx *ctx, int32_t rs, uint64_t seed, const void *init_states);
/* Checkpoint resume: sets a replica set's current states and best-so-far states from host
 * buffers in the layout nmc_replicas_read writes (in->states and in->best_states required; the
 * energy fields are ignored and recomputed from the states). Reading a set after sweeps
 * [0, t1) and restoring the result into a fresh set of the same instance and seed continues
 * the chains exactly: running [t1, t2) there equals running [0, t2) in one set. */
int nmc_replicas_restore(nmc_ctx *ctx, int32_t rs, const nmc_result *in);
/* Frees a replica set. */
int nmc_replicas_destroy(nmc_ctx *ctx, int32_t rs);
/*
 * Runs sweeps (k-SAT) or steps (QAP) t0..t1-1 of the schedule on the resident replica set,
 * asynchronously on the context's stream: the single-variable Metropolis dynamics with each
 * variable (facility) at its own inverse temperature beta[unit][t] of the sampling stage
 * (Sec. "Nonequilibrium inhomogeneous sampling over subgraphs"; the sampling and unlearning
 * sweeps of Algorithm 1; swap moves on the cost of Sec. "Quadratic Assignment Problems"). A k-SAT set that nmc_batch_run accepts runs on that
 * (shared-memory, cluster) kernel, any other on the grid-barrier kernel; the results are the
 * same bit for bit (the environment variable NMC_RUN_PATH=grid forces the grid kernel). t is absolute, so [t0,t1) then [t1,t2) equals
 * [t0,t2) bit for bit. Requires 0 <= t0 <= t1 <= n_steps of the current schedule
 * (NMC_ESTATE otherwise). A device-side wait that expires is reported as NMC_ETIMEOUT by the
 * next synchronising call on this replica set.
 */
int nmc_replicas_run(nmc_ctx *ctx, int32_t rs, int32_t t0, int32_t t1);
/* Copies the replica set's current states, energies, best energies and best states to host
 * buffers (synchronises). */
int nmc_replicas_read(nmc_ctx *ctx, int32_t rs, const nmc_result *out);
/* As nmc_replicas_read, into device buffers, asynchronously on the context's stream. */
int nmc_replicas_read_device(nmc_ctx *ctx, int32_t rs, const nmc_result *out_dev);

/*
 * Batched sweeps: runs sweeps t0[i]..t1[i]-1 of k-SAT replica sets rs[i] (i < n_sets), all in
 * one persistent launch per occurrence width (formulas with k <= 4 and with 4 < k <= 8),
 * asynchronously on the context's stream; when both widths are present the k > 4 launch runs
 * beside the other on an auxiliary stream of the context, forked from and joined back to the
 * context's stream, so work enqueued later on that stream still follows. Each set's result is bit for
 * bit what nmc_replicas_run gives for it alone. Work is split into items of one word (32
 * replicas) of one set; a CTA runs an item with the word vector in shared memory, so each
 * instance needs n_vars <= the limit of nmc_batch_max_vars() and every variable in at most 127
 * clauses (else NMC_EINVAL; use nmc_replicas_run for those). The same set may not appear twice.
 */
int nmc_batch_run(nmc_ctx *ctx, int32_t n_sets, const int32_t *rs, const int32_t *t0,
                  const int32_t *t1);
/*
 * nmc_batch_run for callers that must not allocate device memory during the call. The paper
 * has no counterpart: this serves host programs that cannot call cudaMalloc at this point -
 * code running inside a framework whose allocator owns all free device memory, or a loop
 * that cannot afford the device-wide synchronisation an allocation may cause. It does the
 * same work with the same results as nmc_batch_run on the same arguments, but its work list
 * and counters live in one fixed 1 MiB device array of the library instead of memory the
 * context allocates. Limit: one call takes at most (1 MiB - 256 B) / 136 B = 7708 work items,
 * one per 32-replica word of each set (NMC_EINVAL beyond, with a message). The array is
 * reserved on every GPU that loads the library until the process exits. The first call on a
 * device does the set-up: it looks up the array's device address (cudaGetSymbolAddress, with
 * that device current) and keeps it for the rest of the process, so make that first call
 * before any stream capture, and do not reset the device (cudaDeviceReset) after it. Each call
 * copies its work list into the array from host memory and clears the counters on the stream
 * before its launches. Every call shares the one array, which keeps the last call's work
 * list: calls whose launches overlap on the GPU (other streams, other contexts, other host
 * threads) race on it and must be serialised by the caller.
 */
int nmc_batch_run_noalloc(nmc_ctx *ctx, int32_t n_sets, const int32_t *rs, const int32_t *t0,
                          const int32_t *t1);
/*
 * Autotuner of the batched sweep. Times every launch shape (1, 2, 4 or 8 CTAs per work item x
 * 1, 4 or 8 lanes per variable) on sweeps [t0, t0 + sweeps) of the k-SAT replica sets rs[i]
 * (the batch nmc_batch_run would run), separately for the two occurrence widths (k <= 4,
 * k <= 8), and keeps the fastest on this context: later nmc_batch_run / nmc_replicas_run /
 * replica-exchange launches whose work list has the same width, largest n_vars and number of
 * work items (32-replica words) use it; the variables NMC_BATCH_CTAS / NMC_BATCH_LANES still
 * take precedence. Every shape gives the same results bit for bit, and the sets' states, best
 * states and energies are saved before the trials and restored after them, so the call leaves
 * the sets as it found them. shapes_out (host, nullable): int32 [2][3] = (CTAs per item, lanes,
 * microseconds per sweep) per width, zeros where the width has no items. Synchronises.
 */
int nmc_batch_autotune(nmc_ctx *ctx, int32_t n_sets, const int32_t *rs, int32_t t0,
                       int32_t sweeps, int32_t *shapes_out);
/* Batched QAP steps: runs steps t0[i]..t1[i]-1 of QAP replica sets rs[i], one CTA per block of
 * 32 replicas, one launch per launch shape (the sets' sizes pick the shapes); the shapes run side
 * by side on internal streams forked from the context's stream and joined back to it, so the call
 * stays asynchronous and ordered on that stream. Results as nmc_replicas_run on each set alone. */
int nmc_qap_batch_run(nmc_ctx *ctx, int32_t n_sets, const int32_t *rs, const int32_t *t0,
                      const int32_t *t1);
/* Largest n_vars nmc_batch_run accepts on this context's device. */
int32_t nmc_batch_max_vars(nmc_ctx *ctx);

/*
 * Replica exchange (parallel tempering, App. "Adaptive Parallel Tempering": replicas at
 * adjacent temperatures exchange with probability min{1, exp[(beta_i - beta_j)(E_i - E_j)]}).
 *
 * nmc_replicas_set_ladder attaches a temperature ladder to a replica set whose R is a
 * multiple of n_temps: the set becomes G = R / n_temps independent ladders, replica g*n_temps
 * + i in ladder g. ladder: n_temps floats (host), each finite and in [0, 65535], quantised to
 * Q16 like the schedule (lq[k]). slots (host, nullable): R int32, the slot of every replica
 * within its ladder, each ladder's slots a permutation of 0..n_temps-1; NULL puts replica
 * g*n_temps + i at slot i. A replica at slot k moves at min(2^32-1, (lq[k] bq_v[t]) >> 16)
 * instead of the schedule's bq_v[t] (QAP: of the swap's pair temperature
 * (bq_r[t] + bq_s[t]) >> 1): the schedule gives the spatial profile, the ladder the
 * temperature. Works on k-SAT and QAP sets.
 * Replaces an earlier ladder; reset and restore leave the ladder and slots alone, and
 * nmc_replicas_run / nmc_batch_run ignore it (they sweep at the schedule's beta).
 * A k-SAT instance must be one nmc_batch_run accepts (NMC_EINVAL otherwise).
 */
int nmc_replicas_set_ladder(nmc_ctx *ctx, int32_t rs, int32_t n_temps, const float *ladder,
                            const int32_t *slots);
/*
 * Runs sweeps t0..t1-1 of a set with a ladder, asynchronously on the context's stream, with an
 * exchange round after every sweep t where (t+1) % sweeps_per_round == 0: round
 * q = (t+1)/sweeps_per_round - 1 tries the slot pairs (k, k+1), k = q mod 2, k+2, ..., of
 * every ladder g; replicas a (at k) and b (at k+1) exchange slots when
 * d = (lq[k] - lq[k+1]) (E_a - E_b) >= 0, else when ((-d) >> 8) < L and u < Tab[(-d) >> 8],
 * u = word 0 of the Philox block for counter (k, q, g, 0x50545357) under the set's seed (d is
 * formed exactly: QAP costs reach 2^33). For QAP sets a "sweep" is a step of n swap attempts.
 * Rounds are absolute like t, so [t0, t1) then [t1, t2) equals [t0, t2).
 */
int nmc_replicas_run_pt(nmc_ctx *ctx, int32_t rs, int32_t t0, int32_t t1,
                        int32_t sweeps_per_round);
/* Copies the slot of every replica (R int32) of a set with a ladder to host memory
 * (synchronises). */
int nmc_replicas_read_slots(nmc_ctx *ctx, int32_t rs, int32_t *slots_out);

/*
 * Collective move (the nonlocal flip of a whole backbone, Fig. 1(c) caption; Sec.
 * "Nonequilibrium Nonlocal Monte Carlo"): every replica r of a k-SAT set proposes flipping all
 * variables of its mask at once, x' = x xor m_r, and accepts with the Metropolis rule at inverse
 * temperature beta[r] on dE = E(x') - E(x): dE <= 0 accepts; otherwise bq = Q16(beta[r]) and it
 * accepts iff ((bq dE) >> 8) < L and u < Tab[(bq dE) >> 8], u = word r&3 of the Philox block for
 * counter (move_id, 0, r>>2, 0x434C5354) under the set's seed. Energies follow; the best-so-far
 * is replaced on strictly lower energy. mask: host uint8 [mask_rows][n_vars], 0/1, original
 * variable order; mask_rows = 1 (the same mask for every replica) or R. beta: R host floats,
 * finite and in [0, 65535]. Runs asynchronously on the context's stream; with accepted_out
 * (host, R bytes, nullable) it synchronises and reports which replicas moved. Callers pass a
 * different move_id for every move they want drawn independently.
 */
int nmc_replicas_cluster_flip(nmc_ctx *ctx, int32_t rs, int32_t mask_rows, const uint8_t *mask,
                              const float *beta, uint32_t move_id, uint8_t *accepted_out);

/*
 * Learning stage for k-SAT: loopy belief propagation on the surrogate Hamiltonian around S seed
 * states (Sec. "4-SAT Problems Near Computational Phase Transitions"; App. "Loopy Belief
 * propagation for k-local Hamiltonians over conjugate normal form"), double precision.
 * Spins r = 2x - 1; sigma_ai = +1 for a positive literal of variable i in clause a, -1 for a
 * negated one. Messages: h_{i->a} = sigma_ai (lambda eps_i s*_i + sum_{b != a} sigma_bi u_{b->i}),
 * u_{a->i} = -1/2 ln[1 - (1 - e^{-2 beta}) prod_{j in a, j != i} (1 - tanh h_{j->a}) / 2]. They
 * start from h = sigma lambda_0 eps s* and the u of those h; an iteration recomputes every h
 * from the previous u, then every u; a lambda converges when max |u_new - u_old| < tol. lambda
 * runs through `lambdas` without re-initialising; when one fails to converge in max_iter
 * iterations, the messages of the previous converged lambda are restored and that seed stops.
 * Outputs from the final messages (lambda = the last converged one, else lambda_0):
 * <r_i> = tanh(lambda eps_i s*_i + sum_a sigma_ai u_{a->i}); clause correlations
 * <prod_{i in a} r_i> under mu_a(r) ~ omega_a(r) prod_i (1 + sigma_ai r_i tanh h_{i->a}) / 2
 * with omega_a = e^{-2 beta} on the violating configuration (the full sum over the clause's
 * configurations); p = (1/N) sum s*_i <r_i>, q1 = (1/N) sum <r_i>^2.
 * x_star: host uint8 [S][N] 0/1 (original variable order); eps: host double [N], NULL = the
 * number of clauses of each variable; lambdas: host double [n_lambda]. Outputs (host):
 * marg_out [S][N] (required); corr_out [S][M], iters_out [S][n_lambda] (iterations run at each
 * lambda, 0 where not reached), deltas_out [S][n_lambda] (last max |du|), n_done_out [S]
 * (lambdas that converged), overlap_out [S][2] (p, q1): each nullable. Synchronises.
 */
int nmc_cnf_lbp(nmc_ctx *ctx, int32_t inst, int32_t n_seeds, const uint8_t *x_star,
                const double *eps, double beta, int32_t n_lambda, const double *lambdas,
                double tol, int32_t max_iter, double *marg_out, double *corr_out,
                int32_t *iters_out, double *deltas_out, int32_t *n_done_out,
                double *overlap_out);
/*
 * Backbones (Sec. "Generating backbones of rigid variables") from clause correlations corr
 * (host double [S][M], each in [-1, 1]): effective factor couplings J~_a = atanh|corr_a| / beta;
 * factors with J~ > seed_thr are nuclei; clusters grow through every factor with J~ > cutoff
 * (or > seed_thr) touching them. labels_out (host int32 [S][N], original order): the cluster's
 * smallest variable id, -1 outside every cluster; n_clusters_out (host [S], nullable).
 * beta > 0. Synchronises.
 */
int nmc_cnf_backbone(nmc_ctx *ctx, int32_t inst, int32_t n_seeds, const double *corr,
                     double beta, double seed_thr, double cutoff, int32_t *labels_out,
                     int32_t *n_clusters_out);
/*
 * The sampling stage's schedule of Algorithm 1 built on the device from backbone labels (host
 * int32 [N], original order, -1 = not in a backbone): cycles x (t_hot sweeps with the backbone
 * at beta = base / heat (float) and every other variable held (+inf), t_cold sweeps with the
 * backbone held and the rest at base, t_unlearn homogeneous sweeps at base). Replaces the
 * instance's schedule (n_steps = cycles (t_hot + t_cold + t_unlearn)). base and base / heat in
 * [0, 65535], heat > 0.
 */
int nmc_set_schedule_backbone(nmc_ctx *ctx, int32_t inst, const int32_t *labels, int32_t cycles,
                              int32_t t_hot, int32_t t_cold, int32_t t_unlearn, float base,
                              float heat);

/*
 * Whitening (Sec. "Whitening procedure for low energy states") of every replica of a k-SAT set,
 * on its current states (use_best = 0) or its best states (use_best = 1). A variable turns
 * white when no clause containing it blocks it; a clause blocks v when it is neither satisfied
 * by another of its variables nor holds another white variable, and, with generalized != 0 (the
 * paper's extension to low-energy states), when it is moreover satisfied by v itself, so that
 * violated clauses never report a frozen variable. Whitening runs to its fixed point (the same
 * for any inspection order); frozen = not white. frozen_count_out: host int32 [R] (required);
 * frozen_out: host uint8 [R][N] 0/1, original order (nullable); rounds_out (nullable): parallel
 * rounds run. Synchronises.
 */
int nmc_replicas_whitening(nmc_ctx *ctx, int32_t rs, int32_t use_best, int32_t generalized,
                           int32_t *frozen_count_out, uint8_t *frozen_out, int32_t *rounds_out);

/*
 * Adaptive ladder (App. "Adaptive Parallel Tempering"): beta_0 = beta0; for level i the k-SAT
 * instance's `replicas` chains (a temporary set seeded by `seed`, Philox initial states, each
 * level continuing from the previous level's states) run sweeps_eq + sweeps_meas sweeps
 * (absolute sweeps [i T, (i+1) T), T = sweeps_eq + sweeps_meas) at the homogeneous inverse
 * temperature beta_i (every variable, float32 then Q16 as a schedule). The end-of-sweep
 * energies of the last sweeps_meas sweeps of every replica give
 * sigma_i = sqrt(<E^2> - <E>^2) (exact integer sums, then IEEE double, each operation rounded
 * separately, a negative variance taken as 0). The ladder stops at level i when
 * sigma_i <= sigma_min or i + 1 == max_temps, else beta_{i+1} = beta_i + alpha / sigma_i.
 * betas_out, sigmas_out: max_temps doubles (host); *n_temps_out = levels run. The instance's
 * own schedule is not used or changed. sigma_min must be >= 0 (so sigma = 0 always stops).
 * NMC_EINVAL if a beta leaves [0, 65535].
 * QAP instances: the same with swap steps for sweeps (n attempts each) and every facility at
 * beta_i; the costs (up to 2^33, squares beyond 2^53) are summed in double instead, per replica
 * in step order (E converted exactly, E*E and every sum rounded to nearest), then over the
 * replicas in replica order, so the result is reproducible but not an exact integer moment.
 */
int nmc_adaptive_ladder(nmc_ctx *ctx, int32_t inst, int32_t replicas, uint64_t seed, double beta0,
                        double alpha, double sigma_min, int32_t max_temps, int32_t sweeps_eq,
                        int32_t sweeps_meas, double *betas_out, double *sigmas_out,
                        int32_t *n_temps_out);

/*
 * One-shot anneal through host memory: creates a replica set, runs [t0, t1) of the sampling
 * stage's inhomogeneous Metropolis dynamics (Sec. "Nonequilibrium inhomogeneous sampling over
 * subgraphs"; Algorithm 1's sampling sweeps; as nmc_replicas_run), copies the results to the
 * host buffers in *out and frees the set. Arguments as above.
 */
int nmc_anneal(nmc_ctx *ctx, int32_t inst, int32_t replicas, int32_t t0, int32_t t1,
               uint64_t seed, const void *init_states, const nmc_result *out);

/*
 * Serving: continuous batching of anneal requests on one GPU.
 *
 * A server owns a private context on `device` and one worker thread. Requests are copied at
 * submission and queued; the worker admits them (FIFO) while at most max_active are active and
 * the device memory they will hold stays within memory_budget bytes (a request larger than the
 * whole budget fails with NMC_ENOMEM). Admitted requests keep their instance, schedule and
 * replica state resident on the device until they finish. Every tick advances all active
 * requests by a slice of about 2^slice_log2 units of work each (one unit: one clause
 * occurrence of one variable for 32 replicas; a QAP swap attempt on one replica counts as n/3
 * units), but by no more sweeps than fit about 0.1 s of GPU time by an estimate of the request's
 * time per sweep (small instances are bound by the per-colour-class latency, not by their
 * work), so that requests progress at similar wall-clock rates, k-SAT requests together
 * in one batched launch (nmc_batch_run), so requests that arrive while others run share the
 * following launches. Results are bit for bit those of nmc_anneal on the same inputs
 * (segment invariance). All nmc_server_* calls are thread-safe.
 */
typedef struct nmc_server nmc_server;
/* A request's schedule: either beta ([n_units][n_steps], as nmc_set_schedule) or, when beta is
 * NULL, the factored form base[n_steps] x factor[n_units] (as nmc_set_schedule_factored). */
typedef struct nmc_schedule {
  int32_t n_steps;
  const float *beta;
  const float *base;
  const float *factor;
} nmc_schedule;
typedef struct nmc_server_config {
  int32_t max_active;     /* >= 1 */
  int64_t memory_budget;  /* bytes, >= 1 */
  int32_t slice_log2;     /* 10..40 */
} nmc_server_config;
int nmc_server_create(int device, const nmc_server_config *cfg, nmc_server **out);
/* Stops the worker (requests still queued or running fail with NMC_ESTATE) and frees all. */
void nmc_server_destroy(nmc_server *srv);
/* Queues an anneal of sweeps 0..n_steps-1 (arguments as nmc_load_ksat / nmc_set_schedule(_factored)
 * / nmc_replicas_create with Philox initial states; all inputs are copied). *req_out receives
 * the request id. */
int nmc_server_submit_ksat(nmc_server *srv, int32_t n_vars, int32_t n_clauses, int32_t k_max,
                           const int32_t *lits, const nmc_schedule *sched, int32_t replicas,
                           uint64_t seed, int64_t *req_out);
int nmc_server_submit_qap(nmc_server *srv, int32_t n, const int32_t *F, const int32_t *D,
                          const nmc_schedule *sched, int32_t replicas, uint64_t seed,
                          int64_t *req_out);
/* *status: 0 queued, 1 running, 2 done, or the negative error code of a failed request. Waits
 * up to wait_ms for completion (0: no wait). */
int nmc_server_poll(nmc_server *srv, int64_t req, int32_t wait_ms, int32_t *status);
/* Copies a finished request's results to host buffers (layout as nmc_replicas_read; fields may
 * be NULL), reports its latency in seconds from the start of its submit call (so the host-side
 * build of a k-SAT instance, done inside that call, is included) to completion, and forgets it.
 * Returns the request's error code if it failed, NMC_ESTATE if it is not finished. */
int nmc_server_result(nmc_server *srv, int64_t req, const nmc_result *out, double *latency_s);
/* Asks for a request to be dropped at the next tick (its status becomes NMC_ESTATE). */
int nmc_server_cancel(nmc_server *srv, int64_t req);
/* Counters: ticks, Metropolis attempts executed, seconds spent in ticks, queue and active sizes,
 * device memory held by active requests (estimate). Any pointer may be NULL. */
int nmc_server_stats(nmc_server *srv, int64_t *ticks, int64_t *attempts, double *busy_s,
                     int32_t *queued, int32_t *active, int64_t *mem_in_use);
/* Message of the last failed nmc_server_result. */
const char *nmc_server_last_error(nmc_server *srv);

/* Self-test of the bounded device wait: launches one CTA that waits at the grid barrier the
 * sweep kernel uses, for a second arrival that never comes, with the given limit in
 * milliseconds (1..10000). Returns NMC_ETIMEOUT when the wait expired and was reported as
 * the sweep would report it, NMC_OK if it did not expire (a defect), or an error code. The
 * context stays usable afterwards. */
int nmc_selftest_wait_timeout(nmc_ctx *ctx, int32_t timeout_ms);

/* The library's acceptance-threshold table: writes min(cap, L) entries
 * floor(2^32 exp(-j/256)) (entry 0 capped at 2^32-1) and returns L, the index of the first
 * zero entry. */
int32_t nmc_threshold_table(uint32_t *out, int32_t cap);

#ifdef __cplusplus
}
#endif

#endif /* NMC_H_ */
