// Host side of the C ABI declared in include/nmc.h: argument checks, the instance build
// (DSatur colouring, renumbering, occurrence lists), device residency of instances, schedules
// and replica sets, and the dispatch to the kernels in ksat.cu and qap.cu.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "nmc.h"
#include "nmc_internal.h"

using namespace nmc;

namespace {

struct Instance {
  int kind = 0;
  int32_t n_units = 0;
  KsatDevice ks{};
  QapDevice qp{};
  std::vector<int32_t> colour;  // k-SAT: colour of every original variable
  uint32_t *bq = nullptr;       // [n_steps][n_units] Q16, step-major (new ids for k-SAT)
  int32_t n_steps = 0;
  int users = 0;  // live replica sets
  int32_t *lbp_vptr = nullptr;   // k-SAT: variable -> clause-slot CSR for LBP (built on first use)
  int32_t *lbp_vedge = nullptr;
};

struct ReplicaSet {
  int32_t inst = -1;
  int32_t R = 0;
  uint64_t seed = 0;
  KsatReplicas ks{};
  QapReplicas qp{};
  // temperature ladder (k-SAT replica exchange); pt_L = 0 without one
  int32_t pt_L = 0;
  uint32_t *pt_lq = nullptr;    // pt_L Q16 inverse temperatures of the slots
  int32_t *pt_slot = nullptr;   // R: slot of every replica within its ladder
  int32_t *pt_at = nullptr;     // R: replica at slot k of ladder g (index g*pt_L + k)
  uint32_t *pt_mult = nullptr;  // 32W: Q16 multiplier of every replica (1.0 for padding)
};

const char *kStaticNoCtx = "nmc: no context";

// Acceptance thresholds Tab[j] = min(2^32-1, floor(2^32 exp(-j/256))), computed in IEEE
// double with the host C library's exp; returns the index of the first zero entry.
int32_t build_table(uint32_t *out, int32_t cap) {
  int32_t len = -1;
  for (int32_t j = 0; j < cap; ++j) {
    const double scaled = std::ldexp(std::exp(-static_cast<double>(j) / 256.0), 32);
    const uint32_t t = scaled >= 4294967295.0 ? 0xFFFFFFFFu : static_cast<uint32_t>(std::floor(scaled));
    if (t == 0u) {
      len = j;
      for (int32_t q = j; q < cap; ++q) out[q] = 0u;
      break;
    }
    out[j] = t;
  }
  return len;
}

}  // namespace

struct nmc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  std::map<int32_t, Instance> insts;
  std::map<int32_t, ReplicaSet> sets;
  int32_t next_inst = 1, next_set = 1;
  uint32_t *tab = nullptr;
  int32_t tab_len = 0;
  int32_t *flag = nullptr;  // device scratch flag for schedule validation
  BatchItem *items = nullptr;  // batched-kernel work list (grown on demand)
  size_t items_cap = 0;
  int32_t *next_item = nullptr;  // two work counters (one per occurrence width)
  QapArgs *qitems = nullptr;     // batched QAP work list (grown on demand)
  size_t qitems_cap = 0;
  // auxiliary streams of the batched QAP launches (one per launch shape, created on first use):
  // forked from the context's stream after the work-list upload and joined back by events
  cudaStream_t qaux[kQapShapes] = {};
  cudaEvent_t qfork = nullptr;
  cudaEvent_t qjoin[kQapShapes] = {};
  // auxiliary stream of the batched k-SAT launch of the second occurrence width (created on first
  // use): forked after the work-list upload and joined back, so that the two widths' persistent
  // launches share the SMs (the second fills those the first's tail leaves idle)
  cudaStream_t kaux = nullptr;
  cudaEvent_t kfork = nullptr, kjoin = nullptr;
  // tuned batched-sweep shapes: (occurrence width, largest n, work items) -> (cs, lanes)
  std::map<std::tuple<int, int, int>, std::pair<int, int>> tune;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int fail(nmc_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(nmc_ctx *c, cudaError_t e, const char *what) {
  cudaGetLastError();
  const int code = (e == cudaErrorMemoryAllocation) ? NMC_ENOMEM : NMC_ECUDA;
  return fail(c, code, std::string(what) + ": " + cudaGetErrorString(e));
}

#define NMC_CUDA(call, what)                     \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

template <typename T>
cudaError_t dev_alloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * count);
}

template <typename T>
void dev_free(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_instance(Instance &I) {
  dev_free(I.ks.occ);
  dev_free(I.ks.occ_ptr);
  dev_free(I.ks.col_ptr);
  dev_free(I.ks.orig);
  dev_free(I.ks.newid);
  dev_free(I.ks.clits);
  dev_free(I.ks.occ_t);
  dev_free(I.ks.grp_base);
  dev_free(I.ks.cgrp);
  dev_free(I.qp.F);
  dev_free(I.qp.D);
  dev_free(I.bq);
  dev_free(I.lbp_vptr);
  dev_free(I.lbp_vedge);
}

void free_set(ReplicaSet &S) {
  dev_free(S.ks.S);
  dev_free(S.ks.best);
  dev_free(S.ks.energy);
  dev_free(S.ks.best_energy);
  dev_free(S.ks.imp);
  dev_free(S.ks.bar);
  dev_free(S.qp.perm);
  dev_free(S.qp.best_perm);
  dev_free(S.qp.energy);
  dev_free(S.qp.best_energy);
  dev_free(S.pt_lq);
  dev_free(S.pt_slot);
  dev_free(S.pt_at);
  dev_free(S.pt_mult);
  S.pt_L = 0;
}

Instance *find_inst(nmc_ctx *ctx, int32_t id) {
  auto it = ctx->insts.find(id);
  return it == ctx->insts.end() ? nullptr : &it->second;
}

ReplicaSet *find_set(nmc_ctx *ctx, int32_t id) {
  auto it = ctx->sets.find(id);
  return it == ctx->sets.end() ? nullptr : &it->second;
}

// Checks the sticky timeout word of a k-SAT replica set after its stream was synchronised.
int check_timeout(nmc_ctx *ctx, ReplicaSet &S) {
  if (!S.ks.bar) return NMC_OK;
  int sticky = 0;
  NMC_CUDA(cudaMemcpy(&sticky, &S.ks.bar->sticky, sizeof(int), cudaMemcpyDeviceToHost),
           "read barrier status");
  if (sticky) {
    const int zero = 0;
    cudaMemcpy(&S.ks.bar->sticky, &zero, sizeof(int), cudaMemcpyHostToDevice);
    return fail(ctx, NMC_ETIMEOUT, "a grid barrier wait expired; the sweep stopped early");
  }
  return NMC_OK;
}

// Host-side check of caller-given initial states.
int check_init(nmc_ctx *ctx, const Instance &I, int32_t replicas, const void *init_states) {
  if (!init_states) return NMC_OK;
  if (I.kind == NMC_KIND_KSAT) {
    const uint8_t *p = static_cast<const uint8_t *>(init_states);
    for (size_t i = 0; i < static_cast<size_t>(replicas) * I.ks.n; ++i)
      if (p[i] > 1) return fail(ctx, NMC_EINVAL, "k-SAT initial states must be 0/1");
    return NMC_OK;
  }
  const int32_t n = I.qp.n;
  const int16_t *p = static_cast<const int16_t *>(init_states);
  std::vector<int> seen(n);
  for (int32_t r = 0; r < replicas; ++r) {
    std::fill(seen.begin(), seen.end(), 0);
    for (int32_t k = 0; k < n; ++k) {
      const int16_t x = p[static_cast<size_t>(r) * n + k];
      if (x < 0 || x >= n || seen[x]++)
        return fail(ctx, NMC_EINVAL, "QAP initial states must be permutations");
    }
  }
  return NMC_OK;
}

// Initial states (Philox or given), energies and best-so-far of an allocated replica set.
int init_replicas(nmc_ctx *ctx, const Instance &I, ReplicaSet &S, const void *init_states) {
  cudaError_t e = cudaSuccess;
  void *init_dev = nullptr;
  const size_t n = static_cast<size_t>(I.n_units);
  const size_t bytes = static_cast<size_t>(S.R) * n * (I.kind == NMC_KIND_KSAT ? 1 : 2);
  if (init_states) {
    if ((e = cudaMallocAsync(&init_dev, bytes, ctx->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(init_dev, init_states, bytes, cudaMemcpyHostToDevice, ctx->stream)) != cudaSuccess)
      return cuda_fail(ctx, e, "upload initial states");
  }
  if (I.kind == NMC_KIND_KSAT) {
    e = cudaMemsetAsync(S.ks.imp, 0, sizeof(uint32_t) * S.ks.W, ctx->stream);
    if (e == cudaSuccess)
      e = ksat_init_states(I.ks, S.ks, S.seed, static_cast<const uint8_t *>(init_dev), ctx->stream);
    if (e == cudaSuccess) e = ksat_energies(I.ks, S.ks, ctx->stream);
  } else {
    e = qap_init_states(I.qp, S.qp, S.seed, static_cast<const int16_t *>(init_dev), ctx->stream);
  }
  if (init_dev) cudaFreeAsync(init_dev, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "initialise replicas");
  return NMC_OK;
}

}  // namespace

namespace nmc {

int set_ctx_error(nmc_ctx *ctx, int code, const char *msg) {
  if (ctx) ctx->err = msg;
  return code;
}

// Mean colour-class size of a k-SAT instance (variables per class, rounded up).
int class_size(const Instance &I) { return (I.ks.n + I.ks.n_colours - 1) / std::max(1, I.ks.n_colours); }

double ksat_sweep_us(int32_t n, int32_t n_colours) {
  const double nc = std::max(1, n_colours);
  const double per_class = std::max(1.0, n / nc);
  const double rounds = std::ceil(per_class / 512.0);
  const double last = per_class - 512.0 * (rounds - 1.0);  // variables in the last round
  const double cycles = nc * (2200.0 + 16000.0 * (rounds - 1.0) + 27.0 * last);
  return cycles / 2070.0;  // SM clock in MHz
}

double qap_step_us(int32_t n) { return 0.008 * static_cast<double>(n) * n + 1.0; }

// CTAs per work item: few items are spread over the SMs (each cluster keeps its own copy of the
// word vector), but a colour class is not split below about 32 variables per CTA, where a
// cluster barrier per class costs more than the work it spreads (measured: 4-SAT N = 200 with 64
// replicas, 43 us per sweep on one CTA per word against 78 on eight; N = 1,000 with 256, 82
// against 105 on eight; N = 5,000 with 1,024 keeps four, 132 us).
int choose_ctas(int sms, long long cnt, int per_class) {
  int cs = 1;
  while (cs < 8 && cnt * cs * 2 <= sms && per_class >= 64 * cs) cs *= 2;
  return cs;
}

// Lanes per variable for about per_class / cs variables of a class on each CTA: teams of 8 up
// to ~24, of 4 up to ~100, single threads beyond (the one-thread kernel still runs its smaller
// classes with teams).
int choose_lanes(int cs, int per_class) {
  const int per_cta = per_class / cs;
  return per_cta <= 24 ? 8 : (per_cta <= 100 ? 4 : 1);
}

int batch_plan(nmc_ctx *ctx, int32_t n_sets, const int32_t *rs, const int32_t *t0,
               const int32_t *t1, BatchPlan *plan) {
  if (!ctx || !plan) return NMC_EINVAL;
  if (n_sets < 0 || (n_sets > 0 && (!rs || !t0 || !t1)))
    return fail(ctx, NMC_EINVAL, "bad batch arrays");
  const size_t max_vars = batch_max_vars(ctx->tab_len, ctx->device);
  std::vector<BatchItem> by_kq[2];
  std::vector<long long> cost[2];
  std::map<int32_t, int> seen;
  plan->max_n[0] = plan->max_n[1] = 0;
  int per_class[2] = {0, 0};  // largest mean colour-class size among the items
  for (int32_t i = 0; i < n_sets; ++i) {
    ReplicaSet *S = find_set(ctx, rs[i]);
    if (!S) return fail(ctx, NMC_EINVAL, "unknown replica set in batch");
    if (seen[rs[i]]++) return fail(ctx, NMC_EINVAL, "replica set repeated in batch");
    Instance *I = find_inst(ctx, S->inst);
    if (!I || I->kind != NMC_KIND_KSAT) return fail(ctx, NMC_EINVAL, "batch sets must be k-SAT");
    if (t0[i] < 0 || t1[i] < t0[i]) return fail(ctx, NMC_EINVAL, "need 0 <= t0 <= t1");
    if (t1[i] > t0[i] && (!I->bq || t1[i] > I->n_steps))
      return fail(ctx, NMC_ESTATE, "schedule missing or shorter than t1");
    if (I->ks.nb > 7) return fail(ctx, NMC_EINVAL, "batched sets need every variable in <= 127 clauses");
    if (static_cast<size_t>(I->ks.n) > max_vars)
      return fail(ctx, NMC_EINVAL, "instance too large for the batched kernel");
    if (t1[i] == t0[i]) continue;
    const int q = I->ks.kq == 1 ? 0 : 1;
    for (int32_t w = 0; w < S->ks.W; ++w) {
      BatchItem B{};
      B.occ_t = I->ks.occ_t;
      B.grp_base = I->ks.grp_base;
      B.cgrp = I->ks.cgrp;
      B.col_ptr = I->ks.col_ptr;
      B.orig = I->ks.orig;
      B.bq = I->bq;
      B.S = S->ks.S;
      B.best = S->ks.best;
      B.energy = S->ks.energy;
      B.best_energy = S->ks.best_energy;
      B.n = I->ks.n;
      B.n_colours = I->ks.n_colours;
      B.n_groups = I->ks.n_groups;
      B.W = S->ks.W;
      B.w = w;
      B.t0 = t0[i];
      B.t1 = t1[i];
      B.k0 = static_cast<uint32_t>(S->seed);
      B.k1 = static_cast<uint32_t>(S->seed >> 32);
      by_kq[q].push_back(B);
      // longest-first by estimated time (small instances are bound by the per-class latency,
      // not by their work)
      cost[q].push_back(static_cast<long long>(
          1000.0 * ksat_sweep_us(I->ks.n, I->ks.n_colours) * (t1[i] - t0[i])));
      if (I->ks.n > plan->max_n[q]) plan->max_n[q] = I->ks.n;
    }
    per_class[q] = std::max(per_class[q], class_size(*I));
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, NMC_ECUDA, "query SMs");
  }
  plan->items.clear();
  for (int q = 0; q < 2; ++q) {
    std::vector<size_t> idx(by_kq[q].size());
    for (size_t k = 0; k < idx.size(); ++k) idx[k] = k;
    std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return cost[q][a] > cost[q][b]; });
    plan->off[q] = plan->items.size();
    plan->cnt[q] = static_cast<int>(idx.size());
    for (size_t k : idx) plan->items.push_back(by_kq[q][k]);
    // CTAs per item: spread few items over the SMs (word vectors replicated per cluster)
    int cs = 1, lanes = 0;
    const auto tuned = ctx->tune.find(std::make_tuple(q + 1, plan->max_n[q], plan->cnt[q]));
    if (const char *env = getenv("NMC_BATCH_CTAS")) {
      cs = atoi(env);
    } else if (tuned != ctx->tune.end()) {
      cs = tuned->second.first;
      lanes = tuned->second.second;
    } else {
      cs = choose_ctas(sms, plan->cnt[q], per_class[q]);
      lanes = choose_lanes(cs, per_class[q]);
    }
    if (cs != 1 && cs != 2 && cs != 4 && cs != 8) cs = 1;
    plan->cs[q] = cs;
    plan->lanes[q] = lanes;
  }
  plan->device = ctx->device;
  plan->stream = ctx->stream;
  plan->tab = ctx->tab;
  plan->tab_len = ctx->tab_len;
  return NMC_OK;
}

}  // namespace nmc

namespace {

// Makes room for `total` work items in the context's device work list (waiting for earlier
// launches that may still read it) and allocates the two work counters.
int reserve_items(nmc_ctx *ctx, size_t total) {
  if (total > ctx->items_cap) {
    NMC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    dev_free(ctx->items);
    ctx->items_cap = 0;
    NMC_CUDA(dev_alloc(&ctx->items, total), "allocate batch work list");
    ctx->items_cap = total;
  }
  if (!ctx->next_item) NMC_CUDA(dev_alloc(&ctx->next_item, 2), "allocate batch counters");
  return NMC_OK;
}

// Uploads a work list and launches it: items [off[q], off[q] + cnt[q]) have occurrence width
// q + 1. pt selects the kernels with temperature multipliers and energy statistics.
int launch_items(nmc_ctx *ctx, const std::vector<BatchItem> &items, const size_t off[2],
                 const int cnt[2], const int max_n[2], const int cs[2], bool pt,
                 const int lanes[2]) {
  if (items.empty()) return NMC_OK;
  const int rc = reserve_items(ctx, items.size());
  if (rc != NMC_OK) return rc;
  // cudaMemcpyAsync stages pageable host memory before it returns
  NMC_CUDA(cudaMemcpyAsync(ctx->items, items.data(), sizeof(BatchItem) * items.size(),
                           cudaMemcpyHostToDevice, ctx->stream),
           "upload batch work list");
  if (!cnt[0] || !cnt[1]) {
    const int q = cnt[0] ? 0 : 1;
    NMC_CUDA(ksat_batch(ctx->items + off[q], cnt[q], q + 1, cs[q], max_n[q], ctx->next_item + q,
                        ctx->tab, ctx->tab_len, ctx->device, ctx->stream, pt, lanes[q]),
             "launch batched sweep");
    return NMC_OK;
  }
  // both widths: the two-entry items (k > 4) on the auxiliary stream, launched first, the
  // one-entry items on the context's stream, which then waits for the auxiliary one
  if (!ctx->kaux) {
    NMC_CUDA(cudaStreamCreateWithFlags(&ctx->kaux, cudaStreamNonBlocking), "create batch stream");
    NMC_CUDA(cudaEventCreateWithFlags(&ctx->kfork, cudaEventDisableTiming), "create batch event");
    NMC_CUDA(cudaEventCreateWithFlags(&ctx->kjoin, cudaEventDisableTiming), "create batch event");
  }
  NMC_CUDA(cudaEventRecord(ctx->kfork, ctx->stream), "fork batch stream");
  NMC_CUDA(cudaStreamWaitEvent(ctx->kaux, ctx->kfork, 0), "fork batch stream");
  const cudaError_t e1 = ksat_batch(ctx->items + off[1], cnt[1], 2, cs[1], max_n[1],
                                    ctx->next_item + 1, ctx->tab, ctx->tab_len, ctx->device,
                                    ctx->kaux, pt, lanes[1]);
  // joined whether or not the launch succeeded, so that nothing is left unjoined
  const cudaError_t ej = cudaEventRecord(ctx->kjoin, ctx->kaux);
  const cudaError_t e0 = ksat_batch(ctx->items + off[0], cnt[0], 1, cs[0], max_n[0],
                                    ctx->next_item, ctx->tab, ctx->tab_len, ctx->device,
                                    ctx->stream, pt, lanes[0]);
  cudaError_t ew = ej == cudaSuccess ? cudaStreamWaitEvent(ctx->stream, ctx->kjoin, 0) : ej;
  if (ew != cudaSuccess) cudaStreamSynchronize(ctx->kaux);  // no join: wait on the host instead
  if (e1 != cudaSuccess) return cuda_fail(ctx, e1, "launch batched sweep");
  if (e0 != cudaSuccess) return cuda_fail(ctx, e0, "launch batched sweep");
  if (ew != cudaSuccess) return cuda_fail(ctx, ew, "join batch stream");
  return NMC_OK;
}

// The work item of word w of k-SAT set S for sweeps [t0, t1).
BatchItem ksat_item(const Instance &I, const ReplicaSet &S, int32_t w, int32_t t0, int32_t t1) {
  BatchItem B{};
  B.occ_t = I.ks.occ_t;
  B.grp_base = I.ks.grp_base;
  B.cgrp = I.ks.cgrp;
  B.col_ptr = I.ks.col_ptr;
  B.orig = I.ks.orig;
  B.bq = I.bq;
  B.S = S.ks.S;
  B.best = S.ks.best;
  B.energy = S.ks.energy;
  B.best_energy = S.ks.best_energy;
  B.n = I.ks.n;
  B.n_colours = I.ks.n_colours;
  B.n_groups = I.ks.n_groups;
  B.W = S.ks.W;
  B.w = w;
  B.t0 = t0;
  B.t1 = t1;
  B.k0 = static_cast<uint32_t>(S.seed);
  B.k1 = static_cast<uint32_t>(S.seed >> 32);
  return B;
}

// CTAs per work item and lanes per variable for a launch of the `cnt` items of one instance (a
// tuned shape when the context has one, else as batch_plan chooses).
void tuned_shape(nmc_ctx *ctx, const Instance &I, int cnt, int *cs, int *lanes) {
  *lanes = 0;
  const auto t = ctx->tune.find(std::make_tuple(I.ks.kq, I.ks.n, cnt));
  if (!getenv("NMC_BATCH_CTAS") && t != ctx->tune.end()) {
    *cs = t->second.first;
    *lanes = t->second.second;
    return;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
    cudaGetLastError();
    sms = 1;
  }
  int c = choose_ctas(sms, cnt, class_size(I));
  if (const char *env = getenv("NMC_BATCH_CTAS")) c = atoi(env);
  if (c != 1 && c != 2 && c != 4 && c != 8) c = 1;
  *cs = c;
  *lanes = choose_lanes(c, class_size(I));
}

// The checks every batched-kernel path makes on a k-SAT instance.
int check_batchable(nmc_ctx *ctx, const Instance &I) {
  if (I.kind != NMC_KIND_KSAT) return fail(ctx, NMC_EINVAL, "needs a k-SAT instance");
  if (I.ks.nb > 7) return fail(ctx, NMC_EINVAL, "needs every variable in <= 127 clauses");
  if (static_cast<size_t>(I.ks.n) > batch_max_vars(ctx->tab_len, ctx->device))
    return fail(ctx, NMC_EINVAL, "instance too large for the batched kernel");
  return NMC_OK;
}

}  // namespace

extern "C" {

int nmc_batch_run(nmc_ctx *ctx, int32_t n_sets, const int32_t *rs, const int32_t *t0,
                  const int32_t *t1);

int nmc_create(nmc_ctx **out, int device, void *cuda_stream) {
  if (!out) return NMC_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return NMC_EINVAL;
  }
  nmc_ctx *ctx = new nmc_ctx();
  ctx->device = device;
  DeviceGuard g(device);
  if (!g.ok) {
    delete ctx;
    return NMC_ECUDA;
  }
  if (cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return NMC_ECUDA;
    }
    ctx->own_stream = true;
  }
  std::vector<uint32_t> tab(kTabCap);
  ctx->tab_len = build_table(tab.data(), kTabCap);
  if (cudaMalloc(&ctx->tab, sizeof(uint32_t) * kTabCap) != cudaSuccess ||
      cudaMemcpy(ctx->tab, tab.data(), sizeof(uint32_t) * kTabCap, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMalloc(&ctx->flag, sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    nmc_destroy(ctx);
    return NMC_ENOMEM;
  }
  *out = ctx;
  return NMC_OK;
}

void nmc_destroy(nmc_ctx *ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->kaux) {
    cudaStreamSynchronize(ctx->kaux);
    cudaStreamDestroy(ctx->kaux);
  }
  if (ctx->kfork) cudaEventDestroy(ctx->kfork);
  if (ctx->kjoin) cudaEventDestroy(ctx->kjoin);
  for (auto &kv : ctx->sets) free_set(kv.second);
  for (auto &kv : ctx->insts) free_instance(kv.second);
  dev_free(ctx->tab);
  dev_free(ctx->flag);
  dev_free(ctx->items);
  dev_free(ctx->next_item);
  dev_free(ctx->qitems);
  for (int q = 0; q < kQapShapes; ++q) {
    if (ctx->qaux[q]) {
      cudaStreamSynchronize(ctx->qaux[q]);
      cudaStreamDestroy(ctx->qaux[q]);
    }
    if (ctx->qjoin[q]) cudaEventDestroy(ctx->qjoin[q]);
  }
  if (ctx->qfork) cudaEventDestroy(ctx->qfork);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  cudaGetLastError();
  delete ctx;
}

const char *nmc_last_error(nmc_ctx *ctx) { return ctx ? ctx->err.c_str() : kStaticNoCtx; }

int nmc_sync(nmc_ctx *ctx) {
  if (!ctx) return NMC_EINVAL;
  DeviceGuard g(ctx->device);
  NMC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  for (auto &kv : ctx->sets) {
    const int rc = check_timeout(ctx, kv.second);
    if (rc != NMC_OK) return rc;
  }
  return NMC_OK;
}

int nmc_selftest_wait_timeout(nmc_ctx *ctx, int32_t timeout_ms) {
  if (!ctx) return NMC_EINVAL;
  if (timeout_ms < 1 || timeout_ms > 10000) return fail(ctx, NMC_EINVAL, "timeout_ms out of range");
  DeviceGuard g(ctx->device);
  GridBarrier *gb = nullptr;
  NMC_CUDA(cudaMalloc(&gb, sizeof(GridBarrier)), "allocate barrier");
  cudaError_t e = cudaMemset(gb, 0, sizeof(GridBarrier));
  if (e == cudaSuccess) e = wait_selftest(gb, 1000000ull * (unsigned long long)timeout_ms, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  GridBarrier host{};
  if (e == cudaSuccess) e = cudaMemcpy(&host, gb, sizeof(GridBarrier), cudaMemcpyDeviceToHost);
  cudaFree(gb);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "wait self-test");
  if (host.sticky && host.error) return fail(ctx, NMC_ETIMEOUT, "bounded wait expired as designed");
  return NMC_OK;
}

int32_t nmc_threshold_table(uint32_t *out, int32_t cap) {
  std::vector<uint32_t> tab(kTabCap);
  const int32_t len = build_table(tab.data(), kTabCap);
  if (out)
    for (int32_t j = 0; j < cap; ++j) out[j] = j < kTabCap ? tab[j] : 0u;
  return len;
}

}  // extern "C"

namespace nmc {

int prep_fail(HostKsat *out, int code, const std::string &msg) {
  out->code = code;
  out->err = msg;
  return code;
}

// Runs f(lo, hi) over [0, count) split into contiguous ranges on up to 16 host threads, each
// taking at least per_thread items (inline when there are fewer). Every range writes disjoint
// outputs, so the result does not depend on the split.
int host_threads() {
  const unsigned hw = std::thread::hardware_concurrency();
  return hw == 0 ? 1 : static_cast<int>(std::min<unsigned>(hw, 16u));
}

template <typename F>
void parallel_ranges(int64_t count, F f, int64_t per_thread = 8192) {
  const int64_t T = std::max<int64_t>(1, std::min<int64_t>(host_threads(), count / per_thread));
  if (T <= 1) {
    f(int64_t{0}, count);
    return;
  }
  std::vector<std::thread> th;
  for (int64_t t = 1; t < T; ++t)
    th.emplace_back([&, t] { f(count * t / T, count * (t + 1) / T); });
  f(int64_t{0}, count / T);
  for (auto &x : th) x.join();
}

// Order of the k <= 4 occurrence entries of one group of 32 variables in the warp-interleaved
// layout. The kernel gathers, for occurrence slot j, the word of "other literal" p (p = 1, 2, 3)
// of all 32 lanes with one shared-memory load; the word of variable u sits in bank u mod 32, and
// a load takes as many passes as the largest number of distinct words it needs from one bank.
// The order of a variable's occurrences and of the other literals inside an occurrence does not
// change its energy change (a sum over occurrences of an OR over the other literals), so slot by
// slot every lane takes, from the next 8 of its occurrences not yet placed, the one and the order
// of its three literals that add the fewest distinct words to banks already used in this slot
// (first found on ties; a lane with none left takes an inert entry). Simulated on the
// 50,000-variable bench formula: 3.39 -> 1.98 passes per load on average (1.94 with every
// remaining occurrence a candidate, at several times the host time). A lane's occurrences in
// which its own literal is positive come first, those where it is negated next, so that the
// kernel can count each kind with one bit-sliced counter outside the slots where lanes differ.
struct BankOrder {
  std::vector<int32_t> pend[2][32];  // per lane: own-positive / own-negative occurrences to place
  int32_t addr[3][32][32];           // per literal position and bank: distinct words this slot
  int32_t cnt[3][32];

  int cost(int p, int32_t w) const {
    const int b = w & 31;
    for (int i = 0; i < cnt[p][b]; ++i)
      if (addr[p][b][i] == w) return 0;
    return cnt[p][b];
  }
  void add(int p, int32_t w) {
    const int b = w & 31;
    for (int i = 0; i < cnt[p][b]; ++i)
      if (addr[p][b][i] == w) return;
    addr[p][b][cnt[p][b]++] = w;
  }
  // Writes the group's len x 32 entries (int4 each: sign bytes, three word byte offsets). A
  // lane's own-positive occurrences fill its first npos slots, its own-negative ones the next.
  void build(int32_t g0, int32_t cend, int32_t len, int32_t n, const HostVec &occ,
             const std::vector<int32_t> &occ_ptr, const std::vector<int32_t> &orig,
             const std::vector<int32_t> &deg, const std::vector<int32_t> &npos, int32_t *dst0) {
    static const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    int32_t np[32];
    for (int32_t l = 0; l < 32; ++l) {
      pend[0][l].clear();
      pend[1][l].clear();
      np[l] = 0;
      const int32_t v = g0 + l;
      if (v >= cend) continue;
      np[l] = npos[orig[v]];
      for (int32_t j = 0; j < deg[orig[v]]; ++j) {
        const int32_t e = occ_ptr[v] + j;
        pend[occ[static_cast<size_t>(e) * 4] != 0 ? 1 : 0][l].push_back(e);
      }
    }
    for (int32_t j = 0; j < len; ++j) {
      for (int p = 0; p < 3; ++p)
        for (int b = 0; b < 32; ++b) cnt[p][b] = 0;
      for (int32_t l = 0; l < 32; ++l) {
        int32_t *dst = dst0 + (static_cast<size_t>(j) * 32 + l) * 4;
        std::vector<int32_t> &pool = pend[j < np[l] ? 0 : 1][l];
        if (pool.empty()) {  // inert: own sign 0, one always-true literal (word n)
          dst[0] = static_cast<int32_t>(1u << 15);
          dst[1] = dst[2] = dst[3] = n * 4;
          for (int p = 0; p < 3; ++p) add(p, n);
          continue;
        }
        int best = -1, best_i = 0, best_pm = 0;
        const size_t window = std::min<size_t>(pool.size(), 8);  // next 8 candidates
        for (size_t i = 0; i < window && best != 0; ++i) {
          const int32_t *src = &occ[static_cast<size_t>(pool[i]) * 4];
          int cm[3][3];  // cm[p][k]: cost of literal k at position p
          for (int p = 0; p < 3; ++p)
            for (int k = 0; k < 3; ++k) cm[p][k] = cost(p, src[1 + k] >> 1);
          for (int pm = 0; pm < 6; ++pm) {
            const int c = cm[0][kPerm[pm][0]] + cm[1][kPerm[pm][1]] + cm[2][kPerm[pm][2]];
            if (best < 0 || c < best) {
              best = c;
              best_i = static_cast<int>(i);
              best_pm = pm;
              if (c == 0) break;
            }
          }
        }
        const int32_t *src = &occ[static_cast<size_t>(pool[best_i]) * 4];
        pool.erase(pool.begin() + best_i);
        uint32_t signs = static_cast<uint32_t>(src[0] != 0) << 7;
        for (int p = 0; p < 3; ++p) {
          const int32_t lit = src[1 + kPerm[best_pm][p]];
          signs |= static_cast<uint32_t>(lit & 1) << (8 * (p + 1) + 7);
          dst[1 + p] = (lit >> 1) * 4;
          add(p, lit >> 1);
        }
        dst[0] = static_cast<int32_t>(signs);
      }
    }
  }
};

int prepare_ksat(int32_t n_vars, int32_t n_clauses, int32_t k_max, const int32_t *lits,
                 HostKsat *out) {
  if (n_vars < 1 || n_vars >= (1 << 28)) return prep_fail(out, NMC_EINVAL, "n_vars out of range");
  if (n_clauses < 0) return prep_fail(out, NMC_EINVAL, "n_clauses < 0");
  if (k_max < 1 || k_max > 8) return prep_fail(out, NMC_EINVAL, "k_max must be in [1, 8]");
  if (n_clauses > 0 && !lits) return prep_fail(out, NMC_EINVAL, "lits is NULL");
  const int32_t n = n_vars, m = n_clauses, K = k_max;
  // -- checks, clause ranges in parallel; the first failing clause is the one reported
  {
    std::mutex fm;
    int64_t first = INT64_MAX;
    int first_kind = 0;  // 1 literal out of range, 2 variable repeated, 3 empty clause
    parallel_ranges(m, [&](int64_t a0, int64_t a1) {
      for (int64_t a = a0; a < a1; ++a) {
        int kind = 0, used = 0;
        for (int q = 0; q < K && kind == 0; ++q) {
          const int32_t l = lits[a * K + q];
          if (l == 0) continue;
          if (l < -n || l > n) {
            kind = 1;
            break;
          }
          const int32_t v = (l > 0 ? l : -l) - 1;
          for (int q2 = 0; q2 < q; ++q2) {
            const int32_t l2 = lits[a * K + q2];
            if (l2 != 0 && ((l2 > 0 ? l2 : -l2) - 1) == v) kind = 2;
          }
          ++used;
        }
        if (kind == 0 && used == 0) kind = 3;
        if (kind != 0) {
          std::lock_guard<std::mutex> g(fm);
          if (a < first) {
            first = a;
            first_kind = kind;
          }
          return;
        }
      }
    });
    if (first_kind == 1)
      return prep_fail(out, NMC_EINVAL, "literal out of range in clause " + std::to_string(first));
    if (first_kind == 2)
      return prep_fail(out, NMC_EINVAL, "variable repeated in clause " + std::to_string(first));
    if (first_kind == 3) return prep_fail(out, NMC_EINVAL, "empty clause " + std::to_string(first));
  }
  // -- variable -> clause incidence, clauses in ascending order. Clause ranges in parallel:
  //    thread t counts its clauses' occurrences of every variable; variable v's entries from
  //    thread t follow those of threads 0..t-1, so every list stays in clause order. (One
  //    thread when the per-thread counts would exceed 2^26 entries.)
  int64_t TC = std::max<int64_t>(1, std::min<int64_t>(host_threads(), m / 8192));
  if (TC * static_cast<int64_t>(n) > (int64_t(1) << 26)) TC = 1;
  std::vector<int32_t> cnt(static_cast<size_t>(TC) * n, 0);
  auto by_clause_range = [&](auto &&body) {
    parallel_ranges(TC, [&](int64_t t0, int64_t t1) {
      for (int64_t t = t0; t < t1; ++t) body(t, m * t / TC, m * (t + 1) / TC);
    }, 1);
  };
  by_clause_range([&](int64_t t, int64_t a0, int64_t a1) {
    int32_t *c = &cnt[static_cast<size_t>(t) * n];
    for (int64_t i = a0 * K; i < a1 * K; ++i) {
      const int32_t l = lits[i];
      if (l != 0) ++c[(l > 0 ? l : -l) - 1];
    }
  });
  std::vector<int32_t> deg(n, 0);
  parallel_ranges(n, [&](int64_t v0, int64_t v1) {
    for (int64_t v = v0; v < v1; ++v) {
      int32_t d = 0;
      for (int64_t t = 0; t < TC; ++t) d += cnt[static_cast<size_t>(t) * n + v];
      deg[v] = d;
    }
  }, 4096);
  int32_t dmax = 0;
  for (int32_t v = 0; v < n; ++v) dmax = deg[v] > dmax ? deg[v] : dmax;
  if (dmax > kMaxDegree)
    return prep_fail(out, NMC_EINVAL, "a variable occurs in more than 1023 clauses");
  std::vector<int32_t> vptr(n + 1, 0);
  for (int32_t v = 0; v < n; ++v) vptr[v + 1] = vptr[v] + deg[v];
  parallel_ranges(n, [&](int64_t v0, int64_t v1) {  // counts -> each thread's first slot
    for (int64_t v = v0; v < v1; ++v) {
      int32_t o = vptr[v];
      for (int64_t t = 0; t < TC; ++t) {
        int32_t &c = cnt[static_cast<size_t>(t) * n + v];
        const int32_t k = c;
        c = o;
        o += k;
      }
    }
  }, 4096);
  HostVec vcl(vptr[n] > 0 ? vptr[n] : 1);
  by_clause_range([&](int64_t t, int64_t a0, int64_t a1) {
    int32_t *c = &cnt[static_cast<size_t>(t) * n];
    for (int64_t a = a0; a < a1; ++a)
      for (int q = 0; q < K; ++q) {
        const int32_t l = lits[a * K + q];
        if (l != 0) vcl[c[(l > 0 ? l : -l) - 1]++] = static_cast<int32_t>(a);
      }
  });
  // -- occurrence entries in original ids, one per (variable, clause containing it): slot 0
  //    the variable's own sign (0 or -1), slots 1.. the clause's other literals 2u + neg, the
  //    rest lit_false. One pass of random clause reads, spread over threads; the colouring and
  //    the renumbered lists below stream it.
  const int kq = K <= 4 ? 1 : 2;
  const int slots = 4 * kq;
  const int32_t lit_false = 2 * n, lit_true = 2 * n + 1;
  HostVec occ0(static_cast<size_t>(vptr[n] > 0 ? vptr[n] : 1) * slots);
  parallel_ranges(n, [&](int64_t v0, int64_t v1) {
    for (int64_t ov = v0; ov < v1; ++ov)
      for (int32_t e = vptr[ov]; e < vptr[ov + 1]; ++e) {
        const int64_t a = vcl[e];
        int32_t *slot = &occ0[static_cast<size_t>(e) * slots];
        int s = 1;
        for (int q = 0; q < K; ++q) {
          const int32_t l = lits[a * K + q];
          if (l == 0) continue;
          const int32_t u = (l > 0 ? l : -l) - 1;
          const int32_t neg = l < 0 ? 1 : 0;
          if (u == ov)
            slot[0] = neg ? -1 : 0;
          else
            slot[s++] = 2 * u + neg;
        }
        for (; s < slots; ++s) slot[s] = lit_false;
      }
  }, 1024);
  // the tie order of the colouring: more occurrences first, then the smaller id (a counting
  // sort by degree, stable in id)
  std::vector<int32_t> ord(n);
  {
    std::vector<int32_t> start(dmax + 2, 0);
    for (int32_t v = 0; v < n; ++v) ++start[dmax - deg[v] + 1];
    for (int32_t d = 0; d <= dmax; ++d) start[d + 1] += start[d];
    for (int32_t v = 0; v < n; ++v) ord[start[dmax - deg[v]]++] = v;
  }
  // -- DSatur colouring: repeatedly the uncoloured variable whose coloured neighbours show the
  //    most distinct colours (then the one in more clauses, then the smaller id) takes the
  //    smallest colour none of its neighbours holds. Every variable has a rank in the fixed tie
  //    order, and the uncoloured variables sit in one bucket per saturation: a bitset over
  //    ranks with a summary word per 64 words and the index below which a bucket's summary
  //    words are all zero (the scan for its lowest rank starts there, so a sparse instance
  //    does not rescan empty words on every pick). The buckets are interleaved word by word
  //    (word w of bucket s at w * S + s), so moving a variable from saturation s to s + 1
  //    touches one cache line. A rising saturation only sets the variable's bit in its new
  //    bucket; the old bit goes stale and is dropped when a pick meets it (count[s] counts the
  //    live entries). The pick is the lowest live rank of the highest non-empty bucket.
  //    The colours next to each variable are kept as a 64-bit word for colours 0..63 and,
  //    beyond, in a map of further 64-bit words.
  std::vector<int32_t> colour(n, -1);
  int32_t n_colours = 0;
  {
    // per variable: the colours 0..63 its neighbours hold (all ones once it is coloured
    // itself, so one test skips both cases), and its saturation with its rank in the tie order
    std::vector<uint64_t> low(n, 0u);
    struct SatRank {
      int32_t sat;   // distinct colours among its coloured neighbours
      int32_t rank;  // position in the tie order
    };
    std::vector<SatRank> sr(n);
    for (int32_t r = 0; r < n; ++r) sr[ord[r]] = SatRank{0, r};
    const size_t nw = (static_cast<size_t>(n) + 63) / 64, ns = (nw + 63) / 64;
    size_t S = 16;  // bucket capacity (saturations 0..S-1), doubled on demand
    std::vector<uint64_t> bits(nw * S, 0u), summary(ns * S, 0u);
    std::vector<int64_t> count(S, 0);  // live entries per bucket
    std::vector<size_t> from(S, 0);  // per bucket: its summary words below this index are zero
    auto grow = [&]() {
      const size_t S2 = 2 * S;
      std::vector<uint64_t> b2(nw * S2, 0u), s2(ns * S2, 0u);
      for (size_t w = 0; w < nw; ++w)
        for (size_t s = 0; s < S; ++s) b2[w * S2 + s] = bits[w * S + s];
      for (size_t k = 0; k < ns; ++k)
        for (size_t s = 0; s < S; ++s) s2[k * S2 + s] = summary[k * S + s];
      bits.swap(b2);
      summary.swap(s2);
      count.resize(S2, 0);
      from.resize(S2, 0);
      S = S2;
    };
    auto insert = [&](int32_t s, int32_t r) {
      if (static_cast<size_t>(s) >= S) grow();
      bits[static_cast<size_t>(r >> 6) * S + s] |= uint64_t(1) << (r & 63);
      summary[static_cast<size_t>(r >> 12) * S + s] |= uint64_t(1) << ((r >> 6) & 63);
      if (static_cast<size_t>(r >> 12) < from[s]) from[s] = static_cast<size_t>(r >> 12);
      ++count[s];
    };
    auto clear = [&](int32_t s, int32_t r) {
      uint64_t &w = bits[static_cast<size_t>(r >> 6) * S + s];
      w &= ~(uint64_t(1) << (r & 63));
      if (w == 0u) summary[static_cast<size_t>(r >> 12) * S + s] &= ~(uint64_t(1) << ((r >> 6) & 63));
    };
    auto lowest = [&](int32_t s) -> int32_t {
      for (size_t k = from[s];; ++k)
        if (const uint64_t sw = summary[k * S + s]) {
          from[s] = k;
          const size_t wi = k * 64 + __builtin_ctzll(sw);
          return static_cast<int32_t>(wi * 64 + __builtin_ctzll(bits[wi * S + s]));
        }
    };
    std::unordered_map<int64_t, uint64_t> high;  // (v, block >= 1) -> colours 64 block ..
    auto has_high = [&](int32_t v, int32_t c) -> bool {
      const auto it = high.find(static_cast<int64_t>(v) * 4096 + c / 64);
      return it != high.end() && ((it->second >> (c % 64)) & 1u);
    };
    for (int32_t r = 0; r < n; ++r) insert(0, r);
    int32_t top = 0;  // highest saturation with an uncoloured variable
    for (int32_t left = n; left > 0; --left) {
      while (count[top] == 0) --top;
      int32_t v;
      while (true) {  // stale bits (variables that have moved up since) are dropped here
        const int32_t r = lowest(top);
        clear(top, r);
        v = ord[r];
        if (sr[v].sat == top) break;
      }
      --count[top];
      int32_t c;
      if (low[v] != ~uint64_t(0)) {
        c = __builtin_ctzll(~low[v]);
      } else {
        c = 64;
        while (has_high(v, c)) ++c;
      }
      colour[v] = c;
      low[v] = ~uint64_t(0);
      if (c + 1 > n_colours) n_colours = c + 1;
      const int32_t *p0 = &occ0[static_cast<size_t>(vptr[v]) * slots];
      const int32_t *p1 = &occ0[static_cast<size_t>(vptr[v + 1]) * slots];
      auto raise = [&](int32_t u) {  // its bit at the old saturation stays, now stale
        SatRank &x = sr[u];
        --count[x.sat];
        insert(++x.sat, x.rank);
        if (x.sat > top) top = x.sat;
      };
      if (c < 64) {
        const uint64_t cbit = uint64_t(1) << c;
        for (const int32_t *q = p0; q < p1; q += slots)
          for (int z = 1; z < slots; ++z) {
            const int32_t l = q[z];
            if (l >= lit_false) continue;
            uint64_t &lw = low[l >> 1];
            if (lw & cbit) continue;  // coloured, or colour c already next to it
            lw |= cbit;
            raise(l >> 1);
          }
      } else {
        for (const int32_t *q = p0; q < p1; q += slots)
          for (int z = 1; z < slots; ++z) {
            const int32_t l = q[z];
            if (l >= lit_false || colour[l >> 1] >= 0) continue;
            uint64_t &w = high[static_cast<int64_t>(l >> 1) * 4096 + c / 64];
            if ((w >> (c % 64)) & 1u) continue;
            w |= uint64_t(1) << (c % 64);
            raise(l >> 1);
          }
      }
    }
  }
  // -- renumber: colour-major; inside a colour class by decreasing degree, then original id
  //    (the order inside a class does not change the dynamics; similar degrees side by side
  //    keep the warp-interleaved occurrence groups below nearly free of padding). The tie
  //    order above is already (degree down, id up): a stable counting sort of it by colour.
  std::vector<int32_t> col_ptr(n_colours + 1, 0);
  for (int32_t v = 0; v < n; ++v) ++col_ptr[colour[v] + 1];
  for (int32_t c = 0; c < n_colours; ++c) col_ptr[c + 1] += col_ptr[c];
  std::vector<int32_t> orig(n), newid(n);
  // own-positive occurrences of each variable (k <= 4 layout: a group's lanes keep those first)
  std::vector<int32_t> npos(kq == 1 ? n : 0, 0);
  if (kq == 1)
    parallel_ranges(n, [&](int64_t v0, int64_t v1) {
      for (int64_t v = v0; v < v1; ++v)
        for (int32_t e = vptr[v]; e < vptr[v + 1]; ++e)
          npos[v] += occ0[static_cast<size_t>(e) * slots] == 0 ? 1 : 0;
    });
  {
    std::vector<int32_t> pos(col_ptr.begin(), col_ptr.end() - 1);
    for (int32_t r = 0; r < n; ++r) orig[pos[colour[ord[r]]]++] = ord[r];
    if (kq == 1) {
      // inside a class: degree down, then own-positive count down (a group's lanes then have
      // similar splits between positive and negative occurrences), then id up
      parallel_ranges(n_colours, [&](int64_t c0, int64_t c1) {
        for (int64_t c = c0; c < c1; ++c)
          std::stable_sort(orig.begin() + col_ptr[c], orig.begin() + col_ptr[c + 1],
                           [&](int32_t a, int32_t b) {
                             return deg[a] != deg[b] ? deg[a] > deg[b] : npos[a] > npos[b];
                           });
      }, 1);
    }
    for (int32_t p = 0; p < n; ++p) newid[orig[p]] = p;
  }
  // -- occurrence lists in new ids, each padded to a multiple of 4 occurrences
  std::vector<int32_t> occ_ptr(n + 1, 0);
  for (int32_t v = 0; v < n; ++v) occ_ptr[v + 1] = occ_ptr[v] + ((deg[orig[v]] + 3) & ~3);
  const int64_t n_occ = occ_ptr[n];
  HostVec occ(static_cast<size_t>(n_occ > 0 ? n_occ : 1) * slots);
  if (n_occ == 0) std::fill(occ.begin(), occ.end(), lit_false);
  parallel_ranges(n, [&](int64_t v0, int64_t v1) {
    for (int64_t v = v0; v < v1; ++v) {
      const int32_t ov = orig[v];
      int64_t o = occ_ptr[v];
      for (int32_t e = vptr[ov]; e < vptr[ov + 1]; ++e, ++o) {
        const int32_t *src = &occ0[static_cast<size_t>(e) * slots];
        int32_t *slot = &occ[static_cast<size_t>(o) * slots];
        slot[0] = src[0];
        for (int z = 1; z < slots; ++z) {
          const int32_t l = src[z];
          slot[z] = l >= lit_false ? l : 2 * newid[l >> 1] + (l & 1);
        }
      }
      for (; o < occ_ptr[v + 1]; ++o) {  // padding: a satisfied pseudo-clause (no effect)
        int32_t *slot = &occ[static_cast<size_t>(o) * slots];
        slot[0] = 0;
        slot[1] = lit_true;
        for (int z = 2; z < slots; ++z) slot[z] = lit_false;
      }
    }
  }, 1024);
  // -- the same lists interleaved per group of 32 consecutive variables of a colour class
  //    (group g covers new ids [col_ptr[c] + 32k, +32)): occurrence j of the group's lane l
  //    sits at grp_base[g] + (j*kq + q)*32 + l (int4 units), so one warp load of occurrence j
  //    is contiguous. Each group is padded to its longest list with inert entries. For k <= 4
  //    an entry is {sign bytes, 4u1, 4u2, 4u3}: the other literals as byte offsets of their
  //    variable's word in the shared-memory word vector, and bit 7 of byte 0 / 1 / 2 / 3 of the
  //    first field set when the own literal / literal 1 / 2 / 3 is negated. For k > 4 the two
  //    int4 are {sign bits, 4u1, 4u2, 4u3} and {4u4, 4u5, 4u6, 4u7}: the same byte offsets, the
  //    signs of the own literal and literals 1..3 in bit 7 and those of literals 4..7 in bit 6
  //    of bytes 0..3 of the first field (unused literals: word n, which is always 0, positive).
  std::vector<int32_t> cgrp(n_colours + 1, 0), grp_base(1, 0), grp_v0;
  for (int32_t c = 0; c < n_colours; ++c) {
    const int32_t size = col_ptr[c + 1] - col_ptr[c];
    cgrp[c + 1] = cgrp[c] + (size + 31) / 32;
    for (int32_t g0 = col_ptr[c]; g0 < col_ptr[c + 1]; g0 += 32) {
      int32_t len = 0;
      for (int32_t v = g0; v < std::min(g0 + 32, col_ptr[c + 1]); ++v)
        len = std::max(len, occ_ptr[v + 1] - occ_ptr[v]);
      grp_base.push_back(grp_base.back() + len * kq * 32);
      grp_v0.push_back(g0);
    }
  }
  // sign regions of every group (k <= 4): slots [0, a) hold own-positive occurrences in every
  // lane, slots from b on none; stored as a | b << 16 after the G + 1 offsets
  const int32_t n_groups = static_cast<int32_t>(grp_v0.size());
  grp_base.resize(static_cast<size_t>(2) * n_groups + 1, 0);
  if (kq == 1)
    for (int32_t c = 0; c < n_colours; ++c)
      for (int32_t g = cgrp[c]; g < cgrp[c + 1]; ++g) {
        int32_t lo = INT32_MAX, hi = 0;
        for (int32_t v = grp_v0[g]; v < std::min(grp_v0[g] + 32, col_ptr[c + 1]); ++v) {
          lo = std::min(lo, npos[orig[v]]);
          hi = std::max(hi, npos[orig[v]]);
        }
        grp_base[n_groups + 1 + g] = (lo & ~3) | (((hi + 3) & ~3) << 16);
      }
  // the class end of every group's first variable
  std::vector<int32_t> grp_end(grp_v0.size());
  for (int32_t c = 0; c < n_colours; ++c)
    for (int32_t g = cgrp[c]; g < cgrp[c + 1]; ++g) grp_end[g] = col_ptr[c + 1];
  // every entry of every group is written below (lanes x occurrences x kq int4)
  const int64_t n_rows = grp_base[n_groups];
  HostVec occ_t(static_cast<size_t>(std::max<int64_t>(n_rows, 1)) * 4);
  if (n_rows == 0) std::fill(occ_t.begin(), occ_t.end(), 0);
  parallel_ranges(static_cast<int64_t>(grp_v0.size()), [&](int64_t ga, int64_t gz) {
    BankOrder bo;
    for (int64_t g = ga; g < gz; ++g) {
      const int32_t g0 = grp_v0[g], cend = grp_end[g];
      const int32_t len = (grp_base[g + 1] - grp_base[g]) / (kq * 32);
      if (kq == 1) {
        bo.build(g0, cend, len, n, occ, occ_ptr, orig, deg, npos,
                 &occ_t[static_cast<size_t>(grp_base[g]) * 4]);
        continue;
      }
      // k > 4: two int4 per occurrence (src: {own sign mask, lit1..lit7} in literal ids; inert:
      // own sign 0, literal 1 always true (word n negated), the rest always false (word n))
      for (int32_t l = 0; l < 32; ++l) {
        const int32_t v = g0 + l;
        for (int32_t j = 0; j < len; ++j) {
          int32_t *dst = &occ_t[(static_cast<size_t>(grp_base[g]) + j * kq * 32 + l) * 4];
          int32_t *dst2 = dst + 32 * 4;  // the occurrence's second int4, one warp row further
          const bool real = v < cend && j < occ_ptr[v + 1] - occ_ptr[v];
          const int32_t *src = real ? &occ[static_cast<size_t>(occ_ptr[v] + j) * slots] : nullptr;
          auto lit = [&](int z) { return real ? src[z] : (z == 1 ? lit_true : lit_false); };
          uint32_t signs = static_cast<uint32_t>(real && src[0] != 0) << 7;
          for (int z = 1; z < 4; ++z) signs |= static_cast<uint32_t>(lit(z) & 1) << (8 * z + 7);
          for (int z = 4; z < 8; ++z) signs |= static_cast<uint32_t>(lit(z) & 1) << (8 * (z - 4) + 6);
          dst[0] = static_cast<int32_t>(signs);
          for (int z = 1; z < 4; ++z) dst[z] = (lit(z) >> 1) * 4;
          for (int z = 0; z < 4; ++z) dst2[z] = (lit(4 + z) >> 1) * 4;
        }
      }
    }
  }, 32);  // a group is 32 variables' lists
  HostVec clits(static_cast<size_t>(m > 0 ? m : 1) * K);
  if (m == 0) std::fill(clits.begin(), clits.end(), lit_false);
  parallel_ranges(m, [&](int64_t a0, int64_t a1) {
    for (int64_t a = a0; a < a1; ++a)
      for (int q = 0; q < K; ++q) {
        const int32_t l = lits[a * K + q];
        if (l == 0) {
          clits[a * K + q] = lit_false;
          continue;
        }
        const int32_t u = (l > 0 ? l : -l) - 1;
        clits[a * K + q] = 2 * newid[u] + (l < 0 ? 1 : 0);
      }
  });
  int nb = 2;
  while ((1 << nb) <= dmax) ++nb;
  out->n = n;
  out->m = m;
  out->K = K;
  out->n_colours = n_colours;
  out->kq = kq;
  out->nb = nb;
  out->n_occ = static_cast<int32_t>(n_occ);
  out->occ = std::move(occ);
  out->occ_ptr = std::move(occ_ptr);
  out->col_ptr = std::move(col_ptr);
  out->orig = std::move(orig);
  out->newid = std::move(newid);
  out->clits = std::move(clits);
  out->occ_t = std::move(occ_t);
  out->grp_base = std::move(grp_base);
  out->cgrp = std::move(cgrp);
  out->colour = std::move(colour);
  out->code = NMC_OK;
  return NMC_OK;
}

int upload_ksat(nmc_ctx *ctx, HostKsat &h, int32_t *inst_out) {
  if (!ctx || !inst_out) return NMC_EINVAL;
  if (h.code != NMC_OK) return fail(ctx, h.code, h.err);
  const int32_t n = h.n, m = h.m, K = h.K, n_colours = h.n_colours, kq = h.kq, nb = h.nb;
  const int64_t n_occ = h.n_occ;
  HostVec &occ = h.occ, &clits = h.clits, &occ_t = h.occ_t;
  std::vector<int32_t> &occ_ptr = h.occ_ptr, &col_ptr = h.col_ptr, &orig = h.orig,
                       &newid = h.newid,
                       &grp_base = h.grp_base, &cgrp = h.cgrp, &colour = h.colour;
  DeviceGuard g(ctx->device);
  Instance I;
  I.kind = NMC_KIND_KSAT;
  I.n_units = n;
  I.ks.n = n;
  I.ks.m = m;
  I.ks.kmax = K;
  I.ks.n_colours = n_colours;
  I.ks.n_groups = cgrp.back();
  I.ks.kq = kq;
  I.ks.nb = nb;
  I.ks.n_occ = static_cast<int32_t>(n_occ);
  I.colour = colour;
  cudaError_t e = cudaSuccess;
  if ((e = dev_alloc(&I.ks.occ, occ.size() / 4)) != cudaSuccess ||
      (e = dev_alloc(&I.ks.occ_ptr, n + 1)) != cudaSuccess ||
      (e = dev_alloc(&I.ks.col_ptr, n_colours + 1)) != cudaSuccess ||
      (e = dev_alloc(&I.ks.orig, n)) != cudaSuccess ||
      (e = dev_alloc(&I.ks.newid, n)) != cudaSuccess ||
      (e = dev_alloc(&I.ks.clits, clits.size())) != cudaSuccess ||
      (e = dev_alloc(&I.ks.occ_t, occ_t.size() / 4)) != cudaSuccess ||
      (e = dev_alloc(&I.ks.grp_base, grp_base.size())) != cudaSuccess ||
      (e = dev_alloc(&I.ks.cgrp, cgrp.size())) != cudaSuccess ||
      (e = cudaMemcpy(I.ks.occ_t, occ_t.data(), sizeof(int32_t) * occ_t.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(I.ks.grp_base, grp_base.data(), sizeof(int32_t) * grp_base.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(I.ks.cgrp, cgrp.data(), sizeof(int32_t) * cgrp.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(I.ks.occ, occ.data(), sizeof(int32_t) * occ.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(I.ks.occ_ptr, occ_ptr.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(I.ks.col_ptr, col_ptr.data(), sizeof(int32_t) * (n_colours + 1), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(I.ks.orig, orig.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(I.ks.newid, newid.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(I.ks.clits, clits.data(), sizeof(int32_t) * clits.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    free_instance(I);
    return cuda_fail(ctx, e, "upload k-SAT instance");
  }
  const int32_t id = ctx->next_inst++;
  ctx->insts[id] = I;
  *inst_out = id;
  return NMC_OK;
}


}  // namespace nmc

namespace nmc {

int qap_batch_join(nmc_ctx *ctx, uint32_t joins) {
  if (!ctx) return NMC_EINVAL;
  cudaError_t err = cudaSuccess;
  for (int q = 0; q < kQapShapes; ++q)
    if (joins & (1u << q)) {
      const cudaError_t e = cudaStreamWaitEvent(ctx->stream, ctx->qjoin[q], 0);
      if (err == cudaSuccess) err = e;
    }
  return err == cudaSuccess ? NMC_OK : cuda_fail(ctx, err, "join QAP streams");
}

int qap_batch_enqueue(nmc_ctx *ctx, int32_t n_sets, const int32_t *rs, const int32_t *t0,
                      const int32_t *t1, uint32_t *joins) {
  *joins = 0;
  if (!ctx) return NMC_EINVAL;
  if (n_sets < 0 || (n_sets > 0 && (!rs || !t0 || !t1)))
    return fail(ctx, NMC_EINVAL, "bad batch arrays");
  DeviceGuard g(ctx->device);
  std::vector<QapArgs> by_npl[kQapShapes];
  int max_n[kQapShapes] = {0};
  std::map<int32_t, int> seen;
  for (int32_t i = 0; i < n_sets; ++i) {
    ReplicaSet *S = find_set(ctx, rs[i]);
    if (!S) return fail(ctx, NMC_EINVAL, "unknown replica set in batch");
    if (seen[rs[i]]++) return fail(ctx, NMC_EINVAL, "replica set repeated in batch");
    Instance *I = find_inst(ctx, S->inst);
    if (!I || I->kind != NMC_KIND_QAP) return fail(ctx, NMC_EINVAL, "batch sets must be QAP");
    if (t0[i] < 0 || t1[i] < t0[i]) return fail(ctx, NMC_EINVAL, "need 0 <= t0 <= t1");
    if (t1[i] > t0[i] && (!I->bq || t1[i] > I->n_steps))
      return fail(ctx, NMC_ESTATE, "schedule missing or shorter than t1");
    if (t1[i] == t0[i]) continue;
    const int n = I->qp.n;
    const int q = qap_shape(n);
    for (int b = 0; b < (S->R + 31) / 32; ++b)
      by_npl[q].push_back(qap_block_args(I->qp, S->qp, I->bq, ctx->tab, ctx->tab_len, t0[i], t1[i],
                                         S->seed, b));
    max_n[q] = std::max(max_n[q], n);
  }
  size_t total = 0;
  for (int q = 0; q < kQapShapes; ++q) total += by_npl[q].size();
  if (total == 0) return NMC_OK;
  if (total > ctx->qitems_cap) {
    NMC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    dev_free(ctx->qitems);
    ctx->qitems_cap = 0;
    NMC_CUDA(dev_alloc(&ctx->qitems, total), "allocate QAP work list");
    ctx->qitems_cap = total;
  }
  std::vector<QapArgs> all;
  all.reserve(total);
  size_t off[kQapShapes];
  for (int q = 0; q < kQapShapes; ++q) {
    off[q] = all.size();
    all.insert(all.end(), by_npl[q].begin(), by_npl[q].end());
  }
  NMC_CUDA(cudaMemcpyAsync(ctx->qitems, all.data(), sizeof(QapArgs) * total, cudaMemcpyHostToDevice,
                           ctx->stream),
           "upload QAP work list");
  // every launch shape on its own stream after the upload, so that shapes with few blocks run
  // side by side (and beside whatever the caller enqueues on its stream before the join)
  if (!ctx->qfork) {
    for (int q = 0; q < kQapShapes; ++q) {
      NMC_CUDA(cudaStreamCreateWithFlags(&ctx->qaux[q], cudaStreamNonBlocking), "create QAP stream");
      NMC_CUDA(cudaEventCreateWithFlags(&ctx->qjoin[q], cudaEventDisableTiming), "create QAP event");
    }
    NMC_CUDA(cudaEventCreateWithFlags(&ctx->qfork, cudaEventDisableTiming), "create QAP event");
  }
  NMC_CUDA(cudaEventRecord(ctx->qfork, ctx->stream), "fork QAP streams");
  cudaError_t err = cudaSuccess;
  for (int q = 0; q < kQapShapes && err == cudaSuccess; ++q) {
    if (by_npl[q].empty()) continue;
    if ((err = cudaStreamWaitEvent(ctx->qaux[q], ctx->qfork, 0)) != cudaSuccess) break;
    err = qap_batch(ctx->qitems + off[q], static_cast<int>(by_npl[q].size()), q, max_n[q],
                    ctx->tab_len, ctx->qaux[q]);
    const cudaError_t e2 = cudaEventRecord(ctx->qjoin[q], ctx->qaux[q]);
    if (e2 == cudaSuccess) *joins |= 1u << q;  // launched (or failed): joined all the same
    if (err == cudaSuccess) err = e2;
  }
  return err == cudaSuccess ? NMC_OK : cuda_fail(ctx, err, "launch batched QAP");
}

}  // namespace nmc

extern "C" {

int nmc_load_ksat(nmc_ctx *ctx, int32_t n_vars, int32_t n_clauses, int32_t k_max,
                  const int32_t *lits, int32_t *inst_out) {
  if (!ctx) return NMC_EINVAL;
  if (!inst_out) return fail(ctx, NMC_EINVAL, "inst_out is NULL");
  HostKsat h;
  if (prepare_ksat(n_vars, n_clauses, k_max, lits, &h) != NMC_OK) return fail(ctx, h.code, h.err);
  return upload_ksat(ctx, h, inst_out);
}

int nmc_load_qap(nmc_ctx *ctx, int32_t n, const int32_t *F, const int32_t *D, int32_t *inst_out) {
  if (!ctx) return NMC_EINVAL;
  if (!inst_out || !F || !D) return fail(ctx, NMC_EINVAL, "NULL argument");
  if (n < 1 || n > kMaxQapN) return fail(ctx, NMC_EINVAL, "QAP size must be in [1, 256]");
  std::vector<uint8_t> f(static_cast<size_t>(n) * n), d(static_cast<size_t>(n) * n);
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < n; ++j) {
      const int32_t fij = F[i * n + j], dij = D[i * n + j];
      if (fij < 0 || fij > 255 || dij < 0 || dij > 255)
        return fail(ctx, NMC_EINVAL, "QAP entries must be in [0, 255]");
      if (fij != F[j * n + i] || dij != D[j * n + i])
        return fail(ctx, NMC_EINVAL, "F and D must be symmetric");
      if (i == j && (fij != 0 || dij != 0))
        return fail(ctx, NMC_EINVAL, "F and D must have a zero diagonal");
      f[i * n + j] = static_cast<uint8_t>(fij);
      d[i * n + j] = static_cast<uint8_t>(dij);
    }
  DeviceGuard g(ctx->device);
  Instance I;
  I.kind = NMC_KIND_QAP;
  I.n_units = n;
  I.qp.n = n;
  cudaError_t e = cudaSuccess;
  if ((e = dev_alloc(&I.qp.F, f.size())) != cudaSuccess ||
      (e = dev_alloc(&I.qp.D, d.size())) != cudaSuccess ||
      (e = cudaMemcpy(I.qp.F, f.data(), f.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(I.qp.D, d.data(), d.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    free_instance(I);
    return cuda_fail(ctx, e, "upload QAP instance");
  }
  const int32_t id = ctx->next_inst++;
  ctx->insts[id] = I;
  *inst_out = id;
  return NMC_OK;
}

int nmc_unload(nmc_ctx *ctx, int32_t inst) {
  if (!ctx) return NMC_EINVAL;
  Instance *I = find_inst(ctx, inst);
  if (!I) return fail(ctx, NMC_EINVAL, "unknown instance");
  if (I->users > 0) return fail(ctx, NMC_ESTATE, "instance still has replica sets");
  DeviceGuard g(ctx->device);
  NMC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  free_instance(*I);
  ctx->insts.erase(inst);
  return NMC_OK;
}

int nmc_ksat_colouring(nmc_ctx *ctx, int32_t inst, int32_t *colour_out, int32_t *n_colours) {
  if (!ctx) return NMC_EINVAL;
  Instance *I = find_inst(ctx, inst);
  if (!I || I->kind != NMC_KIND_KSAT) return fail(ctx, NMC_EINVAL, "not a k-SAT instance");
  if (colour_out) std::memcpy(colour_out, I->colour.data(), sizeof(int32_t) * I->colour.size());
  if (n_colours) *n_colours = I->ks.n_colours;
  return NMC_OK;
}

static int set_schedule_impl(nmc_ctx *ctx, int32_t inst, int32_t n_steps, const float *beta,
                             bool on_device) {
  if (!ctx) return NMC_EINVAL;
  Instance *I = find_inst(ctx, inst);
  if (!I) return fail(ctx, NMC_EINVAL, "unknown instance");
  if (n_steps < 1 || !beta) return fail(ctx, NMC_EINVAL, "need n_steps >= 1 and a beta array");
  DeviceGuard g(ctx->device);
  const size_t count = static_cast<size_t>(I->n_units) * static_cast<size_t>(n_steps);
  float *src = nullptr;
  if (on_device) {
    src = const_cast<float *>(beta);
  } else {
    NMC_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&src), sizeof(float) * count, ctx->stream),
             "allocate schedule staging");
    const cudaError_t ce =
        cudaMemcpyAsync(src, beta, sizeof(float) * count, cudaMemcpyHostToDevice, ctx->stream);
    if (ce != cudaSuccess) {
      cudaFreeAsync(src, ctx->stream);
      return cuda_fail(ctx, ce, "copy schedule");
    }
  }
  uint32_t *bq = nullptr;
  cudaError_t e = cudaMalloc(&bq, sizeof(uint32_t) * count);
  if (e != cudaSuccess) {
    if (!on_device) cudaFreeAsync(src, ctx->stream);
    return cuda_fail(ctx, e, "allocate schedule");
  }
  int32_t bad = 0;
  e = cudaMemsetAsync(ctx->flag, 0, sizeof(int32_t), ctx->stream);
  if (e == cudaSuccess)
    e = quantize_schedule(src, I->n_units, n_steps, I->kind == NMC_KIND_KSAT ? I->ks.orig : nullptr,
                          bq, ctx->flag, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&bad, ctx->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
  if (!on_device) cudaFreeAsync(src, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    cudaFree(bq);
    return cuda_fail(ctx, e, "quantise schedule");
  }
  if (bad) {
    cudaFree(bq);
    return fail(ctx, NMC_EINVAL, "beta must be in [0, 65535] or +infinity (held)");
  }
  dev_free(I->bq);
  I->bq = bq;
  I->n_steps = n_steps;
  return NMC_OK;
}

int nmc_set_schedule_factored(nmc_ctx *ctx, int32_t inst, int32_t n_steps, const float *base,
                              const float *factor) {
  if (!ctx) return NMC_EINVAL;
  Instance *I = find_inst(ctx, inst);
  if (!I) return fail(ctx, NMC_EINVAL, "unknown instance");
  if (n_steps < 1 || !base || !factor) return fail(ctx, NMC_EINVAL, "need n_steps >= 1, base and factor");
  DeviceGuard g(ctx->device);
  const size_t count = static_cast<size_t>(I->n_units) * static_cast<size_t>(n_steps);
  float *src = nullptr;
  const size_t nb = sizeof(float) * (static_cast<size_t>(n_steps) + I->n_units);
  NMC_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&src), nb, ctx->stream), "allocate schedule staging");
  uint32_t *bq = nullptr;
  int32_t bad = 0;
  cudaError_t e = cudaMemcpyAsync(src, base, sizeof(float) * n_steps, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(src + n_steps, factor, sizeof(float) * I->n_units, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMalloc(&bq, sizeof(uint32_t) * count);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->flag, 0, sizeof(int32_t), ctx->stream);
  if (e == cudaSuccess)
    e = quantize_schedule_factored(src, src + n_steps, I->n_units, n_steps,
                                   I->kind == NMC_KIND_KSAT ? I->ks.orig : nullptr, bq, ctx->flag,
                                   ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&bad, ctx->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
  cudaFreeAsync(src, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    if (bq) cudaFree(bq);
    return cuda_fail(ctx, e, "factored schedule");
  }
  if (bad) {
    cudaFree(bq);
    return fail(ctx, NMC_EINVAL, "beta must be in [0, 65535] or +infinity (held)");
  }
  dev_free(I->bq);
  I->bq = bq;
  I->n_steps = n_steps;
  return NMC_OK;
}

int nmc_set_schedule(nmc_ctx *ctx, int32_t inst, int32_t n_steps, const float *beta) {
  return set_schedule_impl(ctx, inst, n_steps, beta, false);
}

int nmc_set_schedule_device(nmc_ctx *ctx, int32_t inst, int32_t n_steps, const float *beta_dev) {
  return set_schedule_impl(ctx, inst, n_steps, beta_dev, true);
}

int nmc_replicas_create(nmc_ctx *ctx, int32_t inst, int32_t replicas, uint64_t seed,
                        const void *init_states, int32_t *rs_out) {
  if (!ctx) return NMC_EINVAL;
  if (!rs_out) return fail(ctx, NMC_EINVAL, "rs_out is NULL");
  Instance *I = find_inst(ctx, inst);
  if (!I) return fail(ctx, NMC_EINVAL, "unknown instance");
  if (replicas < 1 || replicas > kMaxReplicas)
    return fail(ctx, NMC_EINVAL, "replicas must be in [1, 4096]");
  {
    const int rc = check_init(ctx, *I, replicas, init_states);
    if (rc != NMC_OK) return rc;
  }
  DeviceGuard g(ctx->device);
  ReplicaSet S;
  S.inst = inst;
  S.R = replicas;
  S.seed = seed;
  cudaError_t e = cudaSuccess;
  if (I->kind == NMC_KIND_KSAT) {
    const int32_t n = I->ks.n;
    const int32_t W = (replicas + 31) / 32;
    S.ks.R = replicas;
    S.ks.W = W;
    if ((e = dev_alloc(&S.ks.S, static_cast<size_t>(2 * n + 2) * W)) != cudaSuccess ||
        (e = dev_alloc(&S.ks.best, static_cast<size_t>(2 * n) * W)) != cudaSuccess ||
        (e = dev_alloc(&S.ks.energy, 32 * W)) != cudaSuccess ||
        (e = dev_alloc(&S.ks.best_energy, 32 * W)) != cudaSuccess ||
        (e = dev_alloc(&S.ks.imp, W)) != cudaSuccess ||
        (e = dev_alloc(&S.ks.bar, 1)) != cudaSuccess ||
        (e = cudaMemsetAsync(S.ks.imp, 0, sizeof(uint32_t) * W, ctx->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(S.ks.bar, 0, sizeof(GridBarrier), ctx->stream)) != cudaSuccess) {
      free_set(S);
      return cuda_fail(ctx, e, "allocate replica set");
    }
    const int rc = init_replicas(ctx, *I, S, init_states);
    if (rc != NMC_OK) {
      free_set(S);
      return rc;
    }
  } else {
    const int32_t n = I->qp.n;
    S.qp.R = replicas;
    const size_t cnt = static_cast<size_t>(replicas) * n;
    if ((e = dev_alloc(&S.qp.perm, cnt)) != cudaSuccess ||
        (e = dev_alloc(&S.qp.best_perm, cnt)) != cudaSuccess ||
        (e = dev_alloc(&S.qp.energy, replicas)) != cudaSuccess ||
        (e = dev_alloc(&S.qp.best_energy, replicas)) != cudaSuccess) {
      free_set(S);
      return cuda_fail(ctx, e, "allocate replica set");
    }
    const int rc = init_replicas(ctx, *I, S, init_states);
    if (rc != NMC_OK) {
      free_set(S);
      return rc;
    }
  }
  const int32_t id = ctx->next_set++;
  ctx->sets[id] = S;
  I->users++;
  *rs_out = id;
  return NMC_OK;
}

int nmc_replicas_reset(nmc_ctx *ctx, int32_t rs, uint64_t seed, const void *init_states) {
  if (!ctx) return NMC_EINVAL;
  ReplicaSet *S = find_set(ctx, rs);
  if (!S) return fail(ctx, NMC_EINVAL, "unknown replica set");
  Instance *I = find_inst(ctx, S->inst);
  if (!I) return fail(ctx, NMC_ESTATE, "instance was unloaded");
  const int rc = check_init(ctx, *I, S->R, init_states);
  if (rc != NMC_OK) return rc;
  DeviceGuard g(ctx->device);
  S->seed = seed;
  return init_replicas(ctx, *I, *S, init_states);
}

int nmc_replicas_restore(nmc_ctx *ctx, int32_t rs, const nmc_result *in) {
  if (!ctx) return NMC_EINVAL;
  if (!in || !in->states || !in->best_states)
    return fail(ctx, NMC_EINVAL, "restore needs states and best_states");
  ReplicaSet *S = find_set(ctx, rs);
  if (!S) return fail(ctx, NMC_EINVAL, "unknown replica set");
  Instance *I = find_inst(ctx, S->inst);
  if (!I) return fail(ctx, NMC_ESTATE, "instance was unloaded");
  int rc = check_init(ctx, *I, S->R, in->states);
  if (rc == NMC_OK) rc = check_init(ctx, *I, S->R, in->best_states);
  if (rc != NMC_OK) return rc;
  DeviceGuard g(ctx->device);
  const size_t bytes = static_cast<size_t>(S->R) * I->n_units * (I->kind == NMC_KIND_KSAT ? 1 : 2);
  void *dev = nullptr;
  NMC_CUDA(cudaMallocAsync(&dev, 2 * bytes, ctx->stream), "allocate restore staging");
  char *bdev = static_cast<char *>(dev), *sdev = bdev + bytes;
  cudaError_t e = cudaMemcpyAsync(bdev, in->best_states, bytes, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sdev, in->states, bytes, cudaMemcpyHostToDevice, ctx->stream);
  // the best states first (their energies become the best energies), then the current states
  if (I->kind == NMC_KIND_KSAT) {
    if (e == cudaSuccess) e = cudaMemsetAsync(S->ks.imp, 0, sizeof(uint32_t) * S->ks.W, ctx->stream);
    if (e == cudaSuccess) e = ksat_init_states(I->ks, S->ks, S->seed, reinterpret_cast<uint8_t *>(bdev), ctx->stream, true);
    if (e == cudaSuccess) e = ksat_energies(I->ks, S->ks, ctx->stream, true);
    if (e == cudaSuccess) e = ksat_init_states(I->ks, S->ks, S->seed, reinterpret_cast<uint8_t *>(sdev), ctx->stream, false);
    if (e == cudaSuccess) e = ksat_energies(I->ks, S->ks, ctx->stream, false);
  } else {
    if (e == cudaSuccess) e = qap_init_states(I->qp, S->qp, S->seed, reinterpret_cast<int16_t *>(bdev), ctx->stream, true);
    if (e == cudaSuccess) e = qap_init_states(I->qp, S->qp, S->seed, reinterpret_cast<int16_t *>(sdev), ctx->stream, false);
  }
  cudaFreeAsync(dev, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "restore replicas");
  return NMC_OK;
}

int nmc_replicas_destroy(nmc_ctx *ctx, int32_t rs) {
  if (!ctx) return NMC_EINVAL;
  ReplicaSet *S = find_set(ctx, rs);
  if (!S) return fail(ctx, NMC_EINVAL, "unknown replica set");
  DeviceGuard g(ctx->device);
  NMC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  Instance *I = find_inst(ctx, S->inst);
  if (I) I->users--;
  free_set(*S);
  ctx->sets.erase(rs);
  return NMC_OK;
}

int nmc_replicas_run(nmc_ctx *ctx, int32_t rs, int32_t t0, int32_t t1) {
  if (!ctx) return NMC_EINVAL;
  ReplicaSet *S = find_set(ctx, rs);
  if (!S) return fail(ctx, NMC_EINVAL, "unknown replica set");
  Instance *I = find_inst(ctx, S->inst);
  if (!I) return fail(ctx, NMC_ESTATE, "instance was unloaded");
  if (t0 < 0 || t1 < t0) return fail(ctx, NMC_EINVAL, "need 0 <= t0 <= t1");
  if (t1 > t0 && (!I->bq || t1 > I->n_steps))
    return fail(ctx, NMC_ESTATE, "schedule missing or shorter than t1");
  if (t1 == t0) return NMC_OK;
  if (I->kind == NMC_KIND_KSAT) {
    // one set through the shared-memory kernel (clusters of CTAs per word) when it fits;
    // the grid-barrier kernel otherwise (or when NMC_RUN_PATH=grid)
    const char *path = getenv("NMC_RUN_PATH");
    const bool force_grid = path && std::strcmp(path, "grid") == 0;
    if (!force_grid && I->ks.nb <= 7 &&
        static_cast<size_t>(I->ks.n) <= batch_max_vars(ctx->tab_len, ctx->device))
      return nmc_batch_run(ctx, 1, &rs, &t0, &t1);
  }
  DeviceGuard g(ctx->device);
  cudaError_t e;
  if (I->kind == NMC_KIND_KSAT)
    e = ksat_sweeps(I->ks, S->ks, I->bq, ctx->tab, ctx->tab_len, t0, t1, S->seed, ctx->device,
                    ctx->stream);
  else
    e = qap_steps(I->qp, S->qp, I->bq, ctx->tab, ctx->tab_len, t0, t1, S->seed, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "launch sweep");
  return NMC_OK;
}

static int read_impl(nmc_ctx *ctx, int32_t rs, const nmc_result *out, bool to_host) {
  if (!ctx) return NMC_EINVAL;
  if (!out) return fail(ctx, NMC_EINVAL, "out is NULL");
  ReplicaSet *S = find_set(ctx, rs);
  if (!S) return fail(ctx, NMC_EINVAL, "unknown replica set");
  Instance *I = find_inst(ctx, S->inst);
  if (!I) return fail(ctx, NMC_ESTATE, "instance was unloaded");
  DeviceGuard g(ctx->device);
  const size_t R = static_cast<size_t>(S->R), n = static_cast<size_t>(I->n_units);
  const size_t elem = I->kind == NMC_KIND_KSAT ? 1 : 2;
  const size_t state_bytes = R * n * elem;
  void *st = out->states, *bst = out->best_states;
  int64_t *en = out->energies, *ben = out->best_energies;
  char *stage = nullptr;
  if (to_host) {
    // staging sections start on 256-byte boundaries (the int64 energies need 8-byte alignment)
    const size_t sec_s = (state_bytes + 255) & ~static_cast<size_t>(255);
    const size_t sec_e = (R * sizeof(int64_t) + 255) & ~static_cast<size_t>(255);
    const size_t total = 2 * sec_s + 2 * sec_e;
    NMC_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&stage), total, ctx->stream), "allocate readback");
    st = out->states ? stage : nullptr;
    bst = out->best_states ? stage + sec_s : nullptr;
    en = out->energies ? reinterpret_cast<int64_t *>(stage + 2 * sec_s) : nullptr;
    ben = out->best_energies ? reinterpret_cast<int64_t *>(stage + 2 * sec_s + sec_e) : nullptr;
  }
  cudaError_t e;
  if (I->kind == NMC_KIND_KSAT)
    e = ksat_unpack(I->ks, S->ks, static_cast<uint8_t *>(st), static_cast<uint8_t *>(bst), en, ben,
                    ctx->stream);
  else
    e = qap_unpack(I->qp, S->qp, static_cast<int16_t *>(st), static_cast<int16_t *>(bst), en, ben,
                   ctx->stream);
  if (e == cudaSuccess && to_host) {
    if (out->states && e == cudaSuccess)
      e = cudaMemcpyAsync(out->states, st, state_bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (out->best_states && e == cudaSuccess)
      e = cudaMemcpyAsync(out->best_states, bst, state_bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (out->energies && e == cudaSuccess)
      e = cudaMemcpyAsync(out->energies, en, R * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream);
    if (out->best_energies && e == cudaSuccess)
      e = cudaMemcpyAsync(out->best_energies, ben, R * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream);
  }
  if (stage) cudaFreeAsync(stage, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "read replicas");
  if (to_host) {
    NMC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    return check_timeout(ctx, *S);
  }
  return NMC_OK;
}

int nmc_replicas_read(nmc_ctx *ctx, int32_t rs, const nmc_result *out) {
  return read_impl(ctx, rs, out, true);
}

int nmc_replicas_read_device(nmc_ctx *ctx, int32_t rs, const nmc_result *out_dev) {
  return read_impl(ctx, rs, out_dev, false);
}

int nmc_qap_batch_run(nmc_ctx *ctx, int32_t n_sets, const int32_t *rs, const int32_t *t0,
                      const int32_t *t1) {
  if (!ctx) return NMC_EINVAL;
  uint32_t joins = 0;
  const int rc = nmc::qap_batch_enqueue(ctx, n_sets, rs, t0, t1, &joins);
  const int rcj = nmc::qap_batch_join(ctx, joins);
  return rc != NMC_OK ? rc : rcj;
}

int32_t nmc_batch_max_vars(nmc_ctx *ctx) {
  if (!ctx) return 0;
  const size_t m = batch_max_vars(ctx->tab_len, ctx->device);
  return m > 0x7FFFFFFF ? 0x7FFFFFFF : static_cast<int32_t>(m);
}

int nmc_batch_run(nmc_ctx *ctx, int32_t n_sets, const int32_t *rs, const int32_t *t0,
                  const int32_t *t1) {
  if (!ctx) return NMC_EINVAL;
  DeviceGuard g(ctx->device);
  BatchPlan plan;
  const int rc = batch_plan(ctx, n_sets, rs, t0, t1, &plan);
  if (rc != NMC_OK) return rc;
  return launch_items(ctx, plan.items, plan.off, plan.cnt, plan.max_n, plan.cs, false, plan.lanes);
}

int nmc_replicas_set_ladder(nmc_ctx *ctx, int32_t rs, int32_t n_temps, const float *ladder,
                            const int32_t *slots) {
  if (!ctx) return NMC_EINVAL;
  ReplicaSet *S = find_set(ctx, rs);
  if (!S) return fail(ctx, NMC_EINVAL, "unknown replica set");
  Instance *I = find_inst(ctx, S->inst);
  if (!I) return fail(ctx, NMC_ESTATE, "instance was unloaded");
  if (I->kind == NMC_KIND_KSAT) {
    const int rc = check_batchable(ctx, *I);
    if (rc != NMC_OK) return rc;
  }
  if (n_temps < 1 || !ladder || S->R % n_temps != 0)
    return fail(ctx, NMC_EINVAL, "need a ladder of n_temps >= 1 temperatures dividing R");
  const int32_t R = S->R, L = n_temps, G = R / L;
  // one multiplier per replica lane: 32W for k-SAT words, R for QAP
  const int32_t W = I->kind == NMC_KIND_KSAT ? S->ks.W : (R + 31) / 32;
  std::vector<uint32_t> lq(L);
  for (int32_t k = 0; k < L; ++k) {
    const float b = ladder[k];
    if (!(b >= 0.0f && b <= 65535.0f))
      return fail(ctx, NMC_EINVAL, "ladder temperatures must be finite and in [0, 65535]");
    lq[k] = static_cast<uint32_t>(std::nearbyint(static_cast<double>(b) * 65536.0));
  }
  std::vector<int32_t> slot(R), at(R);
  std::vector<uint32_t> mult(32 * static_cast<size_t>(W), 65536u);
  std::vector<char> seen(L);
  for (int32_t g = 0; g < G; ++g) {
    std::fill(seen.begin(), seen.end(), 0);
    for (int32_t i = 0; i < L; ++i) {
      const int32_t r = g * L + i;
      const int32_t k = slots ? slots[r] : i;
      if (k < 0 || k >= L || seen[k])
        return fail(ctx, NMC_EINVAL, "each ladder's slots must be a permutation of 0..n_temps-1");
      seen[k] = 1;
      slot[r] = k;
      at[static_cast<size_t>(g) * L + k] = r;
      mult[r] = lq[k];
    }
  }
  DeviceGuard dg(ctx->device);
  // earlier launches may still read the old arrays
  NMC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  if (S->pt_L != L) {
    dev_free(S->pt_lq);
    S->pt_L = 0;
    NMC_CUDA(dev_alloc(&S->pt_lq, L), "allocate ladder");
  }
  if (!S->pt_slot) NMC_CUDA(dev_alloc(&S->pt_slot, R), "allocate ladder slots");
  if (!S->pt_at) NMC_CUDA(dev_alloc(&S->pt_at, R), "allocate ladder slots");
  if (!S->pt_mult) NMC_CUDA(dev_alloc(&S->pt_mult, mult.size()), "allocate ladder multipliers");
  NMC_CUDA(cudaMemcpyAsync(S->pt_lq, lq.data(), sizeof(uint32_t) * L, cudaMemcpyHostToDevice, ctx->stream), "upload ladder");
  NMC_CUDA(cudaMemcpyAsync(S->pt_slot, slot.data(), sizeof(int32_t) * R, cudaMemcpyHostToDevice, ctx->stream), "upload slots");
  NMC_CUDA(cudaMemcpyAsync(S->pt_at, at.data(), sizeof(int32_t) * R, cudaMemcpyHostToDevice, ctx->stream), "upload slots");
  NMC_CUDA(cudaMemcpyAsync(S->pt_mult, mult.data(), sizeof(uint32_t) * mult.size(), cudaMemcpyHostToDevice, ctx->stream), "upload multipliers");
  NMC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  S->pt_L = L;
  return NMC_OK;
}

int nmc_replicas_run_pt(nmc_ctx *ctx, int32_t rs, int32_t t0, int32_t t1,
                        int32_t sweeps_per_round) {
  if (!ctx) return NMC_EINVAL;
  ReplicaSet *S = find_set(ctx, rs);
  if (!S) return fail(ctx, NMC_EINVAL, "unknown replica set");
  Instance *I = find_inst(ctx, S->inst);
  if (!I) return fail(ctx, NMC_ESTATE, "instance was unloaded");
  int rc = I->kind == NMC_KIND_KSAT ? check_batchable(ctx, *I) : NMC_OK;
  if (rc != NMC_OK) return rc;
  if (S->pt_L < 1) return fail(ctx, NMC_ESTATE, "no ladder attached (nmc_replicas_set_ladder)");
  if (sweeps_per_round < 1) return fail(ctx, NMC_EINVAL, "sweeps_per_round must be >= 1");
  if (t0 < 0 || t1 < t0) return fail(ctx, NMC_EINVAL, "need 0 <= t0 <= t1");
  if (t1 > t0 && (!I->bq || t1 > I->n_steps))
    return fail(ctx, NMC_ESTATE, "schedule missing or shorter than t1");
  if (t1 == t0) return NMC_OK;
  DeviceGuard dg(ctx->device);
  if (I->kind == NMC_KIND_QAP) {
    // QAP: per segment one batched launch of the set's 32-replica blocks (with the
    // multipliers), then the exchange round on the 64-bit costs
    const int32_t Lq = S->pt_L, Gq = S->R / Lq, perq = sweeps_per_round;
    const int32_t nblk = (S->R + 31) / 32, n = I->qp.n, shape = qap_shape(n);
    int32_t t = t0;
    std::vector<QapArgs> qitems;
    std::vector<int32_t> ends;
    const int64_t max_chunk = std::max<int64_t>(nblk, 1 << 16);
    while (t < t1) {
      qitems.clear();
      ends.clear();
      while (t < t1 && static_cast<int64_t>(ends.size() + 1) * nblk <= max_chunk) {
        const int64_t te = std::min<int64_t>(t1, (static_cast<int64_t>(t) / perq + 1) * perq);
        for (int32_t b = 0; b < nblk; ++b) {
          QapArgs a = qap_block_args(I->qp, S->qp, I->bq, ctx->tab, ctx->tab_len, t,
                                     static_cast<int32_t>(te), S->seed, b);
          a.mult = S->pt_mult;
          qitems.push_back(a);
        }
        ends.push_back(static_cast<int32_t>(te));
        t = static_cast<int32_t>(te);
      }
      if (qitems.size() > ctx->qitems_cap) {
        NMC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
        dev_free(ctx->qitems);
        ctx->qitems_cap = 0;
        NMC_CUDA(dev_alloc(&ctx->qitems, qitems.size()), "allocate QAP work list");
        ctx->qitems_cap = qitems.size();
      }
      NMC_CUDA(cudaMemcpyAsync(ctx->qitems, qitems.data(), sizeof(QapArgs) * qitems.size(),
                               cudaMemcpyHostToDevice, ctx->stream),
               "upload QAP work list");
      for (size_t i = 0; i < ends.size(); ++i) {
        NMC_CUDA(qap_batch(ctx->qitems + i * nblk, nblk, shape, n, ctx->tab_len, ctx->stream),
                 "launch QAP steps");
        if (ends[i] % perq == 0)
          NMC_CUDA(pt_exchange64(S->pt_lq, Lq, Gq, reinterpret_cast<const long long *>(S->qp.energy),
                                 S->pt_slot, S->pt_at, S->pt_mult, ctx->tab, ctx->tab_len,
                                 static_cast<uint32_t>(ends[i] / perq - 1),
                                 static_cast<uint32_t>(S->seed), static_cast<uint32_t>(S->seed >> 32),
                                 ctx->stream),
                   "launch exchange round");
      }
    }
    return NMC_OK;
  }
  const int32_t W = S->ks.W, L = S->pt_L, G = S->R / L, per = sweeps_per_round;
  const int kq = I->ks.kq;
  int cs = 1, lanes = 0;
  tuned_shape(ctx, *I, W, &cs, &lanes);
  // segments end at t1 or after sweep t with (t+1) % per == 0, where an exchange round follows;
  // their work items are uploaded in chunks
  const int64_t max_chunk_items = std::max<int64_t>(W, 1 << 18);
  std::vector<BatchItem> items;
  std::vector<std::pair<int32_t, int32_t>> seg;
  int32_t t = t0;
  while (t < t1) {
    items.clear();
    seg.clear();
    while (t < t1 && static_cast<int64_t>(seg.size() + 1) * W <= max_chunk_items) {
      const int64_t te = std::min<int64_t>(t1, (static_cast<int64_t>(t) / per + 1) * per);
      seg.push_back({t, static_cast<int32_t>(te)});
      for (int32_t w = 0; w < W; ++w) {
        BatchItem B = ksat_item(*I, *S, w, t, static_cast<int32_t>(te));
        B.mult = S->pt_mult;
        items.push_back(B);
      }
      t = static_cast<int32_t>(te);
    }
    rc = reserve_items(ctx, items.size());
    if (rc != NMC_OK) return rc;
    NMC_CUDA(cudaMemcpyAsync(ctx->items, items.data(), sizeof(BatchItem) * items.size(),
                             cudaMemcpyHostToDevice, ctx->stream),
             "upload work list");
    for (size_t i = 0; i < seg.size(); ++i) {
      NMC_CUDA(ksat_batch(ctx->items + i * W, W, kq, cs, I->ks.n, ctx->next_item, ctx->tab,
                          ctx->tab_len, ctx->device, ctx->stream, true, lanes),
               "launch sweeps");
      const int32_t te = seg[i].second;
      if (te % per == 0)
        NMC_CUDA(pt_exchange(S->pt_lq, L, G, S->ks.energy, S->pt_slot, S->pt_at, S->pt_mult,
                             ctx->tab, ctx->tab_len, static_cast<uint32_t>(te / per - 1),
                             static_cast<uint32_t>(S->seed), static_cast<uint32_t>(S->seed >> 32),
                             ctx->stream),
                 "launch exchange round");
    }
  }
  return NMC_OK;
}

int nmc_replicas_read_slots(nmc_ctx *ctx, int32_t rs, int32_t *slots_out) {
  if (!ctx) return NMC_EINVAL;
  if (!slots_out) return fail(ctx, NMC_EINVAL, "slots_out is NULL");
  ReplicaSet *S = find_set(ctx, rs);
  if (!S) return fail(ctx, NMC_EINVAL, "unknown replica set");
  if (S->pt_L < 1) return fail(ctx, NMC_ESTATE, "no ladder attached (nmc_replicas_set_ladder)");
  DeviceGuard dg(ctx->device);
  NMC_CUDA(cudaMemcpyAsync(slots_out, S->pt_slot, sizeof(int32_t) * S->R, cudaMemcpyDeviceToHost,
                           ctx->stream),
           "read slots");
  NMC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  return NMC_OK;
}

int nmc_replicas_cluster_flip(nmc_ctx *ctx, int32_t rs, int32_t mask_rows, const uint8_t *mask,
                              const float *beta, uint32_t move_id, uint8_t *accepted_out) {
  if (!ctx) return NMC_EINVAL;
  ReplicaSet *S = find_set(ctx, rs);
  if (!S) return fail(ctx, NMC_EINVAL, "unknown replica set");
  Instance *I = find_inst(ctx, S->inst);
  if (!I) return fail(ctx, NMC_ESTATE, "instance was unloaded");
  if (I->kind != NMC_KIND_KSAT) return fail(ctx, NMC_EINVAL, "collective moves need a k-SAT set");
  if (!mask || !beta || (mask_rows != 1 && mask_rows != S->R))
    return fail(ctx, NMC_EINVAL, "need a mask of 1 or R rows and R temperatures");
  const int32_t n = I->ks.n, R = S->R, W = S->ks.W;
  const size_t mask_bytes = static_cast<size_t>(mask_rows) * n;
  for (size_t i = 0; i < mask_bytes; ++i)
    if (mask[i] > 1) return fail(ctx, NMC_EINVAL, "mask entries must be 0 or 1");
  for (int32_t r = 0; r < R; ++r)
    if (!(beta[r] >= 0.0f && beta[r] <= 65535.0f))
      return fail(ctx, NMC_EINVAL, "beta must be finite and in [0, 65535]");
  DeviceGuard dg(ctx->device);
  // staging: mask bytes, beta, accepted flags, then the kernels' scratch (256-byte sections)
  auto up = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
  const size_t off_beta = up(mask_bytes), off_acc = off_beta + up(sizeof(float) * R);
  const size_t off_scr = off_acc + up(static_cast<size_t>(R));
  const size_t total = off_scr + cluster_scratch_bytes(n, W);
  char *dev = nullptr;
  NMC_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&dev), total, ctx->stream), "allocate move scratch");
  cudaError_t e = cudaMemcpyAsync(dev, mask, mask_bytes, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dev + off_beta, beta, sizeof(float) * R, cudaMemcpyHostToDevice, ctx->stream);
  uint8_t *acc_dev = accepted_out ? reinterpret_cast<uint8_t *>(dev + off_acc) : nullptr;
  if (e == cudaSuccess)
    e = ksat_cluster_flip(I->ks, S->ks, reinterpret_cast<const uint8_t *>(dev), mask_rows,
                          reinterpret_cast<const float *>(dev + off_beta), move_id, S->seed,
                          ctx->tab, ctx->tab_len, dev + off_scr, acc_dev, ctx->stream);
  if (e == cudaSuccess && accepted_out)
    e = cudaMemcpyAsync(accepted_out, acc_dev, static_cast<size_t>(R), cudaMemcpyDeviceToHost, ctx->stream);
  cudaFreeAsync(dev, ctx->stream);
  if (e == cudaSuccess && accepted_out) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "collective move");
  return NMC_OK;
}

}  // extern "C"

namespace {

// Variable -> clause-slot incidence (slots e = a * kmax + q in increasing order) of a k-SAT
// instance, built from its device clause literals on first use and kept with the instance.
int ensure_lbp_graph(nmc_ctx *ctx, Instance &I) {
  if (I.lbp_vptr) return NMC_OK;
  const int32_t n = I.ks.n;
  const size_t slots = static_cast<size_t>(I.ks.m) * I.ks.kmax;
  std::vector<int32_t> cl(slots > 0 ? slots : 1);
  if (slots > 0)
    NMC_CUDA(cudaMemcpy(cl.data(), I.ks.clits, sizeof(int32_t) * slots, cudaMemcpyDeviceToHost),
             "read clause literals");
  std::vector<int32_t> vptr(static_cast<size_t>(n) + 1, 0), vedge;
  for (size_t e = 0; e < slots; ++e)
    if (cl[e] < 2 * n) vptr[(cl[e] >> 1) + 1]++;
  for (int32_t v = 0; v < n; ++v) vptr[v + 1] += vptr[v];
  vedge.resize(static_cast<size_t>(vptr[n]) + 1);
  std::vector<int32_t> fill(vptr.begin(), vptr.end() - 1);
  for (size_t e = 0; e < slots; ++e)
    if (cl[e] < 2 * n) vedge[fill[cl[e] >> 1]++] = static_cast<int32_t>(e);
  int32_t *dp = nullptr, *de = nullptr;
  cudaError_t e;
  if ((e = dev_alloc(&dp, vptr.size())) != cudaSuccess || (e = dev_alloc(&de, vedge.size())) != cudaSuccess ||
      (e = cudaMemcpy(dp, vptr.data(), sizeof(int32_t) * vptr.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(de, vedge.data(), sizeof(int32_t) * vedge.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    dev_free(dp);
    dev_free(de);
    return cuda_fail(ctx, e, "build LBP incidence");
  }
  I.lbp_vptr = dp;
  I.lbp_vedge = de;
  return NMC_OK;
}

// Device allocations released when the scope ends (after the stream has drained).
struct DevScratch {
  std::vector<void *> ptrs;
  cudaStream_t st = nullptr;
  ~DevScratch() {
    if (st) cudaStreamSynchronize(st);
    for (void *p : ptrs) cudaFree(p);
  }
  template <typename T>
  cudaError_t get(T **p, size_t count) {
    *p = nullptr;
    const cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (count ? count : 1));
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
};

// The adaptive ladder on a QAP replica set S (fresh, Philox initial states): level i runs steps
// [i T, (i+1) T) of every 32-replica block in one batched launch at the constant schedule beta_i,
// with per-replica double sums of the costs of the last sweeps_meas steps, then the one-thread
// ladder step.
int qap_ladder(nmc_ctx *ctx, const Instance &I, ReplicaSet &S, double beta0, double alpha,
                      double sigma_min, int32_t max_temps, int32_t sweeps_eq, int32_t sweeps_meas,
                      double *betas_out, double *sigmas_out, int32_t *n_temps_out) {
  const int32_t n = I.qp.n, R = S.R, nblk = (R + 31) / 32, shape = qap_shape(n);
  const int64_t T = static_cast<int64_t>(sweeps_eq) + sweeps_meas;
  uint32_t *bq = nullptr;
  double *stats = nullptr, *out_dev = nullptr;
  int rc = NMC_OK;
  cudaError_t e = cudaSuccess;
  if ((e = dev_alloc(&bq, static_cast<size_t>(n) * T)) != cudaSuccess ||
      (e = dev_alloc(&stats, 2 * static_cast<size_t>(R))) != cudaSuccess ||
      (e = dev_alloc(&out_dev, 2)) != cudaSuccess)
    rc = cuda_fail(ctx, e, "allocate ladder scratch");
  if (rc == NMC_OK && static_cast<size_t>(nblk) > ctx->qitems_cap) {
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) {
      rc = cuda_fail(ctx, e, "stream synchronize");
    } else {
      dev_free(ctx->qitems);
      ctx->qitems_cap = 0;
      if ((e = dev_alloc(&ctx->qitems, nblk)) != cudaSuccess)
        rc = cuda_fail(ctx, e, "allocate QAP work list");
      else
        ctx->qitems_cap = nblk;
    }
  }
  std::vector<QapArgs> items(nblk);
  double beta = beta0;
  for (int32_t i = 0; rc == NMC_OK && i < max_temps; ++i) {
    const float bf = static_cast<float>(beta);
    if (!(bf >= 0.0f && bf <= 65535.0f)) {
      rc = fail(ctx, NMC_EINVAL, "a ladder temperature left [0, 65535]");
      break;
    }
    const int32_t ts = static_cast<int32_t>(i * T), te = static_cast<int32_t>(ts + T);
    // the level's schedule holds steps [ts, te) only: the base pointer is moved back by ts steps
    // so that the kernel's index t * n + v lands in it (no access before bq)
    const uint32_t *base = reinterpret_cast<const uint32_t *>(
        reinterpret_cast<uintptr_t>(bq) - sizeof(uint32_t) * static_cast<size_t>(ts) * n);
    for (int32_t b = 0; b < nblk; ++b) {
      items[b] = qap_block_args(I.qp, S.qp, base, ctx->tab, ctx->tab_len, ts, te, S.seed, b);
      items[b].stats = stats;
      items[b].stats_t0 = ts + sweeps_eq;
    }
    double out[2] = {0.0, 0.0};
    if ((e = fill_schedule(bq, static_cast<size_t>(n) * T, beta, ctx->flag, ctx->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(stats, 0, sizeof(double) * 2 * R, ctx->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(ctx->qitems, items.data(), sizeof(QapArgs) * nblk, cudaMemcpyHostToDevice,
                             ctx->stream)) != cudaSuccess ||
        (e = qap_batch(ctx->qitems, nblk, shape, n, ctx->tab_len, ctx->stream)) != cudaSuccess ||
        (e = ladder_step_f64(stats, R, static_cast<long long>(R) * sweeps_meas, beta, alpha, out_dev,
                             ctx->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(out, out_dev, sizeof(out), cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) {
      rc = cuda_fail(ctx, e, "ladder level");
      break;
    }
    betas_out[i] = beta;
    sigmas_out[i] = out[0];
    *n_temps_out = i + 1;
    if (out[0] <= sigma_min) break;
    beta = out[1];
  }
  cudaStreamSynchronize(ctx->stream);
  dev_free(bq);
  dev_free(stats);
  dev_free(out_dev);
  return rc;
}

}  // namespace

extern "C" {

int nmc_batch_autotune(nmc_ctx *ctx, int32_t n_sets, const int32_t *rs, int32_t t0,
                       int32_t sweeps, int32_t *shapes_out) {
  if (!ctx) return NMC_EINVAL;
  if (sweeps < 1 || t0 < 0) return fail(ctx, NMC_EINVAL, "need t0 >= 0 and sweeps >= 1");
  DeviceGuard g(ctx->device);
  std::vector<int32_t> a(n_sets > 0 ? n_sets : 1, t0), b(n_sets > 0 ? n_sets : 1, t0 + sweeps);
  BatchPlan plan;
  int rc = batch_plan(ctx, n_sets, rs, a.data(), b.data(), &plan);
  if (rc != NMC_OK) return rc;
  if (shapes_out) std::fill(shapes_out, shapes_out + 6, 0);
  if (plan.items.empty()) return NMC_OK;
  // snapshot of every set's state, restored before each trial and at the end
  std::vector<std::pair<void *, size_t>> parts;
  for (int32_t i = 0; i < n_sets; ++i) {
    ReplicaSet *S = find_set(ctx, rs[i]);
    Instance *I = find_inst(ctx, S->inst);
    const size_t W = S->ks.W, n = I->ks.n;
    parts.push_back({S->ks.S, sizeof(uint32_t) * (2 * n + 2) * W});
    parts.push_back({S->ks.best, sizeof(uint32_t) * n * W});
    parts.push_back({S->ks.energy, sizeof(int32_t) * 32 * W});
    parts.push_back({S->ks.best_energy, sizeof(int32_t) * 32 * W});
  }
  size_t total = 0;
  for (auto &p : parts) total += (p.second + 255) & ~static_cast<size_t>(255);
  DevScratch d;
  d.st = ctx->stream;
  char *snap = nullptr;
  NMC_CUDA(d.get(&snap, total), "allocate tuning snapshot");
  auto copy_all = [&](bool save) -> cudaError_t {
    size_t off = 0;
    for (auto &p : parts) {
      char *s = snap + off;
      const cudaError_t e = save ? cudaMemcpyAsync(s, p.first, p.second, cudaMemcpyDeviceToDevice, ctx->stream)
                                 : cudaMemcpyAsync(p.first, s, p.second, cudaMemcpyDeviceToDevice, ctx->stream);
      if (e != cudaSuccess) return e;
      off += (p.second + 255) & ~static_cast<size_t>(255);
    }
    return cudaSuccess;
  };
  NMC_CUDA(copy_all(true), "snapshot replica sets");
  rc = reserve_items(ctx, plan.items.size());
  if (rc != NMC_OK) return rc;
  NMC_CUDA(cudaMemcpyAsync(ctx->items, plan.items.data(), sizeof(BatchItem) * plan.items.size(),
                           cudaMemcpyHostToDevice, ctx->stream),
           "upload batch work list");
  cudaEvent_t ev0, ev1;
  NMC_CUDA(cudaEventCreate(&ev0), "create event");
  if (cudaEventCreate(&ev1) != cudaSuccess) {
    cudaEventDestroy(ev0);
    return cuda_fail(ctx, cudaErrorUnknown, "create event");
  }
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
    if (!plan.cnt[q]) continue;
    float best_ms = 1e30f;
    int best_cs = plan.cs[q], best_lanes = 0;
    for (int cs : {1, 2, 4, 8}) {
      for (int lanes : {1, 4, 8}) {
        float ms = 0.0f;
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {  // the first run loads and sizes the kernel
          if ((e = copy_all(false)) != cudaSuccess) break;
          if ((e = cudaEventRecord(ev0, ctx->stream)) != cudaSuccess) break;
          const cudaError_t le = ksat_batch(ctx->items + plan.off[q], plan.cnt[q], q + 1, cs,
                                            plan.max_n[q], ctx->next_item + q, ctx->tab,
                                            ctx->tab_len, ctx->device, ctx->stream, false, lanes);
          if (le != cudaSuccess) {  // a shape this device cannot launch: skip it
            cudaGetLastError();
            ok = false;
            break;
          }
          if ((e = cudaEventRecord(ev1, ctx->stream)) != cudaSuccess ||
              (e = cudaEventSynchronize(ev1)) != cudaSuccess ||
              (e = cudaEventElapsedTime(&ms, ev0, ev1)) != cudaSuccess)
            break;
        }
        if (e != cudaSuccess) break;
        if (ok && ms < best_ms) {
          best_ms = ms;
          best_cs = cs;
          best_lanes = lanes;
        }
      }
      if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess && best_ms < 1e30f) {
      ctx->tune[std::make_tuple(q + 1, plan.max_n[q], plan.cnt[q])] = {best_cs, best_lanes};
      if (shapes_out) {
        shapes_out[3 * q] = best_cs;
        shapes_out[3 * q + 1] = best_lanes;
        shapes_out[3 * q + 2] = static_cast<int32_t>(best_ms * 1000.0f / sweeps);
      }
    }
  }
  if (e == cudaSuccess) e = copy_all(false);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
  return NMC_OK;
}

int nmc_cnf_lbp(nmc_ctx *ctx, int32_t inst, int32_t n_seeds, const uint8_t *x_star,
                const double *eps, double beta, int32_t n_lambda, const double *lambdas,
                double tol, int32_t max_iter, double *marg_out, double *corr_out,
                int32_t *iters_out, double *deltas_out, int32_t *n_done_out,
                double *overlap_out) {
  if (!ctx) return NMC_EINVAL;
  Instance *I = find_inst(ctx, inst);
  if (!I || I->kind != NMC_KIND_KSAT) return fail(ctx, NMC_EINVAL, "needs a k-SAT instance");
  if (n_seeds < 1 || !x_star || !marg_out || n_lambda < 1 || !lambdas || max_iter < 1)
    return fail(ctx, NMC_EINVAL, "need seeds, lambdas, max_iter >= 1 and marg_out");
  if (!std::isfinite(beta) || beta < 0.0 || !std::isfinite(tol) || tol < 0.0)
    return fail(ctx, NMC_EINVAL, "beta and tol must be finite and >= 0");
  const int32_t n = I->ks.n, m = I->ks.m, K = I->ks.kmax, S = n_seeds;
  for (size_t i = 0; i < static_cast<size_t>(S) * n; ++i)
    if (x_star[i] > 1) return fail(ctx, NMC_EINVAL, "seed states must be 0/1");
  for (int32_t k = 0; k < n_lambda; ++k)
    if (!std::isfinite(lambdas[k])) return fail(ctx, NMC_EINVAL, "lambdas must be finite");
  if (eps)
    for (int32_t i = 0; i < n; ++i)
      if (!std::isfinite(eps[i])) return fail(ctx, NMC_EINVAL, "eps must be finite");
  DeviceGuard dg(ctx->device);
  int rc = ensure_lbp_graph(ctx, *I);
  if (rc != NMC_OK) return rc;
  NMC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  DevScratch d;
  d.st = ctx->stream;
  uint8_t *x_in = nullptr, *xs = nullptr;
  double *eps_in = nullptr, *eps_d = nullptr, *marg = nullptr, *corr = nullptr, *deltas = nullptr,
         *overlap = nullptr;
  int32_t *iters = nullptr, *n_done = nullptr;
  char *scratch = nullptr;
  const size_t sn = static_cast<size_t>(S) * n;
  NMC_CUDA(d.get(&x_in, sn), "allocate LBP seeds");
  NMC_CUDA(d.get(&xs, sn), "allocate LBP seeds");
  if (eps) NMC_CUDA(d.get(&eps_in, n), "allocate eps");
  NMC_CUDA(d.get(&eps_d, n), "allocate eps");
  NMC_CUDA(d.get(&marg, sn), "allocate marginals");
  NMC_CUDA(d.get(&corr, static_cast<size_t>(S) * m), "allocate correlations");
  NMC_CUDA(d.get(&iters, static_cast<size_t>(S) * n_lambda), "allocate LBP report");
  NMC_CUDA(d.get(&deltas, static_cast<size_t>(S) * n_lambda), "allocate LBP report");
  NMC_CUDA(d.get(&n_done, S), "allocate LBP report");
  NMC_CUDA(d.get(&overlap, 2 * static_cast<size_t>(S)), "allocate LBP report");
  NMC_CUDA(d.get(&scratch, lbp_scratch_bytes(n, m, K, S, n_lambda)),
           "allocate LBP messages");
  NMC_CUDA(cudaMemcpyAsync(x_in, x_star, sn, cudaMemcpyHostToDevice, ctx->stream), "upload seeds");
  if (eps)
    NMC_CUDA(cudaMemcpyAsync(eps_in, eps, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream),
             "upload eps");
  NMC_CUDA(lbp_prepare(x_in, eps_in, I->ks.orig, I->lbp_vptr, n, S, xs, eps_d, ctx->stream),
           "prepare LBP");
  LbpArgs A{};
  A.clits = I->ks.clits;
  A.vptr = I->lbp_vptr;
  A.vedge = I->lbp_vedge;
  A.orig = I->ks.orig;
  A.n = n;
  A.m = m;
  A.kmax = K;
  A.S = S;
  A.n_lambda = n_lambda;
  A.max_iter = max_iter;
  A.eps = eps_d;
  A.xs = xs;
  A.lambdas = lambdas;
  A.beta = beta;
  A.tol = tol;
  A.scratch = scratch;
  A.marg = marg;
  A.corr = corr;
  A.iters = iters;
  A.deltas = deltas;
  A.n_done = n_done;
  A.overlap = overlap;
  const int err = lbp_run(A, ctx->stream);
  if (err != 0) return cuda_fail(ctx, static_cast<cudaError_t>(err), "LBP");
  NMC_CUDA(cudaMemcpyAsync(marg_out, marg, sizeof(double) * sn, cudaMemcpyDeviceToHost, ctx->stream), "read marginals");
  if (corr_out)
    NMC_CUDA(cudaMemcpyAsync(corr_out, corr, sizeof(double) * S * static_cast<size_t>(m), cudaMemcpyDeviceToHost, ctx->stream), "read correlations");
  if (iters_out)
    NMC_CUDA(cudaMemcpyAsync(iters_out, iters, sizeof(int32_t) * S * static_cast<size_t>(n_lambda), cudaMemcpyDeviceToHost, ctx->stream), "read LBP report");
  if (deltas_out)
    NMC_CUDA(cudaMemcpyAsync(deltas_out, deltas, sizeof(double) * S * static_cast<size_t>(n_lambda), cudaMemcpyDeviceToHost, ctx->stream), "read LBP report");
  if (n_done_out)
    NMC_CUDA(cudaMemcpyAsync(n_done_out, n_done, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, ctx->stream), "read LBP report");
  if (overlap_out)
    NMC_CUDA(cudaMemcpyAsync(overlap_out, overlap, sizeof(double) * 2 * S, cudaMemcpyDeviceToHost, ctx->stream), "read LBP report");
  NMC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  return NMC_OK;
}

int nmc_cnf_backbone(nmc_ctx *ctx, int32_t inst, int32_t n_seeds, const double *corr,
                     double beta, double seed_thr, double cutoff, int32_t *labels_out,
                     int32_t *n_clusters_out) {
  if (!ctx) return NMC_EINVAL;
  Instance *I = find_inst(ctx, inst);
  if (!I || I->kind != NMC_KIND_KSAT) return fail(ctx, NMC_EINVAL, "needs a k-SAT instance");
  if (n_seeds < 1 || !corr || !labels_out) return fail(ctx, NMC_EINVAL, "need correlations and labels_out");
  if (!std::isfinite(beta) || beta <= 0.0 || std::isnan(seed_thr) || std::isnan(cutoff))
    return fail(ctx, NMC_EINVAL, "beta must be finite and > 0, thresholds not NaN");
  const int32_t n = I->ks.n, m = I->ks.m, S = n_seeds;
  for (size_t i = 0; i < static_cast<size_t>(S) * m; ++i)
    if (!(corr[i] >= -1.0 && corr[i] <= 1.0)) return fail(ctx, NMC_EINVAL, "correlations must be in [-1, 1]");
  DeviceGuard dg(ctx->device);
  NMC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  DevScratch d;
  d.st = ctx->stream;
  double *corr_d = nullptr;
  int32_t *lab = nullptr, *ncl = nullptr;
  char *scratch = nullptr;
  NMC_CUDA(d.get(&corr_d, static_cast<size_t>(S) * m), "allocate correlations");
  NMC_CUDA(d.get(&lab, static_cast<size_t>(S) * n), "allocate labels");
  NMC_CUDA(d.get(&ncl, S), "allocate labels");
  NMC_CUDA(d.get(&scratch, backbone_scratch_bytes(n, m, S)), "allocate backbone scratch");
  NMC_CUDA(cudaMemcpyAsync(corr_d, corr, sizeof(double) * S * static_cast<size_t>(m), cudaMemcpyHostToDevice, ctx->stream), "upload correlations");
  BackboneArgs A{};
  A.clits = I->ks.clits;
  A.orig = I->ks.orig;
  A.newid = I->ks.newid;
  A.n = n;
  A.m = m;
  A.kmax = I->ks.kmax;
  A.S = S;
  A.corr = corr_d;
  A.beta = beta;
  A.seed_thr = seed_thr;
  A.cutoff = cutoff;
  A.scratch = scratch;
  A.labels = lab;
  A.n_clusters = ncl;
  const int err = backbone_run(A, ctx->stream);
  if (err != 0) return cuda_fail(ctx, static_cast<cudaError_t>(err), "backbone growth");
  NMC_CUDA(cudaMemcpyAsync(labels_out, lab, sizeof(int32_t) * S * static_cast<size_t>(n), cudaMemcpyDeviceToHost, ctx->stream), "read labels");
  if (n_clusters_out)
    NMC_CUDA(cudaMemcpyAsync(n_clusters_out, ncl, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, ctx->stream), "read labels");
  NMC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  return NMC_OK;
}

int nmc_replicas_whitening(nmc_ctx *ctx, int32_t rs, int32_t use_best, int32_t generalized,
                           int32_t *frozen_count_out, uint8_t *frozen_out, int32_t *rounds_out) {
  if (!ctx) return NMC_EINVAL;
  ReplicaSet *S = find_set(ctx, rs);
  if (!S) return fail(ctx, NMC_EINVAL, "unknown replica set");
  Instance *I = find_inst(ctx, S->inst);
  if (!I) return fail(ctx, NMC_ESTATE, "instance was unloaded");
  if (I->kind != NMC_KIND_KSAT) return fail(ctx, NMC_EINVAL, "whitening needs a k-SAT set");
  if (!frozen_count_out) return fail(ctx, NMC_EINVAL, "frozen_count_out is NULL");
  const int32_t n = I->ks.n, R = S->R, W = S->ks.W;
  DeviceGuard dg(ctx->device);
  DevScratch d;
  d.st = ctx->stream;
  int32_t *count = nullptr;
  uint8_t *frozen = nullptr;
  char *scratch = nullptr;
  NMC_CUDA(d.get(&count, R), "allocate whitening output");
  if (frozen_out) NMC_CUDA(d.get(&frozen, static_cast<size_t>(R) * n), "allocate whitening output");
  NMC_CUDA(d.get(&scratch, whitening_scratch_bytes(n, W)), "allocate whitening scratch");
  int32_t rounds = 0;
  const int err = whitening_run(I->ks, use_best ? S->ks.best : S->ks.S, use_best ? 1 : 2, R, W,
                                generalized ? 1 : 0, scratch, count, frozen, &rounds, ctx->stream);
  if (err != 0) return cuda_fail(ctx, static_cast<cudaError_t>(err), "whitening");
  NMC_CUDA(cudaMemcpyAsync(frozen_count_out, count, sizeof(int32_t) * R, cudaMemcpyDeviceToHost, ctx->stream), "read whitening");
  if (frozen_out)
    NMC_CUDA(cudaMemcpyAsync(frozen_out, frozen, static_cast<size_t>(R) * n, cudaMemcpyDeviceToHost, ctx->stream), "read whitening");
  NMC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  if (rounds_out) *rounds_out = rounds;
  return NMC_OK;
}

int nmc_set_schedule_backbone(nmc_ctx *ctx, int32_t inst, const int32_t *labels, int32_t cycles,
                              int32_t t_hot, int32_t t_cold, int32_t t_unlearn, float base,
                              float heat) {
  if (!ctx) return NMC_EINVAL;
  Instance *I = find_inst(ctx, inst);
  if (!I || I->kind != NMC_KIND_KSAT) return fail(ctx, NMC_EINVAL, "needs a k-SAT instance");
  if (!labels || cycles < 1 || t_hot < 0 || t_cold < 0 || t_unlearn < 0)
    return fail(ctx, NMC_EINVAL, "need labels, cycles >= 1 and phase lengths >= 0");
  const int64_t cyc = static_cast<int64_t>(t_hot) + t_cold + t_unlearn;
  if (cyc < 1 || cyc * cycles > 0x7FFFFFFF) return fail(ctx, NMC_EINVAL, "bad phase lengths");
  const float hot = base / heat;
  if (!(base >= 0.0f && base <= 65535.0f) || !(heat > 0.0f) || !std::isfinite(heat) ||
      !(hot >= 0.0f && hot <= 65535.0f))
    return fail(ctx, NMC_EINVAL, "base and base/heat must be in [0, 65535], heat > 0");
  const int32_t n = I->ks.n, n_steps = static_cast<int32_t>(cyc * cycles);
  DeviceGuard dg(ctx->device);
  int32_t *lab = nullptr;
  uint32_t *bq = nullptr;
  cudaError_t e;
  if ((e = cudaMallocAsync(reinterpret_cast<void **>(&lab), sizeof(int32_t) * n, ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "allocate labels");
  if ((e = cudaMalloc(&bq, sizeof(uint32_t) * static_cast<size_t>(n) * n_steps)) != cudaSuccess) {
    cudaFreeAsync(lab, ctx->stream);
    return cuda_fail(ctx, e, "allocate schedule");
  }
  e = cudaMemcpyAsync(lab, labels, sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = backbone_schedule(lab, I->ks.orig, n, n_steps, base, heat, t_hot, t_cold, t_unlearn, bq,
                          ctx->stream);
  cudaFreeAsync(lab, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    cudaFree(bq);
    return cuda_fail(ctx, e, "backbone schedule");
  }
  dev_free(I->bq);
  I->bq = bq;
  I->n_steps = n_steps;
  return NMC_OK;
}

int nmc_adaptive_ladder(nmc_ctx *ctx, int32_t inst, int32_t replicas, uint64_t seed, double beta0,
                        double alpha, double sigma_min, int32_t max_temps, int32_t sweeps_eq,
                        int32_t sweeps_meas, double *betas_out, double *sigmas_out,
                        int32_t *n_temps_out) {
  if (!ctx) return NMC_EINVAL;
  Instance *I = find_inst(ctx, inst);
  if (!I) return fail(ctx, NMC_EINVAL, "unknown instance");
  const bool qap = I->kind == NMC_KIND_QAP;
  int rc = qap ? NMC_OK : check_batchable(ctx, *I);
  if (rc != NMC_OK) return rc;
  if (!betas_out || !sigmas_out || !n_temps_out) return fail(ctx, NMC_EINVAL, "NULL output");
  if (max_temps < 1 || sweeps_eq < 0 || sweeps_meas < 1)
    return fail(ctx, NMC_EINVAL, "need max_temps >= 1, sweeps_eq >= 0, sweeps_meas >= 1");
  if (!std::isfinite(alpha) || !std::isfinite(sigma_min) || !std::isfinite(beta0) || sigma_min < 0.0)
    return fail(ctx, NMC_EINVAL, "beta0 and alpha must be finite, sigma_min finite and >= 0");
  const int64_t T = static_cast<int64_t>(sweeps_eq) + sweeps_meas;
  if (T * max_temps > 0x7FFFFFFF) return fail(ctx, NMC_EINVAL, "too many sweeps in total");
  // the k-SAT energy sums stay exact: m^2 * replicas * sweeps_meas < 2^62
  const double mm = qap ? 0.0 : static_cast<double>(I->ks.m);
  if (mm * mm * replicas * sweeps_meas >= 4.6e18)
    return fail(ctx, NMC_EINVAL, "energy sums could overflow: fewer replicas or sweeps");
  *n_temps_out = 0;
  int32_t rs = 0;
  rc = nmc_replicas_create(ctx, inst, replicas, seed, nullptr, &rs);
  if (rc != NMC_OK) return rc;
  ReplicaSet *S = find_set(ctx, rs);
  DeviceGuard dg(ctx->device);
  if (qap) {
    rc = qap_ladder(ctx, *I, *S, beta0, alpha, sigma_min, max_temps, sweeps_eq, sweeps_meas,
                    betas_out, sigmas_out, n_temps_out);
    const std::string keep = ctx->err;
    const int rc2 = nmc_replicas_destroy(ctx, rs);
    if (rc != NMC_OK) {
      ctx->err = keep;
      return rc;
    }
    return rc2;
  }
  const int32_t n = I->ks.n, W = S->ks.W;
  uint32_t *bq = nullptr, *mult = nullptr;
  long long *stats = nullptr;
  double *out_dev = nullptr;
  cudaError_t e = cudaSuccess;
  const std::vector<uint32_t> ones(32 * static_cast<size_t>(W), 65536u);
  if ((e = dev_alloc(&bq, static_cast<size_t>(n) * T)) != cudaSuccess ||
      (e = dev_alloc(&mult, ones.size())) != cudaSuccess ||
      (e = dev_alloc(&stats, 64 * static_cast<size_t>(W))) != cudaSuccess ||
      (e = dev_alloc(&out_dev, 2)) != cudaSuccess ||
      (e = cudaMemcpyAsync(mult, ones.data(), sizeof(uint32_t) * ones.size(), cudaMemcpyHostToDevice, ctx->stream)) != cudaSuccess)
    rc = cuda_fail(ctx, e, "allocate ladder scratch");
  double beta = beta0;
  for (int32_t i = 0; rc == NMC_OK && i < max_temps; ++i) {
    const float bf = static_cast<float>(beta);
    if (!(bf >= 0.0f && bf <= 65535.0f)) {
      rc = fail(ctx, NMC_EINVAL, "a ladder temperature left [0, 65535]");
      break;
    }
    const int32_t ts = static_cast<int32_t>(i * T), te = static_cast<int32_t>(ts + T);
    std::vector<BatchItem> items;
    for (int32_t w = 0; w < W; ++w) {
      BatchItem B = ksat_item(*I, *S, w, ts, te);
      // the level's schedule holds sweeps [ts, te) only: the item's base pointer is moved back
      // by ts steps so that the kernel's index t * n + v lands in it (no access before bq)
      B.bq = reinterpret_cast<const uint32_t *>(reinterpret_cast<uintptr_t>(bq) -
                                                sizeof(uint32_t) * static_cast<size_t>(ts) * n);
      B.mult = mult;
      B.stats = stats;
      B.stats_t0 = ts + sweeps_eq;
      items.push_back(B);
    }
    const int q = I->ks.kq == 1 ? 0 : 1;
    size_t off[2] = {0, 0};
    int cnt[2] = {0, 0}, max_n[2] = {0, 0}, cs[2] = {1, 1}, lanes[2] = {0, 0};
    cnt[q] = W;
    max_n[q] = n;
    tuned_shape(ctx, *I, W, &cs[q], &lanes[q]);
    if ((e = fill_schedule(bq, static_cast<size_t>(n) * T, beta, ctx->flag, ctx->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(stats, 0, sizeof(long long) * 64 * W, ctx->stream)) != cudaSuccess) {
      rc = cuda_fail(ctx, e, "prepare ladder level");
      break;
    }
    rc = launch_items(ctx, items, off, cnt, max_n, cs, true, lanes);
    if (rc != NMC_OK) break;
    double out[2] = {0.0, 0.0};
    if ((e = ladder_step(stats, S->R, W, static_cast<long long>(S->R) * sweeps_meas, beta, alpha,
                         out_dev, ctx->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(out, out_dev, sizeof(out), cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) {
      rc = cuda_fail(ctx, e, "ladder level");
      break;
    }
    betas_out[i] = beta;
    sigmas_out[i] = out[0];
    *n_temps_out = i + 1;
    if (out[0] <= sigma_min) break;
    beta = out[1];
  }
  cudaStreamSynchronize(ctx->stream);
  dev_free(bq);
  dev_free(mult);
  dev_free(stats);
  dev_free(out_dev);
  const std::string keep = ctx->err;
  const int rc2 = nmc_replicas_destroy(ctx, rs);
  if (rc != NMC_OK) {
    ctx->err = keep;
    return rc;
  }
  return rc2;
}

int nmc_anneal(nmc_ctx *ctx, int32_t inst, int32_t replicas, int32_t t0, int32_t t1,
               uint64_t seed, const void *init_states, const nmc_result *out) {
  if (!ctx) return NMC_EINVAL;
  int32_t rs = 0;
  int rc = nmc_replicas_create(ctx, inst, replicas, seed, init_states, &rs);
  if (rc != NMC_OK) return rc;
  rc = nmc_replicas_run(ctx, rs, t0, t1);
  if (rc == NMC_OK && out) rc = nmc_replicas_read(ctx, rs, out);
  const std::string keep = ctx->err;
  const int rc2 = nmc_replicas_destroy(ctx, rs);
  if (rc != NMC_OK) {
    ctx->err = keep;
    return rc;
  }
  return rc2;
}

}  // extern "C"

extern "C" int nmc_ksat_colour_host(int32_t n_vars, int32_t n_clauses, int32_t k_max,
                                    const int32_t *lits, int32_t *colour_out, int32_t *n_colours) {
  if (!n_colours) return NMC_EINVAL;
  nmc::HostKsat h;
  if (nmc::prepare_ksat(n_vars, n_clauses, k_max, lits, &h) != NMC_OK) return h.code;
  if (colour_out) std::memcpy(colour_out, h.colour.data(), sizeof(int32_t) * h.colour.size());
  *n_colours = h.n_colours;
  return NMC_OK;
}
