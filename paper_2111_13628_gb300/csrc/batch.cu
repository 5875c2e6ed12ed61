// Batched k-SAT sweep: one persistent launch runs many replica sets of uneven instances
// (sampling stage of Algorithm 1 for many problems at once).
//
// Work item = (replica set, word w of 32 replicas, sweep range). A CTA takes items from a
// device counter, loads the item's word vector x[0..n) into shared memory, runs its sweeps
// with the variables of one colour class spread over the threads (one thread = one variable
// for the 32 replicas of the word) and a CTA barrier between classes, and writes the state
// back. Words are independent chains, so no grid-wide synchronisation is needed and uneven
// instances fill the GPU. The dynamics are identical to the single-instance kernels.
// Occurrence lists are read in a warp-interleaved layout (one coalesced load per occurrence
// for 32 variables); each thread keeps its share of the sweep's energy change as 16
// bit-sliced planes and converts them to per-replica sums once per sweep.
#include <cooperative_groups.h>

#include <map>
#include <mutex>

#include "nmc.h"
#include "nmc_internal.h"
#include "philox.cuh"

namespace cg = cooperative_groups;

namespace nmc {

namespace {

constexpr int kBatchThreads = 768;

__device__ __forceinline__ uint32_t maj3b(uint32_t a, uint32_t b, uint32_t c) {
  return (a & b) | (a & c) | (b & c);
}

template <int NB>
__device__ __forceinline__ void csa4(uint32_t (&c)[NB], uint32_t a0, uint32_t a1, uint32_t a2,
                                     uint32_t a3) {
  const uint32_t s1 = c[0] ^ a0 ^ a1;
  const uint32_t y1 = maj3b(c[0], a0, a1);
  const uint32_t s2 = s1 ^ a2 ^ a3;
  const uint32_t y2 = maj3b(s1, a2, a3);
  c[0] = s2;
  const uint32_t s3 = c[1] ^ y1 ^ y2;
  uint32_t carry = maj3b(c[1], y1, y2);
  c[1] = s3;
#pragma unroll
  for (int j = 2; j < NB; ++j) {
    const uint32_t t = c[j] & carry;
    c[j] ^= carry;
    carry = t;
  }
}

// Transposes the 8x8 bit matrix held as 8 bytes (byte j = row j) so that byte i holds
// column i: with row j = bit plane j of 8 replicas, byte i becomes replica i's value.
__device__ __forceinline__ unsigned long long transpose8(unsigned long long x) {
  unsigned long long t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
  x = x ^ t ^ (t << 7);
  t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
  x = x ^ t ^ (t << 14);
  t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
  x = x ^ t ^ (t << 28);
  return x;
}

// Gathers byte q of each of the 8 planes p[0..7] into one 64-bit word (byte j from plane j).
__device__ __forceinline__ unsigned long long gather_bytes(const uint32_t *p, int q) {
  const uint32_t sel = (uint32_t)q | ((uint32_t)(4 + q) << 4);
  const uint32_t t01 = __byte_perm(p[0], p[1], sel), t23 = __byte_perm(p[2], p[3], sel);
  const uint32_t t45 = __byte_perm(p[4], p[5], sel), t67 = __byte_perm(p[6], p[7], sel);
  return (unsigned long long)__byte_perm(t01, t23, 0x5410) |
         ((unsigned long long)__byte_perm(t45, t67, 0x5410) << 32);
}

constexpr int kAccPlanes = 16;  // per-thread energy accumulator: 16-bit two's complement

// Truth value (32 replicas) of literal id l = 2u + neg from the word vector in shared memory.
__device__ __forceinline__ uint32_t lit_word(const uint32_t *xs, int l) {
  return xs[l >> 1] ^ (0u - (uint32_t)(l & 1));
}

// v = c0 + off is a variable of colour class c (starting at new id c0).
template <int KQ>
__device__ __forceinline__ uint32_t attempt_batch(const BatchItem &B, const uint32_t *xs,
                                                  const uint32_t *tab_s, int tab_len, int c,
                                                  int c0, int v, int t,
                                                  uint32_t (&acc)[kAccPlanes]) {
  constexpr int NB = 7;
  const uint32_t x = xs[v];
  const uint32_t bqv = __ldg(B.bq + (size_t)t * B.n + v);
  uint32_t bc[NB], mc[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    bc[j] = 0u;
    mc[j] = 0u;
  }
  const int off = v - c0;
  const int g = __ldg(B.cgrp + c) + (off >> 5), ln = off & 31;
  const int gb = __ldg(B.grp_base + g);
  const int len = (__ldg(B.grp_base + g + 1) - gb) / (32 * KQ);
  const int4 *ent = B.occ_t + gb + ln;
  for (int e = 0; e < len; e += 4) {
    uint32_t bb[4], mm[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int4 q = __ldg(ent + (size_t)((e + j) * KQ) * 32);
      uint32_t o = lit_word(xs, q.y) | lit_word(xs, q.z) | lit_word(xs, q.w);
      if (KQ == 2) {
        const int4 q2 = __ldg(ent + (size_t)((e + j) * KQ + 1) * 32);
        o |= lit_word(xs, q2.x) | lit_word(xs, q2.y) | lit_word(xs, q2.z) | lit_word(xs, q2.w);
      }
      const uint32_t own = x ^ (uint32_t)q.x;
      bb[j] = own & ~o;
      mm[j] = ~(own | o);
    }
    csa4<NB>(bc, bb[0], bb[1], bb[2], bb[3]);
    csa4<NB>(mc, mm[0], mm[1], mm[2], mm[3]);
  }
  // D = B - U, 8 bit planes (two's complement), then per-replica bytes by 8x8 transposes
  uint32_t s8[8];
  {
    uint32_t br = 0u;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      s8[j] = bc[j] ^ mc[j] ^ br;
      br = maj3b(~bc[j], mc[j], br);
    }
    s8[NB] = br;
  }
  const uint32_t vo = (uint32_t)__ldg(B.orig + v);
  // (bq * dE) >> 8 in 32-bit pieces: bq = 256 hi + lo, so the index is hi dE + (lo dE) >> 8
  // exactly (dE <= 127 keeps both terms below 2^31).
  const uint32_t bq_hi = bqv >> 8, bq_lo = bqv & 255u;
  uint32_t flip = 0u;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const unsigned long long xm = transpose8(gather_bytes(s8, q));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = 2 * q + h;
      int de[4];
      uint32_t th[4];
      bool need = false;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        de[j] = (int)(signed char)(unsigned char)(xm >> (8 * (4 * h + j)));
        th[j] = 0u;
        if (de[j] > 0) {
          const uint32_t idx = bq_hi * (uint32_t)de[j] + ((bq_lo * (uint32_t)de[j]) >> 8);
          th[j] = idx < (uint32_t)tab_len ? tab_s[idx] : 0u;
        }
        need |= th[j] != 0u;
      }
      uint4 u = make_uint4(0u, 0u, 0u, 0u);
      if (need)
        u = philox4x32_10(make_uint4(vo, (uint32_t)t, (uint32_t)(8 * B.w + g), kTagKsatSweep), B.k0, B.k1);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (de[j] <= 0 || uint4_word(u, j) < th[j]) flip |= 1u << (4 * g + j);
    }
  }
  // energy bookkeeping: acc += D on the flipped replicas (bit-sliced, sign-extended add)
  {
    uint32_t carry = 0u;
#pragma unroll
    for (int j = 0; j < kAccPlanes; ++j) {
      const uint32_t b = s8[j < 8 ? j : 7] & flip;
      const uint32_t a = acc[j];
      acc[j] = a ^ b ^ carry;
      carry = maj3b(a, b, carry);
    }
  }
  return x ^ flip;
}

// Synchronises the CS CTAs of a cluster (or the CTA when CS = 1); cluster barriers are
// hardware barriers with release/acquire semantics for distributed shared memory.
template <int CS>
__device__ __forceinline__ void group_sync() {
  if (CS == 1) {
    __syncthreads();
  } else {
    cg::this_cluster().sync();
  }
}

// Stores v at the same shared-memory word of CTA `rank` of the cluster (32-bit addressing).
__device__ __forceinline__ void st_rank(uint32_t saddr, int rank, uint32_t v) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(saddr), "r"(rank));
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(ra), "r"(v) : "memory");
}

template <int CS, typename T>
__device__ __forceinline__ T *rank_ptr(T *p, int r) {
  if (CS == 1) return p;
  return cg::this_cluster().map_shared_rank(p, r);
}

// CS = CTAs per item. With CS > 1 every CTA of the cluster keeps a full copy of the item's
// word vector; each CTA updates its share of every colour class and stores the new words
// into all CS copies (distributed shared memory), then the cluster barrier publishes them.
template <int KQ, int CS>
__global__ void __launch_bounds__(kBatchThreads, 1)
    ksat_batch_kernel(const BatchItem *__restrict__ items, int n_items, int *next_item,
                      const uint32_t *tab, int tab_len) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t *tab_s = smem;
  uint32_t *xs = smem + ((tab_len + 31) & ~31);
  __shared__ int e_s[32], be_s[32], ep_s[32];
  __shared__ uint32_t imp_s;
  __shared__ int item_s;
  __shared__ BatchItem item_b;  // the current item, read from shared memory where needed
  const int rank = CS == 1 ? 0 : (int)cg::this_cluster().block_rank();
  for (int i = threadIdx.x; i < tab_len; i += blockDim.x) tab_s[i] = tab[i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  while (true) {
    if (rank == 0 && threadIdx.x == 0) item_s = atomicAdd(next_item, 1);
    group_sync<CS>();
    const int it = *rank_ptr<CS>(&item_s, 0);
    if (it < n_items && threadIdx.x == 0) item_b = items[it];
    group_sync<CS>();  // every rank has read the item id before any rank moves on or exits
    if (it >= n_items) break;
    const BatchItem &B = item_b;
    const int n = B.n, W = B.W, w = B.w;
    const int share = (n + CS - 1) / CS;
    for (int v = threadIdx.x; v < n; v += blockDim.x) xs[v] = B.S[(size_t)(2 * v) * W + w];
    if (threadIdx.x == 0) xs[n] = 0u;
    if (threadIdx.x < 32) {
      ep_s[threadIdx.x] = 0;
      if (rank == 0) {
        e_s[threadIdx.x] = B.energy[32 * w + threadIdx.x];
        be_s[threadIdx.x] = B.best_energy[32 * w + threadIdx.x];
      }
    }
    group_sync<CS>();
    for (int t = B.t0; t < B.t1; ++t) {
      uint32_t acc[kAccPlanes];
#pragma unroll
      for (int j = 0; j < kAccPlanes; ++j) acc[j] = 0u;
      for (int c = 0; c < B.n_colours; ++c) {
        const int c0 = __ldg(B.col_ptr + c), c1 = __ldg(B.col_ptr + c + 1);
        const int part = ((c1 - c0 + CS - 1) / CS + 31) & ~31;  // whole 32-variable groups
        const int v0 = c0 + rank * part, v1 = min(c1, v0 + part);
        for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
          const uint32_t xn = attempt_batch<KQ>(B, xs, tab_s, tab_len, c, c0, v, t, acc);
          if (CS == 1) {
            xs[v] = xn;
          } else {
            const uint32_t sa = (uint32_t)__cvta_generic_to_shared(xs + v);
#pragma unroll
            for (int r = 0; r < CS; ++r) st_rank(sa, r, xn);
          }
        }
        group_sync<CS>();
      }
      // per-replica sums of this sweep: planes -> 16-bit values (two byte transposes per block
      // of 8 replicas), then a warp reduction per replica
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const unsigned long long lo = transpose8(gather_bytes(acc, q));
        const unsigned long long hi = transpose8(gather_bytes(acc + 8, q));
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int val = (int)(short)(unsigned short)(((lo >> (8 * i)) & 0xFFull) |
                                                       (((hi >> (8 * i)) & 0xFFull) << 8));
          const int s2 = __reduce_add_sync(0xFFFFFFFFu, val);
          if (lane == 0 && s2 != 0) atomicAdd(&ep_s[8 * q + i], s2);
        }
      }
      group_sync<CS>();
      if (rank == 0 && warp == 0) {
        int sum = e_s[lane];
#pragma unroll
        for (int r = 0; r < CS; ++r) sum += rank_ptr<CS>(ep_s, r)[lane];
        e_s[lane] = sum;
        const bool better = sum < be_s[lane];
        if (better) be_s[lane] = sum;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, better);
        if (lane == 0) imp_s = m;
      }
      group_sync<CS>();
      const uint32_t m = *rank_ptr<CS>(&imp_s, 0);
      if (threadIdx.x < 32) ep_s[threadIdx.x] = 0;
      if (m) {
        const int b0 = rank * share, b1 = min(n, b0 + share);
        for (int v = b0 + threadIdx.x; v < b1; v += blockDim.x) {
          const size_t bi = (size_t)v * W + w;
          B.best[bi] = (B.best[bi] & ~m) | (xs[v] & m);
        }
        group_sync<CS>();
      }
    }
    {
      const int b0 = rank * share, b1 = min(n, b0 + share);
      for (int v = b0 + threadIdx.x; v < b1; v += blockDim.x) {
        B.S[(size_t)(2 * v) * W + w] = xs[v];
        B.S[(size_t)(2 * v + 1) * W + w] = ~xs[v];
      }
    }
    if (rank == 0 && threadIdx.x < 32) {
      B.energy[32 * w + threadIdx.x] = e_s[threadIdx.x];
      B.best_energy[32 * w + threadIdx.x] = be_s[threadIdx.x];
    }
    group_sync<CS>();
  }
}

// The launch shape of each kernel instance is queried once per (device, shared-memory size):
// occupancy and cluster queries are slow host calls.
template <int KQ, int CS>
cudaError_t launch_batch(const BatchItem *items, int n_items, int *next_item,
                         const uint32_t *tab, int tab_len, int max_n, int device,
                         cudaStream_t st) {
  const size_t smem = sizeof(uint32_t) * (((tab_len + 31) & ~31) + (size_t)max_n + 1);
  auto kern = ksat_batch_kernel<KQ, CS>;
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, int> shapes;  // (device, smem) -> resident clusters
  static std::map<int, size_t> smem_set;                // device -> largest smem attribute set
  int clusters = 0;
  {
    std::lock_guard<std::mutex> g(mu);
    cudaError_t err;
    size_t &cur = smem_set[device];
    if (smem > cur) {
      err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      cur = smem;
    }
    auto it = shapes.find({device, smem});
    if (it != shapes.end()) {
      clusters = it->second;
    } else {
      int sms = 0;
      err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
      if (err != cudaSuccess) return err;
      if (CS == 1) {
        int per_sm = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchThreads, smem);
        if (err != cudaSuccess) return err;
        clusters = sms * per_sm;
      } else {
        cudaLaunchConfig_t q = {};
        q.blockDim = dim3(kBatchThreads);
        q.dynamicSmemBytes = smem;
        q.gridDim = dim3(CS * sms);
        cudaLaunchAttribute qa[1];
        qa[0].id = cudaLaunchAttributeClusterDimension;
        qa[0].val.clusterDim.x = CS;
        qa[0].val.clusterDim.y = 1;
        qa[0].val.clusterDim.z = 1;
        q.attrs = qa;
        q.numAttrs = 1;
        err = cudaOccupancyMaxActiveClusters(&clusters, kern, &q);
        if (err != cudaSuccess) return err;
      }
      shapes[{device, smem}] = clusters;
    }
  }
  if (clusters < 1) return cudaErrorInvalidConfiguration;
  if (clusters > n_items) clusters = n_items;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kBatchThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(clusters * CS);
  cudaError_t err = cudaMemsetAsync(next_item, 0, sizeof(int), st);
  if (err != cudaSuccess) return err;
  return cudaLaunchKernelEx(&cfg, kern, items, n_items, next_item, tab, tab_len);
}

template <int KQ>
cudaError_t dispatch_batch(int cs, const BatchItem *items, int n_items, int *next_item,
                           const uint32_t *tab, int tab_len, int max_n, int device, cudaStream_t st) {
  switch (cs) {
    case 8: return launch_batch<KQ, 8>(items, n_items, next_item, tab, tab_len, max_n, device, st);
    case 4: return launch_batch<KQ, 4>(items, n_items, next_item, tab, tab_len, max_n, device, st);
    case 2: return launch_batch<KQ, 2>(items, n_items, next_item, tab, tab_len, max_n, device, st);
    default: return launch_batch<KQ, 1>(items, n_items, next_item, tab, tab_len, max_n, device, st);
  }
}

}  // namespace

// ---- batched sweep without any allocation ----------------------------------------------------
//
// Work list and counters live in one fixed device array of this file instead of memory the
// context allocates on demand. kNoAllocBytes bounds one call: two counters, then up to
// kNoAllocItems work items (one item = one 32-replica word of one replica set).
constexpr size_t kNoAllocBytes = 1u << 20;  // 1 MiB on every GPU that loads the library
constexpr size_t kNoAllocHeader = 256;      // two int counters, padded to the item alignment
constexpr size_t kNoAllocItems = (kNoAllocBytes - kNoAllocHeader) / sizeof(BatchItem);
static_assert(sizeof(BatchItem) == 112 && kNoAllocItems == 9360, "limit stated in nmc.h");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

// Device address of g_noalloc_scratch, looked up once per device (with that device current).
// In host code the array's name is only a host-side stand-in, never a device address.
std::mutex g_noalloc_mu;
void *g_noalloc_addr[64] = {};

int noalloc_scratch(int device, void **out) {
  if (device < 0 || device >= 64) return NMC_EINVAL;
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return NMC_ECUDA;
    }
    g_noalloc_addr[device] = p;
  }
  *out = g_noalloc_addr[device];
  return NMC_OK;
}

}  // namespace

}  // namespace nmc

extern "C" int nmc_batch_run_noalloc(nmc_ctx *ctx, int32_t n_sets, const int32_t *rs,
                                     const int32_t *t0, const int32_t *t1) {
  using namespace nmc;
  if (!ctx) return NMC_EINVAL;
  BatchPlan plan;
  int rc = batch_plan(ctx, n_sets, rs, t0, t1, &plan);
  if (rc != NMC_OK) return rc;
  if (plan.items.empty()) return NMC_OK;
  if (plan.items.size() > kNoAllocItems)
    return set_ctx_error(ctx, NMC_EINVAL,
                         "nmc_batch_run_noalloc: more work items (32-replica words) than the "
                         "fixed scratch array holds; split the batch or use nmc_batch_run");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (cudaSetDevice(plan.device) != cudaSuccess) {
    cudaGetLastError();
    return set_ctx_error(ctx, NMC_ECUDA, "nmc_batch_run_noalloc: cannot select the device");
  }
  void *base = nullptr;
  rc = noalloc_scratch(plan.device, &base);
  cudaError_t e = cudaSuccess;
  if (rc == NMC_OK) {
    int *counters = static_cast<int *>(base);
    BatchItem *items = reinterpret_cast<BatchItem *>(static_cast<char *>(base) + kNoAllocHeader);
    e = cudaMemcpyAsync(items, plan.items.data(), sizeof(BatchItem) * plan.items.size(),
                        cudaMemcpyHostToDevice, plan.stream);
    for (int q = 0; q < 2 && e == cudaSuccess; ++q)
      if (plan.cnt[q] > 0)  // the launcher clears counters[q] on the stream before the kernel
        e = ksat_batch(items + plan.off[q], plan.cnt[q], q + 1, plan.cs[q], plan.max_n[q],
                       counters + q, plan.tab, plan.tab_len, plan.device, plan.stream);
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (rc != NMC_OK)
    return set_ctx_error(ctx, rc, "nmc_batch_run_noalloc: cudaGetSymbolAddress failed");
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_ctx_error(ctx, NMC_ECUDA, cudaGetErrorString(e));
  }
  return NMC_OK;
}

namespace nmc {

size_t batch_max_vars(int tab_len, int device) {
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess)
    return 0;
  // dynamic shared memory: table + n+1 words; the static part is under 192 words
  const long long words = (long long)optin / 4 - ((tab_len + 31) & ~31) - 1 - 192;
  return words > 0 ? (size_t)words : 0;
}

cudaError_t ksat_batch(const BatchItem *items_dev, int n_items, int kq, int cs, int max_n,
                       int *next_item, const uint32_t *tab, int tab_len, int device,
                       cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  if (kq == 1) return dispatch_batch<1>(cs, items_dev, n_items, next_item, tab, tab_len, max_n, device, st);
  return dispatch_batch<2>(cs, items_dev, n_items, next_item, tab, tab_len, max_n, device, st);
}

}  // namespace nmc
