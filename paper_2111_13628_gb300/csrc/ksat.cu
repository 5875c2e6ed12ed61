// k-SAT kernels of the inhomogeneous Metropolis sweep (NMC sampling stage, Algorithm 1;
// single-variable Metropolis updates with a per-variable inverse temperature, Sec.
// "Nonequilibrium inhomogeneous sampling over subgraphs"; energy = number of violated
// clauses, Sec. "4-SAT Problems Near Computational Phase Transitions").
//
// Layout. Replicas are multi-spin coded: bit b of word w holds replica 32w+b. Row 2v of S is
// the word vector of x_v and row 2v+1 its complement, so a literal id (2v+neg) addresses its
// truth value directly. Rows 2n (always false) and 2n+1 (always true) pad clauses and
// occurrence lists. A warp's lanes take consecutive words of one variable, so each literal
// gather is one contiguous 128-byte line when W >= 32.
//
// Energy change. For the flip of v, each clause a containing v contributes +1 when v's
// literal is its only true literal ("break") and -1 when it has no true literal ("make").
// Both counts are kept as bit-sliced counters (one bit plane per binary digit), fed four
// clauses at a time through carry-save adders, so one thread evaluates 32 replicas at once.
//
// Sweep. A persistent cooperative kernel walks sweeps t0..t1-1 and colours 0..C-1; each colour
// class is an independent set, updated in parallel, followed by a grid barrier. The barrier's
// waits are bounded (a few seconds); when one expires the kernel records an error and every
// CTA returns.
#include <cooperative_groups.h>
#include <cstdlib>
#include <map>
#include <mutex>

#include "nmc_internal.h"
#include "philox.cuh"

namespace nmc {

namespace {

constexpr unsigned long long kSweepWaitLimitNs = 5ull * 1000ull * 1000ull * 1000ull;
constexpr unsigned kBarrierMaxPolls = 1u << 28;
constexpr int kSweepThreads = 256;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident): each CTA stores its
// barrier count into its own flag (release) and its first warp polls all flags (acquire)
// until every CTA has arrived. No counter is shared, so arrivals do not serialise on one
// address. Returns false when the launch must stop (a wait expired here or in another CTA).
__device__ bool grid_sync(GridBarrier *gb, unsigned nblocks, unsigned &gen,
                          unsigned long long limit_ns) {
  __shared__ int s_ok;
  const unsigned target = gen + 1u;
  __syncthreads();
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(&gb->flags[blockIdx.x], target);
    }
    __syncwarp();
    int ok = 1;
    const unsigned long long start = global_ns();
    unsigned polls = 0;
    while (true) {
      bool mine = true;
      for (unsigned i = threadIdx.x; i < nblocks; i += 32) mine &= ld_acquire(&gb->flags[i]) >= target;
      if (__all_sync(0xFFFFFFFFu, mine)) break;
      ++polls;
      if ((polls & 15u) == 0u) {
        int bad = 0;
        if (threadIdx.x == 0) {
          bad = *(volatile int *)&gb->error;
          if (!bad && (global_ns() - start > limit_ns || polls > kBarrierMaxPolls)) {
            atomicExch(&gb->error, 1);
            atomicExch(&gb->sticky, 1);
            bad = 1;
          }
        }
        if (__shfl_sync(0xFFFFFFFFu, bad, 0)) {
          ok = 0;
          break;
        }
      }
    }
    if (threadIdx.x == 0) s_ok = ok;
  }
  __syncthreads();
  gen = target;
  return s_ok != 0;
}

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) {
  return (a & b) | (a & c) | (b & c);
}

// c += a0 + a1 + a2 + a3, per bit lane, on a bit-sliced counter of NB digits.
template <int NB>
__device__ __forceinline__ void csa_add4(uint32_t (&c)[NB], uint32_t a0, uint32_t a1,
                                         uint32_t a2, uint32_t a3) {
  const uint32_t s1 = c[0] ^ a0 ^ a1;
  const uint32_t y1 = maj3(c[0], a0, a1);
  const uint32_t s2 = s1 ^ a2 ^ a3;
  const uint32_t y2 = maj3(s1, a2, a3);
  c[0] = s2;
  const uint32_t s3 = c[1] ^ y1 ^ y2;
  uint32_t carry = maj3(c[1], y1, y2);
  c[1] = s3;
#pragma unroll
  for (int j = 2; j < NB; ++j) {
    const uint32_t t = c[j] & carry;
    c[j] ^= carry;
    carry = t;
  }
}

template <int NB>
__device__ __forceinline__ int slice_value(const uint32_t (&c)[NB], int b) {
  int v = 0;
#pragma unroll
  for (int j = 0; j < NB; ++j) v |= (int)((c[j] >> b) & 1u) << j;
  return v;
}

struct SweepArgs {
  uint32_t *S;
  uint32_t *best;
  int32_t *energy;
  int32_t *best_energy;
  uint32_t *imp;
  GridBarrier *bar;
  const int4 *occ;
  const int32_t *occ_ptr;
  const int32_t *col_ptr;
  const int32_t *orig;
  const uint32_t *bq;
  const uint32_t *tab;
  int32_t tab_len;
  int32_t n, W, n_colours;
  int32_t t0, t1;
  uint32_t k0, k1;
};

// One Metropolis attempt on variable v for the 32 replicas of word w at sweep t.
template <int NB, int KQ>
__device__ __forceinline__ void attempt(const SweepArgs &a, const uint32_t *__restrict__ tab_s,
                                        int v, int w, int t, int (&acc)[32]) {
  const int W = a.W;
  const uint32_t *Sw = a.S + w;
  const uint32_t x = __ldcg(Sw + (size_t)(2 * v) * W);
  const uint32_t bqv = __ldg(a.bq + (size_t)t * a.n + v);
  const bool frozen = bqv == kFrozenQ16;  // held: no attempt (the pending best copy still runs)
  uint32_t bc[NB], mc[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    bc[j] = 0u;
    mc[j] = 0u;
  }
  const int e0 = __ldg(a.occ_ptr + v), e1 = frozen ? e0 : __ldg(a.occ_ptr + v + 1);
  for (int e = e0; e < e1; e += 4) {
    uint32_t bb[4], mm[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int4 q = __ldg(a.occ + (size_t)(e + j) * KQ);
      uint32_t o = __ldcg(Sw + (size_t)q.y * W) | __ldcg(Sw + (size_t)q.z * W) |
                   __ldcg(Sw + (size_t)q.w * W);
      if (KQ == 2) {
        const int4 q2 = __ldg(a.occ + (size_t)(e + j) * KQ + 1);
        o |= __ldcg(Sw + (size_t)q2.x * W) | __ldcg(Sw + (size_t)q2.y * W) |
             __ldcg(Sw + (size_t)q2.z * W) | __ldcg(Sw + (size_t)q2.w * W);
      }
      const uint32_t own = x ^ (uint32_t)q.x;
      bb[j] = own & ~o;
      mm[j] = ~(own | o);
    }
    csa_add4<NB>(bc, bb[0], bb[1], bb[2], bb[3]);
    csa_add4<NB>(mc, mm[0], mm[1], mm[2], mm[3]);
  }
  const uint32_t vo = (uint32_t)__ldg(a.orig + v);
  uint32_t flip = 0u;
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    int dE[4];
    uint32_t thr[4];
    bool need = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = 4 * g + j;
      dE[j] = slice_value<NB>(bc, b) - slice_value<NB>(mc, b);
      thr[j] = 0u;
      if (dE[j] > 0) {
        const unsigned long long idx = ((unsigned long long)bqv * (unsigned)dE[j]) >> 8;
        thr[j] = idx < (unsigned long long)a.tab_len ? tab_s[idx] : 0u;
        need |= thr[j] != 0u;
      }
    }
    uint4 u = make_uint4(0u, 0u, 0u, 0u);
    if (need) u = philox4x32_10(make_uint4(vo, (uint32_t)t, (uint32_t)(8 * w + g), kTagKsatSweep),
                                a.k0, a.k1);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = 4 * g + j;
      const bool ok = dE[j] <= 0 || uint4_word(u, j) < thr[j];
      if (ok) {
        flip |= 1u << b;
        acc[b] += dE[j];
      }
    }
  }
  if (frozen) flip = 0u;  // zero counters read as dE = 0: cancel those flips
  const uint32_t xn = x ^ flip;
  __stcg(a.S + (size_t)(2 * v) * W + w, xn);
  __stcg(a.S + (size_t)(2 * v + 1) * W + w, ~xn);
  // Pending best-state copy from the previous sweep end: x is still that sweep's state of v.
  const uint32_t m = __ldcg(a.imp + w);
  if (m) {
    const size_t bi = (size_t)v * W + w;
    __stcg(a.best + bi, (__ldcg(a.best + bi) & ~m) | (x & m));
  }
}

template <int NB, int KQ>
__global__ void __launch_bounds__(kSweepThreads) ksat_sweep_kernel(SweepArgs a) {
  extern __shared__ uint32_t smem[];
  uint32_t *tab_s = smem;                                // tab_len entries
  int *eacc = (int *)(smem + ((a.tab_len + 31) & ~31));  // W*33 entries (padded rows)
  const int W = a.W;
  for (int i = threadIdx.x; i < a.tab_len; i += blockDim.x) tab_s[i] = a.tab[i];
  for (int i = threadIdx.x; i < W * 33; i += blockDim.x) eacc[i] = 0;
  __syncthreads();

  const unsigned nblocks = gridDim.x;
  unsigned gen = 0;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = gridDim.x * blockDim.x;
  const int slots = nthreads / W;
  const int w = gtid % W;
  const int slot = gtid / W;
  const bool active = slot < slots;

  for (int t = a.t0; t < a.t1; ++t) {
    int acc[32];
#pragma unroll
    for (int b = 0; b < 32; ++b) acc[b] = 0;
    for (int c = 0; c < a.n_colours; ++c) {
      if (active) {
        const int v0 = __ldg(a.col_ptr + c), v1 = __ldg(a.col_ptr + c + 1);
        for (int v = v0 + slot; v < v1; v += slots) attempt<NB, KQ>(a, tab_s, v, w, t, acc);
      }
      if (!grid_sync(a.bar, nblocks, gen, kSweepWaitLimitNs)) return;
    }
    // Energies: per-thread sums -> CTA sums in shared memory -> device atomics.
    if (active) {
#pragma unroll
      for (int b = 0; b < 32; ++b)
        if (acc[b] != 0) atomicAdd(&eacc[w * 33 + b], acc[b]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < W * 32; i += blockDim.x) {
      const int s = (i >> 5) * 33 + (i & 31);
      const int val = eacc[s];
      if (val != 0) {
        atomicAdd(&a.energy[i], val);
        eacc[s] = 0;
      }
    }
    if (!grid_sync(a.bar, nblocks, gen, kSweepWaitLimitNs)) return;
    // Best-so-far on strictly lower energy; the state copy is deferred to the next visit.
    if (gtid < W * 32) {
      const int e = __ldcg(a.energy + gtid);
      const int be = __ldcg(a.best_energy + gtid);
      const bool better = e < be;
      if (better) __stcg(a.best_energy + gtid, e);
      const unsigned mask = __ballot_sync(0xFFFFFFFFu, better);
      if ((threadIdx.x & 31) == 0) __stcg(a.imp + (gtid >> 5), mask);
    }
    if (!grid_sync(a.bar, nblocks, gen, kSweepWaitLimitNs)) return;
  }
  // Apply the copy still pending from the last sweep, then clear the masks.
  if (a.t1 > a.t0) {
    for (long long i = gtid; i < (long long)a.n * W; i += nthreads) {
      const int ww = (int)(i % W);
      const uint32_t m = __ldcg(a.imp + ww);
      if (m) {
        const long long v = i / W;
        const uint32_t x = __ldcg(a.S + (size_t)(2 * v) * W + ww);
        __stcg(a.best + i, (__ldcg(a.best + i) & ~m) | (x & m));
      }
    }
    if (!grid_sync(a.bar, nblocks, gen, kSweepWaitLimitNs)) return;
    for (int i = gtid; i < W; i += nthreads) __stcg(a.imp + i, 0u);
  }
}

// ---- fast path: W a multiple of 32, counters of at most 7 bits ---------------------------
//
// A team of P consecutive warps takes one variable and one group of 32 words (lane = word):
// the warps split the variable's occurrence list, stage their entries in shared memory with
// one cooperative load, gather the neighbour literal words in batches of CH occurrences, and
// exchange their partial bit-sliced counters through shared memory. Each warp then resolves
// the acceptance of 32/P of the 32 replica bits of its lane's word. With P > 1 the latency
// of one attempt is split P ways, which matters because one colour class is one wave.
constexpr int kFastEntCap = 64;   // occurrences staged per warp per batch
constexpr int kFastMaxTeams = 15; // named barriers 1..15

__device__ __forceinline__ void team_bar(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

struct FastSmem {
  uint32_t *tab;   // acceptance table
  int *eacc;       // W*33 per-CTA energy sums
  int4 *ent;       // per warp: kFastEntCap * KQ entries
  uint32_t *thr;   // per warp: 128 thresholds by energy change 0..127
  uint32_t *part;  // per team: P * 2*NB * 32 partial counters
  uint32_t *flip;  // per team: P * 32 flip masks
  int *acc;        // per warp: (32/P) x 32 lanes, energy change of this sweep per replica bit
};

template <int NB, int KQ, int P>
__host__ __device__ constexpr size_t fast_smem_bytes(int tab_len, int W, int nwarps) {
  return sizeof(uint32_t) * ((tab_len + 31) & ~31) + sizeof(int) * (size_t)W * 33 +
         sizeof(int4) * (size_t)nwarps * kFastEntCap * KQ + sizeof(uint32_t) * (size_t)nwarps * 128 +
         sizeof(uint32_t) * (size_t)(nwarps / P) * P * 2 * NB * 32 +
         sizeof(uint32_t) * (size_t)(nwarps / P) * P * 32 + sizeof(int) * (size_t)nwarps * 32 * (32 / P) +
         64;
}

template <int NB, int KQ, int P>
__device__ __forceinline__ void fast_attempt(const SweepArgs &a, const FastSmem &sm, int v, int w,
                                             int t, int warp, int team_in_cta, int p, int lane) {
  const int W = a.W;
  const uint32_t *Sw = a.S + w;
  const int e0 = __ldg(a.occ_ptr + v), e1 = __ldg(a.occ_ptr + v + 1);
  const uint32_t x = __ldcg(Sw + (size_t)(2 * v) * W);
  const uint32_t bqv = __ldg(a.bq + (size_t)t * a.n + v);
  const bool frozen = bqv == kFrozenQ16;  // uniform over the team (one variable)
  // this warp's share of the occurrences, a multiple of 4 (none when the variable is held)
  const int quads = frozen ? 0 : (e1 - e0) >> 2;
  const int per = (quads + P - 1) / P;
  const int lo = e0 + 4 * min(quads, p * per);
  const int hi = e0 + 4 * min(quads, (p + 1) * per);
  uint32_t bc[NB], mc[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    bc[j] = 0u;
    mc[j] = 0u;
  }
  int4 *ent = sm.ent + (size_t)warp * kFastEntCap * KQ;
  for (int base = lo; base < hi; base += kFastEntCap) {
    const int cnt = min(kFastEntCap, hi - base);
    for (int i = lane; i < cnt * KQ; i += 32) ent[i] = __ldg(a.occ + (size_t)base * KQ + i);
    __syncwarp();
    for (int e = 0; e < cnt; e += 4) {
      uint32_t bb[4], mm[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int4 q = ent[(e + j) * KQ];
        uint32_t o = __ldcg(Sw + (size_t)q.y * W) | __ldcg(Sw + (size_t)q.z * W) |
                     __ldcg(Sw + (size_t)q.w * W);
        if (KQ == 2) {
          const int4 q2 = ent[(e + j) * KQ + 1];
          o |= __ldcg(Sw + (size_t)q2.x * W) | __ldcg(Sw + (size_t)q2.y * W) |
               __ldcg(Sw + (size_t)q2.z * W) | __ldcg(Sw + (size_t)q2.w * W);
        }
        const uint32_t own = x ^ (uint32_t)q.x;
        bb[j] = own & ~o;
        mm[j] = ~(own | o);
      }
      csa_add4<NB>(bc, bb[0], bb[1], bb[2], bb[3]);
      csa_add4<NB>(mc, mm[0], mm[1], mm[2], mm[3]);
    }
    __syncwarp();
  }
  const int bar_id = 1 + team_in_cta;
  if (P > 1) {
    uint32_t *part = sm.part + (size_t)team_in_cta * P * 2 * NB * 32;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      part[((p * 2 + 0) * NB + j) * 32 + lane] = bc[j];
      part[((p * 2 + 1) * NB + j) * 32 + lane] = mc[j];
    }
    team_bar(bar_id, P * 32);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      bc[j] = 0u;
      mc[j] = 0u;
    }
#pragma unroll
    for (int q = 0; q < P; ++q) {  // sum the P partial counters (ripple-carry, bit-sliced)
      uint32_t cb = 0u, cm = 0u;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const uint32_t pb = part[((q * 2 + 0) * NB + j) * 32 + lane];
        const uint32_t pm = part[((q * 2 + 1) * NB + j) * 32 + lane];
        const uint32_t sb = bc[j] ^ pb ^ cb;
        cb = maj3(bc[j], pb, cb);
        bc[j] = sb;
        const uint32_t sm2 = mc[j] ^ pm ^ cm;
        cm = maj3(mc[j], pm, cm);
        mc[j] = sm2;
      }
    }
  }
  // D = B - U in NB+1 bit two's complement, bit-sliced
  uint32_t d[NB + 1];
  {
    uint32_t br = 0u;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      d[j] = bc[j] ^ mc[j] ^ br;
      br = maj3(~bc[j], mc[j], br);
    }
    d[NB] = br;
  }
  // thresholds by energy change for this variable's beta (shared by the warp's lanes)
  uint32_t *thr = sm.thr + warp * 128;
  for (int dv = lane; dv < (1 << NB); dv += 32) {
    const unsigned long long idx = ((unsigned long long)bqv * (unsigned)dv) >> 8;
    thr[dv] = (dv > 0 && idx < (unsigned long long)a.tab_len) ? sm.tab[idx] : 0u;
  }
  __syncwarp();
  const uint32_t vo = (uint32_t)__ldg(a.orig + v);
  uint32_t flip = 0u;
  // Per-replica values: sign-extend D to 8 bit planes and transpose each 8x8 block (8 planes x
  // 8 replicas) so that byte i of the result is replica i's signed energy change.
  uint32_t s8[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) s8[j] = j <= NB ? d[j] : d[NB];
  constexpr int BPW = 4 / P;  // blocks of 8 replicas handled by this warp
#pragma unroll 1
  for (int qi = 0; qi < BPW; ++qi) {
    const int q = p * BPW + qi;
    const uint32_t sel = (uint32_t)q | ((uint32_t)(4 + q) << 4);
    const uint32_t t01 = __byte_perm(s8[0], s8[1], sel), t23 = __byte_perm(s8[2], s8[3], sel);
    const uint32_t t45 = __byte_perm(s8[4], s8[5], sel), t67 = __byte_perm(s8[6], s8[7], sel);
    unsigned long long xm = (unsigned long long)__byte_perm(t01, t23, 0x5410) |
                            ((unsigned long long)__byte_perm(t45, t67, 0x5410) << 32);
    unsigned long long tt = (xm ^ (xm >> 7)) & 0x00AA00AA00AA00AAull;
    xm = xm ^ tt ^ (tt << 7);
    tt = (xm ^ (xm >> 14)) & 0x0000CCCC0000CCCCull;
    xm = xm ^ tt ^ (tt << 14);
    tt = (xm ^ (xm >> 28)) & 0x00000000F0F0F0F0ull;
    xm = xm ^ tt ^ (tt << 28);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = 2 * q + h;  // Philox group: replicas 4g..4g+3
      int de[4];
      uint32_t th[4];
      bool need = false;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        de[j] = (int)(signed char)(unsigned char)(xm >> (8 * (4 * h + j)));
        th[j] = de[j] > 0 ? thr[de[j]] : 0u;
        need |= th[j] != 0u;
      }
      uint4 u = make_uint4(0u, 0u, 0u, 0u);
      if (need)
        u = philox4x32_10(make_uint4(vo, (uint32_t)t, (uint32_t)(8 * w + g), kTagKsatSweep), a.k0, a.k1);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bool ok = de[j] <= 0 || uint4_word(u, j) < th[j];
        if (ok) {
          flip |= 1u << (4 * g + j);
          if (de[j] != 0) sm.acc[(warp * (32 / P) + 8 * qi + 4 * h + j) * 32 + lane] += de[j];
        }
      }
    }
  }
  if (frozen) flip = 0u;  // zero counters read as dE = 0: cancel those flips
  if (P > 1) {
    uint32_t *fl = sm.flip + (size_t)team_in_cta * P * 32;
    fl[p * 32 + lane] = flip;
    team_bar(bar_id, P * 32);
    if (p != 0) return;
    flip = 0u;
#pragma unroll
    for (int q = 0; q < P; ++q) flip |= fl[q * 32 + lane];
  }
  const uint32_t xn = x ^ flip;
  __stcg(a.S + (size_t)(2 * v) * W + w, xn);
  __stcg(a.S + (size_t)(2 * v + 1) * W + w, ~xn);
  const uint32_t m = __ldcg(a.imp + w);
  if (m) {
    const size_t bi = (size_t)v * W + w;
    __stcg(a.best + bi, (__ldcg(a.best + bi) & ~m) | (x & m));
  }
}

template <int NB, int KQ, int P, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) ksat_sweep_fast_kernel(SweepArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int W = a.W;
  const int nwarps = blockDim.x >> 5;
  FastSmem sm;
  {
    char *p = (char *)smem;
    sm.tab = (uint32_t *)p;
    p += sizeof(uint32_t) * ((a.tab_len + 31) & ~31);
    sm.eacc = (int *)p;
    p += sizeof(int) * (size_t)W * 33;
    p = (char *)(((size_t)p + 15) & ~(size_t)15);
    sm.ent = (int4 *)p;
    p += sizeof(int4) * (size_t)nwarps * kFastEntCap * KQ;
    sm.thr = (uint32_t *)p;
    p += sizeof(uint32_t) * (size_t)nwarps * 128;
    sm.part = (uint32_t *)p;
    p += sizeof(uint32_t) * (size_t)(nwarps / P) * P * 2 * NB * 32;
    sm.flip = (uint32_t *)p;
    p += sizeof(uint32_t) * (size_t)(nwarps / P) * P * 32;
    sm.acc = (int *)p;
  }
  for (int i = threadIdx.x; i < a.tab_len; i += blockDim.x) sm.tab[i] = a.tab[i];
  for (int i = threadIdx.x; i < W * 33; i += blockDim.x) sm.eacc[i] = 0;
  for (int i = threadIdx.x; i < nwarps * 32 * (32 / P); i += blockDim.x) sm.acc[i] = 0;
  __syncthreads();

  const unsigned nblocks = gridDim.x;
  unsigned gen = 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int team_in_cta = warp / P, p = warp % P;
  const int teams_per_cta = nwarps / P;
  const int team = blockIdx.x * teams_per_cta + team_in_cta;
  const int nteams = gridDim.x * teams_per_cta;
  const int G = W >> 5;
  const int g = team % G, vslot = team / G, vslots = nteams / G;
  const bool active = team_in_cta < teams_per_cta && vslot < vslots;
  const int w = g * 32 + lane;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = gridDim.x * blockDim.x;

  for (int t = a.t0; t < a.t1; ++t) {
    for (int c = 0; c < a.n_colours; ++c) {
      if (active) {
        const int v0 = __ldg(a.col_ptr + c), v1 = __ldg(a.col_ptr + c + 1);
        for (int v = v0 + vslot; v < v1; v += vslots)
          fast_attempt<NB, KQ, P>(a, sm, v, w, t, warp, team_in_cta, p, lane);
      }
      if (!grid_sync(a.bar, nblocks, gen, kSweepWaitLimitNs)) return;
    }
    if (active) {
#pragma unroll
      for (int b = 0; b < 32 / P; ++b) {
        int *slot = &sm.acc[(warp * (32 / P) + b) * 32 + lane];
        const int val = *slot;
        if (val != 0) {
          atomicAdd(&sm.eacc[w * 33 + p * (32 / P) + b], val);
          *slot = 0;
        }
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < W * 32; i += blockDim.x) {
      const int s = (i >> 5) * 33 + (i & 31);
      const int val = sm.eacc[s];
      if (val != 0) {
        atomicAdd(&a.energy[i], val);
        sm.eacc[s] = 0;
      }
    }
    if (!grid_sync(a.bar, nblocks, gen, kSweepWaitLimitNs)) return;
    if (gtid < W * 32) {
      const int e = __ldcg(a.energy + gtid);
      const int be = __ldcg(a.best_energy + gtid);
      const bool better = e < be;
      if (better) __stcg(a.best_energy + gtid, e);
      const unsigned mask = __ballot_sync(0xFFFFFFFFu, better);
      if ((threadIdx.x & 31) == 0) __stcg(a.imp + (gtid >> 5), mask);
    }
    if (!grid_sync(a.bar, nblocks, gen, kSweepWaitLimitNs)) return;
  }
  if (a.t1 > a.t0) {
    for (long long i = gtid; i < (long long)a.n * W; i += nthreads) {
      const int ww = (int)(i % W);
      const uint32_t m = __ldcg(a.imp + ww);
      if (m) {
        const long long v = i / W;
        const uint32_t x = __ldcg(a.S + (size_t)(2 * v) * W + ww);
        __stcg(a.best + i, (__ldcg(a.best + i) & ~m) | (x & m));
      }
    }
    if (!grid_sync(a.bar, nblocks, gen, kSweepWaitLimitNs)) return;
    for (int i = gtid; i < W; i += nthreads) __stcg(a.imp + i, 0u);
  }
}

// One CTA waits for `expected` arrivals at the barrier; with expected > 1 nothing releases it
// and the bounded wait must expire.
__global__ void wait_selftest_kernel(GridBarrier *gb, unsigned expected,
                                     unsigned long long limit_ns) {
  unsigned gen = 0;
  grid_sync(gb, expected, gen, limit_ns);
}

// ---- initial states, energies, unpacking ---------------------------------------------------
__global__ void ksat_init_kernel(uint32_t *S, uint32_t *best, const int32_t *orig,
                                 const uint8_t *init, int32_t n, int32_t W, int32_t R,
                                 uint32_t k0, uint32_t k1, bool write_best) {
  const long long total = (long long)(n + 1) * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(i / W), w = (int)(i % W);
    if (v == n) {  // dummy rows: literal 2n always false, 2n+1 always true
      S[(size_t)(2 * n) * W + w] = 0u;
      S[(size_t)(2 * n + 1) * W + w] = 0xFFFFFFFFu;
      continue;
    }
    const uint32_t vo = (uint32_t)orig[v];
    uint32_t x = 0u;
    if (init) {
      for (int b = 0; b < 32; ++b) {
        const int r = 32 * w + b;
        if (r < R) x |= (uint32_t)(init[(size_t)r * n + vo] & 1u) << b;
      }
    } else {
      for (int g = 0; g < 8; ++g) {
        const uint4 u = philox4x32_10(make_uint4(vo, 0u, (uint32_t)(8 * w + g), kTagKsatInit), k0, k1);
        x |= (u.x & 1u) << (4 * g) | (u.y & 1u) << (4 * g + 1) | (u.z & 1u) << (4 * g + 2) |
             (u.w & 1u) << (4 * g + 3);
      }
    }
    S[(size_t)(2 * v) * W + w] = x;
    S[(size_t)(2 * v + 1) * W + w] = ~x;
    if (write_best) best[(size_t)v * W + w] = x;
  }
}

// Energy of every replica from scratch: a clause is violated in the replicas where none of its
// literal words has the bit set.
__global__ void ksat_energy_kernel(const uint32_t *S, const int32_t *clits, int32_t m,
                                   int32_t kmax, int32_t W, int32_t *energy) {
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = gridDim.x * blockDim.x;
  const int slots = nthreads / W;
  const int w = gtid % W, slot = gtid / W;
  if (slot >= slots) return;
  int cnt[32];
#pragma unroll
  for (int b = 0; b < 32; ++b) cnt[b] = 0;
  for (int c = slot; c < m; c += slots) {
    uint32_t o = 0u;
    for (int q = 0; q < kmax; ++q) o |= S[(size_t)clits[(size_t)c * kmax + q] * W + w];
    const uint32_t u = ~o;
#pragma unroll
    for (int b = 0; b < 32; ++b) cnt[b] += (int)((u >> b) & 1u);
  }
#pragma unroll
  for (int b = 0; b < 32; ++b)
    if (cnt[b]) atomicAdd(&energy[32 * w + b], cnt[b]);
}

__global__ void ksat_unpack_kernel(const uint32_t *S, const uint32_t *best,
                                   const int32_t *newid, const int32_t *energy,
                                   const int32_t *best_energy, int32_t n, int32_t W, int32_t R,
                                   uint8_t *states, uint8_t *best_states, int64_t *e_out,
                                   int64_t *be_out) {
  const long long total = (long long)R * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / n), vo = (int)(i % n);
    const int v = newid[vo];
    const int w = r >> 5, b = r & 31;
    if (states) states[i] = (uint8_t)((S[(size_t)(2 * v) * W + w] >> b) & 1u);
    if (best_states) best_states[i] = (uint8_t)((best[(size_t)v * W + w] >> b) & 1u);
    if (vo == 0) {
      if (e_out) e_out[r] = energy[r];
      if (be_out) be_out[r] = best_energy[r];
    }
  }
}

// beta[u][t] (float, original unit order) -> bq[t][new(u)] = round_half_even(beta * 2^16).
// Tiles of 32 units x 32 steps keep both the reads and the writes coalesced.
__global__ void quantize_kernel(const float *beta, int32_t n_units, int32_t n_steps,
                                const int32_t *orig, uint32_t *bq, int32_t *bad) {
  __shared__ uint32_t tile[32][33];
  const int t0 = blockIdx.x * 32;
  for (int v0 = blockIdx.y * 32; v0 < n_units; v0 += gridDim.y * 32) {
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int v = v0 + j, t = t0 + threadIdx.x;
    uint32_t q = 0u;
    if (v < n_units && t < n_steps) {
      const int u = orig ? orig[v] : v;
      const float b = beta[(size_t)u * n_steps + t];
      if (isinf(b) && b > 0.0f) {
        q = kFrozenQ16;
      } else if (!(b >= 0.0f && b <= 65535.0f)) {  // also rejects NaN
        atomicExch(bad, 1);
      } else {
        q = __float2uint_rn(b * 65536.0f);  // exact product, ties to even
      }
    }
    tile[j][threadIdx.x] = q;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int t = t0 + j, v = v0 + threadIdx.x;
    if (v < n_units && t < n_steps) bq[(size_t)t * n_units + v] = tile[threadIdx.x][j];
  }
  }
}

// beta[u][t] = base[t] * factor[u] (float32, round to nearest) -> bq[t][new(u)], validated.
__global__ void quantize_factored_kernel(const float *base, const float *factor, int32_t n_units,
                                         int32_t n_steps, const int32_t *orig, uint32_t *bq,
                                         int32_t *bad) {
  const long long total = (long long)n_units * n_steps;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i / n_units), v = (int)(i % n_units);
    const int u = orig ? orig[v] : v;
    const float b = __fmul_rn(base[t], factor[u]);
    uint32_t q = 0u;
    if (isinf(b) && b > 0.0f) {
      q = kFrozenQ16;
    } else if (!(b >= 0.0f && b <= 65535.0f)) {
      atomicExch(bad, 1);
    } else {
      q = __float2uint_rn(b * 65536.0f);
    }
    bq[i] = q;
  }
}

template <int NB, int KQ>
cudaError_t launch_sweeps(const SweepArgs &a, int device, cudaStream_t st) {
  const size_t smem = sizeof(uint32_t) * (((a.tab_len + 31) & ~31) + (size_t)a.W * 33);
  cudaError_t err;
  auto kern = ksat_sweep_kernel<NB, KQ>;
  err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSweepThreads, smem);
  if (err != cudaSuccess) return err;
  int sms = 0;
  err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  while (per_sm > 1 && sms * per_sm > kMaxGridCtas) --per_sm;
  const int blocks = sms * per_sm;
  if (blocks > kMaxGridCtas) return cudaErrorInvalidConfiguration;
  void *args[] = {(void *)&a};
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(blocks), dim3(kSweepThreads), args,
                                     smem, st);
}


template <int NB, int KQ, int P, int THREADS>
cudaError_t launch_fast(const SweepArgs &a, int device, cudaStream_t st) {
  const int threads = THREADS;
  const int nwarps = threads / 32;
  const size_t smem = fast_smem_bytes<NB, KQ, P>(a.tab_len, a.W, nwarps);
  auto kern = ksat_sweep_fast_kernel<NB, KQ, P, THREADS>;
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, int> grids;  // (device, smem) -> co-resident CTAs
  int blocks = 0;
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = grids.find({device, smem});
    if (it != grids.end()) {
      blocks = it->second;
    } else {
      cudaError_t err =
          cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      int per_sm = 0;
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
      if (err != cudaSuccess) return err;
      int sms = 0;
      err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
      if (err != cudaSuccess) return err;
      if (per_sm < 1) return cudaErrorInvalidConfiguration;
      while (per_sm > 1 && sms * per_sm > kMaxGridCtas) --per_sm;
      if (sms * per_sm > kMaxGridCtas) return cudaErrorInvalidConfiguration;
      blocks = sms * per_sm;
      grids[{device, smem}] = blocks;
    }
  }
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  void *args[] = {(void *)&a};
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(blocks), dim3(threads), args, smem, st);
}

// Fast-path shape: warps per variable (teams of P warps; at most 15 teams per CTA).
int g_fast_p = 2;

template <int NB, int KQ>
cudaError_t dispatch_fast(const SweepArgs &a, int device, cudaStream_t st) {
  switch (g_fast_p) {
    case 1: return launch_fast<NB, KQ, 1, 512>(a, device, st);
    case 4: return launch_fast<NB, KQ, 4, 1024>(a, device, st);
    default: return launch_fast<NB, KQ, 2, 896>(a, device, st);
  }
}

int grid_for(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 65535LL * 8) b = 65535LL * 8;
  return (int)b;
}

}  // namespace

void set_sweep_shape(int warps_per_variable) { g_fast_p = warps_per_variable; }

cudaError_t ksat_init_states(const KsatDevice &I, KsatReplicas &Rp, uint64_t seed,
                             const uint8_t *init_dev, cudaStream_t st, bool set_best) {
  const long long work = (long long)(I.n + 1) * Rp.W;
  ksat_init_kernel<<<grid_for(work, 256), 256, 0, st>>>(Rp.S, Rp.best, I.orig, init_dev, I.n,
                                                        Rp.W, Rp.R, (uint32_t)seed,
                                                        (uint32_t)(seed >> 32), set_best);
  return cudaGetLastError();
}

cudaError_t ksat_energies(const KsatDevice &I, KsatReplicas &Rp, cudaStream_t st, bool set_best) {
  cudaError_t err = cudaMemsetAsync(Rp.energy, 0, sizeof(int32_t) * 32 * Rp.W, st);
  if (err != cudaSuccess) return err;
  if (I.m > 0) {
    const long long want = (long long)Rp.W * ((I.m + 63) / 64);
    int blocks = grid_for(want, 256);
    if (blocks > 4096) blocks = 4096;
    ksat_energy_kernel<<<blocks, 256, 0, st>>>(Rp.S, I.clits, I.m, I.kmax, Rp.W, Rp.energy);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (!set_best) return cudaSuccess;
  return cudaMemcpyAsync(Rp.best_energy, Rp.energy, sizeof(int32_t) * 32 * Rp.W,
                         cudaMemcpyDeviceToDevice, st);
}

cudaError_t ksat_sweeps(const KsatDevice &I, KsatReplicas &Rp, const uint32_t *bq,
                        const uint32_t *tab, int32_t tab_len, int32_t t0, int32_t t1,
                        uint64_t seed, int device, cudaStream_t st) {
  if (t1 <= t0) return cudaSuccess;
  cudaError_t err = cudaMemsetAsync(reinterpret_cast<char *>(Rp.bar) + kBarrierResetOffset, 0, kBarrierResetBytes, st);
  if (err != cudaSuccess) return err;
  SweepArgs a;
  a.S = Rp.S;
  a.best = Rp.best;
  a.energy = Rp.energy;
  a.best_energy = Rp.best_energy;
  a.imp = Rp.imp;
  a.bar = Rp.bar;
  a.occ = I.occ;
  a.occ_ptr = I.occ_ptr;
  a.col_ptr = I.col_ptr;
  a.orig = I.orig;
  a.bq = bq;
  a.tab = tab;
  a.tab_len = tab_len;
  a.n = I.n;
  a.W = Rp.W;
  a.n_colours = I.n_colours;
  a.t0 = t0;
  a.t1 = t1;
  a.k0 = (uint32_t)seed;
  a.k1 = (uint32_t)(seed >> 32);
  if (const char *env = getenv("NMC_SWEEP_WARPS")) g_fast_p = atoi(env);  // tuning override
  if (Rp.W % 32 == 0 && I.nb <= 7 && g_fast_p > 0) {
    if (I.kq == 1) return I.nb <= 5 ? dispatch_fast<5, 1>(a, device, st) : dispatch_fast<7, 1>(a, device, st);
    return I.nb <= 5 ? dispatch_fast<5, 2>(a, device, st) : dispatch_fast<7, 2>(a, device, st);
  }
  if (I.kq == 1) {
    if (I.nb <= 5) return launch_sweeps<5, 1>(a, device, st);
    if (I.nb <= 7) return launch_sweeps<7, 1>(a, device, st);
    return launch_sweeps<10, 1>(a, device, st);
  }
  if (I.nb <= 5) return launch_sweeps<5, 2>(a, device, st);
  if (I.nb <= 7) return launch_sweeps<7, 2>(a, device, st);
  return launch_sweeps<10, 2>(a, device, st);
}

cudaError_t ksat_unpack(const KsatDevice &I, const KsatReplicas &Rp, uint8_t *states,
                        uint8_t *best_states, int64_t *energies, int64_t *best_energies,
                        cudaStream_t st) {
  const long long work = (long long)Rp.R * I.n;
  ksat_unpack_kernel<<<grid_for(work, 256), 256, 0, st>>>(Rp.S, Rp.best, I.newid, Rp.energy,
                                                          Rp.best_energy, I.n, Rp.W, Rp.R,
                                                          states, best_states, energies,
                                                          best_energies);
  return cudaGetLastError();
}

cudaError_t wait_selftest(GridBarrier *gb, unsigned long long limit_ns, cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(reinterpret_cast<char *>(gb) + kBarrierResetOffset, 0, kBarrierResetBytes, st);
  if (err != cudaSuccess) return err;
  wait_selftest_kernel<<<1, 32, 0, st>>>(gb, 2u, limit_ns);
  return cudaGetLastError();
}

cudaError_t quantize_schedule_factored(const float *base, const float *factor, int32_t n_units,
                                       int32_t n_steps, const int32_t *orig, uint32_t *bq,
                                       int32_t *bad, cudaStream_t st) {
  const long long work = (long long)n_units * n_steps;
  quantize_factored_kernel<<<grid_for(work, 256), 256, 0, st>>>(base, factor, n_units, n_steps,
                                                                  orig, bq, bad);
  return cudaGetLastError();
}

cudaError_t quantize_schedule(const float *beta, int32_t n_units, int32_t n_steps,
                              const int32_t *orig, uint32_t *bq, int32_t *bad,
                              cudaStream_t st) {
  int gy = (n_units + 31) / 32;
  if (gy > 65535) gy = 65535;
  dim3 grid((n_steps + 31) / 32, gy);
  quantize_kernel<<<grid, dim3(32, 8), 0, st>>>(beta, n_units, n_steps, orig, bq, bad);
  return cudaGetLastError();
}

}  // namespace nmc
