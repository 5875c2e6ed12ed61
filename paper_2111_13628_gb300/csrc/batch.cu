// Batched k-SAT sweep: one persistent launch runs many replica sets of uneven instances
// (sampling stage of Algorithm 1 for many problems at once).
//
// Work item = (replica set, word w of 32 replicas, sweep range). A cluster of CS CTAs takes
// items from a device counter; each CTA loads the item's word vector x[0..n) into its shared
// memory, runs the sweeps with the variables of one colour class spread over the cluster's
// threads (one thread, or a team of 2, 4 or 8 lanes, per variable for the 32 replicas of the
// word), stores every new word into all CS copies, and meets the cluster barrier between
// classes; the next class's bounds are requested before that barrier. Words are independent
// chains, so no grid-wide synchronisation is needed and uneven instances fill the GPU. The
// dynamics are identical to the single-instance kernels. Occurrence lists are read in a
// warp-interleaved layout (one coalesced load per occurrence for 32 variables); each thread
// keeps its share of the sweep's energy change as 16 bit-sliced planes and converts them to
// per-replica sums once per sweep.
#include <cooperative_groups.h>

#include <cstdlib>
#include <map>
#include <mutex>

#include "nmc.h"
#include "nmc_internal.h"
#include "bits.cuh"
#include "philox.cuh"

namespace cg = cooperative_groups;

namespace nmc {

namespace {

// One-thread kernel for k <= 4: 16 warps, up to 128 registers (no spills; a DSatur colour class
// of the 50,000-variable bench instance puts at most ~490 variables on each CTA of a 4-CTA
// cluster, one round of 512 threads: measured 296 us per sweep against 295 with 640 threads and
// 96 registers, and 293 with the next class's loads requested at the barrier, which 640 threads
// cannot hold without spilling). For k <= 8 (two int4 list entries per occurrence, twice the
// prefetched registers) 12 warps with up to 168 registers, so that nothing spills.
template <int KQ>
__host__ __device__ constexpr int one_thread_threads() {
  return KQ == 1 ? 512 : 384;
}
constexpr int kTeamThreads = 384;   // team kernel with teams of 2 or 4: 12 warps, up to 168 registers
constexpr int kTeam8Threads = 512;  // team kernel with teams of 8: up to 128 registers

// Threads of the sweep kernel with TL lanes per variable: 384 for teams of 2 or 4, which then
// prefetch their occurrence entries a group ahead (measured at N = 5,000: 107 -> 102 us per
// sweep); 512 for teams of 8 (the tiny classes of small instances, where 384 threads measured
// slower: N = 200, 37.3 -> 45.3 us; 640 spilled with the replica-exchange multipliers); single
// threads as one_thread_threads.
template <int KQ, int TL>
__host__ __device__ constexpr int sweep_threads() {
  return (TL == 2 || TL == 4) ? kTeamThreads : (TL == 8 ? kTeam8Threads : one_thread_threads<KQ>());
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

// Adds a0..a3 into the weight-1 and weight-2 planes c[0], c[1] of a bit-sliced counter and
// returns the weight-4 carry, which the caller adds from plane 2 up.
template <int NB>
__device__ __forceinline__ uint32_t csa4_low(uint32_t (&c)[NB], uint32_t a0, uint32_t a1,
                                             uint32_t a2, uint32_t a3) {
  const uint32_t s1 = c[0] ^ a0 ^ a1;
  const uint32_t y1 = maj3b(c[0], a0, a1);
  c[0] = s1 ^ a2 ^ a3;
  const uint32_t y2 = maj3b(s1, a2, a3);
  const uint32_t s3 = c[1] ^ y1 ^ y2;
  const uint32_t f = maj3b(c[1], y1, y2);
  c[1] = s3;
  return f;
}

// c += f * 4 (f one bit per replica), carries rippled up to the top plane.
template <int NB>
__device__ __forceinline__ void add_carry(uint32_t (&c)[NB], uint32_t f) {
#pragma unroll
  for (int j = 2; j < NB; ++j) {
    const uint32_t t = c[j] & f;
    c[j] ^= f;
    f = t;
  }
}

// c += (f + g) * 4: a full adder at plane 2, then one ripple from plane 3.
template <int NB>
__device__ __forceinline__ void add_carry_pair(uint32_t (&c)[NB], uint32_t f, uint32_t g) {
  const uint32_t s = c[2] ^ f ^ g;
  uint32_t carry = maj3b(c[2], f, g);
  c[2] = s;
#pragma unroll
  for (int j = 3; j < NB; ++j) {
    const uint32_t t = c[j] & carry;
    c[j] ^= carry;
    carry = t;
  }
}

constexpr int kAccPlanes = 16;  // per-thread energy accumulator: 16-bit two's complement

// k <= 4 entries of the interleaved lists: literal words by byte offset into the word vector
// (which starts at the beginning of dynamic shared memory); sign i is bit 7 of byte i of the
// first field, turned into an all-zeros / all-ones mask.
__device__ __forceinline__ uint32_t xs_at(const uint32_t *xs, int byte_off) {
  return *reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(xs) + byte_off);
}

// prmt with the top bit of every selector nibble set replicates the sign (bit 7) of byte I of
// sg into all four result bytes: one instruction per mask.
template <int I>
__device__ __forceinline__ uint32_t sign_mask(uint32_t sg) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(sg), "r"(0u), "n"(0x8888 + 0x1111 * I));
  return r;
}

// Byte b (0..3) of x as a signed value: prmt replicates the byte's sign into the upper three
// bytes (selector nibbles 8-15).
__device__ __forceinline__ int sext_byte(uint32_t x, int b) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(0u), "r"(0x8880u + 0x1111u * (uint32_t)b));
  return (int)r;
}

// OR over the clause's other literals of their truth values (32 replicas), from an occurrence's
// entry: q = {sign bits, byte offsets of literals 1..3}; for k > 4 also q2 = {byte offsets of
// literals 4..7}, whose signs sit in bit 6 of bytes 0..3 of q.x (shifted up to bit 7 here).
template <int KQ>
__device__ __forceinline__ uint32_t others_or(const uint32_t *xs, const int4 &q, const int4 &q2) {
  const uint32_t sg = (uint32_t)q.x;
  uint32_t o = (xs_at(xs, q.y) ^ sign_mask<1>(sg)) | (xs_at(xs, q.z) ^ sign_mask<2>(sg)) |
               (xs_at(xs, q.w) ^ sign_mask<3>(sg));
  if (KQ == 2) {
    const uint32_t s6 = sg << 1;
    o |= (xs_at(xs, q2.x) ^ sign_mask<0>(s6)) | (xs_at(xs, q2.y) ^ sign_mask<1>(s6)) |
         (xs_at(xs, q2.z) ^ sign_mask<2>(s6)) | (xs_at(xs, q2.w) ^ sign_mask<3>(s6));
  }
  return o;
}

// Adds the bit-sliced counter p into c (ripple carry).
template <int NB>
__device__ __forceinline__ void add_planes(uint32_t (&c)[NB], const uint32_t (&p)[NB]) {
  uint32_t carry = 0u;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const uint32_t a = c[j], b = p[j];
    c[j] = a ^ b ^ carry;
    carry = maj3b(a, b, carry);
  }
}

// The loads of one attempt that do not depend on the replicas' states: the variable's Q16
// inverse temperature, its list length and its first group of occurrence entries. A thread
// requests them for its next variable before it waits at the barrier that ends the current
// colour class, so their L2 / HBM latency overlaps the barrier.
template <int KQ>
struct AttemptPrep {
  int4 q[4 * KQ];
  const int4 *ent;
  int len;
  int regions;  // k <= 4: own-sign regions of the variable's group (a | b << 16)
  uint32_t bq;
};

// v = c0 + off is a variable of colour class c (starting at new id c0; cg: the class's first
// group of 32 variables), attempted at sweep t.
template <int KQ>
__device__ __forceinline__ void prep_attempt(const BatchItem &B, int cg, int c0, int v, int t,
                                             AttemptPrep<KQ> &p) {
  p.bq = __ldg(B.bq + (size_t)t * B.n + v);
  const int off = v - c0;
  const int g = cg + (off >> 5), ln = off & 31;
  const int gb = __ldg(B.grp_base + g);
  p.len = (__ldg(B.grp_base + g + 1) - gb) / (32 * KQ);
  p.ent = B.occ_t + gb + ln;
  p.regions = KQ == 1 ? __ldg(B.grp_base + B.n_groups + 1 + g) : 0;
  if (p.len > 0) {
#pragma unroll
    for (int j = 0; j < 4 * KQ; ++j) p.q[j] = __ldg(p.ent + (size_t)j * 32);
  }
}

// One attempt of variable v at sweep t for the 32 replicas of the word, from the loads in P.
// With PT, replica j of the word moves at min(2^32-1, (mult_s[j] * bq) >> 16) instead of bq.
template <int KQ, bool PT>
__device__ __forceinline__ uint32_t attempt_batch(const BatchItem &B, const uint32_t *xs,
                                                  const uint32_t *tab_s, int tab_len,
                                                  const uint32_t *mult_s, int v, int t,
                                                  AttemptPrep<KQ> &P,
                                                  uint32_t (&acc)[kAccPlanes]) {
  constexpr int NB = 7;
  const uint32_t x = xs[v];
  const uint32_t bqv = P.bq;
  if (bqv == kFrozenQ16) return x;  // held at this step: no attempt
  uint32_t bc[NB], mc[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    bc[j] = 0u;
    mc[j] = 0u;
  }
  const int len = P.len;
  const int4 *ent = P.ent;
  // The entries of the next group of 4 occurrences are requested before the current group is
  // evaluated, so the L2 latency of the list overlaps the shared-memory gathers and counting.
  int4 (&qn)[4 * KQ] = P.q;
  // break / make masks of the 4 occurrences whose entries are in qc
  auto masks4 = [&](const int4 (&qc)[4 * KQ], uint32_t (&bb)[4], uint32_t (&mm)[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int4 q = qc[j * KQ];
      const uint32_t o = others_or<KQ>(xs, q, qc[j * KQ + KQ - 1]);
      const uint32_t own = x ^ sign_mask<0>((uint32_t)q.x);
      bb[j] = own & ~o;
      mm[j] = ~(own | o);
    }
  };
  if constexpr (KQ == 1) {
    // Own-sign split (k <= 4): in a lane's list the occurrences where its own literal is positive
    // come first. With z = "every other literal of the clause false", a replica's energy change
    // is x ? Zp - Zn : Zn - Zp, Zp / Zn counting z over the positive / negated occurrences; slots
    // [0, ra) are positive in every lane of the group and slots from rb on negated (or inert), so
    // only [ra, rb) needs both counters, split by the own sign. bc counts Zp, mc counts Zn; each
    // keeps one weight-4 carry pending so that the carries of two groups enter it together.
    const int ra = P.regions & 0xFFFF, rb = P.regions >> 16;
    uint32_t fp = 0u, fn = 0u;
    bool pp = false, pn = false;
    auto add4 = [&](uint32_t (&c)[NB], uint32_t &f, bool &pend, const uint32_t (&z)[4]) {
      const uint32_t g = csa4_low(c, z[0], z[1], z[2], z[3]);
      if (pend) add_carry_pair<NB>(c, f, g);
      else f = g;
      pend = !pend;
    };
    for (int e = 0; e < len; e += 4) {
      int4 qc[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) qc[j] = qn[j];
      if (e + 4 < len) {
#pragma unroll
        for (int j = 0; j < 4; ++j) qn[j] = __ldg(ent + (size_t)(e + 4 + j) * 32);
      }
      uint32_t z[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t sg = (uint32_t)qc[j].x;
        z[j] = ~((xs_at(xs, qc[j].y) ^ sign_mask<1>(sg)) | (xs_at(xs, qc[j].z) ^ sign_mask<2>(sg)) |
                 (xs_at(xs, qc[j].w) ^ sign_mask<3>(sg)));
      }
      if (e + 4 <= ra) {
        add4(bc, fp, pp, z);
      } else if (e >= rb) {
        add4(mc, fn, pn, z);
      } else {
        uint32_t zp[4], zn[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t neg = sign_mask<0>((uint32_t)qc[j].x);
          zp[j] = z[j] & ~neg;
          zn[j] = z[j] & neg;
        }
        add4(bc, fp, pp, zp);
        add4(mc, fn, pn, zn);
      }
    }
    if (pp) add_carry<NB>(bc, fp);
    if (pn) add_carry<NB>(mc, fn);
    // (bc, mc) <- (Zp, Zn) where x = 1, (Zn, Zp) where x = 0: the subtraction below is the dE
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const uint32_t a = (bc[j] & x) | (mc[j] & ~x), c = (mc[j] & x) | (bc[j] & ~x);
      bc[j] = a;
      mc[j] = c;
    }
  } else {
    // Two groups of 4 per trip: each group's weight-4 carry is kept aside and the pair's carries
    // enter the planes from weight 4 up once (one ripple per 8 occurrences instead of per 4).
    // Every group's entries are still requested one group before they are evaluated.
    for (int e = 0; e < len; e += 8) {
      int4 qc[4 * KQ];
      uint32_t bb[4], mm[4];
#pragma unroll
      for (int j = 0; j < 4 * KQ; ++j) qc[j] = qn[j];
      if (e + 4 < len) {
#pragma unroll
        for (int j = 0; j < 4 * KQ; ++j) qn[j] = __ldg(ent + (size_t)((e + 4) * KQ + j) * 32);
      }
      masks4(qc, bb, mm);
      uint32_t fb = csa4_low(bc, bb[0], bb[1], bb[2], bb[3]);
      uint32_t fm = csa4_low(mc, mm[0], mm[1], mm[2], mm[3]);
      if (e + 4 < len) {
#pragma unroll
        for (int j = 0; j < 4 * KQ; ++j) qc[j] = qn[j];
        if (e + 8 < len) {
#pragma unroll
          for (int j = 0; j < 4 * KQ; ++j) qn[j] = __ldg(ent + (size_t)((e + 8) * KQ + j) * 32);
        }
        masks4(qc, bb, mm);
        add_carry_pair<NB>(bc, fb, csa4_low(bc, bb[0], bb[1], bb[2], bb[3]));
        add_carry_pair<NB>(mc, fm, csa4_low(mc, mm[0], mm[1], mm[2], mm[3]));
      } else {
        add_carry<NB>(bc, fb);
        add_carry<NB>(mc, fm);
      }
    }
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
  // replicas whose dE <= 0 (sign plane set, or every plane zero) accept without a draw
  uint32_t flip = s8[7] | ~(s8[0] | s8[1] | s8[2] | s8[3] | s8[4] | s8[5] | s8[6]);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    // replicas 8q .. 8q+7: Philox groups 2q and 2q+1, drawn together and always (a draw that
    // cannot change an acceptance changes nothing; a branch on whether any lane needs one rarely
    // skips the work for the whole warp and keeps the four pairs from overlapping: 236.5 -> 225.7
    // us per sweep on the 50,000-variable bench instance)
    const unsigned long long xm = transpose8(gather_bytes(s8, q));
    int de[8];
    uint32_t th[8];
    const uint32_t xlo = (uint32_t)xm, xhi = (uint32_t)(xm >> 32);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      de[j] = sext_byte(j < 4 ? xlo : xhi, j & 3);
      uint32_t hi = bq_hi, lo = bq_lo;
      if (PT) {
        const unsigned long long be = ((unsigned long long)mult_s[8 * q + j] * bqv) >> 16;
        const uint32_t b = be > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)be;
        hi = b >> 8;  // below 2^24, so hi dE stays below 2^31
        lo = b & 255u;
      }
      // for dE <= 0 the index is meaningless but clamped into the table; those replicas
      // accept whatever the comparison gives
      const uint32_t idx = hi * (uint32_t)de[j] + ((lo * (uint32_t)de[j]) >> 8);
      th[j] = tab_s[min(idx, (uint32_t)tab_len)];  // entry tab_len is 0
    }
    uint4 u0, u1;
    philox4x32_10_x2(make_uint4(vo, (uint32_t)t, (uint32_t)(8 * B.w + 2 * q), kTagKsatSweep),
                       make_uint4(vo, (uint32_t)t, (uint32_t)(8 * B.w + 2 * q + 1), kTagKsatSweep),
                       B.k0, B.k1, u0, u1);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t u = j < 4 ? uint4_word(u0, j) : uint4_word(u1, j - 4);
      flip |= (uint32_t)(u < th[j]) << (8 * q + j);
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

// ---- team variant: TL lanes per variable --------------------------------------------------------
//
// Same dynamics, shorter critical path: a team of TL consecutive lanes evaluates one variable.
// Lane t of the team takes occurrences t, t+TL, ... of the variable's list, counts its break /
// make masks in bit-sliced counters, and the team adds its TL partial counters with an xor
// butterfly of shuffles, so every lane ends with the totals. Lane t then resolves the
// acceptance of replica groups [t*8/TL, (t+1)*8/TL) (one Philox block per group of 4 replicas)
// and the team ORs the flip bits. A colour class of a few hundred variables then costs the
// latency of a TL-th of one attempt instead of a whole one.
template <int KQ, int TL, bool PT, bool PF = false>
__device__ __forceinline__ uint32_t attempt_team(const BatchItem &B, const uint32_t *xs,
                                                 const uint32_t *tab_s, int tab_len,
                                                 const uint32_t *mult_s, int cg, int c0, int v,
                                                 bool active, int t, int tl,
                                                 int (&acc)[32 / TL]) {
  constexpr int NB = 7;
  const uint32_t x = active ? xs[v] : 0u;
  const uint32_t bqv = active ? __ldg(B.bq + (size_t)t * B.n + v) : 0u;
  // a held variable takes no attempt; the team still joins the shuffles below
  const bool frozen = bqv == kFrozenQ16;
  uint32_t bc[NB], mc[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    bc[j] = 0u;
    mc[j] = 0u;
  }
  int len = 0;
  const int4 *ent = nullptr;
  if (active && !frozen) {
    const int off = v - c0;
    const int g = cg + (off >> 5), ln = off & 31;  // cg: the class's first group
    const int gb = __ldg(B.grp_base + g);
    len = (__ldg(B.grp_base + g + 1) - gb) / (32 * KQ);
    ent = B.occ_t + gb + ln;
  }
  // occurrences j0 + i TL (i < 4) of the lane: break / make masks into the counters
  auto eval4 = [&](const int4 (&qc)[4 * KQ], int j0) {
    uint32_t bb[4], mm[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = j0 + i * TL;
      bb[i] = 0u;
      mm[i] = 0u;
      if (j < len) {
        const int4 q = qc[i * KQ];
        const uint32_t o = others_or<KQ>(xs, q, qc[i * KQ + KQ - 1]);
        const uint32_t own = x ^ sign_mask<0>((uint32_t)q.x);
        bb[i] = own & ~o;
        mm[i] = ~(own | o);
      }
    }
    csa4<NB>(bc, bb[0], bb[1], bb[2], bb[3]);
    csa4<NB>(mc, mm[0], mm[1], mm[2], mm[3]);
  };
  auto load4 = [&](int4 (&q)[4 * KQ], int j0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = j0 + i * TL;
#pragma unroll
      for (int k = 0; k < KQ; ++k)
        q[i * KQ + k] = j < len ? __ldg(ent + (size_t)(j * KQ + k) * 32) : make_int4(0, 0, 0, 0);
    }
  };
  if constexpr (PF) {
    // the next group of the lane's entries is requested before the current one is evaluated
    int4 qn[4 * KQ];
    if (tl < len) load4(qn, tl);
    for (int j0 = tl; j0 < len; j0 += 4 * TL) {
      int4 qc[4 * KQ];
#pragma unroll
      for (int i = 0; i < 4 * KQ; ++i) qc[i] = qn[i];
      if (j0 + 4 * TL < len) load4(qn, j0 + 4 * TL);
      eval4(qc, j0);
    }
  } else {
    // each group's entries loaded where they are evaluated
    for (int j0 = tl; j0 < len; j0 += 4 * TL) {
      uint32_t bb[4], mm[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int j = j0 + i * TL;
        bb[i] = 0u;
        mm[i] = 0u;
        if (j < len) {
          const int4 q = __ldg(ent + (size_t)(j * KQ) * 32);
          const int4 q2 = KQ == 2 ? __ldg(ent + (size_t)(j * KQ + 1) * 32) : q;
          const uint32_t o = others_or<KQ>(xs, q, q2);
          const uint32_t own = x ^ sign_mask<0>((uint32_t)q.x);
          bb[i] = own & ~o;
          mm[i] = ~(own | o);
        }
      }
      csa4<NB>(bc, bb[0], bb[1], bb[2], bb[3]);
      csa4<NB>(mc, mm[0], mm[1], mm[2], mm[3]);
    }
  }
#pragma unroll
  for (int sft = 1; sft < TL; sft <<= 1) {
    uint32_t pb[NB], pm[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      pb[j] = __shfl_xor_sync(0xFFFFFFFFu, bc[j], sft);
      pm[j] = __shfl_xor_sync(0xFFFFFFFFu, mc[j], sft);
    }
    add_planes<NB>(bc, pb);
    add_planes<NB>(mc, pm);
  }
  uint32_t d[NB + 1];
  {
    uint32_t br = 0u;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      d[j] = bc[j] ^ mc[j] ^ br;
      br = maj3b(~bc[j], mc[j], br);
    }
    d[NB] = br;
  }
  const uint32_t vo = active ? (uint32_t)__ldg(B.orig + v) : 0u;
  const uint32_t bq_hi = bqv >> 8, bq_lo = bqv & 255u;
  constexpr int GPL = 8 / TL;             // Philox groups (4 replicas) per lane
  constexpr int NBK = GPL >= 2 ? GPL / 2 : 1;  // blocks of 8 replicas the lane's groups lie in
  // one 8x8 transpose of the 8 planes of D per block gives the replicas' signed bytes
  unsigned long long xmb[NBK];
#pragma unroll
  for (int b = 0; b < NBK; ++b) xmb[b] = transpose8(gather_bytes(d, ((tl * GPL) >> 1) + b));
  uint32_t flip = 0u;
  // the lane's Philox groups, drawn always and two at a time (as in attempt_batch)
  int de[4 * GPL];
  uint32_t th[4 * GPL];
#pragma unroll
  for (int gi = 0; gi < GPL; ++gi) {
    const int g = tl * GPL + gi;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = 4 * g + j;
      const int val = (int)(signed char)(unsigned char)(xmb[gi >> 1] >> (8 * (r & 7)));
      de[4 * gi + j] = val;
      uint32_t hi = bq_hi, lo = bq_lo;
      if (PT) {
        const unsigned long long be = ((unsigned long long)mult_s[r] * bqv) >> 16;
        const uint32_t b = be > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)be;
        hi = b >> 8;
        lo = b & 255u;
      }
      // for dE <= 0 the index is meaningless but clamped into the table; those replicas accept
      const uint32_t idx = hi * (uint32_t)val + ((lo * (uint32_t)val) >> 8);
      th[4 * gi + j] = tab_s[min(idx, (uint32_t)tab_len)];  // entry tab_len is 0
    }
  }
#pragma unroll
  for (int gi = 0; gi < GPL; gi += 2) {
    const int g = tl * GPL + gi;
    uint4 u[2];
    if (gi + 1 < GPL) {
      philox4x32_10_x2(make_uint4(vo, (uint32_t)t, (uint32_t)(8 * B.w + g), kTagKsatSweep),
                       make_uint4(vo, (uint32_t)t, (uint32_t)(8 * B.w + g + 1), kTagKsatSweep),
                       B.k0, B.k1, u[0], u[1]);
    } else {
      u[0] = philox4x32_10(make_uint4(vo, (uint32_t)t, (uint32_t)(8 * B.w + g), kTagKsatSweep),
                           B.k0, B.k1);
      u[1] = u[0];
    }
#pragma unroll
    for (int k = 0; k < 2 && gi + k < GPL; ++k) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int i = 4 * (gi + k) + j;
        const bool ok = de[i] <= 0 || uint4_word(u[k], j) < th[i];
        flip |= (uint32_t)ok << (4 * (g + k) + j);
        if (active) acc[i] += ok ? de[i] : 0;
      }
    }
  }
  if (frozen) flip = 0u;  // zero counters read as dE = 0: cancel those flips
#pragma unroll
  for (int sft = 1; sft < TL; sft <<= 1) flip |= __shfl_xor_sync(0xFFFFFFFFu, flip, sft);
  return x ^ flip;
}

// A colour class [c0, c1) is shared out among the CS CTAs of a cluster by 32-variable groups,
// round-robin: CTA `rank` takes groups rank, rank + CS, ... Variables are degree-descending
// inside a class, so each CTA gets a like mix of long and short occurrence lists (contiguous
// shares would give rank 0 all the longest lists and make every class wait for it).
template <int CS>
__device__ __forceinline__ int share_count(int c0, int c1, int rank) {
  const int ng = (c1 - c0 + 31) >> 5;
  const int mine = ng > rank ? (ng - rank + CS - 1) / CS : 0;
  int cnt = mine * 32;
  if (mine > 0 && rank + (mine - 1) * CS == ng - 1) cnt -= ng * 32 - (c1 - c0);  // last, partial
  return cnt;
}

// Local index li (0 <= li < share_count) -> variable.
template <int CS>
__device__ __forceinline__ int share_var(int c0, int rank, int li) {
  return c0 + 32 * (rank + CS * (li >> 5)) + (li & 31);
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

// The cluster barrier in two halves: arrive (releasing this thread's earlier shared-memory
// stores to the cluster) and wait (acquiring everyone's). Work between the two halves overlaps
// the barrier; it must not touch shared memory that other CTAs read before the wait.
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
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

// A colour class whose share on this CTA is cnt <= blockDim / TT variables: team `team` (TT
// consecutive lanes) updates local variable `team` (the same round-robin share as the one-thread
// path) with attempt_team, stores its new word to every copy of the cluster, and adds its
// replicas' energy changes to ep_s. Warps with no team in range skip the class.
template <int KQ, int CS, int TT, bool PT>
__device__ __forceinline__ void class_teams(const BatchItem &B, uint32_t *xs, const uint32_t *tab_s,
                                            int tab_len, const uint32_t *mult_s, int cg, int c0,
                                            int cnt, int rank, int t, int *ep_s) {
  const int lane = threadIdx.x & 31;
  if ((int)(threadIdx.x & ~31u) / TT >= cnt) return;  // the whole warp
  const int team = threadIdx.x / TT, tl = lane % TT;
  const bool active = team < cnt;
  const int v = active ? share_var<CS>(c0, rank, team) : c0;
  int tacc[32 / TT];
#pragma unroll
  for (int i = 0; i < 32 / TT; ++i) tacc[i] = 0;
  const uint32_t xn = attempt_team<KQ, TT, PT>(B, xs, tab_s, tab_len, mult_s, cg, c0, v, active, t, tl, tacc);
  if (active && tl == 0) {
    if (CS == 1) {
      xs[v] = xn;
    } else {
      const uint32_t sa = (uint32_t)__cvta_generic_to_shared(xs + v);
#pragma unroll
      for (int r = 0; r < CS; ++r) st_rank(sa, r, xn);
    }
  }
#pragma unroll
  for (int i = 0; i < 32 / TT; ++i)
    if (tacc[i] != 0) atomicAdd(&ep_s[4 * (tl * (8 / TT) + i / 4) + (i & 3)], tacc[i]);
}

// CS = CTAs per item. With CS > 1 every CTA of the cluster keeps a full copy of the item's
// word vector; each CTA updates its share of every colour class and stores the new words
// into all CS copies (distributed shared memory), then the cluster barrier publishes them.
// PT: every item carries per-replica temperature multipliers and, optionally, accumulates the
// end-of-sweep energies of sweeps t >= stats_t0 (sums of E and E^2 per replica).
template <int KQ, int CS, bool PT>
__global__ void __launch_bounds__(one_thread_threads<KQ>(), 1)
    ksat_batch_kernel(const BatchItem *__restrict__ items, int n_items, int *next_item,
                      const uint32_t *tab, int tab_len, int xs_words, int small_teams) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t *xs = smem;                               // word vector first (byte offsets in lists)
  uint32_t *tab_s = smem + ((xs_words + 31) & ~31);  // then the acceptance table
  __shared__ int e_s[32], be_s[32], ep_s[32];
  __shared__ uint32_t mult_s[32];
  __shared__ uint32_t imp_s;
  __shared__ int item_s;
  __shared__ BatchItem item_b;  // the current item, read from shared memory where needed
  const int rank = CS == 1 ? 0 : (int)cg::this_cluster().block_rank();
  for (int i = threadIdx.x; i <= tab_len; i += blockDim.x) tab_s[i] = i < tab_len ? tab[i] : 0u;
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
      if (PT) mult_s[threadIdx.x] = B.mult[32 * w + threadIdx.x];
      if (rank == 0) {
        e_s[threadIdx.x] = B.energy[32 * w + threadIdx.x];
        be_s[threadIdx.x] = B.best_energy[32 * w + threadIdx.x];
      }
    }
    long long s1 = 0, s2 = 0;  // energy statistics of this lane's replica (rank 0, warp 0)
    // Best states of the replicas that improve during this item go to a word-major staging row
    // (the second half of the best buffer) at each improving sweep end, and into the [var][word]
    // layout once, at the end of the item: a merge into that layout touches one 32-byte sector
    // per variable, which at every improving sweep cost about 30 us per sweep on the 50,000-
    // variable bench instance.
    uint32_t *best_t = B.best + (size_t)n * W + (size_t)w * n;
    uint32_t m_item = 0;  // replicas improved during this item
    group_sync<CS>();
    for (int t = B.t0; t < B.t1; ++t) {
      uint32_t acc[kAccPlanes];
#pragma unroll
      for (int j = 0; j < kAccPlanes; ++j) acc[j] = 0u;
      // class bounds and first group: those of class c + 1 are requested during class c and
      // arrive behind its barrier
      int c0 = __ldg(B.col_ptr), c1 = __ldg(B.col_ptr + 1), cg = __ldg(B.cgrp);
      // a share of a class with at most this many variables on the CTA runs with teams of lanes
      constexpr int kThreads = one_thread_threads<KQ>();
      const int team_max = small_teams ? kThreads / 2 : -1;
      // the state-independent loads of this thread's first variable of each class: requested
      // for class c + 1 between the two halves of the barrier that ends class c
      // (every thread loads, those without a variable in the class for variable c0, so that
      // P is written before every class and never live across the team path)
      AttemptPrep<KQ> P;
      {
        const int cnt0 = share_count<CS>(c0, c1, rank);
        const bool mine = cnt0 > team_max && (int)threadIdx.x < cnt0;
        prep_attempt<KQ>(B, cg, c0, mine ? share_var<CS>(c0, rank, threadIdx.x) : c0, t, P);
      }
      for (int c = 0; c < B.n_colours; ++c) {
        int c2 = 0, cgn = 0;
        if (c + 1 < B.n_colours) {
          c2 = __ldg(B.col_ptr + c + 2);
          cgn = __ldg(B.cgrp + c + 1);
        }
        // the class's 32-variable groups are dealt round-robin to the cluster's CTAs
        const int cnt = share_count<CS>(c0, c1, rank);
        if (cnt <= team_max) {
          // a smaller share (the later colour classes): teams of 8, 4 or 2 lanes per variable
          // shorten the class's critical path; their energy changes go to ep_s directly
          if (cnt <= kThreads / 8)
            class_teams<KQ, CS, 8, PT>(B, xs, tab_s, tab_len, mult_s, cg, c0, cnt, rank, t, ep_s);
          else if (cnt <= kThreads / 4)
            class_teams<KQ, CS, 4, PT>(B, xs, tab_s, tab_len, mult_s, cg, c0, cnt, rank, t, ep_s);
          else
            class_teams<KQ, CS, 2, PT>(B, xs, tab_s, tab_len, mult_s, cg, c0, cnt, rank, t, ep_s);
        } else {
          auto store = [&](int v, uint32_t xn) {
            if (CS == 1) {
              xs[v] = xn;
            } else {
              const uint32_t sa = (uint32_t)__cvta_generic_to_shared(xs + v);
#pragma unroll
              for (int r = 0; r < CS; ++r) st_rank(sa, r, xn);
            }
          };
          bool first = true;  // the first variable's loads were requested at the barrier
          for (int li = threadIdx.x; li < cnt; li += blockDim.x) {
            const int v = share_var<CS>(c0, rank, li);
            if (!first) prep_attempt<KQ>(B, cg, c0, v, t, P);
            first = false;
            store(v, attempt_batch<KQ, PT>(B, xs, tab_s, tab_len, mult_s, v, t, P, acc));
          }
        }
        // the next class's first attempt of this thread loads its entries during the barrier
        const bool more = c + 1 < B.n_colours;
        const int cntn = more ? share_count<CS>(c1, c2, rank) : 0;
        const int vn = cntn > team_max && (int)threadIdx.x < cntn
                           ? share_var<CS>(c1, rank, threadIdx.x) : c1;
        if (CS == 1) {
          if (more) prep_attempt<KQ>(B, cgn, c1, vn, t, P);
          __syncthreads();
        } else {
          cluster_arrive();
          if (more) prep_attempt<KQ>(B, cgn, c1, vn, t, P);
          cluster_wait();
        }
        c0 = c1;
        c1 = c2;
        cg = cgn;
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
        if (PT && B.stats && t >= B.stats_t0) {
          s1 += sum;
          s2 += (long long)sum * sum;
        }
        const bool better = sum < be_s[lane];
        if (better) be_s[lane] = sum;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, better);
        if (lane == 0) imp_s = m;
      }
      group_sync<CS>();
      const uint32_t m = *rank_ptr<CS>(&imp_s, 0);
      if (threadIdx.x < 32) ep_s[threadIdx.x] = 0;
      __syncthreads();  // cleared before the next sweep's team-path adds
      if (m) {  // the improved replicas' states, into this word's staging row (coalesced)
        const int b0 = rank * share, b1 = min(n, b0 + share);
        for (int v = b0 + threadIdx.x; v < b1; v += blockDim.x)
          best_t[v] = (best_t[v] & ~m) | (xs[v] & m);
        m_item |= m;
        group_sync<CS>();
      }
    }
    {
      const int b0 = rank * share, b1 = min(n, b0 + share);
      for (int v = b0 + threadIdx.x; v < b1; v += blockDim.x) {
        B.S[(size_t)(2 * v) * W + w] = xs[v];
        B.S[(size_t)(2 * v + 1) * W + w] = ~xs[v];
        if (m_item) {  // replicas improved during the item: their last best state from staging
          const size_t bi = (size_t)v * W + w;
          B.best[bi] = (B.best[bi] & ~m_item) | (best_t[v] & m_item);
        }
      }
    }
    if (rank == 0 && threadIdx.x < 32) {
      B.energy[32 * w + threadIdx.x] = e_s[threadIdx.x];
      B.best_energy[32 * w + threadIdx.x] = be_s[threadIdx.x];
      if (PT && B.stats) {  // one item per word in a launch: plain read-modify-write
        B.stats[32 * w + threadIdx.x] += s1;
        B.stats[32 * (B.W + w) + threadIdx.x] += s2;
      }
    }
    group_sync<CS>();
  }
}


template <int KQ, int CS, int TL, bool PT>
__global__ void __launch_bounds__(sweep_threads<KQ, TL>(), 1)
    ksat_team_kernel(const BatchItem *__restrict__ items, int n_items, int *next_item,
                     const uint32_t *tab, int tab_len, int xs_words, int small_teams) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t *xs = smem;                               // word vector first (byte offsets in lists)
  uint32_t *tab_s = smem + ((xs_words + 31) & ~31);  // then the acceptance table
  __shared__ int e_s[32], be_s[32], ep_s[32];
  __shared__ uint32_t mult_s[32];
  __shared__ uint32_t imp_s;
  __shared__ int item_s;
  __shared__ BatchItem item_b;
  const int rank = CS == 1 ? 0 : (int)cg::this_cluster().block_rank();
  for (int i = threadIdx.x; i <= tab_len; i += blockDim.x) tab_s[i] = i < tab_len ? tab[i] : 0u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tl = lane % TL;                       // lane inside the team
  const int team = threadIdx.x / TL;              // team inside the CTA
  const int nteams = blockDim.x / TL;
  while (true) {
    if (rank == 0 && threadIdx.x == 0) item_s = atomicAdd(next_item, 1);
    group_sync<CS>();
    const int it = *rank_ptr<CS>(&item_s, 0);
    if (it < n_items && threadIdx.x == 0) item_b = items[it];
    group_sync<CS>();
    if (it >= n_items) break;
    const BatchItem &B = item_b;
    const int n = B.n, W = B.W, w = B.w;
    const int share = (n + CS - 1) / CS;
    for (int v = threadIdx.x; v < n; v += blockDim.x) xs[v] = B.S[(size_t)(2 * v) * W + w];
    if (threadIdx.x == 0) xs[n] = 0u;
    if (threadIdx.x < 32) {
      ep_s[threadIdx.x] = 0;
      if (PT) mult_s[threadIdx.x] = B.mult[32 * w + threadIdx.x];
      if (rank == 0) {
        e_s[threadIdx.x] = B.energy[32 * w + threadIdx.x];
        be_s[threadIdx.x] = B.best_energy[32 * w + threadIdx.x];
      }
    }
    long long s1 = 0, s2 = 0;  // energy statistics of this lane's replica (rank 0, warp 0)
    // Best states of the replicas that improve during this item go to a word-major staging row
    // (the second half of the best buffer) at each improving sweep end, and into the [var][word]
    // layout once, at the end of the item: a merge into that layout touches one 32-byte sector
    // per variable, which at every improving sweep cost about 30 us per sweep on the 50,000-
    // variable bench instance.
    uint32_t *best_t = B.best + (size_t)n * W + (size_t)w * n;
    uint32_t m_item = 0;  // replicas improved during this item
    group_sync<CS>();
    for (int t = B.t0; t < B.t1; ++t) {
      int acc[32 / TL];
#pragma unroll
      for (int i = 0; i < 32 / TL; ++i) acc[i] = 0;
      // class bounds and first group: for teams of 2 or 4 those of class c + 1 are requested
      // during class c (the tiny classes of teams of 8 measured faster loading their own)
      constexpr bool ahead = sweep_threads<KQ, TL>() == kTeamThreads;
      int c0 = __ldg(B.col_ptr), c1 = __ldg(B.col_ptr + 1), cg = __ldg(B.cgrp);
      for (int c = 0; c < B.n_colours; ++c) {
        int c2 = 0, cgn = 0;
        if (!ahead) {
          c0 = __ldg(B.col_ptr + c);
          c1 = __ldg(B.col_ptr + c + 1);
          cg = __ldg(B.cgrp + c);
        } else if (c + 1 < B.n_colours) {
          c2 = __ldg(B.col_ptr + c + 2);
          cgn = __ldg(B.cgrp + c + 1);
        }
        // contiguous shares here (measured: round-robin groups are slower for the teams)
        const int part = ((c1 - c0 + CS - 1) / CS + 31) & ~31;
        const int v0 = c0 + rank * part, v1 = min(c1, v0 + part);
        // warp-uniform trip count: the warp's teams take consecutive variables each round
        for (int vw = v0 + warp * (32 / TL); vw < v1; vw += nteams) {
          const int v = vw + (lane / TL);
          const bool active = v < v1;
          const uint32_t xn =
              attempt_team<KQ, TL, PT, (sweep_threads<KQ, TL>() == kTeamThreads)>(B, xs, tab_s, tab_len,
                                                                         mult_s, cg, c0, v, active,
                                                                         t, tl, acc);
          if (active && tl == 0) {
            if (CS == 1) {
              xs[v] = xn;
            } else {
              const uint32_t sa = (uint32_t)__cvta_generic_to_shared(xs + v);
#pragma unroll
              for (int r = 0; r < CS; ++r) st_rank(sa, r, xn);
            }
          }
        }
        group_sync<CS>();
        c0 = c1;
        c1 = c2;
        cg = cgn;
      }
#pragma unroll
      for (int i = 0; i < 32 / TL; ++i)
        if (acc[i] != 0) atomicAdd(&ep_s[4 * (tl * (8 / TL) + i / 4) + (i & 3)], acc[i]);
      group_sync<CS>();
      if (rank == 0 && warp == 0) {
        int sum = e_s[lane];
#pragma unroll
        for (int r = 0; r < CS; ++r) sum += rank_ptr<CS>(ep_s, r)[lane];
        e_s[lane] = sum;
        if (PT && B.stats && t >= B.stats_t0) {
          s1 += sum;
          s2 += (long long)sum * sum;
        }
        const bool better = sum < be_s[lane];
        if (better) be_s[lane] = sum;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, better);
        if (lane == 0) imp_s = m;
      }
      group_sync<CS>();
      const uint32_t m = *rank_ptr<CS>(&imp_s, 0);
      if (threadIdx.x < 32) ep_s[threadIdx.x] = 0;
      if (m) {  // the improved replicas' states, into this word's staging row (coalesced)
        const int b0 = rank * share, b1 = min(n, b0 + share);
        for (int v = b0 + threadIdx.x; v < b1; v += blockDim.x)
          best_t[v] = (best_t[v] & ~m) | (xs[v] & m);
        m_item |= m;
        group_sync<CS>();
      }
    }
    {
      const int b0 = rank * share, b1 = min(n, b0 + share);
      for (int v = b0 + threadIdx.x; v < b1; v += blockDim.x) {
        B.S[(size_t)(2 * v) * W + w] = xs[v];
        B.S[(size_t)(2 * v + 1) * W + w] = ~xs[v];
        if (m_item) {  // replicas improved during the item: their last best state from staging
          const size_t bi = (size_t)v * W + w;
          B.best[bi] = (B.best[bi] & ~m_item) | (best_t[v] & m_item);
        }
      }
    }
    if (rank == 0 && threadIdx.x < 32) {
      B.energy[32 * w + threadIdx.x] = e_s[threadIdx.x];
      B.best_energy[32 * w + threadIdx.x] = be_s[threadIdx.x];
      if (PT && B.stats) {  // one item per word in a launch: plain read-modify-write
        B.stats[32 * w + threadIdx.x] += s1;
        B.stats[32 * (B.W + w) + threadIdx.x] += s2;
      }
    }
    group_sync<CS>();
  }
  (void)team;
  (void)small_teams;
}

// The launch shape of each kernel instance is queried once per (device, shared-memory size):
// occupancy and cluster queries are slow host calls.
template <int KQ, int CS, int TL, bool PT = false>
cudaError_t launch_batch(const BatchItem *items, int n_items, int *next_item,
                         const uint32_t *tab, int tab_len, int max_n, int device,
                         cudaStream_t st) {
  const int xs_words = max_n + 1;
  const size_t smem = sizeof(uint32_t) * (((size_t)xs_words + 31) / 32 * 32 + (size_t)tab_len + 1);
  auto kern = TL == 1 ? ksat_batch_kernel<KQ, CS, PT> : ksat_team_kernel<KQ, CS, (TL > 1 ? TL : 4), PT>;
  constexpr int threads = sweep_threads<KQ, TL>();
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, int> shapes;  // (device, smem) -> resident clusters
  static std::map<int, int> sm_count;                    // device -> SMs
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
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        if (err != cudaSuccess) return err;
        clusters = sms * per_sm;
      } else {
        cudaLaunchConfig_t q = {};
        q.blockDim = dim3(threads);
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
  int sms = 0;
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = sm_count.find(device);
    if (it == sm_count.end()) {
      cudaError_t err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
      if (err != cudaSuccess) return err;
      sm_count[device] = sms;
    } else {
      sms = it->second;
    }
  }
  // Teams of lanes for the smaller colour classes shorten a class's critical path; they pay
  // off when each SM runs one CTA of the launch (latency-bound), not when many items queue
  // behind each other (measured on a 256-instance batch: 3% slower with them).
  const int small_teams = (long long)n_items * CS <= sms ? 1 : 0;
  if (clusters > n_items) clusters = n_items;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(threads);
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
  return cudaLaunchKernelEx(&cfg, kern, items, n_items, next_item, tab, tab_len, xs_words, small_teams);
}

// Lanes per variable of the batched kernel: 1 (one thread per variable) or a team of 4 or 8.
// Few variables per CTA per colour class favour teams (latency), many favour single threads.
int batch_lanes(int cs, int max_n, int want) {
  if (const char *env = getenv("NMC_BATCH_LANES")) {
    const int l = atoi(env);
    if (l == 1 || l == 4 || l == 8) return l;
  }
  if (want == 1 || want == 4 || want == 8) return want;  // a tuned shape
  // variables of one colour class per CTA, taking ~32 classes. Measured on 4-SAT (alpha ~9.9,
  // 640 threads): teams of 8 lanes win up to ~24 variables per CTA and class, teams of 4 up to
  // ~100 (5,000 variables over 4-CTA clusters: 151 us per sweep vs 160 with 8 lanes and 227
  // with 1), single threads beyond (20,000 variables over 4-CTA clusters: 253 vs 277 with 4).
  const int per_cta = max_n / (32 * cs);
  if (per_cta <= 24) return 8;
  if (per_cta <= 100) return 4;
  return 1;
}

template <int KQ, int CS>
cudaError_t dispatch_lanes(const BatchItem *items, int n_items, int *next_item, const uint32_t *tab,
                           int tab_len, int max_n, int device, cudaStream_t st, bool pt, int lanes) {
  if (pt) {
    switch (batch_lanes(CS, max_n, lanes)) {
      case 4: return launch_batch<KQ, CS, 4, true>(items, n_items, next_item, tab, tab_len, max_n, device, st);
      case 8: return launch_batch<KQ, CS, 8, true>(items, n_items, next_item, tab, tab_len, max_n, device, st);
      default: return launch_batch<KQ, CS, 1, true>(items, n_items, next_item, tab, tab_len, max_n, device, st);
    }
  }
  switch (batch_lanes(CS, max_n, lanes)) {
    case 4: return launch_batch<KQ, CS, 4>(items, n_items, next_item, tab, tab_len, max_n, device, st);
    case 8: return launch_batch<KQ, CS, 8>(items, n_items, next_item, tab, tab_len, max_n, device, st);
    default: return launch_batch<KQ, CS, 1>(items, n_items, next_item, tab, tab_len, max_n, device, st);
  }
}

template <int KQ>
cudaError_t dispatch_batch(int cs, const BatchItem *items, int n_items, int *next_item,
                           const uint32_t *tab, int tab_len, int max_n, int device, cudaStream_t st,
                           bool pt, int lanes) {
  switch (cs) {
    case 8: return dispatch_lanes<KQ, 8>(items, n_items, next_item, tab, tab_len, max_n, device, st, pt, lanes);
    case 4: return dispatch_lanes<KQ, 4>(items, n_items, next_item, tab, tab_len, max_n, device, st, pt, lanes);
    case 2: return dispatch_lanes<KQ, 2>(items, n_items, next_item, tab, tab_len, max_n, device, st, pt, lanes);
    default: return dispatch_lanes<KQ, 1>(items, n_items, next_item, tab, tab_len, max_n, device, st, pt, lanes);
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
static_assert(sizeof(BatchItem) == 136 && kNoAllocItems == 7708, "limit stated in nmc.h");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

// Device address of g_noalloc_scratch, looked up once per device (with that device current)
// and kept for the rest of the process: a device reset after the first call is not supported.
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
                       counters + q, plan.tab, plan.tab_len, plan.device, plan.stream, false,
                       plan.lanes[q]);
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
  const long long words = (long long)optin / 4 - tab_len - 1 - 32 - 1 - 192;
  return words > 0 ? (size_t)words : 0;
}

cudaError_t ksat_batch(const BatchItem *items_dev, int n_items, int kq, int cs, int max_n,
                       int *next_item, const uint32_t *tab, int tab_len, int device,
                       cudaStream_t st, bool pt, int lanes) {
  if (n_items <= 0) return cudaSuccess;
  if (kq == 1) return dispatch_batch<1>(cs, items_dev, n_items, next_item, tab, tab_len, max_n, device, st, pt, lanes);
  return dispatch_batch<2>(cs, items_dev, n_items, next_item, tab, tab_len, max_n, device, st, pt, lanes);
}

}  // namespace nmc
