// QAP kernels: Metropolis over permutations with pairwise swap moves (Koopmans-Beckmann cost,
// Sec. "Quadratic Assignment Problems"; per-facility inverse temperature as in the sampling
// stage of Algorithm 1).
//
// A CTA runs 32 replicas. Each replica has LPR lanes: LPR = 16 (two replicas per warp, one per
// half) for n <= 128, where the per-attempt broadcasts, reductions and branches are the larger
// part of the work and then serve two replicas at once, and LPR = 32 (one per warp) beyond.
// With NPL = ceil(n / LPR), lane l of a replica owns the locations p[k] of the facilities
// k = NPL l + i (i < NPL) in registers. F and D (entries 0..255, stored as bytes) of the CTA's
// instance sit in shared memory, shared by its replicas; each F row is stored as LPR lane
// chunks of CHB = 4, 8 or 16 bytes (a lane's facilities, zero padded), so a lane reads its part
// of a row with one aligned load. The swap change
//   dC(r,s) = 2 sum_{k != r,s} (F_rk - F_sk)(D_{p(s)p(k)} - D_{p(r)p(k)})
// is an O(n) dot product split over the replica's lanes: the gathered D bytes are packed four
// to a word and the byte products F_r D_s + F_s D_r - F_r D_r - F_s D_s are summed with dp4a,
// then over the lanes. The Philox blocks of LPR consecutive attempts of each replica are drawn
// in parallel, one per lane, and broadcast in turn.
#include "nmc_internal.h"
#include "philox.cuh"

namespace nmc {

namespace {

// Launch shapes: shape q < 8 runs n <= 16 (q + 1) with LPR = 16; shape 8 + q runs
// n <= 32 (q + 5) with LPR = 32.
template <int LPR>
constexpr int qap_threads() { return 32 * 32 / (32 / LPR); }  // 32 replicas per CTA

template <int NPL>
__device__ __forceinline__ void put(int (&p)[NPL], int i, int v) {
#pragma unroll
  for (int q = 0; q < NPL; ++q)
    if (q == i) p[q] = v;
}

template <int NPL>
__device__ __forceinline__ int pick(const int (&p)[NPL], int i) {
  int v = p[0];
#pragma unroll
  for (int q = 1; q < NPL; ++q)
    if (q == i) v = p[q];
  return v;
}

// Shared-memory layout of F: row r at r * LDF, as LPR lane chunks of CHB bytes; facility k
// sits in chunk k / NPL at byte k % NPL (padding bytes zero).
template <int NPL, int LPR>
struct FLayout {
  static constexpr int CHB = NPL <= 4 ? 4 : (NPL <= 8 ? 8 : 16);  // bytes of one lane chunk
  static constexpr int LDF = LPR * CHB;                            // row stride in bytes
  __device__ __forceinline__ static int at(int r, int k) { return r * LDF + CHB * (k / NPL) + k % NPL; }
};

// Four zero-extended bytes (b0 lowest) packed into one word.
__device__ __forceinline__ uint32_t pack4(uint32_t b0, uint32_t b1, uint32_t b2, uint32_t b3) {
  return __byte_perm(__byte_perm(b0, b1, 0x0040), __byte_perm(b2, b3, 0x0040), 0x5410);
}

// Cost of the permutation ps with the whole warp: sum_i sum_j F_ij D_{p(i)p(j)}. The warp's
// 32 / LPR lane groups take rows i in turn; lane l of a group reads its chunk of F row i and the
// bytes D_{p(i)p(k)} of its facilities k = NPL l + q, four to a word, and sums the products with
// dp4a (a row's partial sum stays below 2^22).
template <int NPL, int LPR>
__device__ long long warp_cost(const uint8_t *Fs, const uint8_t *Ds, const uint8_t *ps, int n,
                               int lane) {
  constexpr int CHB = FLayout<NPL, LPR>::CHB, LDF = FLayout<NPL, LPR>::LDF, RPW = 32 / LPR;
  const int hl = lane % LPR;
  int pk[NPL];
#pragma unroll
  for (int q = 0; q < NPL; ++q) {
    const int k = NPL * hl + q;
    pk[q] = k < n ? ps[k] : 0;  // padding facilities: F entries zero
  }
  long long acc = 0;
  for (int i = lane / LPR; i < n; i += RPW) {
    const uint8_t *Drow = Ds + ps[i] * n;
    const uint32_t *Fw = reinterpret_cast<const uint32_t *>(Fs + i * LDF + CHB * hl);
    uint32_t row = 0u;
#pragma unroll
    for (int w4 = 0; w4 < CHB / 4; ++w4) {
      uint32_t b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = 4 * w4 + q;
        b[q] = j < NPL ? (uint32_t)Drow[pk[j < NPL ? j : 0]] : 0u;
      }
      row = __dp4a(Fw[w4], pack4(b[0], b[1], b[2], b[3]), row);
    }
    acc += row;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  return acc;
}

// Initial permutation of replica r into its shared-memory row ps (Fisher-Yates from the
// identity, position q = n-1..1 exchanged with (u (q+1)) >> 32, or a copy of the given state),
// then its cost and the global copies. Whole warp.
template <int NPL, int LPR>
__device__ void qap_init_one(const QapArgs &a, const uint8_t *Fs, const uint8_t *Ds, uint8_t *ps,
                             int r, int lane) {
  const int n = a.n;
  int16_t *gp = a.perm + (size_t)r * n;
  if (a.init_mode == 1) {
    for (int k = lane; k < n; k += 32) ps[k] = (uint8_t)k;
    __syncwarp();
    for (int q0 = n - 1; q0 >= 1; q0 -= 32) {
      const int q = q0 - lane;
      uint32_t u = 0u;
      if (q >= 1)
        u = philox4x32_10(make_uint4((uint32_t)q, 0u, (uint32_t)r, kTagQapInit), a.k0, a.k1).x;
      const int cnt = q0 >= 32 ? 32 : q0;
      for (int j = 0; j < cnt; ++j) {
        const uint32_t uj = __shfl_sync(0xFFFFFFFFu, u, j);
        const int qq = q0 - j;
        const int kk = (int)(((unsigned long long)uj * (unsigned)(qq + 1)) >> 32);
        if (lane == 0) {
          const uint8_t tmp = ps[qq];
          ps[qq] = ps[kk];
          ps[kk] = tmp;
        }
        __syncwarp();
      }
    }
  } else {
    for (int k = lane; k < n; k += 32) ps[k] = (uint8_t)gp[k];
    __syncwarp();
  }
  const long long c = warp_cost<NPL, LPR>(Fs, Ds, ps, n, lane);
  const bool set_best = a.init_mode != 3;
  for (int k = lane; k < n; k += 32) {
    gp[k] = (int16_t)ps[k];
    if (set_best) a.best_perm[(size_t)r * n + k] = (int16_t)ps[k];
  }
  if (lane == 0) {
    a.energy[r] = c;
    if (set_best) a.best_energy[r] = c;
  }
  __syncwarp();
}

// A CTA runs the 32 replicas of one block: lane group h = lane / LPR of warp w runs replica
// 32 block + RPW w + h, its lane l = lane % LPR owning facilities NPL l + i.
template <int NPL, int LPR>
__device__ __forceinline__ void qap_body(const QapArgs &a, int block) {
  constexpr int RPW = 32 / LPR;  // replicas per warp
  extern __shared__ __align__(16) uint32_t smem[];
  const int n = a.n;
  constexpr int CHB = FLayout<NPL, LPR>::CHB, LDF = FLayout<NPL, LPR>::LDF;
  uint32_t *tab_s = smem;
  uint8_t *Fs = (uint8_t *)(smem + ((a.tab_len + 31) & ~31));
  uint8_t *Ds = Fs + ((n * LDF + 15) & ~15);
  uint8_t *pw_all = Ds + ((n * n + 15) & ~15);  // one n-byte row per replica (permutation copy)
  const int pstride = (n + 15) & ~15;
  for (int i = threadIdx.x; i < a.tab_len; i += blockDim.x) tab_s[i] = a.tab[i];
  for (int i = threadIdx.x; i < n * LDF; i += blockDim.x) {
    const int row = i / LDF, col = i % LDF, j = col % CHB, k = NPL * (col / CHB) + j;
    Fs[i] = (j < NPL && k < n) ? a.F[row * n + k] : (uint8_t)0;
  }
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) Ds[i] = a.D[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = block * 32 + RPW * warp;  // the warp's first replica
  if (r0 >= a.R) return;                   // the whole warp
  if (a.init_mode != 0) {
    for (int h = 0; h < RPW && r0 + h < a.R; ++h)
      qap_init_one<NPL, LPR>(a, Fs, Ds, pw_all + (RPW * warp + h) * pstride, r0 + h, lane);
    return;
  }
  const int half = lane / LPR, hl = lane % LPR;
  const int r = r0 + half;
  const bool live = r < a.R;  // the second half of the last warp may have no replica
  uint8_t *pw = pw_all + (RPW * warp + half) * pstride;
  const int16_t *gp = a.perm + (size_t)(live ? r : r0) * n;
  for (int k = hl; k < n; k += LPR) pw[k] = live ? (uint8_t)gp[k] : (uint8_t)0;
  __syncwarp();
  int p[NPL];  // padding facilities (k >= n) sit at location 0; their F entries are zero
#pragma unroll
  for (int i = 0; i < NPL; ++i) {
    const int k = NPL * hl + i;
    p[i] = k < n ? pw[k] : 0;
  }
  long long e = live ? a.energy[r] : 0;
  long long be = live ? a.best_energy[r] : 0;
  const int nm1 = n - 1;
  const unsigned long long mr = (a.mult && live) ? a.mult[r] : 0ull;  // replica exchange multiplier
  // energy statistics: running double sums of the costs after steps t >= stats_t0 (and of their
  // squares), continued from the stored values so that split runs add in step order
  double s1 = 0.0, s2 = 0.0;
  if (a.stats && live) {
    s1 = a.stats[r];
    s2 = a.stats[(size_t)a.R + r];
  }
  for (int t = a.t0; t < a.t1; ++t) {
    if (n >= 2) {
      const uint32_t *bqt = a.bq + (size_t)t * n;
      for (int a0 = 0; a0 < n; a0 += LPR) {
        // lane l of each replica draws its attempt a0 + l
        const int at = a0 + hl;
        int fr = 0, fs = 0, frz = live ? 0 : 1;  // no replica: every attempt rejected
        uint32_t u2 = 0u, bqs = 0u;
        if (at < n && live) {
          const uint4 u =
              philox4x32_10(make_uint4((uint32_t)at, (uint32_t)t, (uint32_t)r, kTagQapStep), a.k0, a.k1);
          fr = (int)(((unsigned long long)u.x * (unsigned)n) >> 32);
          fs = (int)(((unsigned long long)u.y * (unsigned)nm1) >> 32);
          fs += fs >= fr;
          u2 = u.z;
          const uint32_t br = __ldg(bqt + fr), bs = __ldg(bqt + fs);
          frz = (br == kFrozenQ16 || bs == kFrozenQ16) ? 1 : 0;  // a held facility: reject
          bqs = (uint32_t)(((unsigned long long)br + bs) >> 1);
        }
        const int cnt = (n - a0) < LPR ? (n - a0) : LPR;
        // r, s (< 256 each) and the held flag of every lane's attempt in one word: one
        // broadcast per attempt within each replica's lanes
        const int packed = fr | (fs << 9) | (frz << 18);
        for (int j = 0; j < cnt; ++j) {
          const int pj = __shfl_sync(0xFFFFFFFFu, packed, j, LPR);
          const bool held = (pj >> 18) != 0;
          if (__all_sync(0xFFFFFFFFu, held)) continue;  // every replica of the warp held
          const int rr = pj & 511, ss = (pj >> 9) & 511;
          int pr, ps;
          if constexpr (LPR == 32) {  // from the owning lanes' registers
            pr = __shfl_sync(0xFFFFFFFFu, pick<NPL>(p, rr % NPL), rr / NPL);
            ps = __shfl_sync(0xFFFFFFFFu, pick<NPL>(p, ss % NPL), ss / NPL);
          } else {  // from the shared-memory copy
            pr = pw[rr];
            ps = pw[ss];
          }
          const uint8_t *Dr = Ds + pr * n, *Dsr = Ds + ps * n;
          // this lane's chunks of rows r and s of F
          uint32_t fr4[CHB / 4], fs4[CHB / 4];
          if constexpr (CHB == 16) {
            const uint4 a4 = *reinterpret_cast<const uint4 *>(Fs + rr * LDF + 16 * hl);
            const uint4 b4 = *reinterpret_cast<const uint4 *>(Fs + ss * LDF + 16 * hl);
            fr4[0] = a4.x; fr4[1] = a4.y; fr4[2] = a4.z; fr4[3] = a4.w;
            fs4[0] = b4.x; fs4[1] = b4.y; fs4[2] = b4.z; fs4[3] = b4.w;
          } else if constexpr (CHB == 8) {
            const uint2 a2 = *reinterpret_cast<const uint2 *>(Fs + rr * LDF + 8 * hl);
            const uint2 b2 = *reinterpret_cast<const uint2 *>(Fs + ss * LDF + 8 * hl);
            fr4[0] = a2.x; fr4[1] = a2.y;
            fs4[0] = b2.x; fs4[1] = b2.y;
          } else {
            fr4[0] = *reinterpret_cast<const uint32_t *>(Fs + rr * LDF + 4 * hl);
            fs4[0] = *reinterpret_cast<const uint32_t *>(Fs + ss * LDF + 4 * hl);
          }
          // sum over every k (padding bytes of F are zero); the k = r and k = s terms sum to
          // -2 F_rs D_{p(r)p(s)} by symmetry and are added back below. Positive and negative
          // products are summed apart (unsigned, below 2^22) and subtracted at the end.
          uint32_t accp = 0u, accn = 0u;
#pragma unroll
          for (int w4 = 0; w4 < CHB / 4; ++w4) {
            uint32_t dr[4], dsb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int i = 4 * w4 + q;
              dr[q] = i < NPL ? (uint32_t)Dr[p[i < NPL ? i : 0]] : 0u;
              dsb[q] = i < NPL ? (uint32_t)Dsr[p[i < NPL ? i : 0]] : 0u;
            }
            const uint32_t wr = pack4(dr[0], dr[1], dr[2], dr[3]);
            const uint32_t wsv = pack4(dsb[0], dsb[1], dsb[2], dsb[3]);
            accp = __dp4a(fr4[w4], wsv, accp);
            accp = __dp4a(fs4[w4], wr, accp);
            accn = __dp4a(fr4[w4], wr, accn);
            accn = __dp4a(fs4[w4], wsv, accn);
          }
          int acc = (int)(accp - accn);
          if constexpr (LPR == 32) {
            acc = __reduce_add_sync(0xFFFFFFFFu, acc);
          } else {
#pragma unroll
            for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
          }
          acc += 2 * (int)Fs[FLayout<NPL, LPR>::at(rr, ss)] * (int)Dr[ps];  // |sum| < 2^24: exact
          const long long d = 2LL * acc;
          // the draw and pair temperature of the attempt: with two replicas per warp fetched
          // always (the uphill test below may diverge between them)
          uint32_t bj = 0u, uj = 0u;
          if (LPR < 32) {
            bj = __shfl_sync(0xFFFFFFFFu, bqs, j, LPR);
            uj = __shfl_sync(0xFFFFFFFFu, u2, j, LPR);
          }
          bool ok = !held && d <= 0;
          if (!held && d > 0) {
            if (LPR == 32) {  // one replica per warp: a warp-uniform branch
              bj = __shfl_sync(0xFFFFFFFFu, bqs, j);
              uj = __shfl_sync(0xFFFFFFFFu, u2, j);
            }
            if (a.mult) {  // min(2^32 - 1, (mult * bq) >> 16)
              const unsigned long long be2 = (mr * bj) >> 16;
              bj = be2 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)be2;
            }
            const unsigned long long idx = ((unsigned long long)bj * (unsigned long long)d) >> 8;
            ok = idx < (unsigned long long)a.tab_len && uj < tab_s[idx];
          }
          if (ok) {
            if (hl == rr / NPL) put<NPL>(p, rr % NPL, ps);
            if (hl == ss / NPL) put<NPL>(p, ss % NPL, pr);
            if (LPR < 32 && hl == 0) {
              pw[rr] = (uint8_t)ps;
              pw[ss] = (uint8_t)pr;
            }
            e += d;
          }
          if (LPR < 32) __syncwarp();  // the row update is seen by the next attempt
        }
      }
    }
    if (live && e < be) {
      be = e;
#pragma unroll
      for (int i = 0; i < NPL; ++i) {
        const int k = NPL * hl + i;
        if (k < n) a.best_perm[(size_t)r * n + k] = (int16_t)p[i];
      }
    }
    if (a.stats && live && t >= a.stats_t0) {
      const double ed = (double)e;
      s1 = __dadd_rn(s1, ed);
      s2 = __dadd_rn(s2, __dmul_rn(ed, ed));
    }
  }
  if (!live) return;
  int16_t *gq = a.perm + (size_t)r * n;
#pragma unroll
  for (int i = 0; i < NPL; ++i) {
    const int k = NPL * hl + i;
    if (k < n) gq[k] = (int16_t)p[i];
  }
  if (hl == 0) {
    a.energy[r] = e;
    a.best_energy[r] = be;
    if (a.stats) {
      a.stats[r] = s1;
      a.stats[(size_t)a.R + r] = s2;
    }
  }
}

template <int NPL, int LPR>
__global__ void __launch_bounds__(qap_threads<LPR>()) qap_kernel(QapArgs a) {
  qap_body<NPL, LPR>(a, blockIdx.x);
}

// Batched QAP: CTA b runs replica block items[b].block of the replica set items[b] describes.
template <int NPL, int LPR>
__global__ void __launch_bounds__(qap_threads<LPR>()) qap_batch_kernel(const QapArgs *items) {
  const QapArgs a = items[blockIdx.x];
  qap_body<NPL, LPR>(a, a.block);
}

// Shape parameters: NPL and LPR of shape q.
__host__ __device__ constexpr int shape_npl(int q) { return q < 8 ? q + 1 : q - 3; }
__host__ __device__ constexpr int shape_lpr(int q) { return q < 8 ? 16 : 32; }

size_t qap_smem_shape(int n, int q, int tab_len) {
  const int npl = shape_npl(q);
  const int ldf = shape_lpr(q) * (npl <= 4 ? 4 : (npl <= 8 ? 8 : 16));  // FLayout::LDF
  return sizeof(uint32_t) * ((tab_len + 31) & ~31) + (size_t)((n * ldf + 15) & ~15) +
         (size_t)((n * n + 15) & ~15) + (size_t)32 * ((n + 15) & ~15);
}

template <int Q>
cudaError_t launch_qap(const QapArgs &a, cudaStream_t st) {
  constexpr int NPL = shape_npl(Q), LPR = shape_lpr(Q);
  const size_t smem = qap_smem_shape(a.n, Q, a.tab_len);
  auto kern = qap_kernel<NPL, LPR>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int blocks = (a.R + 31) / 32;
  kern<<<blocks, qap_threads<LPR>(), smem, st>>>(a);
  return cudaGetLastError();
}

#define NMC_QAP_CASES(CALL) \
  CALL(0) CALL(1) CALL(2) CALL(3) CALL(4) CALL(5) CALL(6) CALL(7) CALL(8) CALL(9) CALL(10) CALL(11)

cudaError_t dispatch_qap(const QapArgs &a, cudaStream_t st) {
  switch (qap_shape(a.n)) {
#define NMC_CASE(k) case k: return launch_qap<k>(a, st);
    NMC_QAP_CASES(NMC_CASE)
#undef NMC_CASE
    default: return cudaErrorInvalidValue;
  }
}

__global__ void qap_unpack_kernel(const int16_t *perm, const int16_t *best_perm,
                                  const long long *energy, const long long *best_energy,
                                  int32_t n, int32_t R, int16_t *p_out, int16_t *bp_out,
                                  int64_t *e_out, int64_t *be_out) {
  const long long total = (long long)R * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    if (p_out) p_out[i] = perm[i];
    if (bp_out) bp_out[i] = best_perm[i];
    if (i < R) {
      if (e_out) e_out[i] = energy[i];
      if (be_out) be_out[i] = best_energy[i];
    }
  }
}

QapArgs make_args(const QapDevice &I, QapReplicas &Rp, uint64_t seed) {
  QapArgs a;
  a.F = (const uint8_t *)I.F;
  a.D = (const uint8_t *)I.D;
  a.perm = Rp.perm;
  a.best_perm = Rp.best_perm;
  a.energy = (long long *)Rp.energy;
  a.best_energy = (long long *)Rp.best_energy;
  a.bq = nullptr;
  a.tab = nullptr;
  a.tab_len = 0;
  a.n = I.n;
  a.R = Rp.R;
  a.t0 = a.t1 = 0;
  a.k0 = (uint32_t)seed;
  a.k1 = (uint32_t)(seed >> 32);
  a.init_mode = 0;
  a.block = -1;
  a.mult = nullptr;
  a.stats = nullptr;
  a.stats_t0 = 0;
  return a;
}

template <int Q>
cudaError_t launch_qap_batch(const QapArgs *items_dev, int n_blocks, int max_n, int tab_len,
                             cudaStream_t st) {
  constexpr int NPL = shape_npl(Q), LPR = shape_lpr(Q);
  const size_t smem = qap_smem_shape(max_n, Q, tab_len);
  auto kern = qap_batch_kernel<NPL, LPR>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  kern<<<n_blocks, qap_threads<LPR>(), smem, st>>>(items_dev);
  return cudaGetLastError();
}

}  // namespace

QapArgs qap_block_args(const QapDevice &I, QapReplicas &Rp, const uint32_t *bq, const uint32_t *tab,
                       int32_t tab_len, int32_t t0, int32_t t1, uint64_t seed, int block) {
  QapArgs a = make_args(I, Rp, seed);
  a.bq = bq;
  a.tab = tab;
  a.tab_len = tab_len;
  a.t0 = t0;
  a.t1 = t1;
  a.block = block;
  return a;
}

int qap_shape(int n) { return n <= 128 ? (n + 15) / 16 - 1 : 8 + (n + 31) / 32 - 5; }

cudaError_t qap_batch(const QapArgs *items_dev, int n_blocks, int shape, int max_n, int tab_len,
                      cudaStream_t st) {
  if (n_blocks <= 0) return cudaSuccess;
  switch (shape) {
#define NMC_CASE(k) case k: return launch_qap_batch<k>(items_dev, n_blocks, max_n, tab_len, st);
    NMC_QAP_CASES(NMC_CASE)
#undef NMC_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t qap_init_states(const QapDevice &I, QapReplicas &Rp, uint64_t seed,
                            const int16_t *init_dev, cudaStream_t st, bool set_best) {
  QapArgs a = make_args(I, Rp, seed);
  if (init_dev) {
    cudaError_t err = cudaMemcpyAsync(Rp.perm, init_dev, sizeof(int16_t) * (size_t)Rp.R * I.n,
                                      cudaMemcpyDeviceToDevice, st);
    if (err != cudaSuccess) return err;
    a.init_mode = set_best ? 2 : 3;
  } else {
    a.init_mode = 1;
  }
  return dispatch_qap(a, st);
}

cudaError_t qap_steps(const QapDevice &I, QapReplicas &Rp, const uint32_t *bq,
                      const uint32_t *tab, int32_t tab_len, int32_t t0, int32_t t1,
                      uint64_t seed, cudaStream_t st) {
  if (t1 <= t0) return cudaSuccess;
  QapArgs a = make_args(I, Rp, seed);
  a.bq = bq;
  a.tab = tab;
  a.tab_len = tab_len;
  a.t0 = t0;
  a.t1 = t1;
  return dispatch_qap(a, st);
}

cudaError_t qap_unpack(const QapDevice &I, const QapReplicas &Rp, int16_t *perms,
                       int16_t *best_perms, int64_t *energies, int64_t *best_energies,
                       cudaStream_t st) {
  const long long total = (long long)Rp.R * I.n;
  long long blocks = (total + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  if (blocks < 1) blocks = 1;
  qap_unpack_kernel<<<(int)blocks, 256, 0, st>>>(Rp.perm, Rp.best_perm,
                                                 (const long long *)Rp.energy,
                                                 (const long long *)Rp.best_energy, I.n, Rp.R,
                                                 perms, best_perms, energies, best_energies);
  return cudaGetLastError();
}

}  // namespace nmc
