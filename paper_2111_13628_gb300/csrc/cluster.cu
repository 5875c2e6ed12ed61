// Collective (cluster) move on a k-SAT replica set: the nonlocal flip of a whole backbone
// (Fig. 1(c) caption; Sec. "Nonequilibrium Nonlocal Monte Carlo"). Replica r proposes
// x' = x xor m_r and accepts by the Metropolis rule at its own beta on dE = E(x') - E(x).
//
// Three launches on multi-spin-coded words (32 replicas per uint32):
//  1. the mask, host bytes in original variable order, packed to words mb[v][w] (new ids);
//  2. dE of every replica: a warp takes a run of clauses and its lane l the replica word
//     32 gy + l (grid row gy), so every literal's state and mask words are read as one
//     coalesced 128-byte row per warp; each lane evaluates the clauses old and proposed (literal
//     words xor the mask words), counts those that become violated and those that become
//     satisfied in bit-sliced counters, and the per-replica differences are summed in shared
//     memory and added to dE once per block;
//  3. acceptance per replica (Philox counter (move_id, 0, r>>2, "CLST"), word r&3), energies
//     and best energies, then the accepted flips and best-state copies applied word by word.
#include "bits.cuh"
#include "nmc_internal.h"
#include "philox.cuh"

namespace nmc {

namespace {

constexpr int kDeltaWarps = 8;
constexpr int kClausesPerWarp = 128;  // counts <= 128 fit the 8 bit planes below

__global__ void pack_mask_kernel(const uint8_t *__restrict__ mask, int32_t rows, int32_t n,
                                 int32_t R, int32_t W, const int32_t *__restrict__ orig,
                                 uint32_t *mb) {
  const long long total = (long long)(n + 1) * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(i / W), w = (int)(i % W);
    uint32_t bits = 0u;
    if (v < n) {  // row n (the padding literal's variable) stays zero
      const int u = orig[v];
      const int lanes = min(32, R - 32 * w);  // replicas of this word
      if (rows == 1) {
        if (mask[u]) bits = lanes == 32 ? 0xFFFFFFFFu : ((1u << lanes) - 1u);
      } else {
        for (int j = 0; j < lanes; ++j)
          if (mask[(size_t)(32 * w + j) * n + u]) bits |= 1u << j;
      }
    }
    mb[i] = bits;
  }
}

// Adds the one-bit word b to the bit-sliced counter c (8 planes).
__device__ __forceinline__ void inc8(uint32_t (&c)[8], uint32_t b) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t t = c[j] & b;
    c[j] ^= b;
    b = t;
  }
}

// grid (clause runs, ceil(W / 32)): dE[32w + j] += sum over the block's clauses of (becomes
// violated) - (becomes satisfied) for replica j of word w.
__global__ void __launch_bounds__(kDeltaWarps * 32)
    cluster_delta_kernel(const int32_t *__restrict__ clits, int32_t m, int32_t kmax,
                         const uint32_t *__restrict__ S, const uint32_t *__restrict__ mb,
                         int32_t W, int32_t *dE) {
  __shared__ int part[32 * 33];  // [word lane][replica], rows padded against bank conflicts
  for (int i = threadIdx.x; i < 32 * 33; i += blockDim.x) part[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w = 32 * (int)blockIdx.y + lane;
  const bool wok = w < W;
  const long long a0 = ((long long)blockIdx.x * kDeltaWarps + warp) * kClausesPerWarp;
  const long long a1 = a0 + kClausesPerWarp < (long long)m ? a0 + kClausesPerWarp : (long long)m;
  uint32_t up[8], down[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    up[j] = 0u;
    down[j] = 0u;
  }
  for (long long a = a0; a < a1; ++a) {
    uint32_t o = 0u, on = 0u;
    for (int q = 0; q < kmax; ++q) {
      const int l = __ldg(clits + (size_t)a * kmax + q);  // literal id 2v + neg (pad 2n): warp-uniform
      if (wok) {
        const uint32_t lw = __ldg(S + (size_t)l * W + w);
        o |= lw;
        on |= lw ^ __ldg(mb + (size_t)(l >> 1) * W + w);
      }
    }
    inc8(up, o & ~on);    // satisfied -> violated: +1
    inc8(down, ~o & on);  // violated -> satisfied: -1
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const unsigned long long xu = transpose8(gather_bytes(up, q));
    const unsigned long long xd = transpose8(gather_bytes(down, q));
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int val = (int)((xu >> (8 * i)) & 0xFFull) - (int)((xd >> (8 * i)) & 0xFFull);
      if (val != 0) atomicAdd(&part[lane * 33 + 8 * q + i], val);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
    const int wl = i >> 5, j = i & 31, ww = 32 * (int)blockIdx.y + wl;
    const int v = part[wl * 33 + j];
    if (ww < W && v != 0) atomicAdd(&dE[32 * ww + j], v);
  }
}

// One thread per replica lane of every word (whole warps = whole words).
__global__ void cluster_accept_kernel(const int32_t *__restrict__ dE, const float *__restrict__ beta,
                                      int32_t R, int32_t W, const uint32_t *__restrict__ tab,
                                      int32_t tab_len, uint32_t move_id, uint32_t k0, uint32_t k1,
                                      int32_t *energy, int32_t *best_energy, uint32_t *accw,
                                      uint32_t *impw, uint8_t *acc_out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= 32 * W) return;  // 32W and blockDim are multiples of 32: whole warps leave
  bool acc = false, better = false;
  if (r < R) {
    const int d = dE[r];
    acc = d <= 0;
    if (!acc) {
      const uint32_t bq = __float2uint_rn(beta[r] * 65536.0f);  // exact product, ties to even
      const unsigned long long idx = ((unsigned long long)bq * (unsigned)d) >> 8;
      const uint4 u = philox4x32_10(make_uint4(move_id, 0u, (uint32_t)r >> 2, kTagCluster), k0, k1);
      acc = idx < (unsigned long long)tab_len && uint4_word(u, r & 3) < tab[idx];
    }
    if (acc) {
      const int e = energy[r] + d;
      energy[r] = e;
      better = e < best_energy[r];
      if (better) best_energy[r] = e;
    }
    if (acc_out) acc_out[r] = acc ? 1 : 0;
  }
  const unsigned am = __ballot_sync(0xFFFFFFFFu, acc), im = __ballot_sync(0xFFFFFFFFu, better);
  if ((threadIdx.x & 31) == 0) {
    accw[r >> 5] = am;
    impw[r >> 5] = im;
  }
}

__global__ void cluster_apply_kernel(uint32_t *S, uint32_t *best, const uint32_t *__restrict__ mb,
                                     const uint32_t *__restrict__ accw,
                                     const uint32_t *__restrict__ impw, int32_t n, int32_t W) {
  const long long total = (long long)n * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long v = i / W;
    const int w = (int)(i % W);
    const uint32_t f = mb[i] & accw[w];
    uint32_t x = S[(size_t)(2 * v) * W + w];
    if (f) {
      x ^= f;
      S[(size_t)(2 * v) * W + w] = x;
      S[(size_t)(2 * v + 1) * W + w] = ~x;
    }
    const uint32_t im = impw[w];
    if (im) best[i] = (best[i] & ~im) | (x & im);
  }
}

unsigned grid_for(long long work, int block) {
  long long g = (work + block - 1) / block;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

size_t cluster_scratch_bytes(int32_t n, int32_t W) {
  // mb (n+1)W words, dE 32W, accw W, impw W; sections on 256-byte boundaries
  auto up = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
  return up(sizeof(uint32_t) * (size_t)(n + 1) * W) + up(sizeof(int32_t) * 32 * (size_t)W) +
         2 * up(sizeof(uint32_t) * (size_t)W);
}

cudaError_t ksat_cluster_flip(const KsatDevice &I, KsatReplicas &Rp, const uint8_t *mask_dev,
                              int32_t rows, const float *beta_dev, uint32_t move_id,
                              uint64_t seed, const uint32_t *tab, int32_t tab_len, void *scratch,
                              uint8_t *acc_dev, cudaStream_t st) {
  const int32_t n = I.n, W = Rp.W;
  auto up = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
  char *p = static_cast<char *>(scratch);
  uint32_t *mb = reinterpret_cast<uint32_t *>(p);
  p += up(sizeof(uint32_t) * (size_t)(n + 1) * W);
  int32_t *dE = reinterpret_cast<int32_t *>(p);
  p += up(sizeof(int32_t) * 32 * (size_t)W);
  uint32_t *accw = reinterpret_cast<uint32_t *>(p);
  p += up(sizeof(uint32_t) * (size_t)W);
  uint32_t *impw = reinterpret_cast<uint32_t *>(p);
  cudaError_t e = cudaMemsetAsync(dE, 0, sizeof(int32_t) * 32 * (size_t)W, st);
  if (e != cudaSuccess) return e;
  pack_mask_kernel<<<grid_for((long long)(n + 1) * W, 256), 256, 0, st>>>(mask_dev, rows, n, Rp.R,
                                                                         W, I.orig, mb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (I.m > 0) {
    const long long per_block = (long long)kDeltaWarps * kClausesPerWarp;
    const dim3 grid((unsigned)((I.m + per_block - 1) / per_block), (unsigned)((W + 31) / 32));
    cluster_delta_kernel<<<grid, kDeltaWarps * 32, 0, st>>>(I.clits, I.m, I.kmax, Rp.S, mb, W, dE);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  cluster_accept_kernel<<<(unsigned)((32 * (long long)W + 255) / 256), 256, 0, st>>>(
      dE, beta_dev, Rp.R, W, tab, tab_len, move_id, static_cast<uint32_t>(seed),
      static_cast<uint32_t>(seed >> 32), Rp.energy, Rp.best_energy, accw, impw, acc_dev);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cluster_apply_kernel<<<grid_for((long long)n * W, 256), 256, 0, st>>>(Rp.S, Rp.best, mb, accw,
                                                                       impw, n, W);
  return cudaGetLastError();
}

}  // namespace nmc
