// Replica exchange (parallel tempering) and the adaptive temperature ladder (App. "Adaptive
// Parallel Tempering"). The sweeps themselves run in the batched kernel with per-replica
// temperature multipliers; this file holds the small kernels between those launches.
//
// Exchange (swap probability min{1, exp[(beta_i - beta_j)(E_i - E_j)]} for adjacent
// temperatures): ladder g has L slots with Q16 inverse temperatures lq[0..L); replica g*L + i
// belongs to it. Round q pairs the slots (k, k+1) for k = q mod 2, k+2, ...; the replicas a at
// k and b at k+1 exchange slots when d = (lq[k] - lq[k+1]) (E_a - E_b) >= 0, else when
// u < Tab[(-d) >> 8] with u = word 0 of Philox(k, q, g, "PTSW"). Pairs are disjoint, so one
// thread per pair needs no synchronisation.
//
// Ladder step: sigma(beta)^2 = <E^2> - <E>^2 over the sampled sweeps of all replicas, from
// exact integer sums (k-SAT) or per-replica double sums (QAP), then beta_next = beta +
// alpha / sigma, in IEEE double with every operation rounded on its own (no fused
// multiply-add), so the ladder is reproducible.
#include "nmc_internal.h"
#include "philox.cuh"

namespace nmc {

namespace {

// E: int (k-SAT) or long long (QAP). The product (lq[k] - lq[k+1]) (E_a - E_b) is tested from
// its sign and the 128-bit product of the magnitudes (QAP costs reach 2^33, lq 2^32).
template <typename E>
__global__ void pt_exchange_kernel(const uint32_t *__restrict__ lq, int32_t L, int32_t G,
                                   const E *__restrict__ energy, int32_t *slot, int32_t *at,
                                   uint32_t *mult, const uint32_t *__restrict__ tab,
                                   int32_t tab_len, uint32_t round, uint32_t k0, uint32_t k1) {
  const int pairs = L / 2 + 1;  // upper bound of the pairs of one ladder in either parity
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)pairs * G) return;
  const int g = (int)(id / pairs);
  const int k = (int)(round & 1u) + 2 * (int)(id % pairs);
  if (k + 1 >= L) return;
  int32_t *atg = at + (size_t)g * L;
  const int a = atg[k], b = atg[k + 1];
  const long long dl = (long long)lq[k] - (long long)lq[k + 1];
  const long long de = (long long)energy[a] - (long long)energy[b];
  bool acc = true;
  if ((dl < 0 && de > 0) || (dl > 0 && de < 0)) {  // a negative product
    const unsigned long long ma = (unsigned long long)(dl < 0 ? -dl : dl);
    const unsigned long long mb = (unsigned long long)(de < 0 ? -de : de);
    const unsigned long long hi = __umul64hi(ma, mb), lo = ma * mb;
    const unsigned long long idx = (lo >> 8) | (hi << 56);  // exact when hi < 2^8
    const uint32_t u = philox4x32_10(make_uint4((uint32_t)k, round, (uint32_t)g, kTagPtSwap), k0, k1).x;
    acc = (hi >> 8) == 0 && idx < (unsigned long long)tab_len && u < tab[idx];
  }
  if (acc) {
    atg[k] = b;
    atg[k + 1] = a;
    slot[a] = k + 1;
    slot[b] = k;
    mult[a] = lq[k + 1];
    mult[b] = lq[k];
  }
}

// Q16 of float(beta) with the schedule quantiser's rounding (exact product, ties to even).
__global__ void fill_schedule_kernel(uint32_t *bq, size_t count, double beta, int32_t *bad) {
  const float b = __double2float_rn(beta);
  if (!(b >= 0.0f && b <= 65535.0f)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(bad, 1);
    return;
  }
  const uint32_t q = __float2uint_rn(b * 65536.0f);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    bq[i] = q;
}

__global__ void ladder_step_kernel(const long long *__restrict__ stats, int32_t R, int32_t W,
                                   long long samples, double beta, double alpha, double *out) {
  __shared__ long long p1[32], p2[32];
  long long s1 = 0, s2 = 0;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    s1 += stats[r];
    s2 += stats[32 * W + r];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, o);
    s2 += __shfl_xor_sync(0xFFFFFFFFu, s2, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    p1[warp] = s1;
    p2[warp] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t1 = 0, t2 = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      t1 += p1[i];
      t2 += p2[i];
    }
    const double nn = (double)samples;
    const double mean = __ddiv_rn((double)t1, nn);
    double var = __dsub_rn(__ddiv_rn((double)t2, nn), __dmul_rn(mean, mean));
    if (var < 0.0) var = 0.0;
    const double sigma = __dsqrt_rn(var);
    out[0] = sigma;
    out[1] = __dadd_rn(beta, __ddiv_rn(alpha, sigma));
  }
}

// One thread: the per-replica double sums are added in replica order, as one sequential sum
// (a tree would round differently), then the same sigma and beta step as above.
__global__ void ladder_step_f64_kernel(const double *__restrict__ stats, int32_t R, long long samples,
                                       double beta, double alpha, double *out) {
  double t1 = 0.0, t2 = 0.0;
  for (int r = 0; r < R; ++r) {
    t1 = __dadd_rn(t1, stats[r]);
    t2 = __dadd_rn(t2, stats[(size_t)R + r]);
  }
  const double nn = (double)samples;
  const double mean = __ddiv_rn(t1, nn);
  double var = __dsub_rn(__ddiv_rn(t2, nn), __dmul_rn(mean, mean));
  if (var < 0.0) var = 0.0;
  const double sigma = __dsqrt_rn(var);
  out[0] = sigma;
  out[1] = __dadd_rn(beta, __ddiv_rn(alpha, sigma));
}

}  // namespace

cudaError_t pt_exchange(const uint32_t *lq, int32_t L, int32_t G, const int32_t *energy,
                        int32_t *slot, int32_t *at, uint32_t *mult, const uint32_t *tab,
                        int32_t tab_len, uint32_t round, uint32_t k0, uint32_t k1,
                        cudaStream_t st) {
  if (L < 2 || G < 1) return cudaSuccess;
  const long long threads = (long long)(L / 2 + 1) * G;
  const int block = 128;
  const unsigned grid = (unsigned)((threads + block - 1) / block);
  pt_exchange_kernel<int><<<grid, block, 0, st>>>(lq, L, G, energy, slot, at, mult, tab, tab_len,
                                                  round, k0, k1);
  return cudaGetLastError();
}

cudaError_t pt_exchange64(const uint32_t *lq, int32_t L, int32_t G, const long long *energy,
                          int32_t *slot, int32_t *at, uint32_t *mult, const uint32_t *tab,
                          int32_t tab_len, uint32_t round, uint32_t k0, uint32_t k1,
                          cudaStream_t st) {
  if (L < 2 || G < 1) return cudaSuccess;
  const long long threads = (long long)(L / 2 + 1) * G;
  const int block = 128;
  const unsigned grid = (unsigned)((threads + block - 1) / block);
  pt_exchange_kernel<long long><<<grid, block, 0, st>>>(lq, L, G, energy, slot, at, mult, tab,
                                                        tab_len, round, k0, k1);
  return cudaGetLastError();
}

cudaError_t fill_schedule(uint32_t *bq, size_t count, double beta, int32_t *bad, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const int block = 256;
  size_t blocks = (count + block - 1) / block;
  if (blocks > 4096) blocks = 4096;
  fill_schedule_kernel<<<(unsigned)blocks, block, 0, st>>>(bq, count, beta, bad);
  return cudaGetLastError();
}

cudaError_t ladder_step(const long long *stats, int32_t R, int32_t W, long long samples,
                        double beta, double alpha, double *out, cudaStream_t st) {
  ladder_step_kernel<<<1, 1024, 0, st>>>(stats, R, W, samples, beta, alpha, out);
  return cudaGetLastError();
}

cudaError_t ladder_step_f64(const double *stats, int32_t R, long long samples, double beta,
                            double alpha, double *out, cudaStream_t st) {
  ladder_step_f64_kernel<<<1, 1, 0, st>>>(stats, R, samples, beta, alpha, out);
  return cudaGetLastError();
}

}  // namespace nmc
