// Whitening of k-SAT states (Sec. "Whitening procedure for low energy states"), 32 replicas per
// word. A variable turns white (star) when no clause containing it blocks it; a clause blocks v
// when it is neither satisfied by another of its variables nor holds another white variable
// (generalized form: and it is satisfied by v itself, so violated clauses never report a frozen
// variable). White sets only grow and the blocking test is monotone in them, so the parallel
// rounds used here (every variable tested against the white set as it stands, the words updated
// in place, so a round may already use bits set earlier in it) reach the same least fixed point
// as inspecting one variable at a time: every bit set is justified by bits of that fixed point,
// and a round that sets nothing certifies it. Frozen = not white at the fixed point.
//
// Per (variable v, word w) and occurrence (clause a): own = truth word of v's literal in a, o =
// OR of the other literals' truth words (rows of the state array S), so = OR of the other
// variables' white words; block = ~o & ~so (& own when generalized). Padding entries of the
// occurrence lists read as always-true literals (o = ~0) and never block.
#include "nmc_internal.h"

namespace nmc {

namespace {

constexpr int kWhiteBlock = 256;

// star: the white words, read and updated in place (one writer per word; a read sees the old or
// the new word, both below the fixed point).
template <int KQ>
__global__ void white_round_kernel(const int4 *__restrict__ occ, const int32_t *__restrict__ occ_ptr,
                                   const uint32_t *__restrict__ X, int32_t xrows2, int32_t n,
                                   int32_t W, uint32_t *star, int generalized, int32_t *changed) {
  const long long total = (long long)n * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(i / W), w = (int)(i % W);
    const uint32_t s0 = star[i];
    if (s0 == 0xFFFFFFFFu) continue;
    // truth word of literal id l (2u + neg): the state row of u, complemented when negated; the
    // padding literals 2n (false) and 2n+1 (true) address the constant rows / zero star row n
    auto lit = [&](int l) -> uint32_t {
      const int u = l >> 1;
      const uint32_t xu = u < n ? X[(size_t)u * xrows2 * W + w] : 0u;
      return (l & 1) ? ~xu : xu;
    };
    auto st = [&](int l) -> uint32_t { return (l >> 1) < n ? star[(size_t)(l >> 1) * W + w] : 0u; };
    const uint32_t x = X[(size_t)v * xrows2 * W + w];
    uint32_t blocked = 0u;
    for (int e = occ_ptr[v]; e < occ_ptr[v + 1]; ++e) {
      const int4 q = occ[(size_t)e * KQ];
      uint32_t o = lit(q.y) | lit(q.z) | lit(q.w);
      uint32_t so = st(q.y) | st(q.z) | st(q.w);
      if (KQ == 2) {
        const int4 q2 = occ[(size_t)e * KQ + 1];
        o |= lit(q2.x) | lit(q2.y) | lit(q2.z) | lit(q2.w);
        so |= st(q2.x) | st(q2.y) | st(q2.z) | st(q2.w);
      }
      uint32_t b = ~o & ~so;
      if (generalized) b &= x ^ (uint32_t)q.x;  // v's own literal is true
      blocked |= b;
    }
    const uint32_t s1 = s0 | ~blocked;
    if (s1 != s0) {
      star[i] = s1;
      *changed = 1;
    }
  }
}

// frozen count of replica 32w + j: variables whose white bit j stays clear. A warp takes a
// (32-variable group, word) pair at a time: lane l loads variable 32g + l's frozen bits, and one
// ballot per replica bit counts them; lane j keeps replica j's sum. count must start at zero.
__global__ void white_count_kernel(const uint32_t *__restrict__ star, int32_t n, int32_t R, int32_t W,
                                   int32_t *count) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long groups = (n + 31) / 32;
  int mine = 0, w_cur = -1;
  for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < groups * W; i += warps) {
    const int w = (int)(i % W);
    const long long g = i / W;
    if (w != w_cur) {  // flush the running sum when the word changes (warp-uniform)
      if (w_cur >= 0 && 32 * w_cur + lane < R && mine) atomicAdd(&count[32 * w_cur + lane], mine);
      mine = 0;
      w_cur = w;
    }
    const long long v = 32 * g + lane;
    const uint32_t x = v < n ? ~star[(size_t)v * W + w] : 0u;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int c = __popc(__ballot_sync(0xFFFFFFFFu, (x >> r) & 1u));
      if (lane == r) mine += c;
    }
  }
  if (w_cur >= 0 && 32 * w_cur + lane < R && mine) atomicAdd(&count[32 * w_cur + lane], mine);
}

// frozen[r][orig v] = 1 - white bit.
__global__ void white_unpack_kernel(const uint32_t *__restrict__ star, const int32_t *__restrict__ orig,
                                    int32_t n, int32_t R, int32_t W, uint8_t *frozen) {
  const long long total = (long long)n * R;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / n), v = (int)(i % n);
    frozen[(size_t)r * n + orig[v]] = (star[(size_t)v * W + (r >> 5)] >> (r & 31)) & 1u ? 0 : 1;
  }
}

unsigned white_blocks(long long work) {
  long long g = (work + kWhiteBlock - 1) / kWhiteBlock;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

size_t whitening_scratch_bytes(int32_t n, int32_t W) {
  auto up = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
  return up(sizeof(uint32_t) * (size_t)(n + 1) * W) + up(sizeof(int32_t));
}

int whitening_run(const KsatDevice &I, const uint32_t *X, int32_t xrows2, int32_t R, int32_t W,
                  int generalized, void *scratch, int32_t *count, uint8_t *frozen, int32_t *rounds,
                  cudaStream_t st) {
  auto up = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
  const int32_t n = I.n;
  char *p = static_cast<char *>(scratch);
  uint32_t *a = reinterpret_cast<uint32_t *>(p); p += up(sizeof(uint32_t) * (size_t)(n + 1) * W);
  int32_t *changed = reinterpret_cast<int32_t *>(p);
  cudaError_t e;
  // rows 0..n start clear (row n: the padding literals' variable, never white)
  if ((e = cudaMemsetAsync(a, 0, sizeof(uint32_t) * (size_t)(n + 1) * W, st)) != cudaSuccess)
    return (int)e;
  int32_t r = 0;
  for (; r <= n + 1; ++r) {
    if ((e = cudaMemsetAsync(changed, 0, sizeof(int32_t), st)) != cudaSuccess) return (int)e;
    if (I.kq == 1)
      white_round_kernel<1><<<white_blocks((long long)n * W), kWhiteBlock, 0, st>>>(
          I.occ, I.occ_ptr, X, xrows2, n, W, a, generalized, changed);
    else
      white_round_kernel<2><<<white_blocks((long long)n * W), kWhiteBlock, 0, st>>>(
          I.occ, I.occ_ptr, X, xrows2, n, W, a, generalized, changed);
    if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    int32_t ch = 0;
    if ((e = cudaMemcpyAsync(&ch, changed, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return (int)e;
    if (!ch) break;
  }
  *rounds = r + 1;
  if ((e = cudaMemsetAsync(count, 0, sizeof(int32_t) * R, st)) != cudaSuccess) return (int)e;
  white_count_kernel<<<white_blocks((long long)(n + 31) / 32 * W * 32), kWhiteBlock, 0, st>>>(
      a, n, R, W, count);
  if (frozen)
    white_unpack_kernel<<<white_blocks((long long)n * R), kWhiteBlock, 0, st>>>(a, I.orig, n, R, W, frozen);
  return (int)cudaGetLastError();
}

}  // namespace nmc
