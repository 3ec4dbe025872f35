// k_merge.cu -- sum-min of listed gene pairs by merging their sorted
// multiplicity vectors: the similarity of Algorithm 2 ("Best Hit detection
// phase"), Eq. (5) numerator and denominator, for an explicit list of pairs.
//
// The all-against-all path finds the pairs that share a k-mer by walking the
// inverted index (k_summin.cu).  When the pairs are known beforehand -- the
// similarity of every BBH pair, a candidate list from elsewhere -- the paper's
// own form applies: walk the two vectors, sorted by k-mer, side by side and
// add min(mult_a, mult_b) at every k-mer they share.
//
//   1. the genes named by the list are marked and listed;
//   2. each listed gene's vector (stored unordered in the profiles) is
//      sorted by k-mer id into a workspace: one block per gene, a bitonic
//      network in shared memory (genes up to 16384 distinct k-mers) or, for
//      longer genes, the same network on a global-memory copy;
//   3. one warp per pair merges the two sorted vectors: the merged sequence
//      (ties taken from a first) is cut into 32 equal diagonals by the merge
//      path, each lane walks its part with two pointers, and a k-mer shared
//      by both genes is counted by the lane that consumes its b entry (whose
//      predecessor in the merged order is the equal a entry); a warp sum
//      gives s, and den = La + Lb - s (the Eq. (5) identity sum max = La + Lb
//      - sum min).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "pd.h"
#include "pd_host.cuh"
#include "pd_internal.cuh"

using namespace pdh;

namespace {

__global__ void k_mark_genes(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b, uint64_t n,
                             uint32_t n_genes, uint32_t* __restrict__ flag, pdg::DevErr* err) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = a[i], y = b[i];
    if (x >= n_genes || y >= n_genes) {
      pdg::raise_error(err, PD_ERR_ARG, i);
      continue;
    }
    flag[x] = 1u;
    flag[y] = 1u;
  }
}

// listed gene of each marked gene: slot[g] = its index in `genes`
__global__ void k_list_genes(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos, uint32_t n_genes,
                             const uint32_t* __restrict__ mv_n, uint32_t* __restrict__ genes,
                             uint32_t* __restrict__ slot, uint32_t* __restrict__ len) {
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n_genes; g += gridDim.x * blockDim.x) {
    if (!flag[g]) continue;
    const uint32_t x = pos[g];
    genes[x] = g;
    slot[g] = x;
    len[x] = mv_n[g];
  }
}

// Sorts gene genes[x]'s vector by k-mer id into keys[off[x] ..): key = id <<
// 32 | multiplicity.  n_pad = next_pow2(length) <= kSmem: in shared memory;
// longer vectors use `spill` (a global copy padded to its power of two).
constexpr uint32_t kSortThreads = 1024, kSortSmem = 16384;

__global__ void __launch_bounds__(kSortThreads)
    k_sort_vectors(pdg::ProfilesView P, const uint32_t* __restrict__ genes, uint32_t n_listed,
                   const unsigned long long* __restrict__ off, unsigned long long* __restrict__ keys,
                   unsigned long long* __restrict__ spill, const unsigned long long* __restrict__ spill_off) {
  extern __shared__ unsigned long long sk[];
  for (uint32_t x = blockIdx.x; x < n_listed; x += gridDim.x) {
    const uint32_t g = genes[x];
    const uint32_t n = P.mv_n[g], m0 = P.win_off[g];
    const uint32_t n_pad = pdg::next_pow2(n);
    unsigned long long* a = n_pad <= kSortSmem ? sk : spill + spill_off[x];
    for (uint32_t i = threadIdx.x; i < n_pad; i += blockDim.x)
      a[i] = i < n ? ((unsigned long long)P.mv_id[m0 + i] << 32) | P.mv_cnt[m0 + i] : ~0ull;
    __syncthreads();
    pdg::block_bitonic_sort(a, n_pad);
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) keys[off[x] + i] = a[i];
    __syncthreads();
  }
}

// First position of the merged sequence of A (m) and B (n) at diagonal d that
// comes from B: the number of A entries before it (ties: A first).
__device__ __forceinline__ uint32_t merge_path(const unsigned long long* __restrict__ A, uint32_t m,
                                               const unsigned long long* __restrict__ B, uint32_t n, uint32_t d) {
  uint32_t lo = d > n ? d - n : 0u, hi = d < m ? d : m;
  while (lo < hi) {
    const uint32_t i = (lo + hi) >> 1;  // i from A, d - i from B
    if ((A[i] >> 32) <= (B[d - i - 1] >> 32)) lo = i + 1; else hi = i;
  }
  return lo;
}

__global__ void __launch_bounds__(256)
    k_merge_pairs(pdg::ProfilesView P, const uint32_t* __restrict__ a, const uint32_t* __restrict__ b, uint64_t n,
                  const uint32_t* __restrict__ slot, const unsigned long long* __restrict__ off,
                  const uint32_t* __restrict__ len, const unsigned long long* __restrict__ keys,
                  uint32_t* __restrict__ s_out, uint32_t* __restrict__ den_out) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const uint32_t ga = a[i], gb = b[i];
    const uint32_t xa = slot[ga], xb = slot[gb];
    const unsigned long long* A = keys + off[xa];
    const unsigned long long* B = keys + off[xb];
    const uint32_t m = len[xa], nb = len[xb], total = m + nb;
    const uint32_t d0 = (uint32_t)(((unsigned long long)total * lane) / 32u);
    const uint32_t d1 = (uint32_t)(((unsigned long long)total * (lane + 1u)) / 32u);
    uint32_t ia = merge_path(A, m, B, nb, d0);
    uint32_t ib = d0 - ia;
    uint32_t s = 0;
    for (uint32_t d = d0; d < d1; ++d) {
      // take from A when B is exhausted or A's id is not larger (ties: A first)
      if (ib >= nb || (ia < m && (A[ia] >> 32) <= (B[ib] >> 32))) {
        ++ia;
      } else {
        const unsigned long long kb = B[ib];
        if (ia > 0 && (A[ia - 1] >> 32) == (kb >> 32)) s += min((uint32_t)A[ia - 1], (uint32_t)kb);
        ++ib;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const uint32_t La = P.La[ga], Lb = P.La[gb];
      if (s_out) s_out[i] = s;
      if (den_out) den_out[i] = La + Lb - s;
    }
  }
}

unsigned grid_of(uint64_t items, unsigned per_block, unsigned cap) {
  uint64_t g = (items + per_block - 1) / per_block;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(g, cap));
}

pd_status summin_list_impl(pd_ctx* c, const pd_profiles* P, const uint32_t* a, const uint32_t* b, uint64_t n,
                           uint32_t* s, uint32_t* den) {
  PhaseRange range_("pd: sum-min of listed pairs (merge)");
  pdg::Launcher* L = &c->L;
  const pdg::ProfilesView& v = P->view;
  const uint32_t G = v.n_genes;
  if (n == 0) return PD_OK;
  Buf d_a, d_b, flag, pos, tmp, genes, slot, len, off, keys, spill, spill_off, d_s, d_den;
  const uint32_t* pa = a;
  const uint32_t* pb = b;
  if (!is_device_ptr(a)) {
    ALLOC(d_a, sizeof(uint32_t) * n);
    CK(cudaMemcpyAsync(d_a.p, a, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, c->stream));
    pa = d_a.as<uint32_t>();
  }
  if (!is_device_ptr(b)) {
    ALLOC(d_b, sizeof(uint32_t) * n);
    CK(cudaMemcpyAsync(d_b.p, b, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, c->stream));
    pb = d_b.as<uint32_t>();
  }
  // ---- the genes of the list, compacted
  ALLOC(flag, sizeof(uint32_t) * std::max<uint32_t>(G, 1));
  ALLOC(pos, sizeof(uint32_t) * (G + 1));
  ALLOC(tmp, pdg::scan_temp_bytes(G + 1) + 64);
  CK(cudaMemsetAsync(flag.p, 0, sizeof(uint32_t) * std::max<uint32_t>(G, 1), c->stream));
  CK(pdg::launch_begin(L, "merge_mark"));
  k_mark_genes<<<grid_of(n, 256, 152u * 16u), 256, 0, c->stream>>>(pa, pb, n, G, flag.as<uint32_t>(), c->d_err);
  CK(pdg::launch_end(L, "merge_mark"));
  pd_status st = check_dev_err(c);
  if (st != PD_OK) return fail(c, st, "pd_summin_list: a gene index is not below n_genes");
  CK(pdg::scan_u32(L, flag.as<uint32_t>(), G, pos.as<uint32_t>(), tmp.p, c->stream));
  uint32_t n_listed = 0;
  CK(cudaMemcpyAsync(&n_listed, pos.as<uint32_t>() + G, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  ALLOC(genes, sizeof(uint32_t) * std::max<uint32_t>(n_listed, 1));
  ALLOC(slot, sizeof(uint32_t) * std::max<uint32_t>(G, 1));
  ALLOC(len, sizeof(uint32_t) * std::max<uint32_t>(n_listed, 1));
  CK(pdg::launch_begin(L, "merge_list"));
  k_list_genes<<<grid_of(G, 256, 152u * 16u), 256, 0, c->stream>>>(flag.as<uint32_t>(), pos.as<uint32_t>(), G,
                                                                   v.mv_n, genes.as<uint32_t>(), slot.as<uint32_t>(),
                                                                   len.as<uint32_t>());
  CK(pdg::launch_end(L, "merge_list"));
  // ---- workspace offsets (host: the listed genes' lengths)
  std::vector<uint32_t> h_len(n_listed);
  CK(cudaMemcpyAsync(h_len.data(), len.p, sizeof(uint32_t) * n_listed, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  std::vector<unsigned long long> h_off(n_listed + 1), h_spill(n_listed + 1);
  h_off[0] = h_spill[0] = 0;
  for (uint32_t x = 0; x < n_listed; ++x) {
    const uint32_t p2 = pdg::next_pow2(h_len[x]);
    h_off[x + 1] = h_off[x] + h_len[x];
    h_spill[x + 1] = h_spill[x] + (p2 > kSortSmem ? p2 : 0u);
  }
  ALLOC(off, sizeof(unsigned long long) * (n_listed + 1));
  ALLOC(spill_off, sizeof(unsigned long long) * (n_listed + 1));
  ALLOC(keys, sizeof(unsigned long long) * std::max<unsigned long long>(h_off[n_listed], 1));
  ALLOC(spill, sizeof(unsigned long long) * std::max<unsigned long long>(h_spill[n_listed], 1));
  CK(cudaMemcpyAsync(off.p, h_off.data(), sizeof(unsigned long long) * (n_listed + 1), cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaMemcpyAsync(spill_off.p, h_spill.data(), sizeof(unsigned long long) * (n_listed + 1),
                     cudaMemcpyHostToDevice, c->stream));
  // ---- sorted vectors, then one warp per pair
  const size_t smem = sizeof(unsigned long long) * kSortSmem;
  CK(cudaFuncSetAttribute(k_sort_vectors, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (n_listed) {
    CK(pdg::launch_begin(L, "merge_sort"));
    k_sort_vectors<<<grid_of(n_listed, 1, 152u * 2u), kSortThreads, smem, c->stream>>>(
        v, genes.as<uint32_t>(), n_listed, off.as<unsigned long long>(), keys.as<unsigned long long>(),
        spill.as<unsigned long long>(), spill_off.as<unsigned long long>());
    CK(pdg::launch_end(L, "merge_sort"));
  }
  uint32_t* ps = s;
  uint32_t* pden = den;
  if (s && !is_device_ptr(s)) {
    ALLOC(d_s, sizeof(uint32_t) * n);
    ps = d_s.as<uint32_t>();
  }
  if (den && !is_device_ptr(den)) {
    ALLOC(d_den, sizeof(uint32_t) * n);
    pden = d_den.as<uint32_t>();
  }
  CK(pdg::launch_begin(L, "merge_pairs"));
  k_merge_pairs<<<grid_of(n * 32, 256, 152u * 16u), 256, 0, c->stream>>>(
      v, pa, pb, n, slot.as<uint32_t>(), off.as<unsigned long long>(), len.as<uint32_t>(),
      keys.as<unsigned long long>(), ps, pden);
  CK(pdg::launch_end(L, "merge_pairs"));
  if (ps != s) CK(cudaMemcpyAsync(s, ps, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, c->stream));
  if (pden != den) CK(cudaMemcpyAsync(den, pden, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, c->stream));
  return check_dev_err(c);  // synchronizes: the workspace ends here
}

}  // namespace

PD_API pd_status pd_summin_list(pd_ctx* c, const pd_profiles* P, const uint32_t* a, const uint32_t* b, uint64_t n,
                                uint32_t* s, uint32_t* den) {
  if (!c || !P || (n && (!a || !b))) return PD_ERR_ARG;
  try {
    CK(cudaSetDevice(c->device));
    return summin_list_impl(c, P, a, b, n, s, den);
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_summin_list");
  }
}
